// Operator set-up for the PAW finite-element problem (Sec. 2.2, Sec. 4.1).
//
// Host: 1D Gauss / Gauss-Lobatto-Legendre rules by Newton iteration on the
// Legendre recurrence, Lagrange basis tables, the reference kinetic and mass
// cell matrices as Kronecker sums of 1D matrices (exact for affine cubes with
// tensor-product Gauss rules), the lumped GLL mass in closed form, the mesh
// numbering and the projector support lists.
// Device: the potential at the quadrature points, per-cell H^e = 1/2 K^e + V^e
// (Eq. FEM Ham entries), projector cell matrices C^{e,a} (Eq. FEM Cmatrix)
// assembled into P^a, and the projector Gram matrices G_a = P^a^T M_D^-1 P^a.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "common.cuh"

namespace pawfe {

// ============================================================== 1D rules
static void legendre_eval(int n, double x, double &P, double &Pm1) {
  // P_n(x) and P_{n-1}(x) by the three-term recurrence
  double a = 1.0, b = x;
  if (n == 0) { P = 1.0; Pm1 = 0.0; return; }
  for (int k = 1; k < n; ++k) {
    double c = ((2.0 * k + 1.0) * x * b - k * a) / (k + 1.0);
    a = b;
    b = c;
  }
  P = b;
  Pm1 = a;
}

static void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double t = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double P, Pm1;
      legendre_eval(n, t, P, Pm1);
      double dP = n * (t * P - Pm1) / (t * t - 1.0);
      double dt = P / dP;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    double P, Pm1;
    legendre_eval(n, t, P, Pm1);
    double dP = n * (t * P - Pm1) / (t * t - 1.0);
    x[n - 1 - i] = t;
    w[n - 1 - i] = 2.0 / ((1.0 - t * t) * dP * dP);
  }
}

static void gauss_lobatto(int p, std::vector<double> &x, std::vector<double> &w) {
  x.assign(p + 1, 0.0);
  w.assign(p + 1, 0.0);
  x[0] = -1.0;
  x[p] = 1.0;
  for (int i = 1; i < p; ++i) {
    // interior nodes are the roots of P_p'; start from Chebyshev-Lobatto points
    double t = -std::cos(M_PI * i / p);
    for (int it = 0; it < 100; ++it) {
      double P, Pm1;
      legendre_eval(p, t, P, Pm1);
      double d1 = p * (t * P - Pm1) / (t * t - 1.0);
      double d2 = (2.0 * t * d1 - p * (p + 1.0) * P) / (1.0 - t * t);
      double dt = d1 / d2;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    x[i] = t;
  }
  for (int i = 0; i <= p; ++i) {
    double P, Pm1;
    legendre_eval(p, x[i], P, Pm1);
    w[i] = 2.0 / (p * (p + 1.0) * P * P);
  }
}

// Lagrange polynomials on `nodes` and their derivatives at the points `t`.
static void lagrange_tables(const std::vector<double> &nodes, const std::vector<double> &t,
                            std::vector<double> &phi, std::vector<double> &dphi) {
  const int n = (int)nodes.size(), m = (int)t.size();
  phi.assign((size_t)m * n, 0.0);
  dphi.assign((size_t)m * n, 0.0);
  for (int q = 0; q < m; ++q) {
    for (int a = 0; a < n; ++a) {
      double v = 1.0;
      for (int b = 0; b < n; ++b)
        if (b != a) v *= (t[q] - nodes[b]) / (nodes[a] - nodes[b]);
      phi[(size_t)q * n + a] = v;
      double d = 0.0;
      for (int c = 0; c < n; ++c) {
        if (c == a) continue;
        double term = 1.0 / (nodes[a] - nodes[c]);
        for (int b = 0; b < n; ++b)
          if (b != a && b != c) term *= (t[q] - nodes[b]) / (nodes[a] - nodes[b]);
        d += term;
      }
      dphi[(size_t)q * n + a] = d;
    }
  }
}

void build_tables(paw_context *c) {
  const int p = c->p, np1 = c->np1, nc = c->nc;
  std::vector<double> xi, wgll;
  gauss_lobatto(p, xi, wgll);
  // 1D reference matrices with the (p+1)-point Gauss rule
  std::vector<double> g1, w1, phi, dphi;
  gauss_legendre(p + 1, g1, w1);
  lagrange_tables(xi, g1, phi, dphi);
  std::vector<double> M1((size_t)np1 * np1, 0.0), D1((size_t)np1 * np1, 0.0);
  for (int a = 0; a < np1; ++a)
    for (int b = 0; b < np1; ++b) {
      double m = 0, d = 0;
      for (int q = 0; q < p + 1; ++q) {
        m += w1[q] * phi[(size_t)q * np1 + a] * phi[(size_t)q * np1 + b];
        d += w1[q] * dphi[(size_t)q * np1 + a] * dphi[(size_t)q * np1 + b];
      }
      M1[(size_t)a * np1 + b] = m;
      D1[(size_t)a * np1 + b] = d;
    }
  c->M1 = M1;
  c->D1 = D1;
  // C1[a][b] = int l_a l_b' dxi (exact with p+1 Gauss points); its skew part is
  // centro-antisymmetric and carries the k . grad term of Eq. hij
  c->C1s.assign((size_t)np1 * np1, 0.0);
  {
    std::vector<double> C1((size_t)np1 * np1, 0.0);
    for (int a = 0; a < np1; ++a)
      for (int b = 0; b < np1; ++b) {
        double acc = 0.0;
        for (int q = 0; q < p + 1; ++q) acc += w1[q] * phi[(size_t)q * np1 + a] * dphi[(size_t)q * np1 + b];
        C1[(size_t)a * np1 + b] = acc;
      }
    for (int a = 0; a < np1; ++a)
      for (int b = 0; b < np1; ++b)
        c->C1s[(size_t)a * np1 + b] = 0.5 * (C1[(size_t)a * np1 + b] - C1[(size_t)b * np1 + a]);
  }
  const double hh = c->h / 2.0;
  c->K_ref.assign((size_t)nc * nc, 0.0);
  c->M_ref.assign((size_t)nc * nc, 0.0);
  for (int I = 0; I < nc; ++I) {
    const int a = I % np1, b = (I / np1) % np1, cc = I / (np1 * np1);
    for (int J = 0; J < nc; ++J) {
      const int a2 = J % np1, b2 = (J / np1) % np1, c2 = J / (np1 * np1);
      const double mx = M1[a * np1 + a2], my = M1[b * np1 + b2], mz = M1[cc * np1 + c2];
      const double dx = D1[a * np1 + a2], dy = D1[b * np1 + b2], dz = D1[cc * np1 + c2];
      c->K_ref[(size_t)I * nc + J] = 0.5 * hh * (dx * my * mz + mx * dy * mz + mx * my * dz);
      c->M_ref[(size_t)I * nc + J] = hh * hh * hh * mx * my * mz;
    }
  }
  // Bloch cell matrix B^e = sum_d k_d G_d, G_x = (h/2)^2 C1s (x) M1 (x) M1 (and
  // cyclic): the skew form of int N_I dN_J/dx_d per cell, whose assembly equals
  // that of int N_I dN_J/dx_d on the periodic box (Eq. hij: H_loc(k) = A - i B)
  if (c->kc) {
    std::vector<double> B((size_t)nc * nc);
    std::vector<float> Bf((size_t)nc * nc);
    const double s2 = hh * hh;
    const std::vector<double> &Cs = c->C1s;
    for (int I = 0; I < nc; ++I) {
      const int a = I % np1, b = (I / np1) % np1, cc = I / (np1 * np1);
      for (int J = 0; J < nc; ++J) {
        const int a2 = J % np1, b2 = (J / np1) % np1, c2 = J / (np1 * np1);
        const double mx = M1[a * np1 + a2], my = M1[b * np1 + b2], mz = M1[cc * np1 + c2];
        const double gx = Cs[a * np1 + a2] * my * mz, gy = mx * Cs[b * np1 + b2] * mz, gz = mx * my * Cs[cc * np1 + c2];
        const double v = s2 * (c->kvec[0] * gx + c->kvec[1] * gy + c->kvec[2] * gz);
        B[(size_t)I * nc + J] = v;
        Bf[(size_t)I * nc + J] = (float)v;
      }
    }
    c->Bk64.ensure(sizeof(double) * B.size(), &c->dev_bytes);
    c->Bk32.ensure(sizeof(float) * Bf.size(), &c->dev_bytes);
    PAW_CUDA(cudaMemcpy(c->Bk64.ptr, B.data(), sizeof(double) * B.size(), cudaMemcpyHostToDevice));
    PAW_CUDA(cudaMemcpy(c->Bk32.ptr, Bf.data(), sizeof(float) * Bf.size(), cudaMemcpyHostToDevice));
  }
  // (p+2)-point rule: interpolation matrix node -> quadrature point and weights
  std::vector<double> g2, w2, phi2, dphi2;
  gauss_legendre(p + 2, g2, w2);
  lagrange_tables(xi, g2, phi2, dphi2);
  const int nq1 = p + 2, nq = nq1 * nq1 * nq1;
  c->gq = g2;
  c->phiq = phi2;   // phiq[i * np1 + a] = phi_a(g_i)
  c->Nq.assign((size_t)nq * nc, 0.0);
  c->wq.assign(nq, 0.0);
  for (int q = 0; q < nq; ++q) {
    const int i = q % nq1, j = (q / nq1) % nq1, k = q / (nq1 * nq1);
    c->wq[q] = w2[i] * w2[j] * w2[k] * c->detJ;
    for (int I = 0; I < nc; ++I) {
      const int a = I % np1, b = (I / np1) % np1, cc = I / (np1 * np1);
      c->Nq[(size_t)q * nc + I] =
          phi2[(size_t)i * np1 + a] * phi2[(size_t)j * np1 + b] * phi2[(size_t)k * np1 + cc];
    }
  }
  // lumped GLL mass: lattice point i has weight 2 w_0 on cell faces, w_{i mod p} inside
  std::vector<double> what(c->N1);
  for (int i = 0; i < c->N1; ++i) what[i] = (i % p == 0) ? 2.0 * wgll[0] : wgll[i % p];
  std::vector<double> mdi(c->ndof);
  std::vector<float> mdf(c->ndof);
  for (int64_t d = 0; d < c->ndof; ++d) {
    const int i = (int)(d % c->N1), j = (int)((d / c->N1) % c->N1), k = (int)(d / ((int64_t)c->N1 * c->N1));
    mdi[d] = 1.0 / (hh * hh * hh * what[i] * what[j] * what[k]);
    mdf[d] = (float)mdi[d];
  }
  c->mdinv_h = mdi;
  c->md_inv64.ensure(sizeof(double) * c->ndof, &c->dev_bytes);
  c->md_inv32.ensure(sizeof(float) * c->ndof, &c->dev_bytes);
  PAW_CUDA(cudaMemcpy(c->md_inv64.ptr, mdi.data(), sizeof(double) * c->ndof, cudaMemcpyHostToDevice));
  PAW_CUDA(cudaMemcpy(c->md_inv32.ptr, mdf.data(), sizeof(float) * c->ndof, cudaMemcpyHostToDevice));
  // cell -> DoF map
  std::vector<int> dofs((size_t)c->ncells * nc);
  for (int e = 0; e < c->ncells; ++e) {
    const int cx = e % c->n, cy = (e / c->n) % c->n, cz = e / (c->n * c->n);
    for (int I = 0; I < nc; ++I) {
      const int a = I % np1, b = (I / np1) % np1, cc = I / (np1 * np1);
      const int i = (cx * p + a) % c->N1, j = (cy * p + b) % c->N1, k = (cz * p + cc) % c->N1;
      dofs[(size_t)e * nc + I] = i + c->N1 * (j + c->N1 * k);
    }
  }
  c->cell_dofs.ensure(sizeof(int) * dofs.size(), &c->dev_bytes);
  PAW_CUDA(cudaMemcpy(c->cell_dofs.ptr, dofs.data(), sizeof(int) * dofs.size(), cudaMemcpyHostToDevice));
  // shared matrices to the device
  std::vector<float> tmp((size_t)nc * nc);
  c->K64.ensure(sizeof(double) * nc * nc, &c->dev_bytes);
  c->Me64.ensure(sizeof(double) * nc * nc, &c->dev_bytes);
  c->Me32.ensure(sizeof(float) * nc * nc, &c->dev_bytes);
  PAW_CUDA(cudaMemcpy(c->K64.ptr, c->K_ref.data(), sizeof(double) * nc * nc, cudaMemcpyHostToDevice));
  PAW_CUDA(cudaMemcpy(c->Me64.ptr, c->M_ref.data(), sizeof(double) * nc * nc, cudaMemcpyHostToDevice));
  for (size_t i = 0; i < tmp.size(); ++i) tmp[i] = (float)c->M_ref[i];
  PAW_CUDA(cudaMemcpy(c->Me32.ptr, tmp.data(), sizeof(float) * nc * nc, cudaMemcpyHostToDevice));
  c->Nq64.ensure(sizeof(double) * c->Nq.size(), &c->dev_bytes);
  c->wq64.ensure(sizeof(double) * c->wq.size(), &c->dev_bytes);
  PAW_CUDA(cudaMemcpy(c->Nq64.ptr, c->Nq.data(), sizeof(double) * c->Nq.size(), cudaMemcpyHostToDevice));
  PAW_CUDA(cudaMemcpy(c->wq64.ptr, c->wq.data(), sizeof(double) * c->wq.size(), cudaMemcpyHostToDevice));
}

// ============================================================== device kernels
__global__ void k_potential(int ncells, int n, int nq1, double h, double L, const double *gq,
                            int ng, const double *cen, const double *A, const double *w,
                            double *Vq) {
  const int nq = nq1 * nq1 * nq1;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)ncells * nq) return;
  const int e = (int)(idx / nq), q = (int)(idx % nq);
  const int cx = e % n, cy = (e / n) % n, cz = e / (n * n);
  const int i = q % nq1, j = (q / nq1) % nq1, k = q / (nq1 * nq1);
  const double x = cx * h + (gq[i] + 1.0) * 0.5 * h;
  const double y = cy * h + (gq[j] + 1.0) * 0.5 * h;
  const double z = cz * h + (gq[k] + 1.0) * 0.5 * h;
  double v = 0.0;
  for (int g = 0; g < ng; ++g) {
    const double rc = 8.0 * w[g];
    const int nim = (int)ceil(rc / L);
    const double inv2w2 = 1.0 / (2.0 * w[g] * w[g]);
    for (int ix = -nim; ix <= nim; ++ix)
      for (int iy = -nim; iy <= nim; ++iy)
        for (int iz = -nim; iz <= nim; ++iz) {
          const double dx = x - (cen[3 * g] + L * ix);
          const double dy = y - (cen[3 * g + 1] + L * iy);
          const double dz = z - (cen[3 * g + 2] + L * iz);
          const double r2 = dx * dx + dy * dy + dz * dz;
          if (r2 < rc * rc) v -= A[g] * exp(-r2 * inv2w2);
        }
  }
  Vq[idx] = v;
}

// H^e[I][J] = K[I][J] + kmass Me[I][J] + sum_q Nq[q][I] Nq[q][J] wq[q] V[e][q], tiles of 32 x 32
// (kmass = 1/2 |k|^2 at a Bloch wavevector k, Eq. hij)
__global__ void __launch_bounds__(256) k_build_He(int nc, int nq, const double *__restrict__ K,
                                                  const double *__restrict__ Me, double kmass,
                                                  const double *__restrict__ Nq,
                                                  const double *__restrict__ wq,
                                                  const double *__restrict__ Vq,
                                                  double *__restrict__ He64,
                                                  float *__restrict__ He32) {
  __shared__ double As[32][33];
  __shared__ double Bs[32][33];
  const int e = blockIdx.z;
  const int I0 = blockIdx.y * 32, J0 = blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // ty in 0..7
  double acc[4] = {0, 0, 0, 0};
  const double *V = Vq + (size_t)e * nq;
  for (int q0 = 0; q0 < nq; q0 += 32) {
    for (int r = ty; r < 32; r += 8) {
      const int q = q0 + r;
      const bool ok = q < nq;
      const double wv = ok ? wq[q] * V[q] : 0.0;
      As[r][tx] = (ok && I0 + tx < nc) ? Nq[(size_t)q * nc + I0 + tx] * wv : 0.0;
      Bs[r][tx] = (ok && J0 + tx < nc) ? Nq[(size_t)q * nc + J0 + tx] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int r = 0; r < 32; ++r) {
      const double b = Bs[r][tx];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] += As[r][ty * 4 + u] * b;
    }
    __syncthreads();
  }
  const int J = J0 + tx;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int I = I0 + ty * 4 + u;
    if (I < nc && J < nc) {
      const double v = acc[u] + K[(size_t)I * nc + J] + kmass * Me[(size_t)I * nc + J];
      He64[((size_t)e * nc + I) * nc + J] = v;
      if (He32) He32[((size_t)e * nc + I) * nc + J] = (float)v;
    }
  }
}

struct ShellTable {
  int nshells;
  int l[16];
  double w[16], norm[16], rc2[16];
};

__device__ __forceinline__ void projector_values(const ShellTable &S, double dx, double dy,
                                                 double dz, double *out) {
  const double r2 = dx * dx + dy * dy + dz * dz;
  int k = 0;
  for (int s = 0; s < S.nshells; ++s) {
    const double g = (r2 < S.rc2[s]) ? S.norm[s] * exp(-r2 / (2.0 * S.w[s] * S.w[s])) : 0.0;
    if (S.l[s] == 0) {
      out[k++] = g * 0.28209479177387814;           // 1 / (2 sqrt(pi))
    } else if (S.l[s] == 1) {
      const double c1 = 0.48860251190291992 * g;    // sqrt(3 / (4 pi))
      out[k++] = c1 * dy;
      out[k++] = c1 * dz;
      out[k++] = c1 * dx;
    } else {
      const double a = 1.0925484305920792 * g;      // (1/2) sqrt(15 / pi)
      const double b = 0.31539156525252005 * g;     // (1/4) sqrt(5 / pi)
      const double d = 0.54627421529603959 * g;     // (1/4) sqrt(15 / pi)
      out[k++] = a * dx * dy;
      out[k++] = a * dy * dz;
      out[k++] = b * (2.0 * dz * dz - dx * dx - dy * dy);
      out[k++] = a * dx * dz;
      out[k++] = d * (dx * dx - dy * dy);
    }
  }
}

__device__ __forceinline__ double min_image(double d, double L) {
  return d - L * rint(d / L);
}

// One block per (cell, atom) support pair: C^{e,a} = Nq^T diag(wq) p(x_q - R_a),
// accumulated into the assembled P^a entries (FP64 atomics).
__global__ void __launch_bounds__(256) k_projector_cells(
    int npairs, const int *__restrict__ pair_cell, const int *__restrict__ pair_atom,
    const int *__restrict__ pair_ent, int n, int nq1, int nc, int npj, double h, double L,
    const double *__restrict__ gq, const double *__restrict__ pos, ShellTable S,
    const double *__restrict__ Nq, const double *__restrict__ wq, double *__restrict__ P, int npjp, double kx,
    double ky, double kz, int cplx) {
  extern __shared__ double pv[];   // [nq][npj]
  const int pr = blockIdx.x;
  const int e = pair_cell[pr], a = pair_atom[pr];
  const int nq = nq1 * nq1 * nq1;
  const int cx = e % n, cy = (e / n) % n, cz = e / (n * n);
  const double Rx = pos[3 * a], Ry = pos[3 * a + 1], Rz = pos[3 * a + 2];
  for (int q = threadIdx.x; q < nq; q += blockDim.x) {
    const int i = q % nq1, j = (q / nq1) % nq1, k = q / (nq1 * nq1);
    const double x = cx * h + (gq[i] + 1.0) * 0.5 * h;
    const double y = cy * h + (gq[j] + 1.0) * 0.5 * h;
    const double z = cz * h + (gq[k] + 1.0) * 0.5 * h;
    double vals[32];
    const double dx = min_image(x - Rx, L), dy = min_image(y - Ry, L), dz = min_image(z - Rz, L);
    projector_values(S, dx, dy, dz, vals);
    if (cplx) {
      // Bloch phase e^{-i k.(x - L_r)}, x - L_r = R_a + d (Eq. FEM Cmatrix): real and
      // imaginary parts stored as projectors 2 al and 2 al + 1 (so that the stored
      // projectors keep the order of decreasing width in pairs)
      const double th = kx * (Rx + dx) + ky * (Ry + dy) + kz * (Rz + dz);
      const double cr = cos(th), sn = sin(th);
      for (int al = 0; al < npjp; ++al) {
        pv[(size_t)q * npj + 2 * al] = vals[al] * wq[q] * cr;
        pv[(size_t)q * npj + 2 * al + 1] = -vals[al] * wq[q] * sn;
      }
    } else {
      for (int al = 0; al < npj; ++al) pv[(size_t)q * npj + al] = vals[al] * wq[q];
    }
  }
  __syncthreads();
  for (int o = threadIdx.x; o < nc * npj; o += blockDim.x) {
    const int I = o / npj, al = o % npj;
    double acc = 0.0;
    for (int q = 0; q < nq; ++q) acc += Nq[(size_t)q * nc + I] * pv[(size_t)q * npj + al];
    if (acc != 0.0) atomicAdd(&P[(size_t)pair_ent[(size_t)pr * nc + I] * npj + al], acc);
  }
}

// G_a[al][be] = sum_s P[s][al] P[s][be] / M_D[dof_s]  (one block per atom)
__global__ void k_gram(int npj, const int64_t *__restrict__ off, const int *__restrict__ dof,
                       const double *__restrict__ P, const double *__restrict__ mdinv,
                       double *__restrict__ G) {
  const int a = blockIdx.x;
  const int64_t b = off[a], en = off[a + 1];
  for (int o = threadIdx.x; o < npj * npj; o += blockDim.x) {
    const int al = o / npj, be = o % npj;
    double acc = 0.0;
    for (int64_t s = b; s < en; ++s) acc += P[s * npj + al] * P[s * npj + be] * mdinv[dof[s]];
    G[(size_t)a * npj * npj + o] = acc;
  }
}

// ============================================================== host drivers
static double radial_norm(int l, double w) {
  return std::sqrt(2.0 / (std::tgamma(l + 1.5) * std::pow(w, 2 * l + 3)));
}

void rebuild_hamiltonian(paw_context *c) {
  const int nc = c->nc;
  c->He64.ensure(sizeof(double) * (size_t)c->ncells * nc * nc, &c->dev_bytes);
  c->He32.ensure(sizeof(float) * (size_t)c->ncells * nc * nc, &c->dev_bytes);
  dim3 grid((nc + 31) / 32, (nc + 31) / 32, c->ncells);
  k_build_He<<<grid, 256>>>(nc, c->nq, c->K64.as<double>(), c->Me64.as<double>(), c->kmass, c->Nq64.as<double>(),
                            c->wq64.as<double>(), c->Vq.as<double>(), c->He64.as<double>(),
                            c->He32.as<float>());
  PAW_LAUNCH_CHECK("k_build_He");
  c->tc_tf32.valid = 0;
  c->tc_bf16.valid = 0;
  c->wV_valid = 0;
  c->wVx2_valid = 0;
  PAW_CUDA(cudaDeviceSynchronize());
}

void build_operators(paw_context *c, const paw_vloc *vloc) {
  // ---- potential at quadrature points
  c->Vq.ensure(sizeof(double) * (size_t)c->ncells * c->nq, &c->dev_bytes);
  {
    const int ng = vloc ? vloc->ngauss : 0;
    DevBuf dg;
    int64_t dummy = 0;
    std::vector<double> packed;
    packed.insert(packed.end(), c->vg_c.begin(), c->vg_c.end());
    packed.insert(packed.end(), c->vg_A.begin(), c->vg_A.end());
    packed.insert(packed.end(), c->vg_w.begin(), c->vg_w.end());
    DevBuf gqd;
    gqd.ensure(sizeof(double) * c->gq.size(), &dummy);
    PAW_CUDA(cudaMemcpy(gqd.ptr, c->gq.data(), sizeof(double) * c->gq.size(), cudaMemcpyHostToDevice));
    if (ng > 0) {
      dg.ensure(sizeof(double) * packed.size(), &dummy);
      PAW_CUDA(cudaMemcpy(dg.ptr, packed.data(), sizeof(double) * packed.size(), cudaMemcpyHostToDevice));
    }
    const double *base = dg.as<double>();
    const int64_t tot = (int64_t)c->ncells * c->nq;
    k_potential<<<(unsigned)((tot + 255) / 256), 256>>>(
        c->ncells, c->n, c->nq1, c->h, c->L, gqd.as<double>(), ng, base, base ? base + 3 * ng : nullptr,
        base ? base + 4 * ng : nullptr, c->Vq.as<double>());
    PAW_LAUNCH_CHECK("k_potential");
    PAW_CUDA(cudaDeviceSynchronize());
    dg.release(&dummy);
    gqd.release(&dummy);
  }
  rebuild_hamiltonian(c);

  // ---- projector supports
  const int natoms = c->natoms, npj = c->npjr, nc = c->nc;   // stored projectors (2 npj with k != 0)
  c->ent_off.assign(natoms + 1, 0);
  if (natoms == 0 || npj == 0) {
    c->nent = 0;
    c->npairs = 0;
    c->nown_pairs = 0;
    return;
  }
  double rmax = 0.0;
  for (double w : c->shell_w) rmax = std::max(rmax, w * std::sqrt(2.0 * std::log(1e8)));
  const double reach = rmax + c->h * std::sqrt(3.0) / 2.0 + 1e-12;
  std::vector<int> dofs_h((size_t)c->ncells * nc);
  PAW_CUDA(cudaMemcpy(dofs_h.data(), c->cell_dofs.ptr, sizeof(int) * dofs_h.size(), cudaMemcpyDeviceToHost));
  std::vector<int> pair_cell, pair_atom;
  std::vector<std::vector<int>> sup(natoms);
  for (int a = 0; a < natoms; ++a) {
    for (int e = 0; e < c->ncells; ++e) {
      const int cx = e % c->n, cy = (e / c->n) % c->n, cz = e / (c->n * c->n);
      double d2 = 0.0;
      const int cidx[3] = {cx, cy, cz};
      for (int k = 0; k < 3; ++k) {
        double d = (cidx[k] + 0.5) * c->h - c->pos[3 * a + k];
        d -= c->L * std::nearbyint(d / c->L);
        d2 += d * d;
      }
      if (d2 < reach * reach) {
        pair_cell.push_back(e);
        pair_atom.push_back(a);
        sup[a].insert(sup[a].end(), dofs_h.begin() + (size_t)e * nc, dofs_h.begin() + (size_t)(e + 1) * nc);
      }
    }
    std::sort(sup[a].begin(), sup[a].end());
    sup[a].erase(std::unique(sup[a].begin(), sup[a].end()), sup[a].end());
    c->ent_off[a + 1] = c->ent_off[a] + (int64_t)sup[a].size();
  }
  c->nent = c->ent_off[natoms];
  c->npairs = (int64_t)pair_cell.size();
  PAW_REQUIRE(c->nent < (1ll << 31) && c->npairs * nc < (1ll << 31), PAW_ERR_UNSUPPORTED,
              "projector supports exceed 2^31 entries");
  std::vector<int> ent_dof(c->nent);
  for (int a = 0; a < natoms; ++a)
    std::copy(sup[a].begin(), sup[a].end(), ent_dof.begin() + c->ent_off[a]);
  std::vector<int> pair_ent((size_t)c->npairs * nc);
  for (int64_t pr = 0; pr < c->npairs; ++pr) {
    const int e = pair_cell[pr], a = pair_atom[pr];
    for (int I = 0; I < nc; ++I) {
      const int d = dofs_h[(size_t)e * nc + I];
      const auto it = std::lower_bound(sup[a].begin(), sup[a].end(), d);
      pair_ent[(size_t)pr * nc + I] = (int)(c->ent_off[a] + (it - sup[a].begin()));
    }
  }
  // device copies
  int64_t tmpc = 0;
  DevBuf d_pc, d_pa, d_pe, d_pos, d_gq;
  d_pc.ensure(sizeof(int) * pair_cell.size(), &tmpc);
  d_pa.ensure(sizeof(int) * pair_atom.size(), &tmpc);
  d_pe.ensure(sizeof(int) * pair_ent.size(), &tmpc);
  d_pos.ensure(sizeof(double) * c->pos.size(), &tmpc);
  d_gq.ensure(sizeof(double) * c->gq.size(), &tmpc);
  PAW_CUDA(cudaMemcpy(d_pc.ptr, pair_cell.data(), sizeof(int) * pair_cell.size(), cudaMemcpyHostToDevice));
  PAW_CUDA(cudaMemcpy(d_pa.ptr, pair_atom.data(), sizeof(int) * pair_atom.size(), cudaMemcpyHostToDevice));
  PAW_CUDA(cudaMemcpy(d_pe.ptr, pair_ent.data(), sizeof(int) * pair_ent.size(), cudaMemcpyHostToDevice));
  PAW_CUDA(cudaMemcpy(d_pos.ptr, c->pos.data(), sizeof(double) * c->pos.size(), cudaMemcpyHostToDevice));
  PAW_CUDA(cudaMemcpy(d_gq.ptr, c->gq.data(), sizeof(double) * c->gq.size(), cudaMemcpyHostToDevice));
  c->ent_dof.ensure(sizeof(int) * c->nent, &c->dev_bytes);
  PAW_CUDA(cudaMemcpy(c->ent_dof.ptr, ent_dof.data(), sizeof(int) * c->nent, cudaMemcpyHostToDevice));
  c->P64.ensure(sizeof(double) * c->nent * npj, &c->dev_bytes);
  c->P32.ensure(sizeof(float) * c->nent * npj, &c->dev_bytes);
  PAW_CUDA(cudaMemset(c->P64.ptr, 0, sizeof(double) * c->nent * npj));

  ShellTable S{};
  S.nshells = (int)c->shell_l.size();
  for (int s = 0; s < S.nshells; ++s) {
    S.l[s] = c->shell_l[s];
    S.w[s] = c->shell_w[s];
    S.norm[s] = radial_norm(S.l[s], S.w[s]);
    const double rc = S.w[s] * std::sqrt(2.0 * std::log(1e8));
    S.rc2[s] = rc * rc;
  }
  const size_t shm = sizeof(double) * c->nq * npj;
  PAW_CUDA(cudaFuncSetAttribute(k_projector_cells, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  if (c->npairs > 0) {
    k_projector_cells<<<(unsigned)c->npairs, 256, shm>>>(
        (int)c->npairs, d_pc.as<int>(), d_pa.as<int>(), d_pe.as<int>(), c->n, c->nq1, nc, npj, c->h, c->L,
        d_gq.as<double>(), d_pos.as<double>(), S, c->Nq64.as<double>(), c->wq64.as<double>(),
        c->P64.as<double>(), c->npj, c->kvec[0], c->kvec[1], c->kvec[2], c->kc);
    PAW_LAUNCH_CHECK("k_projector_cells");
  }
  PAW_CUDA(cudaDeviceSynchronize());
  {
    std::vector<double> P((size_t)c->nent * npj);
    PAW_CUDA(cudaMemcpy(P.data(), c->P64.ptr, sizeof(double) * P.size(), cudaMemcpyDeviceToHost));
    std::vector<float> Pf(P.size());
    for (size_t i = 0; i < P.size(); ++i) Pf[i] = (float)P[i];
    PAW_CUDA(cudaMemcpy(c->P32.ptr, Pf.data(), sizeof(float) * Pf.size(), cudaMemcpyHostToDevice));
  }
  d_pc.release(&tmpc);
  d_pa.release(&tmpc);
  d_pe.release(&tmpc);
  d_pos.release(&tmpc);
  d_gq.release(&tmpc);

  // ---- owner-cell pairs with assembled projector values on owned nodes
  {
    const int p = c->p, N1 = c->N1;
    c->own = p * p * p;
    c->npad = npj <= 16 ? 16 : 32;
    std::vector<double> P((size_t)c->nent * npj);
    PAW_CUDA(cudaMemcpy(P.data(), c->P64.ptr, sizeof(double) * P.size(), cudaMemcpyDeviceToHost));
    std::vector<int64_t> keys;   // cell * natoms + atom
    keys.reserve(c->nent / 16 + 16);
    std::vector<int> ent_owner(c->nent), ent_slot(c->nent);
    for (int a = 0; a < natoms; ++a)
      for (int64_t s = c->ent_off[a]; s < c->ent_off[a + 1]; ++s) {
        const int d = ent_dof[s];
        const int i = d % N1, j = (d / N1) % N1, k = d / (N1 * N1);
        const int e = (i / p) + c->n * ((j / p) + c->n * (k / p));
        ent_owner[s] = e;
        ent_slot[s] = (i % p) + p * ((j % p) + p * (k % p));
        keys.push_back((int64_t)e * natoms + a);
      }
    std::sort(keys.begin(), keys.end());
    keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
    c->nown_pairs = (int64_t)keys.size();
    std::vector<int> off(c->ncells + 1, 0), oatom(keys.size());
    for (size_t k = 0; k < keys.size(); ++k) {
      off[keys[k] / natoms + 1]++;
      oatom[k] = (int)(keys[k] % natoms);
    }
    for (int e = 0; e < c->ncells; ++e) {
      c->max_own_pairs = std::max(c->max_own_pairs, off[e + 1]);
      off[e + 1] += off[e];
    }
    PAW_REQUIRE(c->max_own_pairs <= PAIRS_PER_CELL_MAX, PAW_ERR_UNSUPPORTED,
                "more than " + std::to_string(PAIRS_PER_CELL_MAX) +
                    " atoms have projector support on the nodes of one cell");
    const size_t blk = (size_t)c->own * c->npad;
    std::vector<double> oP(keys.size() * blk, 0.0);
    for (int a = 0; a < natoms; ++a)
      for (int64_t s = c->ent_off[a]; s < c->ent_off[a + 1]; ++s) {
        const int64_t key = (int64_t)ent_owner[s] * natoms + a;
        const size_t k = std::lower_bound(keys.begin(), keys.end(), key) - keys.begin();
        double *dst = oP.data() + k * blk + (size_t)ent_slot[s] * c->npad;
        for (int al = 0; al < npj; ++al) dst[al] = P[(size_t)s * npj + al];
      }
    std::vector<float> oPf(oP.size());
    for (size_t i = 0; i < oP.size(); ++i) oPf[i] = (float)oP[i];
    // groups of 4 projectors up to the last one with a nonzero value on the pair
    std::vector<int> ngrp(std::max<size_t>(1, keys.size()), 0);
    c->proj_nnz = 0;
    for (size_t i = 0; i < oP.size(); ++i) c->proj_nnz += (oP[i] != 0.0) ? 1 : 0;
    for (size_t k = 0; k < keys.size(); ++k) {
      int last = -1;
      for (int o = 0; o < c->own; ++o)
        for (int al = c->npad - 1; al > last; --al)
          if (oP[k * blk + (size_t)o * c->npad + al] != 0.0) {
            last = al;
            break;
          }
      ngrp[k] = (last + 4) / 4;
    }
    c->own_ngrp.ensure(sizeof(int) * ngrp.size(), &c->dev_bytes);
    PAW_CUDA(cudaMemcpy(c->own_ngrp.ptr, ngrp.data(), sizeof(int) * ngrp.size(), cudaMemcpyHostToDevice));
    // last nonzero group per (pair, owned node), nodes sorted by it, prefix counts per group
    {
      const int ng4 = c->npad / OWN_GROUP, own = c->own;
      std::vector<int8_t> lg(std::max<size_t>(1, keys.size() * own), -1);
      std::vector<int16_t> sidx(std::max<size_t>(1, keys.size() * own), 0);
      std::vector<int> cnt(std::max<size_t>(1, keys.size() * ng4), 0);
      for (size_t k = 0; k < keys.size(); ++k) {
        int8_t *L = lg.data() + k * own;
        for (int o = 0; o < own; ++o) {
          const double *row = oP.data() + k * blk + (size_t)o * c->npad;
          int last = -1;
          for (int al = c->npad - 1; al >= 0; --al)
            if (row[al] != 0.0) {
              last = al;
              break;
            }
          L[o] = (int8_t)(last >= 0 ? last / OWN_GROUP : -1);
          for (int g = 0; g <= L[o]; ++g) cnt[k * ng4 + g]++;
        }
        int16_t *S = sidx.data() + k * own;
        for (int o = 0; o < own; ++o) S[o] = (int16_t)o;
        std::stable_sort(S, S + own, [L](int16_t x, int16_t y) { return L[x] > L[y]; });
      }
      c->own_lg.ensure(lg.size(), &c->dev_bytes);
      c->own_sidx.ensure(sizeof(int16_t) * sidx.size(), &c->dev_bytes);
      c->own_cnt.ensure(sizeof(int) * cnt.size(), &c->dev_bytes);
      PAW_CUDA(cudaMemcpy(c->own_lg.ptr, lg.data(), lg.size(), cudaMemcpyHostToDevice));
      PAW_CUDA(cudaMemcpy(c->own_sidx.ptr, sidx.data(), sizeof(int16_t) * sidx.size(), cudaMemcpyHostToDevice));
      PAW_CUDA(cudaMemcpy(c->own_cnt.ptr, cnt.data(), sizeof(int) * cnt.size(), cudaMemcpyHostToDevice));
    }
    c->own_off.ensure(sizeof(int) * off.size(), &c->dev_bytes);
    c->own_atom.ensure(sizeof(int) * std::max<size_t>(1, oatom.size()), &c->dev_bytes);
    c->ownP64.ensure(sizeof(double) * std::max<size_t>(1, oP.size()), &c->dev_bytes);
    c->ownP32.ensure(sizeof(float) * std::max<size_t>(1, oPf.size()), &c->dev_bytes);
    PAW_CUDA(cudaMemcpy(c->own_off.ptr, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice));
    PAW_CUDA(cudaMemcpy(c->own_atom.ptr, oatom.data(), sizeof(int) * oatom.size(), cudaMemcpyHostToDevice));
    PAW_CUDA(cudaMemcpy(c->ownP64.ptr, oP.data(), sizeof(double) * oP.size(), cudaMemcpyHostToDevice));
    PAW_CUDA(cudaMemcpy(c->ownP32.ptr, oPf.data(), sizeof(float) * oPf.size(), cudaMemcpyHostToDevice));

    // atom-major index of the pairs (for the deterministic per-atom reduction)
    {
      std::vector<int> aoff(natoms + 1, 0), ap(keys.size());
      for (size_t k = 0; k < keys.size(); ++k) aoff[oatom[k] + 1]++;
      for (int a = 0; a < natoms; ++a) aoff[a + 1] += aoff[a];
      std::vector<int> fill(aoff.begin(), aoff.end() - 1);
      for (size_t k = 0; k < keys.size(); ++k) ap[fill[oatom[k]]++] = (int)k;
      c->apair_off.ensure(sizeof(int) * aoff.size(), &c->dev_bytes);
      c->apair.ensure(sizeof(int) * std::max<size_t>(1, ap.size()), &c->dev_bytes);
      PAW_CUDA(cudaMemcpy(c->apair_off.ptr, aoff.data(), sizeof(int) * aoff.size(), cudaMemcpyHostToDevice));
      PAW_CUDA(cudaMemcpy(c->apair.ptr, ap.data(), sizeof(int) * ap.size(), cudaMemcpyHostToDevice));
    }

    // atom pairs sharing an owned node somewhere, and G_ab accumulated cell by cell
    std::vector<std::vector<int>> nb(natoms);
    for (int e = 0; e < c->ncells; ++e)
      for (int k1 = off[e]; k1 < off[e + 1]; ++k1)
        for (int k2 = off[e]; k2 < off[e + 1]; ++k2) nb[oatom[k1]].push_back(oatom[k2]);
    std::vector<int> goff(natoms + 1, 0), gatom;
    for (int a = 0; a < natoms; ++a) {
      std::sort(nb[a].begin(), nb[a].end());
      nb[a].erase(std::unique(nb[a].begin(), nb[a].end()), nb[a].end());
      gatom.insert(gatom.end(), nb[a].begin(), nb[a].end());
      goff[a + 1] = (int)gatom.size();
    }
    c->ngpairs = (int64_t)gatom.size();
    const int np = c->npad;
    std::vector<double> Gf((size_t)c->ngpairs * np * np, 0.0);
    const int p3 = c->own;
    for (int e = 0; e < c->ncells; ++e) {
      std::vector<double> w(p3);
      for (int o = 0; o < p3; ++o) {
        const int a0 = o % p, b0 = (o / p) % p, c0 = o / (p * p);
        const int cx = e % c->n, cy = (e / c->n) % c->n, cz = e / (c->n * c->n);
        const int64_t d = (int64_t)(cx * p + a0) + (int64_t)N1 * ((cy * p + b0) + (int64_t)N1 * (cz * p + c0));
        w[o] = c->mdinv_h[d];
      }
      for (int k1 = off[e]; k1 < off[e + 1]; ++k1)
        for (int k2 = off[e]; k2 < off[e + 1]; ++k2) {
          const int a1 = oatom[k1], a2 = oatom[k2];
          const int slot = goff[a1] + (int)(std::lower_bound(nb[a1].begin(), nb[a1].end(), a2) - nb[a1].begin());
          double *G = Gf.data() + (size_t)slot * np * np;
          const double *P1 = oP.data() + (size_t)k1 * blk, *P2 = oP.data() + (size_t)k2 * blk;
          for (int o = 0; o < p3; ++o) {
            const double *r1 = P1 + (size_t)o * np, *r2 = P2 + (size_t)o * np;
            for (int al = 0; al < npj; ++al) {
              const double f = w[o] * r1[al];
              if (f == 0.0) continue;
              for (int be = 0; be < npj; ++be) G[al * np + be] += f * r2[be];
            }
          }
        }
    }
    c->gnb_off.ensure(sizeof(int) * goff.size(), &c->dev_bytes);
    c->gnb_atom.ensure(sizeof(int) * std::max<size_t>(1, gatom.size()), &c->dev_bytes);
    c->Gfull.ensure(sizeof(double) * std::max<size_t>(1, Gf.size()), &c->dev_bytes);
    PAW_CUDA(cudaMemcpy(c->gnb_off.ptr, goff.data(), sizeof(int) * goff.size(), cudaMemcpyHostToDevice));
    PAW_CUDA(cudaMemcpy(c->gnb_atom.ptr, gatom.data(), sizeof(int) * gatom.size(), cudaMemcpyHostToDevice));
    PAW_CUDA(cudaMemcpy(c->Gfull.ptr, Gf.data(), sizeof(double) * Gf.size(), cudaMemcpyHostToDevice));
    std::vector<float> Gf32(Gf.begin(), Gf.end());
    c->Gfull32.ensure(sizeof(float) * std::max<size_t>(1, Gf32.size()), &c->dev_bytes);
    PAW_CUDA(cudaMemcpy(c->Gfull32.ptr, Gf32.data(), sizeof(float) * Gf32.size(), cudaMemcpyHostToDevice));
  }

  // ---- G_a
  {
    DevBuf d_off, d_G;
    d_off.ensure(sizeof(int64_t) * (natoms + 1), &tmpc);
    d_G.ensure(sizeof(double) * natoms * npj * npj, &tmpc);
    PAW_CUDA(cudaMemcpy(d_off.ptr, c->ent_off.data(), sizeof(int64_t) * (natoms + 1), cudaMemcpyHostToDevice));
    k_gram<<<natoms, 256>>>(npj, d_off.as<int64_t>(), c->ent_dof.as<int>(), c->P64.as<double>(),
                            c->md_inv64.as<double>(), d_G.as<double>());
    PAW_LAUNCH_CHECK("k_gram");
    c->G.assign((size_t)natoms * npj * npj, 0.0);
    PAW_CUDA(cudaMemcpy(c->G.data(), d_G.ptr, sizeof(double) * c->G.size(), cudaMemcpyDeviceToHost));
    d_off.release(&tmpc);
    d_G.release(&tmpc);
  }
}

// Delta_Sinv^a = dS^a (I + G_a dS^a)^-1 and the positivity check of I + G^1/2 dS G^1/2.
// Positivity check of I + G^1/2 dS G^1/2 (G symmetric positive semi-definite)
// and Dsinv = dS (I + G dS)^-1 (Eq. Delta Sinv) for one atom, n x n row-major.
static void dsinv_block(int n, const double *G, const double *dS, double *Dsinv, int atom) {
  std::vector<double> Gm(G, G + (size_t)n * n), ev, V;
  jacobi_eigh(n, Gm, ev, V);
  std::vector<double> Gh((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int k = 0; k < n; ++k) s += V[(size_t)i * n + k] * std::sqrt(std::max(ev[k], 0.0)) * V[(size_t)j * n + k];
      Gh[(size_t)i * n + j] = s;
    }
  std::vector<double> Ms((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = (i == j) ? 1.0 : 0.0;
      for (int k = 0; k < n; ++k)
        for (int l = 0; l < n; ++l) s += Gh[(size_t)i * n + k] * dS[(size_t)k * n + l] * Gh[(size_t)l * n + j];
      Ms[(size_t)i * n + j] = s;
    }
  std::vector<double> ev2, V2;
  jacobi_eigh(n, Ms, ev2, V2);
  PAW_REQUIRE(ev2[0] > 0.0, PAW_ERR_NOT_SPD,
              "overlap block I + G^1/2 dS G^1/2 of atom " + std::to_string(atom) + " is not positive definite");
  std::vector<double> A((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = (i == j) ? 1.0 : 0.0;
      for (int k = 0; k < n; ++k) s += G[(size_t)i * n + k] * dS[(size_t)k * n + j];
      A[(size_t)i * n + j] = s;
    }
  PAW_REQUIRE(invert_small(n, A), PAW_ERR_NOT_SPD, "I + G dS is singular");
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int k = 0; k < n; ++k) s += dS[(size_t)i * n + k] * A[(size_t)k * n + j];
      Dsinv[(size_t)i * n + j] = s;
    }
}

void build_couplings(paw_context *c) {
  const int na = c->natoms, n = c->npj, nr = c->npjr;
  c->Dsinv.assign((size_t)na * n * n * (c->kc ? 2 : 1), 0.0);
  std::vector<double> Gpp;
  if (c->opts.pp_overlap) {
    // G_a = <p_al | p_be> for projectors on one centre (untruncated Gaussians;
    // the Bloch phases of one centre cancel, so it stays real at k != 0)
    std::vector<int> ls, ms;
    std::vector<double> ws;
    for (size_t s = 0; s < c->shell_l.size(); ++s)
      for (int m = -c->shell_l[s]; m <= c->shell_l[s]; ++m) {
        ls.push_back(c->shell_l[s]);
        ms.push_back(m);
        ws.push_back(c->shell_w[s]);
      }
    Gpp.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j)
        if (ls[i] == ls[j] && ms[i] == ms[j]) {
          const int l = ls[i];
          const double w1 = ws[i], w2 = ws[j];
          const double we2 = 2.0 * w1 * w1 * w2 * w2 / (w1 * w1 + w2 * w2);
          Gpp[(size_t)i * n + j] = radial_norm(l, w1) * radial_norm(l, w2) * 0.5 *
                                   std::tgamma(l + 1.5) * std::pow(we2, l + 1.5);
        }
    if (!c->kc)
      for (int a = 0; a < na; ++a) std::copy(Gpp.begin(), Gpp.end(), c->G.begin() + (size_t)a * n * n);
  }
  for (int a = 0; a < na; ++a) {
    const double *dS = c->dS.data() + (size_t)a * n * n;
    if (!c->kc) {
      const double *G = c->opts.pp_overlap ? Gpp.data() : c->G.data() + (size_t)a * n * n;
      dsinv_block(n, G, dS, c->Dsinv.data() + (size_t)a * n * n, a);
      continue;
    }
    // k != 0: the Gram matrix of the stored projectors (Re C_al, Im C_al at 2 al,
    // 2 al + 1) gives G_a = C^dagger M_D^-1 C = (G_rr + G_ii) + i (G_ri - G_ir); the
    // Hermitian algebra runs on the real 2n x 2n forms [[Re, -Im], [Im, Re]]
    // (sums, products and inverses map to the same forms; eigenvalues double)
    const int n2 = 2 * n;
    std::vector<double> Gc((size_t)n2 * n2, 0.0), dS2((size_t)n2 * n2, 0.0), D2((size_t)n2 * n2, 0.0);
    const double *Gs = c->G.data() + (size_t)a * nr * nr;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double gr, gi;
        if (c->opts.pp_overlap) {
          gr = Gpp[(size_t)i * n + j];
          gi = 0.0;
        } else {
          gr = Gs[(size_t)(2 * i) * nr + 2 * j] + Gs[(size_t)(2 * i + 1) * nr + 2 * j + 1];
          gi = Gs[(size_t)(2 * i) * nr + 2 * j + 1] - Gs[(size_t)(2 * i + 1) * nr + 2 * j];
        }
        Gc[(size_t)i * n2 + j] = gr;
        Gc[(size_t)(n + i) * n2 + n + j] = gr;
        Gc[(size_t)i * n2 + n + j] = -gi;
        Gc[(size_t)(n + i) * n2 + j] = gi;
        dS2[(size_t)i * n2 + j] = dS2[(size_t)(n + i) * n2 + n + j] = dS[(size_t)i * n + j];
      }
    dsinv_block(n2, Gc.data(), dS2.data(), D2.data(), a);
    double *out = c->Dsinv.data() + (size_t)a * n * n * 2;   // interleaved (re, im)
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        out[2 * ((size_t)i * n + j)] = D2[(size_t)i * n2 + j];
        out[2 * ((size_t)i * n + j) + 1] = D2[(size_t)(n + i) * n2 + j];
      }
  }
  const size_t bytes = sizeof(double) * std::max<size_t>(1, (size_t)na * n * n);
  c->DH64.ensure(bytes, &c->dev_bytes);
  c->DS64.ensure(bytes, &c->dev_bytes);
  c->DSinv64.ensure(bytes * (c->kc ? 2 : 1), &c->dev_bytes);
  if (na * n > 0) {
    PAW_CUDA(cudaMemcpy(c->DH64.ptr, c->D.data(), sizeof(double) * c->D.size(), cudaMemcpyHostToDevice));
    PAW_CUDA(cudaMemcpy(c->DS64.ptr, c->dS.data(), sizeof(double) * c->dS.size(), cudaMemcpyHostToDevice));
    PAW_CUDA(cudaMemcpy(c->DSinv64.ptr, c->Dsinv.data(), sizeof(double) * c->Dsinv.size(), cudaMemcpyHostToDevice));
  }
  build_couple_f(c);
}

// ============================================================== small host linear algebra
// Cyclic Jacobi rotations for a symmetric n x n matrix (row-major, destroyed).
// evals ascending; evecs[i*n + k] = component i of eigenvector k.
void jacobi_eigh(int n, std::vector<double> &A, std::vector<double> &evals,
                 std::vector<double> &evecs) {
  evecs.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) evecs[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        const double v = A[(size_t)i * n + j] * A[(size_t)i * n + j];
        tot += v;
        if (i != j) off += v;
      }
    if (off <= 1e-30 * std::max(tot, 1e-300)) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[(size_t)p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double cs = 1.0 / std::sqrt(t * t + 1.0), sn = t * cs;
        for (int k = 0; k < n; ++k) {
          const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
          A[(size_t)k * n + p] = cs * akp - sn * akq;
          A[(size_t)k * n + q] = sn * akp + cs * akq;
        }
        for (int k = 0; k < n; ++k) {
          const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
          A[(size_t)p * n + k] = cs * apk - sn * aqk;
          A[(size_t)q * n + k] = sn * apk + cs * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = evecs[(size_t)k * n + p], vkq = evecs[(size_t)k * n + q];
          evecs[(size_t)k * n + p] = cs * vkp - sn * vkq;
          evecs[(size_t)k * n + q] = sn * vkp + cs * vkq;
        }
      }
  }
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int i, int j) { return A[(size_t)i * n + i] < A[(size_t)j * n + j]; });
  evals.assign(n, 0.0);
  std::vector<double> V2((size_t)n * n);
  for (int k = 0; k < n; ++k) {
    evals[k] = A[(size_t)order[k] * n + order[k]];
    for (int i = 0; i < n; ++i) V2[(size_t)i * n + k] = evecs[(size_t)i * n + order[k]];
  }
  evecs.swap(V2);
}

// Gauss-Jordan inversion with partial pivoting; returns false if singular.
bool invert_small(int n, std::vector<double> &A) {
  std::vector<double> Inv((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Inv[(size_t)i * n + i] = 1.0;
  double scale = 0.0;
  for (double v : A) scale = std::max(scale, std::fabs(v));
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(A[(size_t)r * n + col]) > std::fabs(A[(size_t)piv * n + col])) piv = r;
    if (std::fabs(A[(size_t)piv * n + col]) <= 1e-14 * scale) return false;
    if (piv != col)
      for (int k = 0; k < n; ++k) {
        std::swap(A[(size_t)piv * n + k], A[(size_t)col * n + k]);
        std::swap(Inv[(size_t)piv * n + k], Inv[(size_t)col * n + k]);
      }
    const double d = 1.0 / A[(size_t)col * n + col];
    for (int k = 0; k < n; ++k) {
      A[(size_t)col * n + k] *= d;
      Inv[(size_t)col * n + k] *= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      const double f = A[(size_t)r * n + col];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) {
        A[(size_t)r * n + k] -= f * A[(size_t)col * n + k];
        Inv[(size_t)r * n + k] -= f * Inv[(size_t)col * n + k];
      }
    }
  }
  A.swap(Inv);
  return true;
}

}  // namespace pawfe
