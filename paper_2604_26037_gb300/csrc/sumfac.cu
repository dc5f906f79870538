// FP64 local operator by sum factorisation (Sec. 4.1 cell matrices applied
// without forming them):
//
//   Y += alpha * sum_e Q_e^T (cK K^e + cV V^e + c_j M^e) Q_e X
//
// For affine cubic cells with tensor-product Gauss rules the cell matrices
// factor into 1D matrices:
//   K^e = (1/2)(h/2) [D (x) M (x) M + M (x) D (x) M + M (x) M (x) D]   ((p+1)-point Gauss)
//   M^e = (h/2)^3 M (x) M (x) M
//   V^e = Phi^T diag(w_q detJ V_q) Phi,  Phi = phi (x) phi (x) phi    ((p+2)-point Gauss)
// with M, D the 1D reference mass and stiffness matrices and phi the Lagrange
// basis at the 1D Gauss points.  Each application is a chain of 1D
// contractions of the (p+1)^3 nodal tensor: about 36k FMA per cell and vector
// at p = 6 instead of 2 x 343^2 = 235k for the dense H^e and M^e products.
// GB300 has little FP64 throughput, so the FP64 paths (Y = H X - S X Lambda,
// the FP64 filter form, Rayleigh-Ritz products, residuals) use this form.
//
// Block: one cell, VT vectors, 256 threads.  Shared-memory tensors are stored
// [node][vector] so that consecutive threads touch consecutive words.
#include "common.cuh"

namespace pawfe {

namespace {

template <int NP>
constexpr int sf_vt() { return NP >= 9 ? 4 : 8; }

struct SfTables {
  double M1[81], D1[81], phi[90];   // M1, D1: [np1][np1]; phi: [nq1][np1]
  double kfac, mfac;
};

template <int NP>
__global__ void __launch_bounds__(256) k_local_sf(SfTables tab, int ncells, const int *__restrict__ cell_dofs,
                                                  const double *__restrict__ wV,   // ncells x NQ^3 (w_q V_q)
                                                  const double *__restrict__ X, int ldx, double *__restrict__ Y,
                                                  int ldy, int ncols, double alpha, double cK, double cV,
                                                  double cM, const double *__restrict__ cMcol) {
  constexpr int NQ = NP + 1;
  constexpr int VT = sf_vt<NP>();
  constexpr int N3 = NP * NP * NP;
  constexpr int S1 = (NQ * NP * NP > N3) ? NQ * NP * NP : N3;
  constexpr int S2 = (NQ * NQ * NP > N3) ? NQ * NQ * NP : N3;
  constexpr int S3 = (NQ * NQ * NQ > N3) ? NQ * NQ * NQ : N3;
  __shared__ double sM[NP * NP], sD[NP * NP], sphi[NQ * NP];
  __shared__ int dofs[N3];
  extern __shared__ double sm[];
  double *A0 = sm;                 // x                  [N3][VT]
  double *A1 = A0 + N3 * VT;       // P, then y          [N3][VT]
  double *A2 = A1 + N3 * VT;       // Q, then U1, B1     [S1][VT]
  double *A3 = A2 + S1 * VT;       // S, then U2, B2     [S2][VT]
  double *A4 = A3 + S2 * VT;       // R, then U3         [S3][VT]
  double *sw = A4 + S3 * VT;       // w_q V_q            [NQ^3]
  const int e = blockIdx.x, v0 = blockIdx.y * VT, tid = threadIdx.x;
  for (int i = tid; i < NP * NP; i += 256) {
    sM[i] = tab.M1[i];
    sD[i] = tab.D1[i];
  }
  for (int i = tid; i < NQ * NP; i += 256) sphi[i] = tab.phi[i];
  for (int i = tid; i < N3; i += 256) dofs[i] = cell_dofs[(size_t)e * N3 + i];
  const bool doV = cV != 0.0;
  if (doV)
    for (int i = tid; i < NQ * NQ * NQ; i += 256) sw[i] = cV * wV[(size_t)e * NQ * NQ * NQ + i];
  __syncthreads();
  for (int idx = tid; idx < N3 * VT; idx += 256) {
    const int r = idx / VT, v = idx - r * VT;
    A0[idx] = (v0 + v < ncols) ? X[(size_t)dofs[r] * ldx + v0 + v] : 0.0;
  }
  __syncthreads();
  const double kf = cK * tab.kfac, mf = tab.mfac;
  // c-contractions: P = M_c x, Q = D_c x
  for (int idx = tid; idx < N3 * VT; idx += 256) {
    const int r = idx / VT, v = idx - r * VT;
    const int ab = r % (NP * NP), c2 = r / (NP * NP);
    double p = 0.0, q = 0.0;
#pragma unroll
    for (int c = 0; c < NP; ++c) {
      const double xv = A0[(c * NP * NP + ab) * VT + v];
      p = fma(sM[c2 * NP + c], xv, p);
      q = fma(sD[c2 * NP + c], xv, q);
    }
    A1[idx] = p;
    A2[idx] = q;
  }
  __syncthreads();
  // b-contractions: S = M_b P, R = kf (D_b P + M_b Q) + c_j mf S
  for (int idx = tid; idx < N3 * VT; idx += 256) {
    const int r = idx / VT, v = idx - r * VT;
    const int a = r % NP, b2 = (r / NP) % NP, c = r / (NP * NP);
    double s = 0.0, t = 0.0;
#pragma unroll
    for (int b = 0; b < NP; ++b) {
      const int src = ((c * NP + b) * NP + a) * VT + v;
      const double pv = A1[src];
      s = fma(sM[b2 * NP + b], pv, s);
      t = fma(sD[b2 * NP + b], pv, t);
      t = fma(sM[b2 * NP + b], A2[src], t);
    }
    const double cmv = cM + (cMcol ? ((v0 + v < ncols) ? cMcol[v0 + v] : 0.0) : 0.0);
    A3[idx] = s;
    A4[idx] = kf * t + cmv * mf * s;
  }
  __syncthreads();
  // a-contractions: y = kf D_a S + M_a R
  for (int idx = tid; idx < N3 * VT; idx += 256) {
    const int r = idx / VT, v = idx - r * VT;
    const int a2 = r % NP, bc = r / NP;
    double y = 0.0;
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      const int src = (bc * NP + a) * VT + v;
      y = fma(kf * sD[a2 * NP + a], A3[src], y);
      y = fma(sM[a2 * NP + a], A4[src], y);
    }
    A1[idx] = y;
  }
  if (doV) {
    __syncthreads();
    // U1[c][b][i] = sum_a phi[i][a] x[c][b][a]
    for (int idx = tid; idx < NQ * NP * NP * VT; idx += 256) {
      const int r = idx / VT, v = idx - r * VT;
      const int i = r % NQ, bc = r / NQ;
      double u = 0.0;
#pragma unroll
      for (int a = 0; a < NP; ++a) u = fma(sphi[i * NP + a], A0[(bc * NP + a) * VT + v], u);
      A2[idx] = u;
    }
    __syncthreads();
    // U2[c][j][i] = sum_b phi[j][b] U1[c][b][i]
    for (int idx = tid; idx < NQ * NQ * NP * VT; idx += 256) {
      const int r = idx / VT, v = idx - r * VT;
      const int i = r % NQ, j = (r / NQ) % NQ, c = r / (NQ * NQ);
      double u = 0.0;
#pragma unroll
      for (int b = 0; b < NP; ++b) u = fma(sphi[j * NP + b], A2[((c * NP + b) * NQ + i) * VT + v], u);
      A3[idx] = u;
    }
    __syncthreads();
    // U3[k][j][i] = w_q V_q sum_c phi[k][c] U2[c][j][i]
    for (int idx = tid; idx < NQ * NQ * NQ * VT; idx += 256) {
      const int r = idx / VT, v = idx - r * VT;
      const int ji = r % (NQ * NQ), k = r / (NQ * NQ);
      double u = 0.0;
#pragma unroll
      for (int c = 0; c < NP; ++c) u = fma(sphi[k * NP + c], A3[(c * NQ * NQ + ji) * VT + v], u);
      A4[idx] = u * sw[r];
    }
    __syncthreads();
    // B2[c][j][i] = sum_k phi[k][c] U3[k][j][i]
    for (int idx = tid; idx < NQ * NQ * NP * VT; idx += 256) {
      const int r = idx / VT, v = idx - r * VT;
      const int ji = r % (NQ * NQ), c = r / (NQ * NQ);
      double u = 0.0;
#pragma unroll
      for (int k = 0; k < NQ; ++k) u = fma(sphi[k * NP + c], A4[(k * NQ * NQ + ji) * VT + v], u);
      A3[idx] = u;
    }
    __syncthreads();
    // B1[c][b][i] = sum_j phi[j][b] B2[c][j][i]
    for (int idx = tid; idx < NQ * NP * NP * VT; idx += 256) {
      const int r = idx / VT, v = idx - r * VT;
      const int i = r % NQ, b = (r / NQ) % NP, c = r / (NQ * NP);
      double u = 0.0;
#pragma unroll
      for (int j = 0; j < NQ; ++j) u = fma(sphi[j * NP + b], A3[((c * NQ + j) * NQ + i) * VT + v], u);
      A2[idx] = u;
    }
    __syncthreads();
    // y[c][b][a] += sum_i phi[i][a] B1[c][b][i]
    for (int idx = tid; idx < N3 * VT; idx += 256) {
      const int r = idx / VT, v = idx - r * VT;
      const int a = r % NP, bc = r / NP;
      double u = 0.0;
#pragma unroll
      for (int i = 0; i < NQ; ++i) u = fma(sphi[i * NP + a], A2[(bc * NQ + i) * VT + v], u);
      A1[idx] += u;
    }
  }
  __syncthreads();
  for (int idx = tid; idx < N3 * VT; idx += 256) {
    const int r = idx / VT, v = idx - r * VT;
    if (v0 + v < ncols) atomicAdd(&Y[(size_t)dofs[r] * ldy + v0 + v], alpha * A1[idx]);
  }
}

template <int NP>
size_t sf_smem() {
  constexpr int NQ = NP + 1;
  constexpr int N3 = NP * NP * NP;
  constexpr int S1 = (NQ * NP * NP > N3) ? NQ * NP * NP : N3;
  constexpr int S2 = (NQ * NQ * NP > N3) ? NQ * NQ * NP : N3;
  constexpr int S3 = (NQ * NQ * NQ > N3) ? NQ * NQ * NQ : N3;
  return sizeof(double) * ((size_t)(2 * N3 + S1 + S2 + S3) * sf_vt<NP>() + NQ * NQ * NQ);
}

template <int NP>
void launch_sf(paw_context *c, const SfTables &t, const double *wV, const double *X, int ldx, double *Y, int ldy,
               int ncols, double alpha, double cK, double cV, double cM, const double *cMcol, cudaStream_t s) {
  const size_t shm = sf_smem<NP>();
  PAW_CUDA(cudaFuncSetAttribute(k_local_sf<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  dim3 g(c->ncells, (ncols + sf_vt<NP>() - 1) / sf_vt<NP>());
  k_local_sf<NP><<<g, 256, shm, s>>>(t, c->ncells, c->cell_dofs.as<int>(), wV, X, ldx, Y, ldy, ncols, alpha, cK, cV,
                                     cM, cMcol);
  PAW_LAUNCH_CHECK("k_local_sf");
}

__global__ void k_wV(int64_t n, int nq, const double *__restrict__ wq, const double *__restrict__ Vq,
                     double *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = wq[i % nq] * Vq[i];
}

}  // namespace

void local_sf(paw_context *c, const double *X, int ldx, double *Y, int ldy, int ncols, double alpha, double cK,
              double cV, double cM, const double *cMcol, cudaStream_t s) {
  if (ncols <= 0) return;
  SfTables t{};
  const int np1 = c->np1, nq1 = c->nq1;
  for (int i = 0; i < np1 * np1; ++i) {
    t.M1[i] = c->M1[i];
    t.D1[i] = c->D1[i];
  }
  for (int i = 0; i < nq1 * np1; ++i) t.phi[i] = c->phiq[i];
  const double hh = c->h / 2.0;
  t.kfac = 0.5 * hh;
  t.mfac = hh * hh * hh;
  // w_q V_q per cell (rebuilt lazily after a potential change)
  const size_t nwv = (size_t)c->ncells * c->nq;
  if (!c->wV_valid) {
    c->wV.ensure(sizeof(double) * nwv, &c->dev_bytes);
    k_wV<<<(unsigned)((nwv + 255) / 256), 256, 0, s>>>((int64_t)nwv, c->nq, c->wq64.as<double>(), c->Vq.as<double>(),
                                                       c->wV.as<double>());
    PAW_LAUNCH_CHECK("k_wV");
    c->wV_valid = 1;
  }
  const double *wV = c->wV.as<double>();
  switch (np1) {
    case 2: launch_sf<2>(c, t, wV, X, ldx, Y, ldy, ncols, alpha, cK, cV, cM, cMcol, s); break;
    case 3: launch_sf<3>(c, t, wV, X, ldx, Y, ldy, ncols, alpha, cK, cV, cM, cMcol, s); break;
    case 4: launch_sf<4>(c, t, wV, X, ldx, Y, ldy, ncols, alpha, cK, cV, cM, cMcol, s); break;
    case 5: launch_sf<5>(c, t, wV, X, ldx, Y, ldy, ncols, alpha, cK, cV, cM, cMcol, s); break;
    case 6: launch_sf<6>(c, t, wV, X, ldx, Y, ldy, ncols, alpha, cK, cV, cM, cMcol, s); break;
    case 7: launch_sf<7>(c, t, wV, X, ldx, Y, ldy, ncols, alpha, cK, cV, cM, cMcol, s); break;
    case 8: launch_sf<8>(c, t, wV, X, ldx, Y, ldy, ncols, alpha, cK, cV, cM, cMcol, s); break;
    case 9: launch_sf<9>(c, t, wV, X, ldx, Y, ldy, ncols, alpha, cK, cV, cM, cMcol, s); break;
    default: throw Error{PAW_ERR_UNSUPPORTED, "degree out of range for the sum-factorised kernel"};
  }
}

}  // namespace pawfe
