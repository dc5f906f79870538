// Nonlocal PAW terms on the GPU (Eq. FE nonlocal contribution, Eqs. Sinvapprox
// and Delta Sinv) in an owner-cell formulation.
//
// Every DoF is owned by exactly one cell (its local indices a, b, c < p).  A
// block handles the p^3 owned nodes of one cell for a tile of vectors and the
// (cell, atom) pairs k whose P^a is nonzero on those nodes (assembled values
// P[k][o][al], padded to npad projectors):
//   projection  U[k][al][v]  = sum_o P[k][o][al] s(o) X[o][v]       (per-pair partials,
//               then a fixed-order sum over the pairs of each atom)
//   coupling    W[a] = C[a] U[a]                                    (small dense npj x npj)
//   expansion   S[o][v]      = sum_k sum_al P[k][o][al] W[a_k][al][v] (no atomics: rows are owned)
// so each owned row is read once per pass instead of once per atom whose
// support contains it.  One filter step needs one projection: with
// T = M_D^-1 (R - sum_b P^b W_S[b]) the coefficients of the nonlocal H term
// follow from P^a^T T = U^a - sum_b G_ab W_S[b], G_ab = P^a^T M_D^-1 P^b.
//
// The recurrence expansion adds the term (2 zeta/e) Y Lambda_Y "in full
// precision" without FP64 instructions: Y is split once per block into two
// FP32 words (hi + lo) and the product and sum are formed with error-free
// FP32 transformations (about 48 significant bits), then rounded once to FP32.
#include <mutex>
#include <string>

#include "common.cuh"
#include "f32x2.cuh"
#include "nonlocal_common.cuh"

namespace pawfe {

template <typename T>
struct ProjCfg;
template <>
struct ProjCfg<float> {
  static constexpr int VT = 64;
};
template <typename T>
struct ExpCfg;
template <>
struct ExpCfg<float> {
  static constexpr int VT = 32;       // vectors per CTA; 4 when the W of a cell's pairs would not fit
};

constexpr int OWN_MAX = 512;   // p <= 8

// Offsets of the owned nodes of cell e relative to its first owned DoF.
__device__ __forceinline__ int64_t owned_table(int e, int n, int p, int N1, int *ooff, int own) {
  for (int o = threadIdx.x; o < own; o += blockDim.x) ooff[o] = owned_offset(o, p, N1);
  return owned_base(e, n, p, N1);
}

// 4 consecutive elements, 16-byte aligned (one 16-byte access for float, two for double)
__device__ __forceinline__ void ld4(const float *p, float (&r)[4]) {
  const float4 q = *reinterpret_cast<const float4 *>(p);
  r[0] = q.x;
  r[1] = q.y;
  r[2] = q.z;
  r[3] = q.w;
}
__device__ __forceinline__ void ld4(const double *p, double (&r)[4]) {
  const double2 a = reinterpret_cast<const double2 *>(p)[0];
  const double2 b = reinterpret_cast<const double2 *>(p)[1];
  r[0] = a.x;
  r[1] = a.y;
  r[2] = b.x;
  r[3] = b.y;
}
__device__ __forceinline__ void st4(float *p, const float (&r)[4]) {
  *reinterpret_cast<float4 *>(p) = make_float4(r[0], r[1], r[2], r[3]);
}
__device__ __forceinline__ void st4(double *p, const double (&r)[4]) {
  reinterpret_cast<double2 *>(p)[0] = make_double2(r[0], r[1]);
  reinterpret_cast<double2 *>(p)[1] = make_double2(r[2], r[3]);
}

// ------------------------------------------------------------------ projection
// FP32 SIMT form (the FP64 form is k_own_project64 below).
// Thread tile 4 projectors x 4 vectors; the owned nodes are split over OG
// thread groups whose partial sums are reduced through shared memory.
template <typename T, int NPAD>
__global__ void __launch_bounds__(256) k_own_project(int n, int p, int N1, const int *__restrict__ own_off,
                                                     const int *__restrict__ own_ngrp, const T *__restrict__ oP,
                                                     const T *__restrict__ X, int ldx, int ncols,
                                                     const T *__restrict__ rowscale, int npj, T *__restrict__ U,
                                                     int x_aligned) {
  constexpr int VT = ProjCfg<T>::VT;
  constexpr int TPG = (NPAD / 4) * (VT / 4);   // threads per node group
  constexpr int OG = 256 / TPG;                // node groups
  __shared__ int ooff[OWN_MAX];
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int e = blockIdx.y, v0 = blockIdx.x * VT;   // vector tiles of one cell are adjacent: P reused from L2
  const int k0 = own_off[e], k1 = own_off[e + 1];
  if (k0 == k1) return;
  const int own = p * p * p;
  T *Xs = reinterpret_cast<T *>(sm_raw);          // [own][VT]
  T *red = Xs + (size_t)own * VT;                 // [OG][NPAD][VT]
  const int tid = threadIdx.x;
  const int64_t base = owned_table(e, n, p, N1, ooff, own);
  __syncthreads();
  const bool vec = x_aligned != 0;   // base and row pitch of X 16-byte aligned (checked on the host)
  for (int idx = tid; idx < own * (VT / 4); idx += 256) {
    const int o = idx / (VT / 4), q = idx - o * (VT / 4);
    const int64_t d = base + ooff[o];
    const int v = v0 + 4 * q;
    T x[4];
    if (vec && v + 3 < ncols) {
      ld4(X + d * ldx + v, x);
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) x[j] = (v + j < ncols) ? X[d * ldx + v + j] : T(0);
    }
    if (rowscale) {
      const T s = rowscale[d];
#pragma unroll
      for (int j = 0; j < 4; ++j) x[j] *= s;
    }
    st4(Xs + (size_t)o * VT + 4 * q, x);
  }
  __syncthreads();
  // vector quad fastest, then node group, projector quad slowest: the threads of
  // one projector quad form whole warps, so a quad that is zero on a pair is
  // skipped by entire warps
  const int vq = tid % (VT / 4);
  const int og = (tid / (VT / 4)) % OG;
  const int aq = tid / ((VT / 4) * OG);
  static_assert(((VT / 4) * OG) % 32 == 0, "one projector quad must cover whole warps");
  for (int k = k0; k < k1; ++k) {
    const T *Pk = oP + (size_t)k * own * NPAD + aq * 4;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    // projector groups past the pair's last nonzero one contribute zeros
    const int olim = (aq < own_ngrp[k]) ? own : 0;
    for (int o = og; o < olim; o += OG) {
      T pv[4], xv[4];
      ld4(Pk + (size_t)o * NPAD, pv);
      ld4(Xs + (size_t)o * VT + vq * 4, xv);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(pv[i], xv[j], acc[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) st4(red + ((size_t)og * NPAD + aq * 4 + i) * VT + vq * 4, acc[i]);
    __syncthreads();
    // per-pair partial sums: plain coalesced stores, reduced per atom by k_pair_reduce
    for (int idx = tid; idx < NPAD * VT; idx += 256) {
      const int al = idx / VT, v = idx - al * VT;
      if (v0 + v < ncols) {
        T sum = T(0);
#pragma unroll
        for (int g = 0; g < OG; ++g) sum += red[(size_t)g * NPAD * VT + idx];
        U[((size_t)k * NPAD + al) * ncols + v0 + v] = sum;
      }
    }
    __syncthreads();
  }
}

// U[a][al][v] = sum over the pairs k of atom a (fixed order) of partial[k][al][v]
// One warp per (atom, projector, 32 vectors); eight interleaved partial sums keep
// eight loads in flight, combined in a fixed order.
template <typename T>
__global__ void __launch_bounds__(32) k_pair_reduce(const int *__restrict__ aoff, const int *__restrict__ apair,
                                                    const T *__restrict__ partial, int npad, int ncols,
                                                    T *__restrict__ U) {
  constexpr int R = 8;
  const int v = blockIdx.x * 32 + threadIdx.x;
  const int al = blockIdx.y, a = blockIdx.z;
  if (v >= ncols) return;
  T acc[R];
#pragma unroll
  for (int u = 0; u < R; ++u) acc[u] = T(0);
  const int s0 = aoff[a], s1 = aoff[a + 1];
  int s = s0;
  for (; s + R - 1 < s1; s += R) {
    T x[R];
#pragma unroll
    for (int u = 0; u < R; ++u) x[u] = partial[((size_t)apair[s + u] * npad + al) * ncols + v];
#pragma unroll
    for (int u = 0; u < R; ++u) acc[u] += x[u];
  }
  for (; s < s1; ++s) acc[0] += partial[((size_t)apair[s] * npad + al) * ncols + v];
  U[((size_t)a * npad + al) * ncols + v] =
      ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
}

// ------------------------------------------------------------------ coupling
// W[a][al][v] = coup_scale * sum_be (C[a][al][be] + cs[v] C2[a][al][be]) U[a][be][v]
// (C NULL: identity; C2, cs optional); rows al >= npj are zero.
template <typename T, int NPAD>
__global__ void k_own_couple(int npj, const T *__restrict__ U, const double *__restrict__ C,
                             const double *__restrict__ C2, const double *__restrict__ cs, double coup_scale,
                             T *__restrict__ W, int ncols) {
  const int a = blockIdx.x;
  const int v = blockIdx.y * blockDim.x + threadIdx.x;
  if (v >= ncols) return;
  double u[NPAD];
#pragma unroll
  for (int be = 0; be < NPAD; ++be) u[be] = (be < npj) ? (double)U[((size_t)a * NPAD + be) * ncols + v] : 0.0;
  const double *Ca = C ? C + (size_t)a * npj * npj : nullptr;
  const double *C2a = C2 ? C2 + (size_t)a * npj * npj : nullptr;
  const double sv = cs ? cs[v] : 0.0;
  for (int al = 0; al < NPAD; ++al) {
    double w = 0.0;
    if (al < npj) {
      if (Ca) {
#pragma unroll
        for (int be = 0; be < NPAD; ++be)
          if (be < npj) w += (Ca[al * npj + be] + (C2a ? sv * C2a[al * npj + be] : 0.0)) * u[be];
      } else {
#pragma unroll
        for (int be = 0; be < NPAD; ++be)
          if (be == al) w = u[be];
      }
    }
    W[((size_t)a * NPAD + al) * ncols + v] = (T)(coup_scale * w);
  }
}

// W_H[a] = scale * D_H[a] (U[a] - sum_b G_ab W_S[b])  (= scale D_H P^a^T Shat^-1 R)
// accumulated in the arithmetic of T (FP32 for the FP32 / TF32 / BF16 filter).
// Block = (atom a, 32 vectors), warp be = projector be: t[be][v] over the atoms
// b that share support nodes with a (G rows read as warp broadcasts), then
// W_H = D_H t through shared memory.
template <typename T, int NPAD>
__global__ void __launch_bounds__(NPAD * 32) k_own_couple_h(int npj, const int *__restrict__ goff,
                                                            const int *__restrict__ gatom, const T *__restrict__ G,
                                                            const T *__restrict__ U, const T *__restrict__ WS,
                                                            const double *__restrict__ DH, double scale,
                                                            T *__restrict__ WH, int ncols) {
  __shared__ T ts[NPAD][32];
  const int a = blockIdx.x, lane = threadIdx.x & 31, be = threadIdx.x >> 5;
  const int v = blockIdx.y * 32 + lane;
  const int vc = v < ncols ? v : ncols - 1;   // in-range column for the loads of idle lanes
  T t = T(0);
  if (be < npj) {
    t = U[((size_t)a * NPAD + be) * ncols + vc];
    for (int s = goff[a]; s < goff[a + 1]; ++s) {
      const T *Gr = G + ((size_t)s * NPAD + be) * NPAD;
      const T *w = WS + (size_t)gatom[s] * NPAD * ncols + vc;
      T acc = T(0);
      for (int ga = 0; ga < npj; ++ga) acc = fma(Gr[ga], w[(size_t)ga * ncols], acc);
      t -= acc;
    }
  }
  ts[be][lane] = t;
  __syncthreads();
  const int al = be;
  T w = T(0);
  if (al < npj) {
    const double *Da = DH + ((size_t)a * npj + al) * npj;
    for (int b2 = 0; b2 < npj; ++b2) w = fma(T(Da[b2]), ts[b2][lane], w);
  }
  if (v < ncols) WH[((size_t)a * NPAD + al) * ncols + v] = (T)(scale * (double)w);
}

// Fused coupling of the FP32 filter loop.  Both outputs follow from U alone:
//   W_S[a] = DeltaSinv_a U[a],
//   W_H[a] = alpha D_H,a (U[a] - sum_b G_ab W_S[b]) = alpha sum_s F_s U[b_s],
//   F_s    = D_H,a (delta_{a b_s} I - G_{a b_s} DeltaSinv_{b_s})
// over the Gram slots s of atom a (its list holds a itself).  The blocks F_s are
// formed once in FP64 (k_couple_f) and rounded to FP32, so one launch replaces
// the chain W_S -> sum_b G_ab W_S[b] -> D_H (.), whose steps each waited on
// global-memory latency.
//
// k_couple_f: block = atom a, thread (r, col) of an npad x npad tile.
template <int NPAD>
__global__ void __launch_bounds__(NPAD * NPAD) k_couple_f(int npj, const int *__restrict__ goff,
                                                          const int *__restrict__ gatom, const double *__restrict__ G,
                                                          const double *__restrict__ Dsinv,
                                                          const double *__restrict__ DH, float *__restrict__ F,
                                                          float *__restrict__ Ds32) {
  __shared__ double M[NPAD][NPAD + 1];
  const int a = blockIdx.x;
  const int r = threadIdx.x / NPAD, col = threadIdx.x % NPAD;
  const bool in = r < npj && col < npj;
  const double *Da = DH + (size_t)a * npj * npj;
  Ds32[((size_t)a * NPAD + r) * NPAD + col] = in ? (float)Dsinv[(size_t)a * npj * npj + r * npj + col] : 0.f;
  for (int s = goff[a]; s < goff[a + 1]; ++s) {
    const int b = gatom[s];
    const double *Gs = G + (size_t)s * NPAD * NPAD;
    const double *Db = Dsinv + (size_t)b * npj * npj;
    double m = 0.0;   // (G_ab DeltaSinv_b)[r][col]
    if (in)
      for (int ga = 0; ga < npj; ++ga) m = fma(Gs[r * NPAD + ga], Db[ga * npj + col], m);
    __syncthreads();   // the previous slot's readers of M are done
    M[r][col] = m;
    __syncthreads();
    double f = 0.0;
    if (in) {
      f = (b == a) ? Da[r * npj + col] : 0.0;
      for (int be = 0; be < npj; ++be) f = fma(-Da[r * npj + be], M[be][col], f);
    }
    F[((size_t)s * NPAD + r) * NPAD + col] = (float)f;
  }
}

// k_own_couple_sh: block = (atom a, 32 vectors), lane = vector; warp w sums the
// slots s = goff[a] + w, + NW, ... into all npj rows, the NW partial sums meet in
// shared memory.  F rows are warp-uniform float4 loads (padded columns are zero),
// U columns coalesced 128-byte loads.  Rows al >= npj of W_S and W_H are zero.
template <int NPAD, int NW>
__global__ void __launch_bounds__(NW * 32) k_own_couple_sh(int npj, const int *__restrict__ goff,
                                                           const int *__restrict__ gatom, const float *__restrict__ F,
                                                           const float *__restrict__ Ds, const float *__restrict__ U,
                                                           float alpha, float *__restrict__ WS,
                                                           float *__restrict__ WH, int ncols) {
  __shared__ float red[NW][NPAD][32];
  const int a = blockIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int v = blockIdx.y * 32 + lane;
  const int vc = v < ncols ? v : ncols - 1;   // in-range column for the loads of idle lanes
  float acc[NPAD];
#pragma unroll
  for (int al = 0; al < NPAD; ++al) acc[al] = 0.f;
  for (int s = goff[a] + w; s < goff[a + 1]; s += NW) {
    const float *Ub = U + (size_t)gatom[s] * NPAD * ncols + vc;
    float u[NPAD];
#pragma unroll
    for (int g = 0; g < NPAD; ++g) u[g] = g < npj ? Ub[(size_t)g * ncols] : 0.f;
    const float4 *Fs = reinterpret_cast<const float4 *>(F + (size_t)s * NPAD * NPAD);
#pragma unroll
    for (int al = 0; al < NPAD; ++al) {
      if (al < npj) {
        float t = acc[al];
#pragma unroll
        for (int q = 0; q < NPAD / 4; ++q) {
          const float4 f = __ldg(Fs + al * (NPAD / 4) + q);
          t = fmaf(f.x, u[4 * q], t);
          t = fmaf(f.y, u[4 * q + 1], t);
          t = fmaf(f.z, u[4 * q + 2], t);
          t = fmaf(f.w, u[4 * q + 3], t);
        }
        acc[al] = t;
      }
    }
  }
#pragma unroll
  for (int al = 0; al < NPAD; ++al) red[w][al][lane] = acc[al];
  __syncthreads();
  const float *Ua = U + (size_t)a * NPAD * ncols + vc;
  for (int al = w; al < NPAD; al += NW) {
    float h = 0.f, sv = 0.f;
    if (al < npj) {
#pragma unroll
      for (int k = 0; k < NW; ++k) h += red[k][al][lane];
      const float *Dr = Ds + ((size_t)a * NPAD + al) * NPAD;
      for (int g = 0; g < npj; ++g) sv = fmaf(Dr[g], Ua[(size_t)g * ncols], sv);
    }
    if (v < ncols) {
      WS[((size_t)a * NPAD + al) * ncols + v] = sv;
      WH[((size_t)a * NPAD + al) * ncols + v] = alpha * h;
    }
  }
}

// ------------------------------------------------------------------ Bloch wavevector (k != 0)
// Complex multivectors are split blocks [Re X | Im X] (nb = ncols / 2 columns
// each) and the projectors C^{a,k} are stored as 2 np real projectors,
// Re C_al at 2 al and Im C_al at 2 al + 1.  A projection of the split block then
// holds, per atom and complex column v, a = Re C^T Re x, b = Im C^T Re x
// (column v) and c = Re C^T Im x, d = Im C^T Im x (column v + nb), so that
// U = C^dagger x = (a + d) + i (c - b).  An expansion of coefficients W'
// gives C W = (Re C Re W - Im C Im W) + i (Re C Im W + Im C Re W) when
// W'[2 al] = Re W, W'[2 al + 1] = -Im W (column v) and W'[2 al] = Im W,
// W'[2 al + 1] = Re W (column v + nb).
// (arithmetic in T, as in the real coupling kernels: FP32 for the FP32 / TF32 /
// BF16 filter)
template <typename T>
__device__ __forceinline__ void cplx_u(const T *U, int npad, int ncols, int a, int np, int al, int v, int nb,
                                       T &ur, T &ui) {
  const size_t r0 = ((size_t)a * npad + 2 * al) * ncols, r1 = r0 + ncols;
  ur = U[r0 + v] + U[r1 + v + nb];
  ui = U[r0 + v + nb] - U[r1 + v];
}

template <typename T>
__device__ __forceinline__ void cplx_w_store(T *W, int npad, int ncols, int a, int np, int al, int v, int nb, T wr,
                                             T wi) {
  const size_t r0 = ((size_t)a * npad + 2 * al) * ncols, r1 = r0 + ncols;
  W[r0 + v] = wr;
  W[r1 + v] = -wi;
  W[r0 + v + nb] = wi;
  W[r1 + v + nb] = wr;
}

// W = coup_scale (C + cs[v] C2) U per atom and complex column: C complex
// (interleaved re, im; cplxC = 1) or real, C2 real (may be NULL), C NULL:
// identity.  Rows 2 np .. npad - 1 of W are zero.
template <typename T, int NPAD>
__global__ void k_couple_c(int np, const T *__restrict__ U, const double *__restrict__ C, int cplxC,
                           const double *__restrict__ C2, const double *__restrict__ cs, double coup_scale,
                           T *__restrict__ W, int ncols) {
  const int a = blockIdx.x, nb = ncols / 2;
  const int v = blockIdx.y * blockDim.x + threadIdx.x;
  if (v >= nb) return;
  T ur[NPAD / 2], ui[NPAD / 2];
#pragma unroll
  for (int be = 0; be < NPAD / 2; ++be) {
    ur[be] = ui[be] = T(0);
    if (be < np) cplx_u(U, NPAD, ncols, a, np, be, v, nb, ur[be], ui[be]);
  }
  const double sv = cs ? cs[v] : 0.0;
  for (int al = 0; al < np; ++al) {
    T wr = T(0), wi = T(0);
    if (C) {
#pragma unroll
      for (int be = 0; be < NPAD / 2; ++be) {
        if (be >= np) break;
        T kr, ki;
        if (cplxC) {
          kr = (T)C[2 * (((size_t)a * np + al) * np + be)];
          ki = (T)C[2 * (((size_t)a * np + al) * np + be) + 1];
        } else {
          kr = (T)(C[((size_t)a * np + al) * np + be] + (C2 ? sv * C2[((size_t)a * np + al) * np + be] : 0.0));
          ki = T(0);
        }
        wr += kr * ur[be] - ki * ui[be];
        wi += kr * ui[be] + ki * ur[be];
      }
    } else {
#pragma unroll
      for (int be = 0; be < NPAD / 2; ++be)
        if (be == al) {
          wr = ur[be];
          wi = ui[be];
        }
    }
    cplx_w_store(W, NPAD, ncols, a, np, al, v, nb, (T)(coup_scale * (double)wr), (T)(coup_scale * (double)wi));
  }
  for (int j = 2 * np; j < NPAD; ++j) {
    W[((size_t)a * NPAD + j) * ncols + v] = T(0);
    W[((size_t)a * NPAD + j) * ncols + v + nb] = T(0);
  }
}

// W_H = scale D_H (U - sum_b G_ab W_S[b]) with complex U, W_S and G_ab =
// C^a^dagger M_D^-1 C^b (from the Gram block of the stored projectors, rows and
// columns 2 al (real part) and 2 al + 1 (imaginary part): (G_rr + G_ii) +
// i (G_ri - G_ir)); W_S in expansion form, W_H written in it.
// Block = (atom, 32 complex columns), warp al = projector al.
template <typename T, int NPAD>
__global__ void __launch_bounds__(NPAD / 2 * 32) k_couple_h_c(int np, const int *__restrict__ goff,
                                                              const int *__restrict__ gatom,
                                                              const T *__restrict__ G, const T *__restrict__ U,
                                                              const T *__restrict__ WS,
                                                              const double *__restrict__ DH, double scale,
                                                              T *__restrict__ WH, int ncols) {
  __shared__ T tr_s[NPAD / 2][32], ti_s[NPAD / 2][32];
  const int a = blockIdx.x, lane = threadIdx.x & 31, al = threadIdx.x >> 5, nb = ncols / 2;
  const int v = blockIdx.y * 32 + lane;
  const int vc = v < nb ? v : nb - 1;
  T tr = T(0), ti = T(0);
  if (al < np) {
    cplx_u(U, NPAD, ncols, a, np, al, vc, nb, tr, ti);
    for (int s = goff[a]; s < goff[a + 1]; ++s) {
      const int b = gatom[s];
      const T *Gs = G + (size_t)s * NPAD * NPAD;
      const T *wb = WS + (size_t)b * NPAD * ncols + vc;
      const T *g0 = Gs + (2 * al) * NPAD, *g1 = g0 + NPAD;
      for (int be = 0; be < np; ++be) {
        const T gr = g0[2 * be] + g1[2 * be + 1];
        const T gi = g0[2 * be + 1] - g1[2 * be];
        const T wr = wb[(size_t)(2 * be) * ncols], wi = wb[(size_t)(2 * be) * ncols + nb];
        tr -= gr * wr - gi * wi;
        ti -= gr * wi + gi * wr;
      }
    }
    tr_s[al][lane] = tr;
    ti_s[al][lane] = ti;
  }
  __syncthreads();
  if (al < np && v < nb) {
    T wr = T(0), wi = T(0);
    const double *Da = DH + ((size_t)a * np + al) * np;
    for (int be = 0; be < np; ++be) {
      wr = fma(T(Da[be]), tr_s[be][lane], wr);
      wi = fma(T(Da[be]), ti_s[be][lane], wi);
    }
    cplx_w_store(WH, NPAD, ncols, a, np, al, v, nb, (T)(scale * (double)wr), (T)(scale * (double)wi));
  }
  if (v < nb)
    for (int j = 2 * np + al; j < NPAD; j += NPAD / 2) {
      WH[((size_t)a * NPAD + j) * ncols + v] = T(0);
      WH[((size_t)a * NPAD + j) * ncols + v + nb] = T(0);
    }
}

// ------------------------------------------------------------------ expansion
// FP32 SIMT form (the FP64 form is k_own_expand64 below).
// Expansion with a fused output stage.  W of every pair of the cell is staged
// in shared memory (VT vectors of each: 32, or 4 for cells with many pairs);
// a thread owns 4 vectors of one node row at a time.
//   EXP_ADD        Y += cs[v] * S1
//   EXP_SINV       Y  = md_inv * (X - S1)                                         (Eq. Sinvapprox)
//   EXP_RECURRENCE T  = md_inv * (R_Y - S1)
//                  R_X = [-beta R_Y - gamma R_X + S2] + alpha Y Lambda_Y   (S2: nonlocal part of alpha H T)
// with S1 = sum_k P[k][o] . W1[a_k], S2 = sum_k P[k][o] . W2[a_k].
template <typename T, int NPAD, int MODE, int VT>
__global__ void __launch_bounds__(256, 2) k_own_expand(ExpArgs A, const T *__restrict__ oP, const T *__restrict__ W1,
                                                    const T *__restrict__ W2) {
  constexpr int G = VT / 4;               // groups of 4 vectors
  constexpr int OR = 256 / G;             // node rows per pass
  constexpr int NW = (MODE == EXP_RECURRENCE) ? 2 : 1;
  __shared__ int ooff[OWN_MAX];
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int e = blockIdx.y, v0 = blockIdx.x * VT;   // vector tiles of one cell are adjacent: P reused from L2
  const int k0 = A.own_off[e], k1 = A.own_off[e + 1];
  if (MODE == EXP_ADD && k0 == k1) return;
  const int own = A.p * A.p * A.p;
  const int np = k1 - k0;
  const int ncols = A.ncols;
  T *Ws = reinterpret_cast<T *>(sm_raw);   // [NW][np][NPAD][VT]
  const int tid = threadIdx.x;
  const int64_t base = owned_table(e, A.n, A.p, A.N1, ooff, own);
  for (int idx = tid; idx < NW * np * (NPAD * VT / 4); idx += 256) {
    const int q = idx % (VT / 4), rest = idx / (VT / 4), al = rest % NPAD, r2 = rest / NPAD, kk = r2 % np,
              w = r2 / np;
    const T *Wsrc = (w == 0) ? W1 : W2;
    const int v = v0 + 4 * q;
    const T *src = Wsrc + ((size_t)A.own_atom[k0 + kk] * NPAD + al) * ncols + v;
    T x[4];
    if (ncols % 4 == 0 && v + 3 < ncols) {
      ld4(src, x);
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) x[j] = (v + j < ncols) ? src[j] : T(0);
    }
    st4(Ws + (((size_t)w * np + kk) * NPAD + al) * VT + 4 * q, x);
  }
  __syncthreads();
  const int g = tid % G, orow = tid / G;
  const int v = v0 + g * 4;
  const bool full4 = (v + 3 < ncols);
  const T *Xin = static_cast<const T *>(A.Xin);
  T *Y = static_cast<T *>(A.Y);
  T *RX = static_cast<T *>(A.RX);
  const T *mdinv = static_cast<const T *>(A.mdinv);
  const bool vec = full4 && A.vec_ok;
  // output stage of one node row o with its sums s1, s2 over the 4 vectors v .. v+3
  auto emit = [&](int o, const T (&s1)[4], const T (&s2)[4]) {
    const int64_t d = base + ooff[o];
    if (MODE == EXP_ADD) {
      T *yp = Y + d * A.ldy + v;
      if (vec) {
        T y[4];
        ld4(yp, y);
#pragma unroll
        for (int j = 0; j < 4; ++j) y[j] += (A.cs ? T(A.cs[v + j]) : T(1)) * s1[j];
        st4(yp, y);
      } else {
        for (int j = 0; j < 4; ++j)
          if (v + j < ncols) yp[j] += (A.cs ? T(A.cs[v + j]) : T(1)) * s1[j];
      }
    } else if (MODE == EXP_SINV) {
      const T m = mdinv[d];
      const T *xp = Xin + d * A.ldx + v;
      T *yp = Y + d * A.ldy + v;
      if (vec) {
        T x[4], y[4];
        ld4(xp, x);
#pragma unroll
        for (int j = 0; j < 4; ++j) y[j] = m * (x[j] - s1[j]);
        st4(yp, y);
      } else {
        for (int j = 0; j < 4; ++j)
          if (v + j < ncols) yp[j] = m * (xp[j] - s1[j]);
      }
    } else {
      const T m = mdinv[d];
      const T *rp = Xin + d * A.ldx + v;
      T *rxp = RX + d * A.ldx + v;
      T *tp = Y + d * A.ldy + v;
      T ry[4], rx[4], t[4], out[4];
      if (vec) {
        ld4(rp, ry);
        ld4(rxp, rx);
      } else {
        for (int j = 0; j < 4; ++j) {
          ry[j] = (v + j < ncols) ? rp[j] : T(0);
          rx[j] = (v + j < ncols) ? rxp[j] : T(0);
        }
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        t[j] = m * (ry[j] - s1[j]);
        const T bracket = -T(A.beta) * ry[j] - T(A.gamma) * rx[j] + s2[j];
        const int vj = min(v + j, ncols - 1);
        const float *yh = static_cast<const float *>(A.Y0);
        const float *yl = static_cast<const float *>(A.Y0lo);
        const float yhv = yh[d * A.ldy0 + vj];
        const float ylv = yl ? yl[d * A.ldy0 + vj] : 0.f;
        out[j] = add_product_df(bracket, A.chi[vj], A.clo[vj], yhv, ylv);
      }
      if (vec) {
        st4(tp, t);
        st4(rxp, out);
      } else {
        for (int j = 0; j < 4; ++j)
          if (v + j < ncols) {
            tp[j] = t[j];
            rxp[j] = out[j];
          }
      }
    }
  };
  // RB node rows per thread and pass: every W fragment read from shared memory
  // feeds RB x 4 FMAs per sum
  constexpr int RB = 4;
  for (int o0 = orow; o0 < own; o0 += OR * RB) {
    T s1[RB][4], s2[RB][4];
    int orr[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      orr[r] = min(o0 + r * OR, own - 1);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        s1[r][j] = T(0);
        s2[r][j] = T(0);
      }
    }
    for (int kk = 0; kk < np; ++kk) {
      const T *Pb = oP + (size_t)(k0 + kk) * own * NPAD;
      const T *W1k = Ws + (size_t)kk * NPAD * VT + g * 4;
      const T *W2k = Ws + ((size_t)np + kk) * NPAD * VT + g * 4;
      const int ng = A.own_ngrp[k0 + kk];   // the remaining projector groups are zero on this pair
#pragma unroll
      for (int aq = 0; aq < NPAD / 4; ++aq) {
        if (aq >= ng) break;
        T pv[RB][4];
#pragma unroll
        for (int r = 0; r < RB; ++r) ld4(Pb + (size_t)orr[r] * NPAD + aq * 4, pv[r]);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          T w1[4];
          ld4(W1k + (aq * 4 + i) * VT, w1);
#pragma unroll
          for (int r = 0; r < RB; ++r)
#pragma unroll
            for (int j = 0; j < 4; ++j) s1[r][j] = fma(pv[r][i], w1[j], s1[r][j]);
          if (NW == 2) {
            T w2[4];
            ld4(W2k + (aq * 4 + i) * VT, w2);
#pragma unroll
            for (int r = 0; r < RB; ++r)
#pragma unroll
              for (int j = 0; j < 4; ++j) s2[r][j] = fma(pv[r][i], w2[j], s2[r][j]);
          }
        }
      }
    }
#pragma unroll
    for (int r = 0; r < RB; ++r)
      if (o0 + r * OR < own) emit(o0 + r * OR, s1[r], s2[r]);
  }
}

// ------------------------------------------------------------------ FP64 forms
// GB300 retires about one warp-wide FP64 FMA per 16 SM clocks, so the FP64
// kernels spend FP64 instructions only where a projector can be nonzero: lane
// = vector (32 per CTA), and every FP64 instruction of a warp belongs to one
// owned node and one group of OWN_GROUP projectors (warp-uniform control flow),
// taken only up to the last group with a nonzero value on that node (own_lg).
// (Groups of 2 multiply 1.08 times the nonzero entries of P on the workloads
// here, groups of 4 1.23 times.)
// The same kernels run in pair-of-FP32 arithmetic (R = f32x2, f32x2.cuh) for
// the FP64-class step 2 on the FP32 pipes: projector values and coefficients
// then come as pairs, X and Y stay FP64.

// two consecutive numbers through the read-only path
__device__ __forceinline__ void ldg2(const double *p, double &a, double &b) {
  const double2 v = __ldg(reinterpret_cast<const double2 *>(p));
  a = v.x;
  b = v.y;
}
__device__ __forceinline__ void ldg2(const f32x2 *p, f32x2 &a, f32x2 &b) {
  const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
  a = {v.x, v.y};
  b = {v.z, v.w};
}
__device__ __forceinline__ double ldg1(const double *p) { return __ldg(p); }
__device__ __forceinline__ f32x2 ldg1(const f32x2 *p) {
  const float2 v = __ldg(reinterpret_cast<const float2 *>(p));
  return {v.x, v.y};
}

// Projection: warp w takes positions w, w + 8, ... of each pair's node list
// sorted by descending last nonzero group, so the eight warps share every pair
// evenly; their partial sums are added in a fixed order through shared memory.
template <int NPAD, typename R>
__global__ void __launch_bounds__(256) k_own_project64(int n, int p, int N1, const int *__restrict__ own_off,
                                                       const int *__restrict__ own_cnt,
                                                       const int16_t *__restrict__ own_sidx,
                                                       const R *__restrict__ oP, const double *__restrict__ X,
                                                       int ldx, int ncols, const double *__restrict__ rowscale,
                                                       double *__restrict__ U) {
  using A = Ar<R>;
  constexpr int G = OWN_GROUP, NG = NPAD / G, NWARP = 8;
  static_assert(G % 2 == 0 && NPAD % G == 0, "groups of an even number of projectors");
  __shared__ int ooff[OWN_MAX];
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int e = blockIdx.y, v0 = blockIdx.x * 32;   // vector tiles of one cell are adjacent: P reused from L2
  const int k0 = own_off[e], k1 = own_off[e + 1];
  if (k0 == k1) return;
  const int own = p * p * p;
  R *Xs = reinterpret_cast<R *>(sm_raw);   // [own][32]
  R *red = Xs + (size_t)own * 32;          // [NWARP][NPAD][32]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t base = owned_table(e, n, p, N1, ooff, own);
  __syncthreads();
  const int v = v0 + lane;
  for (int o = warp; o < own; o += NWARP) {
    const int64_t d = base + ooff[o];
    double x = (v < ncols) ? X[d * ldx + v] : 0.0;
    if (rowscale) x *= rowscale[d];
    Xs[o * 32 + lane] = A::from(x);
  }
  __syncthreads();
  for (int k = k0; k < k1; ++k) {
    int cg[NG];
#pragma unroll
    for (int g = 0; g < NG; ++g) cg[g] = own_cnt[(size_t)k * NG + g];
    const int16_t *sidx = own_sidx + (size_t)k * own;
    const R *Pk = oP + (size_t)k * own * NPAD;
    R acc[NPAD];
#pragma unroll
    for (int al = 0; al < NPAD; ++al) acc[al] = A::zero();
    int o = (warp < cg[0]) ? sidx[warp] : 0;
    for (int i = warp; i < cg[0]; i += NWARP) {
      const int onext = (i + NWARP < cg[0]) ? sidx[i + NWARP] : 0;   // index of the next node in flight
      const R x = Xs[o * 32 + lane];
      const R *Pr = Pk + (size_t)o * NPAD;
      // the loads of every nonzero group first (predicated, all in flight at
      // once), then the arithmetic behind a real branch: the FMAs of groups
      // that are zero on the node would still occupy the FP64 pipe (or the
      // issue slots of the pair form) under predication
      R pv[NPAD];
#pragma unroll
      for (int g = 0; g < NG; ++g)
        if (i < cg[g]) {
#pragma unroll
          for (int h = 0; h < G; h += 2) ldg2(Pr + G * g + h, pv[G * g + h], pv[G * g + h + 1]);
        }
#pragma unroll
      for (int g = 0; g < NG; ++g) {
        if (i >= cg[g]) break;   // this and the later groups are zero on the node
#pragma unroll
        for (int j = 0; j < G; ++j) acc[G * g + j] = A::fma(pv[G * g + j], x, acc[G * g + j]);
      }
      o = onext;
    }
    // only the warps that met a node and the groups that are nonzero somewhere
    // on the pair take part in the reduction; the other rows are zero
    const int nwk = min(NWARP, cg[0]);
    int nact = 0;
#pragma unroll
    for (int g = 0; g < NG; ++g) nact += (cg[g] > 0) ? G : 0;
    if (warp < nwk) {
#pragma unroll
      for (int al = 0; al < NPAD; ++al)
        if (al < nact) red[((size_t)warp * NPAD + al) * 32 + lane] = acc[al];
    }
    __syncthreads();
    // per-pair partial sums: plain coalesced stores, reduced per atom by k_pair_reduce
    for (int idx = tid; idx < NPAD * 32; idx += 256) {
      const int al = idx >> 5, l = idx & 31;
      if (v0 + l < ncols) {
        R sum = A::zero();
        if (al < nact) {
          sum = red[idx];
          for (int w = 1; w < nwk; ++w) sum = A::add(sum, red[(size_t)w * NPAD * 32 + idx]);
        }
        U[((size_t)k * NPAD + al) * ncols + v0 + l] = A::to(sum);
      }
    }
    __syncthreads();
  }
}

// Expansion: warp w takes the owned nodes w, w + 8, ...; for each pair of the
// cell the groups up to the node's last nonzero one are multiplied (four
// accumulators, one per projector of a group, added in a fixed order), then the
// output stage of k_own_expand (MODE) is applied to the node row.
template <int NPAD, int MODE, typename R>
__global__ void __launch_bounds__(256) k_own_expand64(ExpArgs A, const R *__restrict__ oP,
                                                      const int8_t *__restrict__ own_lg,
                                                      const R *__restrict__ W1, const R *__restrict__ W2) {
  using Q = Ar<R>;
  constexpr int G = OWN_GROUP, NG = NPAD / G, NWARP = 8;
  static_assert(G % 2 == 0 && 4 % G == 0, "groups of 2 or 4 projectors");
  constexpr int NW = (MODE == EXP_RECURRENCE) ? 2 : 1;
  __shared__ int ooff[OWN_MAX];
  __shared__ int patom[PAIRS_PER_CELL_MAX];
  const int e = blockIdx.y, v0 = blockIdx.x * 32;
  const int k0 = A.own_off[e], k1 = A.own_off[e + 1];
  if (MODE == EXP_ADD && k0 == k1) return;
  const int own = A.p * A.p * A.p;
  const int np = k1 - k0;
  const int ncols = A.ncols;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t base = owned_table(e, A.n, A.p, A.N1, ooff, own);
  for (int i = tid; i < np; i += 256) patom[i] = A.own_atom[k0 + i];
  __syncthreads();
  const int v = v0 + lane;
  const bool vok = v < ncols;
  const int vc = vok ? v : ncols - 1;   // in-range column for the loads of idle lanes
  const int8_t *lgc = own_lg + (size_t)k0 * own;
  for (int o = warp; o < own; o += NWARP) {
    R s1[4] = {Q::zero(), Q::zero(), Q::zero(), Q::zero()};   // four independent FMA chains per sum
    R s2[4] = {Q::zero(), Q::zero(), Q::zero(), Q::zero()};
    for (int kk = 0; kk < np; ++kk) {
      const int lg = lgc[(size_t)kk * own + o];   // warp-uniform
      if (lg < 0) continue;
      const R *Pr = oP + ((size_t)(k0 + kk) * own + o) * NPAD;
      const R *w1 = W1 + (size_t)patom[kk] * NPAD * ncols + vc;
      const R *w2 = (NW == 2) ? W2 + (size_t)patom[kk] * NPAD * ncols + vc : nullptr;
#pragma unroll
      for (int g = 0; g < NG; ++g) {
        if (g > lg) break;
        R pv[G];
#pragma unroll
        for (int h = 0; h < G; h += 2) ldg2(Pr + G * g + h, pv[h], pv[h + 1]);
        // the four chains take the projectors of the group in turn (static indices)
        constexpr int CH = 4 / G;
        const int c0 = (g % CH) * G;
#pragma unroll
        for (int j = 0; j < G; ++j)
          s1[c0 + j] = Q::fma(pv[j], ldg1(w1 + (size_t)(G * g + j) * ncols), s1[c0 + j]);
        if constexpr (NW == 2) {
#pragma unroll
          for (int j = 0; j < G; ++j)
            s2[c0 + j] = Q::fma(pv[j], ldg1(w2 + (size_t)(G * g + j) * ncols), s2[c0 + j]);
        }
      }
    }
    const double S1 = Q::to(Q::add(Q::add(s1[0], s1[1]), Q::add(s1[2], s1[3])));
    const double S2 = (NW == 2) ? Q::to(Q::add(Q::add(s2[0], s2[1]), Q::add(s2[2], s2[3]))) : 0.0;
    if (!vok) continue;
    const int64_t d = base + ooff[o];
    const double *Xin = static_cast<const double *>(A.Xin);
    double *Y = static_cast<double *>(A.Y);
    if (MODE == EXP_ADD) {
      Y[d * A.ldy + v] += (A.cs ? A.cs[v] : 1.0) * S1;
    } else if (MODE == EXP_SINV) {
      const double m = static_cast<const double *>(A.mdinv)[d];
      Y[d * A.ldy + v] = m * (Xin[d * A.ldx + v] - S1);
    } else {
      const double m = static_cast<const double *>(A.mdinv)[d];
      double *RX = static_cast<double *>(A.RX);
      const double ry = Xin[d * A.ldx + v], rx = RX[d * A.ldx + v];
      Y[d * A.ldy + v] = m * (ry - S1);
      const double bracket = -A.beta * ry - A.gamma * rx + S2;
      RX[d * A.ldx + v] = fma(A.c64[v], static_cast<const double *>(A.Y0)[d * A.ldy0 + v], bracket);
    }
  }
}

// ------------------------------------------------------------------ host side
// true when p (may be NULL) and the row pitch allow 16-byte vector access
static bool aligned16(const void *p, size_t pitch_bytes) {
  return (reinterpret_cast<uintptr_t>(p) % 16 == 0) && (pitch_bytes % 16 == 0);
}

template <typename T>
static const T *ownP(paw_context *c);
template <>
const float *ownP<float>(paw_context *c) { return c->ownP32.as<float>(); }

template <typename T, int NPAD>
static void project_impl(paw_context *c, const T *X, int ldx, int ncols, const T *rowscale, T *U, cudaStream_t s) {
  if constexpr (sizeof(T) == 8) {
    const size_t shm = sizeof(double) * ((size_t)c->own * 32 + (size_t)8 * NPAD * 32);
    PAW_REQUIRE(shm <= 200 * 1024 && c->own <= OWN_MAX, PAW_ERR_UNSUPPORTED,
                "projection tile exceeds shared memory (degree too high)");
    PAW_CUDA(cudaFuncSetAttribute(k_own_project64<NPAD, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)shm));
    if (c->sf_lean)   // step 2 sharing the SMs with a lean loop kernel: whole shared memory configured
      PAW_CUDA(cudaFuncSetAttribute(k_own_project64<NPAD, double>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                    cudaSharedmemCarveoutMaxShared));
    dim3 g((ncols + 31) / 32, c->ncells);
    k_own_project64<NPAD, double><<<g, 256, shm, s>>>(c->n, c->p, c->N1, c->own_off.as<int>(), c->own_cnt.as<int>(),
                                             c->own_sidx.as<int16_t>(), c->ownP64.as<double>(), X, ldx, ncols,
                                             rowscale, U);
    PAW_LAUNCH_CHECK("k_own_project64");
  } else {
    constexpr int VT = ProjCfg<T>::VT;
    constexpr int TPG = (NPAD / 4) * (VT / 4);
    constexpr int OG = 256 / TPG;
    const size_t shm = sizeof(T) * ((size_t)c->own * VT + (size_t)OG * NPAD * VT);
    PAW_REQUIRE(shm <= 200 * 1024 && c->own <= OWN_MAX, PAW_ERR_UNSUPPORTED,
                "projection tile exceeds shared memory (degree too high)");
    PAW_CUDA(cudaFuncSetAttribute(k_own_project<T, NPAD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    dim3 g1((ncols + VT - 1) / VT, c->ncells);
    const int xa = aligned16(X, ldx * sizeof(T)) ? 1 : 0;
    k_own_project<T, NPAD><<<g1, 256, shm, s>>>(c->n, c->p, c->N1, c->own_off.as<int>(), c->own_ngrp.as<int>(),
                                                ownP<T>(c), X, ldx, ncols, rowscale, c->npjr, U, xa);
    PAW_LAUNCH_CHECK("k_own_project");
  }
}

// U = P^T (rowscale .* X) into c->scr->partial (natoms x npad x ncols): per-pair
// partials, then a fixed-order sum per atom (deterministic, no atomics)
// tensor-core form: FP32 data, TF32 or BF16 filter precision, supported layout
template <typename T>
static bool use_tc(const paw_context *c, paw_precision prec) {
  return sizeof(T) == 4 && (prec == PAW_TF32 || prec == PAW_BF16) && nltc_supported(c);
}

template <typename T>
static T *project_U(paw_context *c, paw_precision prec, const T *X, int ldx, int ncols, const T *rowscale,
                    cudaStream_t s) {
  const size_t ub = sizeof(T) * (size_t)c->natoms * c->npad * ncols;
  c->scr->partial.ensure(ub, &c->dev_bytes);
  c->scr->pp.ensure(sizeof(T) * (size_t)c->nown_pairs * c->npad * ncols, &c->dev_bytes);
  T *U = c->scr->partial.as<T>(), *PP = c->scr->pp.as<T>();
  if constexpr (sizeof(T) == 4) {
    if (use_tc<T>(c, prec)) {
      if (nltc_project(c, X, ldx, ncols, rowscale, PP, U, s)) return U;   // reduced in the epilogue
      dim3 g((ncols + 31) / 32, c->npad, c->natoms);
      k_pair_reduce<T><<<g, 32, 0, s>>>(c->apair_off.as<int>(), c->apair.as<int>(), PP, c->npad, ncols, U);
      PAW_LAUNCH_CHECK("k_pair_reduce");
      return U;
    }
  }
  if (c->npad == 16)
    project_impl<T, 16>(c, X, ldx, ncols, rowscale, PP, s);
  else
    project_impl<T, 32>(c, X, ldx, ncols, rowscale, PP, s);
  dim3 g((ncols + 31) / 32, c->npad, c->natoms);
  k_pair_reduce<T><<<g, 32, 0, s>>>(c->apair_off.as<int>(), c->apair.as<int>(), PP, c->npad, ncols, U);
  PAW_LAUNCH_CHECK("k_pair_reduce");
  return U;
}

template <typename T>
static void couple(paw_context *c, const T *U, const double *C, const double *C2, const double *cs,
                   double scale, T *W, int ncols, cudaStream_t s) {
  if (c->kc) {   // complex coefficients: Delta_Sinv is complex, D_H and dS are real
    PAW_REQUIRE(ncols % 2 == 0 && 2 * c->npj <= c->npad, PAW_ERR_UNSUPPORTED, "complex coupling layout");
    const int cplxC = (C != nullptr && C == c->DSinv64.as<double>()) ? 1 : 0;
    dim3 gc(c->natoms, (ncols / 2 + 63) / 64);
    if (c->npad == 16)
      k_couple_c<T, 16><<<gc, 64, 0, s>>>(c->npj, U, C, cplxC, C2, cs, scale, W, ncols);
    else
      k_couple_c<T, 32><<<gc, 64, 0, s>>>(c->npj, U, C, cplxC, C2, cs, scale, W, ncols);
    PAW_LAUNCH_CHECK("k_couple_c");
    return;
  }
  dim3 g2(c->natoms, (ncols + 63) / 64);
  if (c->npad == 16)
    k_own_couple<T, 16><<<g2, 64, 0, s>>>(c->npj, U, C, C2, cs, scale, W, ncols);
  else
    k_own_couple<T, 32><<<g2, 64, 0, s>>>(c->npj, U, C, C2, cs, scale, W, ncols);
  PAW_LAUNCH_CHECK("k_own_couple");
}

template <typename T>
void nl_project(paw_context *c, paw_precision prec, const T *X, int ldx, int ncols, const T *rowscale,
                const double *coup, double coup_scale, T *W, cudaStream_t s) {
  if (c->nown_pairs == 0 || ncols <= 0) return;
  const T *U = project_U<T>(c, prec, X, ldx, ncols, rowscale, s);
  couple<T>(c, U, coup, nullptr, nullptr, coup_scale, W, ncols, s);
}

template <typename T>
void nl_project_residual(paw_context *c, const T *X, int ldx, int ncols, const double *cs, T *W, cudaStream_t s) {
  if (c->nown_pairs == 0 || ncols <= 0) return;
  const T *U = project_U<T>(c, PAW_FP64, X, ldx, ncols, nullptr, s);
  couple<T>(c, U, c->DH64.as<double>(), c->DS64.as<double>(), cs, 1.0, W, ncols, s);
}

// FP64 values to pairs of FP32 numbers (the tables and coefficients of the pair form)
__global__ void k_to_pair(int64_t n, const double *__restrict__ x, f32x2 *__restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = x2_from(x[i]);
}

static void to_pair(const double *x, int64_t n, f32x2 *y, cudaStream_t s) {
  if (n <= 0) return;
  k_to_pair<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, x, y);
  PAW_LAUNCH_CHECK("k_to_pair");
}

static ExpArgs exp_args(paw_context *c, int ncols);

// Nonlocal part of step 2 in pair-of-FP32 arithmetic:
//   Y += sum_a P^a (C^a + cs_j C2^a) P^a^T x_j   (step 2: C = D_H, C2 = dS, cs = -lambda)
// projection and expansion (the FP64 kernels with R = f32x2) on the owner-cell
// layout; per-atom sums and the 13 x 13 couplings stay FP64 (a small share).
void nl_residual_pair(paw_context *c, const double *X, int ldx, int ncols, const double *C, const double *C2,
                      const double *cs, double *Y, int ldy, cudaStream_t s) {
  if (c->nown_pairs == 0 || ncols <= 0) return;
  PAW_REQUIRE(!c->kc, PAW_ERR_UNSUPPORTED, "pair-of-FP32 arithmetic is implemented for real vectors (k = 0)");
  PAW_REQUIRE(c->max_own_pairs <= PAIRS_PER_CELL_MAX && c->own <= OWN_MAX, PAW_ERR_UNSUPPORTED,
              "too many atoms on one cell for the expansion kernel");
  const int64_t ntab = (int64_t)c->nown_pairs * c->own * c->npad;
  if (!c->ownPx2.ptr) {   // built on first use from the FP64 table
    c->ownPx2.ensure(sizeof(f32x2) * std::max<int64_t>(1, ntab), &c->dev_bytes);
    to_pair(c->ownP64.as<double>(), ntab, c->ownPx2.as<f32x2>(), s);
  }
  const f32x2 *oP = c->ownPx2.as<f32x2>();
  const size_t ub = sizeof(double) * (size_t)c->natoms * c->npad * ncols;
  c->scr->partial.ensure(ub, &c->dev_bytes);
  c->scr->pp.ensure(sizeof(double) * (size_t)c->nown_pairs * c->npad * ncols, &c->dev_bytes);
  double *U = c->scr->partial.as<double>(), *PP = c->scr->pp.as<double>();
  const size_t shm = sizeof(f32x2) * ((size_t)c->own * 32 + (size_t)8 * c->npad * 32);
  PAW_REQUIRE(shm <= 200 * 1024 && c->own <= OWN_MAX, PAW_ERR_UNSUPPORTED,
              "projection tile exceeds shared memory (degree too high)");
  dim3 gp((ncols + 31) / 32, c->ncells);
  auto proj = (c->npad == 16) ? k_own_project64<16, f32x2> : k_own_project64<32, f32x2>;
  PAW_CUDA(cudaFuncSetAttribute(proj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  proj<<<gp, 256, shm, s>>>(c->n, c->p, c->N1, c->own_off.as<int>(), c->own_cnt.as<int>(), c->own_sidx.as<int16_t>(),
                            oP, X, ldx, ncols, nullptr, PP);
  PAW_LAUNCH_CHECK("k_own_project64");
  dim3 gr((ncols + 31) / 32, c->npad, c->natoms);
  k_pair_reduce<double><<<gr, 32, 0, s>>>(c->apair_off.as<int>(), c->apair.as<int>(), PP, c->npad, ncols, U);
  PAW_LAUNCH_CHECK("k_pair_reduce");
  const int64_t nw = (int64_t)c->natoms * c->npad * ncols;
  c->scr->W2.ensure(sizeof(double) * std::max<int64_t>(1, nw), &c->dev_bytes);
  c->scr->Wx2.ensure(sizeof(f32x2) * std::max<int64_t>(1, nw), &c->dev_bytes);
  double *W = c->scr->W2.as<double>();
  couple<double>(c, U, C, C2, cs, 1.0, W, ncols, s);
  to_pair(W, nw, c->scr->Wx2.as<f32x2>(), s);
  ExpArgs A = exp_args(c, ncols);
  A.Y = Y;
  A.ldy = ldy;
  A.ldx = ldy;
  A.ldy0 = 4;
  dim3 ge((ncols + 31) / 32, c->ncells);
  const f32x2 *Wx = c->scr->Wx2.as<f32x2>();
  if (c->npad == 16)
    k_own_expand64<16, EXP_ADD, f32x2><<<ge, 256, 0, s>>>(A, oP, c->own_lg.as<int8_t>(), Wx, nullptr);
  else
    k_own_expand64<32, EXP_ADD, f32x2><<<ge, 256, 0, s>>>(A, oP, c->own_lg.as<int8_t>(), Wx, nullptr);
  PAW_LAUNCH_CHECK("k_own_expand64");
}

void build_couple_f(paw_context *c) {
  if (c->kc || c->natoms == 0 || c->ngpairs == 0) return;
  PAW_REQUIRE(c->npad == 16 || c->npad == 32, PAW_ERR_UNSUPPORTED, "projector padding must be 16 or 32");
  c->Fsh32.ensure(sizeof(float) * (size_t)c->ngpairs * c->npad * c->npad, &c->dev_bytes);
  c->DSinv32.ensure(sizeof(float) * (size_t)c->natoms * c->npad * c->npad, &c->dev_bytes);
  const int *go = c->gnb_off.as<int>(), *ga = c->gnb_atom.as<int>();
  if (c->npad == 16)
    k_couple_f<16><<<c->natoms, 16 * 16>>>(c->npj, go, ga, c->Gfull.as<double>(), c->DSinv64.as<double>(),
                                           c->DH64.as<double>(), c->Fsh32.as<float>(), c->DSinv32.as<float>());
  else
    k_couple_f<32><<<c->natoms, 32 * 32>>>(c->npj, go, ga, c->Gfull.as<double>(), c->DSinv64.as<double>(),
                                           c->DH64.as<double>(), c->Fsh32.as<float>(), c->DSinv32.as<float>());
  PAW_LAUNCH_CHECK("k_couple_f");
  PAW_CUDA(cudaDeviceSynchronize());
}

// atom-pair Gram blocks in the element type of the filter
template <typename T>
static const T *gram(paw_context *c);
template <>
const double *gram<double>(paw_context *c) { return c->Gfull.as<double>(); }
template <>
const float *gram<float>(paw_context *c) { return c->Gfull32.as<float>(); }

template <typename T>
void nl_project_filter(paw_context *c, paw_precision prec, const T *RY, int ldr, int ncols, const T *mdinv,
                       double alpha, T *WS, T *WH, cudaStream_t s) {
  if (c->nown_pairs == 0 || ncols <= 0) return;
  const T *U = project_U<T>(c, prec, RY, ldr, ncols, mdinv, s);
  if constexpr (sizeof(T) == 4) {
    if (!c->kc && c->Fsh32.ptr) {   // W_S and W_H in one launch
      dim3 g(c->natoms, (ncols + 31) / 32);
      const int *go = c->gnb_off.as<int>(), *ga = c->gnb_atom.as<int>();
      if (c->npad == 16)
        k_own_couple_sh<16, 8><<<g, 8 * 32, 0, s>>>(c->npj, go, ga, c->Fsh32.as<float>(), c->DSinv32.as<float>(), U,
                                                    (float)alpha, WS, WH, ncols);
      else
        k_own_couple_sh<32, 4><<<g, 4 * 32, 0, s>>>(c->npj, go, ga, c->Fsh32.as<float>(), c->DSinv32.as<float>(), U,
                                                    (float)alpha, WS, WH, ncols);
      PAW_LAUNCH_CHECK("k_own_couple_sh");
      return;
    }
  }
  couple<T>(c, U, c->DSinv64.as<double>(), nullptr, nullptr, 1.0, WS, ncols, s);
  if (c->kc) {
    dim3 gc(c->natoms, (ncols / 2 + 31) / 32);
    if (c->npad == 16)
      k_couple_h_c<T, 16><<<gc, 8 * 32, 0, s>>>(c->npj, c->gnb_off.as<int>(), c->gnb_atom.as<int>(), gram<T>(c), U,
                                                WS, c->DH64.as<double>(), alpha, WH, ncols);
    else
      k_couple_h_c<T, 32><<<gc, 16 * 32, 0, s>>>(c->npj, c->gnb_off.as<int>(), c->gnb_atom.as<int>(), gram<T>(c), U,
                                                 WS, c->DH64.as<double>(), alpha, WH, ncols);
    PAW_LAUNCH_CHECK("k_couple_h_c");
    return;
  }
  dim3 g2(c->natoms, (ncols + 31) / 32);
  const T *G = gram<T>(c);
  if (c->npad == 16)
    k_own_couple_h<T, 16><<<g2, 16 * 32, 0, s>>>(c->npj, c->gnb_off.as<int>(), c->gnb_atom.as<int>(), G, U, WS,
                                                  c->DH64.as<double>(), alpha, WH, ncols);
  else
    k_own_couple_h<T, 32><<<g2, 32 * 32, 0, s>>>(c->npj, c->gnb_off.as<int>(), c->gnb_atom.as<int>(), G, U, WS,
                                                  c->DH64.as<double>(), alpha, WH, ncols);
  PAW_LAUNCH_CHECK("k_own_couple_h");
}

template <typename T, int MODE>
static void own_expand(paw_context *c, paw_precision prec, ExpArgs A, const T *W1, const T *W2, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (use_tc<T>(c, prec)) {
      nltc_expand(c, MODE, A, W1, W2, s);
      return;
    }
  }
  if constexpr (sizeof(T) == 8) {
    PAW_REQUIRE(c->max_own_pairs <= PAIRS_PER_CELL_MAX && c->own <= OWN_MAX, PAW_ERR_UNSUPPORTED,
                "too many atoms on one cell for the expansion kernel");
    dim3 g((A.ncols + 31) / 32, c->ncells);
    if (c->npad == 16)
      k_own_expand64<16, MODE, double><<<g, 256, 0, s>>>(A, c->ownP64.as<double>(), c->own_lg.as<int8_t>(), W1, W2);
    else
      k_own_expand64<32, MODE, double><<<g, 256, 0, s>>>(A, c->ownP64.as<double>(), c->own_lg.as<int8_t>(), W1, W2);
    PAW_LAUNCH_CHECK("k_own_expand64");
  } else {
    A.vec_ok = aligned16(A.Y, A.ldy * sizeof(T)) && aligned16(A.Xin, A.ldx * sizeof(T)) &&
               aligned16(A.RX, A.ldx * sizeof(T)) && aligned16(A.Y0, A.ldy0 * sizeof(float)) &&
               aligned16(A.Y0lo, A.ldy0 * sizeof(float));
    constexpr int NW = (MODE == EXP_RECURRENCE) ? 2 : 1;
    constexpr size_t SHM_MAX = 200 * 1024;
    // W of every pair of a cell for VT vectors: 32 vectors per CTA, or 4 when that exceeds the budget
    const size_t per_vec = sizeof(T) * (size_t)NW * std::max(1, c->max_own_pairs) * c->npad;
    const bool wide = per_vec * ExpCfg<T>::VT <= SHM_MAX;
    const int VT = wide ? ExpCfg<T>::VT : 4;
    const size_t shm = per_vec * VT;
    PAW_REQUIRE(shm <= SHM_MAX && c->own <= OWN_MAX, PAW_ERR_UNSUPPORTED,
                "too many atoms on one cell for the expansion kernel");
    dim3 g((A.ncols + VT - 1) / VT, c->ncells);
    auto launch = [&](auto kern) {
      PAW_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
      kern<<<g, 256, shm, s>>>(A, ownP<T>(c), W1, W2);
    };
    if (c->npad == 16)
      wide ? launch(k_own_expand<T, 16, MODE, ExpCfg<T>::VT>) : launch(k_own_expand<T, 16, MODE, 4>);
    else
      wide ? launch(k_own_expand<T, 32, MODE, ExpCfg<T>::VT>) : launch(k_own_expand<T, 32, MODE, 4>);
    PAW_LAUNCH_CHECK("k_own_expand");
  }
}

static ExpArgs exp_args(paw_context *c, int ncols) {
  ExpArgs A{};
  A.n = c->n;
  A.p = c->p;
  A.N1 = c->N1;
  A.own_off = c->own_off.as<int>();
  A.own_atom = c->own_atom.as<int>();
  A.own_ngrp = c->own_ngrp.as<int>();
  A.ncols = ncols;
  return A;
}

template <typename T>
void nl_expand(paw_context *c, paw_precision prec, const T *W, int ncols, T *Y, int ldy, const double *colscale,
               cudaStream_t s) {
  if (c->nown_pairs == 0 || ncols <= 0) return;
  ExpArgs A = exp_args(c, ncols);
  A.Y = Y;
  A.ldy = ldy;
  A.ldx = ldy;
  A.ldy0 = 4;
  A.cs = colscale;
  own_expand<T, EXP_ADD>(c, prec, A, W, nullptr, s);
}

template <typename T>
void nl_sinv_out(paw_context *c, paw_precision prec, const T *W, int ncols, const T *X, int ldx, T *Y, int ldy,
                 const T *mdinv, cudaStream_t s) {
  ExpArgs A = exp_args(c, ncols);
  A.Xin = X;
  A.ldx = ldx;
  A.Y = Y;
  A.ldy = ldy;
  A.ldy0 = 4;
  A.mdinv = mdinv;
  own_expand<T, EXP_SINV>(c, prec, A, W, nullptr, s);
}

void nl_recurrence_f32(paw_context *c, paw_precision prec, const float *WS, const float *WH, int ncols,
                       const float *RY, float *RX, float *Tout, int ldr, const float *mdinv, const float *Y0hi,
                       const float *Y0lo, int ldy0, const float *chi, const float *clo, double beta, double gamma,
                       cudaStream_t s) {
  ExpArgs A = exp_args(c, ncols);
  A.Xin = RY;
  A.ldx = ldr;
  A.Y = Tout;
  A.ldy = ldr;
  A.mdinv = mdinv;
  A.RX = RX;
  A.Y0 = Y0hi;
  A.Y0lo = Y0lo;
  A.ldy0 = ldy0;
  A.chi = chi;
  A.clo = clo;
  A.beta = beta;
  A.gamma = gamma;
  own_expand<float, EXP_RECURRENCE>(c, prec, A, WS, WH, s);
}

void nl_recurrence_f64(paw_context *c, const double *WS, const double *WH, int ncols, const double *RY, double *RX,
                       double *Tout, int ldr, const double *mdinv, const double *Y0, int ldy0, const double *c64,
                       double beta, double gamma, cudaStream_t s) {
  ExpArgs A = exp_args(c, ncols);
  A.Xin = RY;
  A.ldx = ldr;
  A.Y = Tout;
  A.ldy = ldr;
  A.mdinv = mdinv;
  A.RX = RX;
  A.Y0 = Y0;
  A.ldy0 = ldy0;
  A.c64 = c64;
  A.beta = beta;
  A.gamma = gamma;
  own_expand<double, EXP_RECURRENCE>(c, PAW_FP64, A, WS, WH, s);
}

template void nl_project<double>(paw_context *, paw_precision, const double *, int, int, const double *,
                                 const double *, double, double *, cudaStream_t);
template void nl_project<float>(paw_context *, paw_precision, const float *, int, int, const float *,
                                const double *, double, float *, cudaStream_t);
template void nl_project_residual<double>(paw_context *, const double *, int, int, const double *, double *,
                                          cudaStream_t);
template void nl_project_filter<double>(paw_context *, paw_precision, const double *, int, int, const double *,
                                        double, double *, double *, cudaStream_t);
template void nl_project_filter<float>(paw_context *, paw_precision, const float *, int, int, const float *,
                                       double, float *, float *, cudaStream_t);
template void nl_expand<double>(paw_context *, paw_precision, const double *, int, double *, int, const double *,
                                cudaStream_t);
template void nl_expand<float>(paw_context *, paw_precision, const float *, int, float *, int, const double *,
                               cudaStream_t);
template void nl_sinv_out<double>(paw_context *, paw_precision, const double *, int, const double *, int, double *,
                                  int, const double *, cudaStream_t);
template void nl_sinv_out<float>(paw_context *, paw_precision, const float *, int, const float *, int, float *, int,
                                 const float *, cudaStream_t);

}  // namespace pawfe

// ====================================================================== no-allocation variant
// Shat^-1 X with every scratch buffer carved out of one static device array,
// for callers that cannot allocate device memory at the point of use.
namespace pawfe {

static __device__ __align__(256) unsigned char g_noalloc_scratch[PAW_NOALLOC_SCRATCH_BYTES];

// The driver context current on the calling thread (NULL if the driver entry
// point cannot be found: then only the device ordinal keys the cache).
static CUcontext current_context() {
  typedef CUresult (*GetCurrent)(CUcontext *);
  static GetCurrent fn = [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    const cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q);
    return (e == cudaSuccess && q == cudaDriverEntryPointSuccess) ? reinterpret_cast<GetCurrent>(f) : nullptr;
  }();
  CUcontext ctx = nullptr;
  if (fn && fn(&ctx) != CUDA_SUCCESS) ctx = nullptr;
  return ctx;
}

// Device address of g_noalloc_scratch on the current device, looked up once per
// device and context (a device reset makes a new primary context, and the
// address is looked up again).  In host code the symbol itself is only a
// host-side handle.
static void *noalloc_scratch() {
  static std::mutex mu;
  static void *addr[128] = {};
  static CUcontext ctx_of[128] = {};
  int dev = 0;
  PAW_CUDA(cudaGetDevice(&dev));
  PAW_REQUIRE(dev >= 0 && dev < 128, PAW_ERR_UNSUPPORTED, "device ordinal above 127");
  const CUcontext ctx = current_context();
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev] || ctx == nullptr || ctx_of[dev] != ctx) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);   // binds the primary context
    PAW_REQUIRE(e == cudaSuccess && p != nullptr, PAW_ERR_CUDA,
                std::string("cudaGetSymbolAddress(no-allocation scratch): ") + cudaGetErrorString(e));
    addr[dev] = p;
    ctx_of[dev] = current_context();
  }
  return addr[dev];
}

template <typename T>
static void sinv_noalloc(paw_context *c, const T *X, int ldx, T *Y, int ldy, int ncols, cudaStream_t s) {
  const T *mdinv = (sizeof(T) == 8) ? reinterpret_cast<const T *>(c->md_inv64.ptr)
                                    : reinterpret_cast<const T *>(c->md_inv32.ptr);
  if (c->nown_pairs == 0) {   // M_D^-1 X only
    scale_rows<T>(X, ldx, Y, ldy, c->ndof, ncols, mdinv, s);
    return;
  }
  const size_t need = sizeof(T) * (size_t)c->npad * ncols * ((size_t)c->nown_pairs + 2 * (size_t)c->natoms);
  PAW_REQUIRE(need <= PAW_NOALLOC_SCRATCH_BYTES, PAW_ERR_INVALID_ARG,
              "no-allocation scratch too small: " + std::to_string(need) + " bytes needed, " +
                  std::to_string((size_t)PAW_NOALLOC_SCRATCH_BYTES) + " available (at most " +
                  std::to_string(PAW_NOALLOC_SCRATCH_BYTES /
                                 (sizeof(T) * (size_t)c->npad * ((size_t)c->nown_pairs + 2 * (size_t)c->natoms))) +
                  " columns per call for this problem)");
  T *PP = static_cast<T *>(noalloc_scratch());
  T *U = PP + (size_t)c->nown_pairs * c->npad * ncols;
  T *W = U + (size_t)c->natoms * c->npad * ncols;
  // projection partials, fixed-order reduction per atom, coupling, expansion:
  // every scratch value is written before it is read
  if (c->npad == 16)
    project_impl<T, 16>(c, X, ldx, ncols, mdinv, PP, s);
  else
    project_impl<T, 32>(c, X, ldx, ncols, mdinv, PP, s);
  dim3 g((ncols + 31) / 32, c->npad, c->natoms);
  k_pair_reduce<T><<<g, 32, 0, s>>>(c->apair_off.as<int>(), c->apair.as<int>(), PP, c->npad, ncols, U);
  PAW_LAUNCH_CHECK("k_pair_reduce");
  couple<T>(c, U, c->DSinv64.as<double>(), nullptr, nullptr, 1.0, W, ncols, s);
  nl_sinv_out<T>(c, (sizeof(T) == 8) ? PAW_FP64 : PAW_FP32, W, ncols, X, ldx, Y, ldy, mdinv, s);
}

}  // namespace pawfe

extern "C" paw_status paw_apply_Sinv_approx_noalloc(paw_handle c, paw_precision prec, const void *X, void *Y,
                                                    int ncols, int ldx, int ldy, void *stream) {
  using namespace pawfe;
  try {
    // the same checks, in the same order and with the same codes, as paw_apply_Sinv_approx
    check_prec(prec);
    check_block_args(c, X, Y, ncols, ldx, ldy);
    PAW_REQUIRE(!c->kc, PAW_ERR_UNSUPPORTED, "the allocation-free entry point has no Bloch-wavevector form");
    if (ncols == 0) return PAW_OK;
    auto s = (cudaStream_t)stream;
    c->last_stream = s;
    if (prec == PAW_FP64)
      sinv_noalloc<double>(c, (const double *)X, ldx, (double *)Y, ldy, ncols, s);
    else
      sinv_noalloc<float>(c, (const float *)X, ldx, (float *)Y, ldy, ncols, s);
    return PAW_OK;
  } catch (const Error &err) {
    return fail(err.code, err.msg);
  } catch (const std::exception &ex) {
    return fail(PAW_ERR_CUDA, ex.what());
  }
}
