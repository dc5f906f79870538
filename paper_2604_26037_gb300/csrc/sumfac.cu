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
// Block: one cell, VT vectors; each 1D contraction handles one line (all
// points along the contracted direction) per thread, in the even/odd split of
// the centro-symmetric 1D matrices (about 26.3k FP64 instructions, 44.6k flops,
// per cell and vector at p = 6 instead of 35.7k instructions).  Terms that
// share an output line are summed on the halves before the one recombination
// (the kinetic factor is folded into the tables kD, kM); the potential part
// runs first, so that the last contraction of the kinetic and mass part and the
// last one of the potential part share their output lines, which are added into
// Y straight from the registers.  Shared-memory
// tensors are stored [node][vector] so that consecutive threads touch
// consecutive words.
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "f32x2.cuh"

namespace pawfe {

namespace {

template <int NP>
constexpr int sf_vt() { return NP >= 9 ? 4 : 8; }
// 512 threads at <= 128 registers: one block of 16 warps per SM (shared memory
// allows one), so that every line of a contraction stage runs in one pass and
// the FP64 pipe sees twice the warps of a 256-thread block
constexpr int SF_THREADS = 512;
// The pair-of-FP32 form issues about 12 FP32 instructions per FP64 FMA, so
// issue slots, not a pipe, bound it: several blocks of 256 threads (half the
// vectors each) per SM, whose gathers, barriers and scatters overlap the
// contractions of the others (the FP64 form measured 1-1.5% slower with two or
// three such blocks than with one block of 512 threads).
template <int NP, typename R>
constexpr int sf_vt_r() { return std::is_same<R, double>::value ? sf_vt<NP>() : sf_vt<NP>() / 2; }
template <typename R>
constexpr int sf_threads() { return std::is_same<R, double>::value ? SF_THREADS : SF_THREADS / 2; }
// (three blocks up to degree 6: 80 registers without spills; two above)
template <int NP, typename R>
constexpr int sf_min_blocks() { return std::is_same<R, double>::value ? 1 : (NP <= 7 ? 3 : 2); }

// Even/odd halves of a centro-symmetric 1D matrix A (m x n, A[m-1-i][n-1-j] = A[i][j]):
//   Ae[i][j] = (A[i][j] + A[i][n-1-j]) / 2   (j < n/2),  Ae[i][n/2] = A[i][n/2] for odd n,
//   Ao[i][j] = (A[i][j] - A[i][n-1-j]) / 2   (i < m/2, j < n/2),
// so that with e[j] = x[j] + x[n-1-j] (e[n/2] = x[n/2]) and o[j] = x[j] - x[n-1-j]:
//   y[i] = E[i] + O[i],  y[m-1-i] = E[i] - O[i],  E = Ae e,  O = Ao o   (y[m/2] = E[m/2] for odd m).
// The GLL nodes and Gauss points are symmetric about the cell centre, so the 1D mass and
// stiffness matrices and the Lagrange values at the Gauss points are all of this form.
constexpr int EOMAX = 5;   // ceil(10 / 2): up to 10 points per direction
template <typename R = double>
struct EoMatT {
  R e[EOMAX * EOMAX];   // [i < ceil(m/2)][j < ceil(n/2)]
  R o[EOMAX * EOMAX];   // [i < m/2][j < n/2]
};
using EoMat = EoMatT<double>;

template <typename R>
struct SfTablesT {
  EoMatT<R> M, D, phi, phit;   // M, D: np1 x np1; phi: nq1 x np1 (Lagrange at Gauss points); phit = phi^T
  EoMatT<R> kD, kM;            // kf D and kf M, kf = cK (h/4) of the call (the kinetic factor folded in)
  double kfac, mfac;
};
using SfTables = SfTablesT<double>;

// The number type R of the contractions is double (the FP64 form) or f32x2
// (pair-of-FP32 arithmetic with about 48 significant bits on the FP32 pipes);
// Ar<R> supplies the operations.
template <int N, typename R = double>
struct Split {
  static constexpr int NE = (N + 1) / 2, NO = N / 2;
  R e[NE], o[NO > 0 ? NO : 1];
};

// split the line x[0], x[s], ..., x[(N-1) s]
template <int N, typename R = double>
__device__ __forceinline__ Split<N, R> split_line(const R *x, int s) {
  using A = Ar<R>;
  Split<N, R> r;
#pragma unroll
  for (int j = 0; j < N / 2; ++j) {
    const R a = x[j * s], b = x[(N - 1 - j) * s];
    r.e[j] = A::add(a, b);
    r.o[j] = A::sub(a, b);
  }
  if (N & 1) r.e[N / 2] = x[(N / 2) * s];
  return r;
}

// E[i] += sum_j Ae[i][j] e[j],  O[i] += sum_j Ao[i][j] o[j]  for A of size M x N (in shared memory)
template <int M, int N, typename R = double>
__device__ __forceinline__ void eo_acc(const EoMatT<R> &A, const Split<N, R> &x, R (&E)[(M + 1) / 2],
                                       R (&O)[M / 2 > 0 ? M / 2 : 1]) {
  using Q = Ar<R>;
  constexpr int NE = (N + 1) / 2, NO = N / 2;
#pragma unroll
  for (int i = 0; i < (M + 1) / 2; ++i)
#pragma unroll
    for (int j = 0; j < NE; ++j) E[i] = Q::fma(A.e[i * NE + j], x.e[j], E[i]);
#pragma unroll
  for (int i = 0; i < M / 2; ++i)
#pragma unroll
    for (int j = 0; j < NO; ++j) O[i] = Q::fma(A.o[i * NO + j], x.o[j], O[i]);
}

template <int M, typename R = double>
struct Half {
  using A = Ar<R>;
  R E[(M + 1) / 2], O[M / 2 > 0 ? M / 2 : 1];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < (M + 1) / 2; ++i) E[i] = A::zero();
#pragma unroll
    for (int i = 0; i < (M / 2 > 0 ? M / 2 : 1); ++i) O[i] = A::zero();
  }
  // output i of the line (normalised)
  __device__ __forceinline__ R out(int i) const {
    if (2 * i + 1 == M) return A::norm(E[i]);
    return (i < M / 2) ? A::add(E[i], O[i]) : A::sub(E[M - 1 - i], O[M - 1 - i]);
  }
};

// cK reaches the kernel folded into tab.kD and tab.kM (the host scales the tables);
// the parameter stays in the launch signature for the call sites.
template <int NP, typename R, int VT, int NT>
__device__ __forceinline__ void sf_body(const SfTablesT<R> &tab, int ncells, const int *__restrict__ cell_dofs,
                                        const R *__restrict__ wV,   // ncells x NQ^3 (w_q V_q)
                                        const double *__restrict__ X, int ldx, double *__restrict__ Y, int ldy,
                                        int ncols, double alpha, double cK, double cV, double cM,
                                        const double *__restrict__ cMcol) {
  constexpr int NQ = NP + 1;
  constexpr int N3 = NP * NP * NP;
  constexpr int S1 = (NQ * NP * NP > N3) ? NQ * NP * NP : N3;
  constexpr int S2 = (NQ * NQ * NP > N3) ? NQ * NQ * NP : N3;
  constexpr int S3 = (NQ * NQ * NQ > N3) ? NQ * NQ * NQ : N3;
  using A = Ar<R>;
  static_assert(sizeof(R) == sizeof(double), "shared-memory layout assumes 8-byte numbers");
  __shared__ SfTablesT<R> st;
  __shared__ int dofs[N3];
  extern __shared__ double sm[];
  R *A0 = reinterpret_cast<R *>(sm);   // x, then R          [N3][VT]
  R *A1 = A0 + N3 * VT;                // P                  [N3][VT]
  R *A2 = A1 + N3 * VT;                // U1, then B1        [S1][VT]
  R *A3 = A2 + S1 * VT;                // U2, B2, then Q     [S2][VT]
  R *A4 = A3 + S2 * VT;                // U3, then S         [S3][VT]
  R *sw = A4 + S3 * VT;                // w_q V_q            [NQ^3]
  const int e = blockIdx.x, v0 = blockIdx.y * VT, tid = threadIdx.x;
  {
    const double *src = reinterpret_cast<const double *>(&tab);
    double *dst = reinterpret_cast<double *>(&st);
    for (int i = tid; i < (int)(sizeof(SfTablesT<R>) / sizeof(double)); i += NT) dst[i] = src[i];
  }
  for (int i = tid; i < N3; i += NT) dofs[i] = cell_dofs[(size_t)e * N3 + i];
  const bool doV = cV != 0.0;
  if (doV)
    for (int i = tid; i < NQ * NQ * NQ; i += NT) {
      const R w = wV[(size_t)e * NQ * NQ * NQ + i];
      sw[i] = (cV == 1.0) ? w : A::mul(A::from(cV), w);
    }
  __syncthreads();
  {
    // gather: every load of the thread in flight before the first use
    constexpr int NPER = (N3 * VT + NT - 1) / NT;
    double xv[NPER];
#pragma unroll
    for (int k = 0; k < NPER; ++k) {
      const int idx = tid + k * NT;
      const int r = idx / VT, v = idx - r * VT;
      xv[k] = (idx < N3 * VT && v0 + v < ncols) ? X[(size_t)dofs[r] * ldx + v0 + v] : 0.0;
    }
#pragma unroll
    for (int k = 0; k < NPER; ++k)
      if (tid + k * NT < N3 * VT) A0[tid + k * NT] = A::from(xv[k]);
  }
  __syncthreads();
  const double mf = st.mfac;
  // Potential part first (x stays in A0): U1, U2, U3 = w V interpolated values, back to
  // B1 = Phi^T-contracted along z and y (B1 in A2 until the last stage)
  if (doV) {
    // U1[c][b][i] = sum_a phi[i][a] x[c][b][a]            (line (b, c), NP -> NQ)
    for (int idx = tid; idx < NP * NP * VT; idx += NT) {
      const int bc = idx / VT, v = idx - bc * VT;
      const Split<NP, R> x = split_line<NP, R>(A0 + bc * NP * VT + v, VT);
      Half<NQ, R> U;
      U.zero();
      eo_acc<NQ, NP, R>(st.phi, x, U.E, U.O);
#pragma unroll
      for (int i = 0; i < NQ; ++i) A2[(bc * NQ + i) * VT + v] = U.out(i);
    }
    __syncthreads();
    // U2[c][j][i] = sum_b phi[j][b] U1[c][b][i]           (line (i, c))
    for (int idx = tid; idx < NQ * NP * VT; idx += NT) {
      const int ic = idx / VT, v = idx - ic * VT;
      const int i = ic % NQ, c = ic / NQ;
      const Split<NP, R> x = split_line<NP, R>(A2 + (c * NP * NQ + i) * VT + v, NQ * VT);
      Half<NQ, R> U;
      U.zero();
      eo_acc<NQ, NP, R>(st.phi, x, U.E, U.O);
#pragma unroll
      for (int j = 0; j < NQ; ++j) A3[((c * NQ + j) * NQ + i) * VT + v] = U.out(j);
    }
    __syncthreads();
    // U3[k][j][i] = w_q V_q sum_c phi[k][c] U2[c][j][i]    (line (i, j))
    for (int idx = tid; idx < NQ * NQ * VT; idx += NT) {
      const int ji = idx / VT, v = idx - ji * VT;
      const Split<NP, R> x = split_line<NP, R>(A3 + ji * VT + v, NQ * NQ * VT);
      Half<NQ, R> U;
      U.zero();
      eo_acc<NQ, NP, R>(st.phi, x, U.E, U.O);
#pragma unroll
      for (int k = 0; k < NQ; ++k) A4[(k * NQ * NQ + ji) * VT + v] = A::mul(U.out(k), sw[k * NQ * NQ + ji]);
    }
    __syncthreads();
    // B2[c][j][i] = sum_k phi[k][c] U3[k][j][i]            (line (i, j), NQ -> NP)
    for (int idx = tid; idx < NQ * NQ * VT; idx += NT) {
      const int ji = idx / VT, v = idx - ji * VT;
      const Split<NQ, R> x = split_line<NQ, R>(A4 + ji * VT + v, NQ * NQ * VT);
      Half<NP, R> B;
      B.zero();
      eo_acc<NP, NQ, R>(st.phit, x, B.E, B.O);
#pragma unroll
      for (int c = 0; c < NP; ++c) A3[(c * NQ * NQ + ji) * VT + v] = B.out(c);
    }
    __syncthreads();
    // B1[c][b][i] = sum_j phi[j][b] B2[c][j][i]            (line (i, c))
    for (int idx = tid; idx < NQ * NP * VT; idx += NT) {
      const int ic = idx / VT, v = idx - ic * VT;
      const int i = ic % NQ, c = ic / NQ;
      const Split<NQ, R> x = split_line<NQ, R>(A3 + (c * NQ * NQ + i) * VT + v, NQ * VT);
      Half<NP, R> B;
      B.zero();
      eo_acc<NP, NQ, R>(st.phit, x, B.E, B.O);
#pragma unroll
      for (int b = 0; b < NP; ++b) A2[((c * NP + b) * NQ + i) * VT + v] = B.out(b);
    }
    __syncthreads();
  }
  // kinetic and mass part.  c-contractions, one (a, b) line per thread: P = M_c x (A1), Q = D_c x (A3)
  for (int idx = tid; idx < NP * NP * VT; idx += NT) {
    const int ab = idx / VT, v = idx - ab * VT;
    const Split<NP, R> x = split_line<NP, R>(A0 + ab * VT + v, NP * NP * VT);
    Half<NP, R> P, Q;
    P.zero();
    Q.zero();
    eo_acc<NP, NP, R>(st.M, x, P.E, P.O);
    eo_acc<NP, NP, R>(st.D, x, Q.E, Q.O);
#pragma unroll
    for (int c2 = 0; c2 < NP; ++c2) {
      A1[(c2 * NP * NP + ab) * VT + v] = P.out(c2);
      A3[(c2 * NP * NP + ab) * VT + v] = Q.out(c2);
    }
  }
  __syncthreads();
  // b-contractions, one (a, c) line per thread: S = M_b P (A4), R = kf (D_b P + M_b Q) + c_j mf S
  // (A0: x is no longer needed), R formed on the even/odd halves (kf folded into the tables kD, kM)
  for (int idx = tid; idx < NP * NP * VT; idx += NT) {
    const int ac = idx / VT, v = idx - ac * VT;
    const int a = ac % NP, c = ac / NP;
    const int base = (c * NP * NP + a) * VT + v;
    const Split<NP, R> p = split_line<NP, R>(A1 + base, NP * VT);
    const Split<NP, R> q = split_line<NP, R>(A3 + base, NP * VT);
    Half<NP, R> S, T;
    S.zero();
    T.zero();
    eo_acc<NP, NP, R>(st.M, p, S.E, S.O);
    eo_acc<NP, NP, R>(st.kD, p, T.E, T.O);
    eo_acc<NP, NP, R>(st.kM, q, T.E, T.O);
    const R cmv = A::from((cM + (cMcol ? ((v0 + v < ncols) ? cMcol[v0 + v] : 0.0) : 0.0)) * mf);
#pragma unroll
    for (int i = 0; i < (NP + 1) / 2; ++i) T.E[i] = A::fma(cmv, A::norm(S.E[i]), T.E[i]);
#pragma unroll
    for (int i = 0; i < NP / 2; ++i) T.O[i] = A::fma(cmv, A::norm(S.O[i]), T.O[i]);
#pragma unroll
    for (int b2 = 0; b2 < NP; ++b2) {
      A4[base + b2 * NP * VT] = S.out(b2);
      A0[base + b2 * NP * VT] = T.out(b2);
    }
  }
  __syncthreads();
  // a-contractions, one (b, c) line per thread, every term of the line in one accumulator:
  // y = kf D_a S + M_a R (+ Phi_a^T B1), added into Y straight from the registers
  for (int idx = tid; idx < NP * NP * VT; idx += NT) {
    const int bc = idx / VT, v = idx - bc * VT;
    const int base = bc * NP * VT + v;
    const Split<NP, R> sl = split_line<NP, R>(A4 + base, VT);
    const Split<NP, R> rl = split_line<NP, R>(A0 + base, VT);
    Half<NP, R> Yl;
    Yl.zero();
    eo_acc<NP, NP, R>(st.kD, sl, Yl.E, Yl.O);
    eo_acc<NP, NP, R>(st.M, rl, Yl.E, Yl.O);
    if (doV) {
      const Split<NQ, R> bl = split_line<NQ, R>(A2 + bc * NQ * VT + v, VT);
      eo_acc<NP, NQ, R>(st.phit, bl, Yl.E, Yl.O);
    }
    if (v0 + v < ncols) {
#pragma unroll
      for (int a2 = 0; a2 < NP; ++a2)
        atomicAdd(&Y[(size_t)dofs[bc * NP + a2] * ldy + v0 + v], alpha * A::to(Yl.out(a2)));
    }
  }
}

template <int NP, typename R>
__global__ void __launch_bounds__(sf_threads<R>(), sf_min_blocks<NP, R>())
    k_local_sf(SfTablesT<R> tab, int ncells, const int *__restrict__ cell_dofs, const R *__restrict__ wV,
               const double *__restrict__ X, int ldx, double *__restrict__ Y, int ldy, int ncols, double alpha,
               double cK, double cV, double cM, const double *__restrict__ cMcol) {
  sf_body<NP, R, sf_vt_r<NP, R>(), sf_threads<R>()>(tab, ncells, cell_dofs, wV, X, ldx, Y, ldy, ncols, alpha, cK, cV,
                                                    cM, cMcol);
}

// Lean FP64 form (4 vectors, 256 threads, at most 120 registers, about 69 KB of
// shared memory at degree 6): small enough to share an SM with a persistent
// cell-product or projection kernel in its lean form when step 2 of one block
// overlaps the loop of another (paw_cheb_filter).  (A 2-vector form, several
// per SM, measured slower: 305 against 291 ms per mid filter call.)
constexpr int SF_LEAN_VT = 4, SF_LEAN_THREADS = 256;
template <int NP>
__global__ void __maxnreg__(120)
    k_local_sf_lean(SfTablesT<double> tab, int ncells, const int *__restrict__ cell_dofs,
                    const double *__restrict__ wV, const double *__restrict__ X, int ldx, double *__restrict__ Y,
                    int ldy, int ncols, double alpha, double cK, double cV, double cM,
                    const double *__restrict__ cMcol) {
  sf_body<NP, double, SF_LEAN_VT, SF_LEAN_THREADS>(tab, ncells, cell_dofs, wV, X, ldx, Y, ldy, ncols, alpha, cK, cV,
                                                   cM, cMcol);
}

// Bloch term at a wavevector k: y = (h/2)^2 [k_x C (x) M (x) M + k_y M (x) C (x) M
// + k_z M (x) M (x) C] x per cell (C = the skew 1D matrix (C1 - C1^T)/2,
// C1[a][b] = int l_a l_b' dxi; M the 1D reference mass), accumulated into
// Y with factor alpha.  Same chain of 1D contractions as the kinetic part of
// k_local_sf (z, then y, then x), in the even/odd split: M is centro-symmetric,
// C centro-antisymmetric (C[n-1-i][n-1-j] = -C[i][j]), which maps the odd part
// of a line to the even part of the result and the even part to the odd one.
struct BlochTables {
  EoMat M, C;   // C: halves of the antisymmetric form (eo_acc_anti)
  double kx, ky, kz, scale;
};

// E[i] += sum_j Ae[i][j] o[j] (i < ceil(M/2), j < N/2),  O[i] += sum_j Ao[i][j] e[j]
// (i < M/2, j < ceil(N/2)) for a centro-antisymmetric M x N matrix
template <int M, int N>
__device__ __forceinline__ void eo_acc_anti(const EoMat &A, const Split<N> &x, double (&E)[(M + 1) / 2],
                                            double (&O)[M / 2 > 0 ? M / 2 : 1]) {
  constexpr int NE = (N + 1) / 2, NO = N / 2;
#pragma unroll
  for (int i = 0; i < (M + 1) / 2; ++i)
#pragma unroll
    for (int j = 0; j < NO; ++j) E[i] = fma(A.e[i * NO + j], x.o[j], E[i]);
#pragma unroll
  for (int i = 0; i < M / 2; ++i)
#pragma unroll
    for (int j = 0; j < NE; ++j) O[i] = fma(A.o[i * NE + j], x.e[j], O[i]);
}

template <int NP>
__global__ void __launch_bounds__(SF_THREADS, 1) k_bloch_sf(BlochTables tab, const int *__restrict__ cell_dofs,
                                                        const double *__restrict__ X, int ldx,
                                                        double *__restrict__ Y, int ldy, int ncols, double alpha) {
  constexpr int VT = sf_vt<NP>();
  constexpr int N3 = NP * NP * NP;
  __shared__ BlochTables st;
  __shared__ int dofs[N3];
  extern __shared__ double sm[];
  double *A0 = sm;               // x, then T
  double *A1 = A0 + N3 * VT;     // P, then y
  double *A2 = A1 + N3 * VT;     // Q
  double *A3 = A2 + N3 * VT;     // S
  const int e = blockIdx.x, v0 = blockIdx.y * VT, tid = threadIdx.x;
  {
    const double *src = reinterpret_cast<const double *>(&tab);
    double *dst = reinterpret_cast<double *>(&st);
    for (int i = tid; i < (int)(sizeof(BlochTables) / sizeof(double)); i += SF_THREADS) dst[i] = src[i];
  }
  for (int i = tid; i < N3; i += SF_THREADS) dofs[i] = cell_dofs[(size_t)e * N3 + i];
  __syncthreads();
  for (int idx = tid; idx < N3 * VT; idx += SF_THREADS) {
    const int r = idx / VT, v = idx - r * VT;
    A0[idx] = (v0 + v < ncols) ? X[(size_t)dofs[r] * ldx + v0 + v] : 0.0;
  }
  __syncthreads();
  // z lines: P = M_c x, Q = C_c x
  for (int idx = tid; idx < NP * NP * VT; idx += SF_THREADS) {
    const int ab = idx / VT, v = idx - ab * VT;
    const Split<NP> x = split_line<NP>(A0 + ab * VT + v, NP * NP * VT);
    Half<NP> P, Q;
    P.zero();
    Q.zero();
    eo_acc<NP, NP>(st.M, x, P.E, P.O);
    eo_acc_anti<NP, NP>(st.C, x, Q.E, Q.O);
#pragma unroll
    for (int c2 = 0; c2 < NP; ++c2) {
      A1[(c2 * NP * NP + ab) * VT + v] = P.out(c2);
      A2[(c2 * NP * NP + ab) * VT + v] = Q.out(c2);
    }
  }
  __syncthreads();
  // y lines: S = M_b P, T = k_y C_b P + k_z M_b Q
  for (int idx = tid; idx < NP * NP * VT; idx += SF_THREADS) {
    const int ac = idx / VT, v = idx - ac * VT;
    const int a = ac % NP, c = ac / NP;
    const int base = (c * NP * NP + a) * VT + v;
    const Split<NP> pl = split_line<NP>(A1 + base, NP * VT);
    const Split<NP> ql = split_line<NP>(A2 + base, NP * VT);
    Half<NP> S, T1, T2;
    S.zero();
    T1.zero();
    T2.zero();
    eo_acc<NP, NP>(st.M, pl, S.E, S.O);
    eo_acc_anti<NP, NP>(st.C, pl, T1.E, T1.O);
    eo_acc<NP, NP>(st.M, ql, T2.E, T2.O);
#pragma unroll
    for (int b2 = 0; b2 < NP; ++b2) {
      A3[base + b2 * NP * VT] = S.out(b2);
      A0[base + b2 * NP * VT] = fma(st.ky, T1.out(b2), st.kz * T2.out(b2));
    }
  }
  __syncthreads();
  // x lines: y = k_x C_a S + M_a T
  for (int idx = tid; idx < NP * NP * VT; idx += SF_THREADS) {
    const int bc = idx / VT, v = idx - bc * VT;
    const int base = bc * NP * VT + v;
    const Split<NP> sl = split_line<NP>(A3 + base, VT);
    const Split<NP> tl = split_line<NP>(A0 + base, VT);
    Half<NP> Y1, Y2;
    Y1.zero();
    Y2.zero();
    eo_acc_anti<NP, NP>(st.C, sl, Y1.E, Y1.O);
    eo_acc<NP, NP>(st.M, tl, Y2.E, Y2.O);
#pragma unroll
    for (int a2 = 0; a2 < NP; ++a2) A1[base + a2 * VT] = st.scale * fma(st.kx, Y1.out(a2), Y2.out(a2));
  }
  __syncthreads();
  for (int idx = tid; idx < N3 * VT; idx += SF_THREADS) {
    const int r = idx / VT, v = idx - r * VT;
    if (v0 + v < ncols) atomicAdd(&Y[(size_t)dofs[r] * ldy + v0 + v], alpha * A1[idx]);
  }
}

template <int NP>
void launch_bloch(paw_context *c, const BlochTables &t, const double *X, int ldx, double *Y, int ldy, int ncols,
                  double alpha, cudaStream_t s) {
  constexpr int VT = sf_vt<NP>();
  const size_t shm = sizeof(double) * 4 * (size_t)NP * NP * NP * VT;
  PAW_CUDA(cudaFuncSetAttribute(k_bloch_sf<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  dim3 g(c->ncells, (ncols + VT - 1) / VT);
  k_bloch_sf<NP><<<g, SF_THREADS, shm, s>>>(t, c->cell_dofs.as<int>(), X, ldx, Y, ldy, ncols, alpha);
  PAW_LAUNCH_CHECK("k_bloch_sf");
}

template <int NP, typename R, int VT = sf_vt_r<NP, R>()>
size_t sf_smem() {
  constexpr int NQ = NP + 1;
  constexpr int N3 = NP * NP * NP;
  constexpr int S1 = (NQ * NP * NP > N3) ? NQ * NP * NP : N3;
  constexpr int S2 = (NQ * NQ * NP > N3) ? NQ * NQ * NP : N3;
  constexpr int S3 = (NQ * NQ * NQ > N3) ? NQ * NQ * NQ : N3;
  return sizeof(double) * ((size_t)(2 * N3 + S1 + S2 + S3) * VT + NQ * NQ * NQ);
}

template <int NP, typename R>
void launch_sf(paw_context *c, const SfTablesT<R> &t, const R *wV, const double *X, int ldx, double *Y, int ldy,
               int ncols, double alpha, double cK, double cV, double cM, const double *cMcol, cudaStream_t s) {
  if constexpr (std::is_same<R, double>::value) {
    if (c->sf_lean) {
      const size_t shm = sf_smem<NP, double, SF_LEAN_VT>();
      PAW_CUDA(cudaFuncSetAttribute(k_local_sf_lean<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
      PAW_CUDA(cudaFuncSetAttribute(k_local_sf_lean<NP>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                    cudaSharedmemCarveoutMaxShared));
      dim3 g(c->ncells, (ncols + SF_LEAN_VT - 1) / SF_LEAN_VT);
      k_local_sf_lean<NP><<<g, SF_LEAN_THREADS, shm, s>>>(t, c->ncells, c->cell_dofs.as<int>(), wV, X, ldx, Y, ldy,
                                                            ncols, alpha, cK, cV, cM, cMcol);
      PAW_LAUNCH_CHECK("k_local_sf_lean");
      return;
    }
  }
  const size_t shm = sf_smem<NP, R>();
  PAW_CUDA(cudaFuncSetAttribute(k_local_sf<NP, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  dim3 g(c->ncells, (ncols + sf_vt_r<NP, R>() - 1) / sf_vt_r<NP, R>());
  k_local_sf<NP, R><<<g, sf_threads<R>(), shm, s>>>(t, c->ncells, c->cell_dofs.as<int>(), wV, X, ldx, Y, ldy, ncols, alpha,
                                              cK, cV, cM, cMcol);
  PAW_LAUNCH_CHECK("k_local_sf");
}

template <typename R>
void dispatch_sf(paw_context *c, const SfTablesT<R> &t, const R *wV, const double *X, int ldx, double *Y,
                 int ldy, int ncols, double alpha, double cK, double cV, double cM, const double *cMcol,
                 cudaStream_t s) {
  switch (c->np1) {
    case 2: launch_sf<2, R>(c, t, wV, X, ldx, Y, ldy, ncols, alpha, cK, cV, cM, cMcol, s); break;
    case 3: launch_sf<3, R>(c, t, wV, X, ldx, Y, ldy, ncols, alpha, cK, cV, cM, cMcol, s); break;
    case 4: launch_sf<4, R>(c, t, wV, X, ldx, Y, ldy, ncols, alpha, cK, cV, cM, cMcol, s); break;
    case 5: launch_sf<5, R>(c, t, wV, X, ldx, Y, ldy, ncols, alpha, cK, cV, cM, cMcol, s); break;
    case 6: launch_sf<6, R>(c, t, wV, X, ldx, Y, ldy, ncols, alpha, cK, cV, cM, cMcol, s); break;
    case 7: launch_sf<7, R>(c, t, wV, X, ldx, Y, ldy, ncols, alpha, cK, cV, cM, cMcol, s); break;
    case 8: launch_sf<8, R>(c, t, wV, X, ldx, Y, ldy, ncols, alpha, cK, cV, cM, cMcol, s); break;
    case 9: launch_sf<9, R>(c, t, wV, X, ldx, Y, ldy, ncols, alpha, cK, cV, cM, cMcol, s); break;
    default: throw Error{PAW_ERR_UNSUPPORTED, "degree out of range for the sum-factorised kernel"};
  }
}

// nearest pair of FP32 numbers to each table entry (hi = fl32(x), lo = fl32(x - hi))
static f32x2 host_pair(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}

static EoMatT<f32x2> pair_table(const EoMat &m) {
  EoMatT<f32x2> r{};
  for (int i = 0; i < EOMAX * EOMAX; ++i) {
    r.e[i] = host_pair(m.e[i]);
    r.o[i] = host_pair(m.o[i]);
  }
  return r;
}

__global__ void k_wV(int64_t n, int nq, const double *__restrict__ wq, const double *__restrict__ Vq,
                     double *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = wq[i % nq] * Vq[i];
}

__global__ void k_wV_pair(int64_t n, const double *__restrict__ wV, f32x2 *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = x2_from(wV[i]);
}

}  // namespace

// even/odd halves of a row-major m x n matrix (see EoMat); the matrix is
// centro-symmetric up to rounding, and the halves use its symmetrised form
static void eo_halves(const double *A, int m, int n, EoMat &out) {
  const int ne = (n + 1) / 2, no = n / 2;
  for (int i = 0; i < (m + 1) / 2; ++i) {
    for (int j = 0; j < no; ++j)
      out.e[i * ne + j] = 0.5 * (A[(size_t)i * n + j] + A[(size_t)i * n + (n - 1 - j)]);
    if (n & 1) out.e[i * ne + no] = A[(size_t)i * n + no];
  }
  for (int i = 0; i < m / 2; ++i)
    for (int j = 0; j < no; ++j)
      out.o[i * no + j] = 0.5 * (A[(size_t)i * n + j] - A[(size_t)i * n + (n - 1 - j)]);
}

// even/odd halves of a centro-antisymmetric m x n matrix A (A[m-1-i][n-1-j] = -A[i][j]),
// in the layout of eo_acc_anti:
//   e[i][j] = (A[i][j] - A[i][n-1-j]) / 2      (i < ceil(m/2), j < n/2; pairs with o-lines),
//   o[i][j] = (A[i][j] + A[i][n-1-j]) / 2      (i < m/2, j < n/2),  o[i][n/2] = A[i][n/2] for odd n.
static void eo_halves_anti(const double *A, int m, int n, EoMat &out) {
  const int ne = (n + 1) / 2, no = n / 2;
  for (int i = 0; i < (m + 1) / 2; ++i)
    for (int j = 0; j < no; ++j)
      out.e[i * no + j] = 0.5 * (A[(size_t)i * n + j] - A[(size_t)i * n + (n - 1 - j)]);
  for (int i = 0; i < m / 2; ++i) {
    for (int j = 0; j < no; ++j)
      out.o[i * ne + j] = 0.5 * (A[(size_t)i * n + j] + A[(size_t)i * n + (n - 1 - j)]);
    if (n & 1) out.o[i * ne + no] = A[(size_t)i * n + no];
  }
}

void bloch_sf(paw_context *c, const double *X, int ldx, double *Y, int ldy, int ncols, double alpha,
              cudaStream_t s) {
  if (ncols <= 0 || !c->kc) return;
  const int np1 = c->np1;
  PAW_REQUIRE(np1 <= 10, PAW_ERR_UNSUPPORTED, "degree out of range for the Bloch kernel");
  BlochTables t{};
  eo_halves(c->M1.data(), np1, np1, t.M);
  eo_halves_anti(c->C1s.data(), np1, np1, t.C);
  t.kx = c->kvec[0];
  t.ky = c->kvec[1];
  t.kz = c->kvec[2];
  t.scale = (c->h / 2.0) * (c->h / 2.0);
  switch (np1) {
    case 2: launch_bloch<2>(c, t, X, ldx, Y, ldy, ncols, alpha, s); break;
    case 3: launch_bloch<3>(c, t, X, ldx, Y, ldy, ncols, alpha, s); break;
    case 4: launch_bloch<4>(c, t, X, ldx, Y, ldy, ncols, alpha, s); break;
    case 5: launch_bloch<5>(c, t, X, ldx, Y, ldy, ncols, alpha, s); break;
    case 6: launch_bloch<6>(c, t, X, ldx, Y, ldy, ncols, alpha, s); break;
    case 7: launch_bloch<7>(c, t, X, ldx, Y, ldy, ncols, alpha, s); break;
    case 8: launch_bloch<8>(c, t, X, ldx, Y, ldy, ncols, alpha, s); break;
    case 9: launch_bloch<9>(c, t, X, ldx, Y, ldy, ncols, alpha, s); break;
    default: throw Error{PAW_ERR_UNSUPPORTED, "degree out of range for the Bloch kernel"};
  }
}

void local_sf(paw_context *c, const double *X, int ldx, double *Y, int ldy, int ncols, double alpha, double cK,
              double cV, double cM, const double *cMcol, cudaStream_t s, bool pair32) {
  if (ncols <= 0) return;
  SfTables t{};
  const int np1 = c->np1, nq1 = c->nq1;
  std::vector<double> phit((size_t)np1 * nq1);
  for (int q = 0; q < nq1; ++q)
    for (int a = 0; a < np1; ++a) phit[(size_t)a * nq1 + q] = c->phiq[(size_t)q * np1 + a];
  eo_halves(c->M1.data(), np1, np1, t.M);
  eo_halves(c->D1.data(), np1, np1, t.D);
  eo_halves(c->phiq.data(), nq1, np1, t.phi);
  eo_halves(phit.data(), np1, nq1, t.phit);
  const double hh = c->h / 2.0;
  t.kfac = 0.5 * hh;
  t.mfac = hh * hh * hh;
  {
    const double kf = cK * t.kfac;
    std::vector<double> kD(c->D1), kM(c->M1);
    for (double &x : kD) x *= kf;
    for (double &x : kM) x *= kf;
    eo_halves(kD.data(), np1, np1, t.kD);
    eo_halves(kM.data(), np1, np1, t.kM);
  }
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
  if (!pair32) {
    dispatch_sf<double>(c, t, wV, X, ldx, Y, ldy, ncols, alpha, cK, cV, cM, cMcol, s);
    return;
  }
  if (!c->wVx2_valid) {   // w_q V_q as pairs of FP32 numbers, rebuilt with wV
    c->wVx2.ensure(sizeof(f32x2) * nwv, &c->dev_bytes);
    k_wV_pair<<<(unsigned)((nwv + 255) / 256), 256, 0, s>>>((int64_t)nwv, wV, c->wVx2.as<f32x2>());
    PAW_LAUNCH_CHECK("k_wV_pair");
    c->wVx2_valid = 1;
  }
  SfTablesT<f32x2> tp{};
  tp.M = pair_table(t.M);
  tp.D = pair_table(t.D);
  tp.phi = pair_table(t.phi);
  tp.phit = pair_table(t.phit);
  tp.kD = pair_table(t.kD);
  tp.kM = pair_table(t.kM);
  tp.kfac = t.kfac;
  tp.mfac = t.mfac;
  dispatch_sf<f32x2>(c, tp, c->wVx2.as<f32x2>(), X, ldx, Y, ldy, ncols, alpha, cK, cV, cM, cMcol, s);
}

}  // namespace pawfe
