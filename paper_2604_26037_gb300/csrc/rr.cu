// Rayleigh-Ritz contractions (Algorithm 1 steps 4 and 6; Sec. 4.5
// "RR-Projection" and "RR-SR"):
//   * projection: A^p = X^T Y for Y = H X or S X, only the lower triangle,
//     one column block of the block vectors at a time (N x B_v blocks);
//   * rotation X <- X Q, in FP64 or in the mixed form of the RR-SR step
//     (X diag(Q) in FP64 plus fl32(X) fl32(Q - diag(Q)) with FP32
//     accumulation: Q tends to the identity as the iteration converges, so
//     its off-diagonal part is small).
// At a Bloch wavevector the complex blocks are read as real blocks of 2N
// interleaved columns: one real Gram matrix holds the four real products of
// X^H Y, and a complex Q acts as a real 2N x 2N matrix.
//
// All are FP64-pipe (or FP32-pipe) bound: 64 x 64 output tiles, 256 threads
// holding 4 x 4 accumulators each, operands staged through shared memory in
// chunks of 32 along the contraction.  The projection's contraction runs over
// all DoFs (M ~ 10^6), so it is split into slices written as partial tiles and
// summed in a fixed order (deterministic).
#include <algorithm>

#include "common.cuh"

namespace pawfe {
namespace {

constexpr int TM = 64, TN = 64, KC = 32, THREADS = 256;

// part[s][r][c] = sum over rows i of slice s of A[i][r] * B[i][c]
// (r < R, c < C; A row pitch lda, B row pitch ldb; tile rows r0.. and
// columns c0..).  lower = 1: tiles whose every entry has r + doff < c are
// skipped (strictly above the diagonal; doff = global row offset of r = 0
// minus that of c = 0, here 0).
__global__ void __launch_bounds__(THREADS) k_gram_part(int64_t K, int nslice, const double *__restrict__ A, int lda,
                                                       int R, const double *__restrict__ B, int ldb, int C,
                                                       int lower, int Rp, int Cp, double *__restrict__ part) {
  __shared__ double As[KC][TM + 1];
  __shared__ double Bs[KC][TN + 1];
  const int a0 = blockIdx.x * TM, b0 = blockIdx.y * TN, sl = blockIdx.z;
  if (lower && a0 + TM - 1 < b0) return;   // never read by the eigensolver
  const int64_t per = (K + nslice - 1) / nslice;
  const int64_t k0 = (int64_t)sl * per, k1 = min(K, k0 + per);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;
  for (int64_t kb = k0; kb < k1; kb += KC) {
#pragma unroll
    for (int j = 0; j < KC * TM / THREADS; ++j) {
      const int idx = threadIdx.x + THREADS * j;
      const int kk = idx / TM, cc = idx % TM;
      const int64_t i = kb + kk;
      As[kk][cc] = (i < k1 && a0 + cc < R) ? A[i * lda + a0 + cc] : 0.0;
      Bs[kk][cc] = (i < k1 && b0 + cc < C) ? B[i * ldb + b0 + cc] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < KC; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
  double *P = part + (size_t)sl * Rp * Cp;
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) P[(size_t)(a0 + ty + 16 * r) * Cp + b0 + tx + 16 * c] = acc[r][c];
}

// G[c * ldg + r] (column-major) = sum_s part[s][r][c] in slice order, for the
// entries of tiles k_gram_part computed
__global__ void k_gram_reduce(int nslice, int R, int C, int lower, int Rp, int Cp, const double *__restrict__ part,
                              double *__restrict__ G, int ldg) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)R * C) return;
  const int r = (int)(idx % R), c = (int)(idx / R);
  if (lower && (r / TM) * TM + TM - 1 < (c / TN) * TN) return;
  double s = 0.0;
  for (int k = 0; k < nslice; ++k) s += part[((size_t)k * Rp + r) * Cp + c];
  G[(size_t)c * ldg + r] = s;
}

// Hermitian A^p (column-major complex, lower part used) from the real Gram
// matrix G (column-major, 2N x 2N) of interleaved (re, im) columns:
// A^p[a][b] = (G[2a][2b] + G[2a+1][2b+1]) + i (G[2a][2b+1] - G[2a+1][2b]).
__global__ void k_gram_to_hermitian(int N, const double *__restrict__ G, double2 *__restrict__ Ap) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)N * N) return;
  const int a = (int)(idx % N), b = (int)(idx / N);
  const int64_t ld = 2 * (int64_t)N;
  auto g = [&](int r, int c) { return G[(int64_t)c * ld + r]; };
  Ap[(size_t)b * N + a] = make_double2(g(2 * a, 2 * b) + g(2 * a + 1, 2 * b + 1), g(2 * a, 2 * b + 1) - g(2 * a + 1, 2 * b));
}

// Real 2N x 2N form (column-major) of a complex N x N matrix Q (column-major):
// for interleaved rows z = (re, im) of X, z Q_real = interleaved rows of X Q.
__global__ void k_complex_to_real(int N, const double2 *__restrict__ Q, double *__restrict__ Qr) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)N * N) return;
  const int l = (int)(idx % N), j = (int)(idx / N);
  const double2 q = Q[(size_t)j * N + l];
  const int64_t ld = 2 * (int64_t)N;
  Qr[(int64_t)(2 * j) * ld + 2 * l] = q.x;
  Qr[(int64_t)(2 * j) * ld + 2 * l + 1] = -q.y;
  Qr[(int64_t)(2 * j + 1) * ld + 2 * l] = q.y;
  Qr[(int64_t)(2 * j + 1) * ld + 2 * l + 1] = q.x;
}

// out[i][j] = sum_l X[i][l] Q[l][j] for rows i < nr of X (pitch ldx) and
// columns j < N; Q column-major (Q[l + j ldq]).  TA = double: FP64 products
// and sums.  TA = float: the mixed rotation, operands rounded to FP32 (X on
// load, Q given as FP32 with a zero diagonal), FP32 sums, then
// out = X[i][j] qd[j] + sum in FP64.  out has pitch ldo (FP64).
template <typename TA>
__global__ void __launch_bounds__(THREADS) k_rotate(int nr, int N, const double *__restrict__ X, int ldx,
                                                    const TA *__restrict__ Q, int ldq,
                                                    const double *__restrict__ qd, double *__restrict__ out,
                                                    int ldo) {
  __shared__ TA Xs[TM][KC + 1];
  __shared__ TA Qs[KC][TN + 1];
  const int i0 = blockIdx.x * TM, j0 = blockIdx.y * TN;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  TA acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = TA(0);
  for (int l0 = 0; l0 < N; l0 += KC) {
#pragma unroll
    for (int j = 0; j < KC * TM / THREADS; ++j) {
      const int idx = threadIdx.x + THREADS * j;
      // X tile: row rr, contraction index ll (ll fastest: a row segment is contiguous)
      const int rr = idx / KC, ll = idx % KC;
      Xs[rr][ll] = (i0 + rr < nr && l0 + ll < N) ? TA(X[(int64_t)(i0 + rr) * ldx + l0 + ll]) : TA(0);
      // Q tile: contraction index ll2 fastest (Q is column-major)
      const int cc = idx / KC, ll2 = idx % KC;
      Qs[ll2][cc] = (j0 + cc < N && l0 + ll2 < N) ? Q[(int64_t)(j0 + cc) * ldq + l0 + ll2] : TA(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < KC; ++kk) {
      TA a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = Xs[ty + 16 * r][kk];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Qs[kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = i0 + ty + 16 * r;
    if (i >= nr) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = j0 + tx + 16 * c;
      if (j >= N) continue;
      if constexpr (sizeof(TA) == 8)
        out[(int64_t)i * ldo + j] = acc[r][c];
      else
        out[(int64_t)i * ldo + j] = fma(X[(int64_t)i * ldx + j], qd[j], (double)acc[r][c]);
    }
  }
}

// q32 = fl32(Q) with a zero diagonal, qd = diag(Q) (FP64), Q column-major N x N
__global__ void k_split_q(int N, const double *__restrict__ Q, float *__restrict__ q32, double *__restrict__ qd) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)N * N) return;
  const int r = (int)(i % N), col = (int)(i / N);
  q32[i] = (r == col) ? 0.f : (float)Q[i];
  if (r == col) qd[col] = Q[i];
}

int sm_count() {
  int dev = 0, n = 0;
  PAW_CUDA(cudaGetDevice(&dev));
  PAW_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
  return std::max(1, n);
}

}  // namespace

void rr_gram(paw_context *c, const double *A, int lda, int R, const double *B, int ldb, int C, int64_t K, bool lower,
             double *G, int ldg, cudaStream_t s) {
  if (R <= 0 || C <= 0) return;
  const int tr = (R + TM - 1) / TM, tc = (C + TN - 1) / TN;
  int tiles = 0;
  for (int a = 0; a < tr; ++a)
    for (int b = 0; b < tc; ++b) tiles += (!lower || a * TM + TM - 1 >= b * TN) ? 1 : 0;
  // about four resident CTAs per SM over all active tiles; every slice at least one chunk
  int nslice = std::max(1, (4 * sm_count() + tiles - 1) / tiles);
  nslice = (int)std::min<int64_t>(nslice, std::max<int64_t>(1, K / KC));
  const int Rp = tr * TM, Cp = tc * TN;
  c->ws_gram.ensure(sizeof(double) * (size_t)nslice * Rp * Cp, &c->dev_bytes);
  double *part = c->ws_gram.as<double>();
  k_gram_part<<<dim3(tr, tc, nslice), THREADS, 0, s>>>(K, nslice, A, lda, R, B, ldb, C, lower ? 1 : 0, Rp, Cp, part);
  PAW_LAUNCH_CHECK("k_gram_part");
  const int64_t n = (int64_t)R * C;
  k_gram_reduce<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(nslice, R, C, lower ? 1 : 0, Rp, Cp, part, G, ldg);
  PAW_LAUNCH_CHECK("k_gram_reduce");
}

void rr_gram_to_hermitian(int N, const double *G, void *Ap, cudaStream_t s) {
  const int64_t n = (int64_t)N * N;
  k_gram_to_hermitian<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(N, G, static_cast<double2 *>(Ap));
  PAW_LAUNCH_CHECK("k_gram_to_hermitian");
}

void rr_complex_to_real(int N, const void *Q, double *Qr, cudaStream_t s) {
  const int64_t n = (int64_t)N * N;
  k_complex_to_real<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(N, static_cast<const double2 *>(Q), Qr);
  PAW_LAUNCH_CHECK("k_complex_to_real");
}

void rr_rotate(paw_context *c, double *X, int ld, int64_t M, int N, const double *Q, bool mixed, cudaStream_t s) {
  // rows per chunk: the rotated chunk goes to a temporary (at most 1 GiB), then back into X
  const int64_t rows = std::min<int64_t>(M, std::max<int64_t>(1024, ((int64_t)1 << 27) / N));
  size_t bytes = sizeof(double) * (size_t)rows * N;
  if (mixed) bytes += sizeof(float) * (size_t)N * N + sizeof(double) * N;
  c->ws_rot.ensure(bytes, &c->dev_bytes);
  double *tmp = c->ws_rot.as<double>();
  float *q32 = nullptr;
  double *qd = nullptr;
  if (mixed) {
    qd = tmp + (size_t)rows * N;
    q32 = reinterpret_cast<float *>(qd + N);
    const int64_t n = (int64_t)N * N;
    k_split_q<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(N, Q, q32, qd);
    PAW_LAUNCH_CHECK("k_split_q");
  }
  for (int64_t r0 = 0; r0 < M; r0 += rows) {
    const int nr = (int)std::min<int64_t>(rows, M - r0);
    const dim3 g((nr + TM - 1) / TM, (N + TN - 1) / TN);
    if (mixed)
      k_rotate<float><<<g, THREADS, 0, s>>>(nr, N, X + r0 * ld, ld, q32, N, qd, tmp, N);
    else
      k_rotate<double><<<g, THREADS, 0, s>>>(nr, N, X + r0 * ld, ld, Q, N, nullptr, tmp, N);
    PAW_LAUNCH_CHECK("k_rotate");
    PAW_CUDA(cudaMemcpy2DAsync(X + r0 * ld, sizeof(double) * ld, tmp, sizeof(double) * N, sizeof(double) * N, nr,
                               cudaMemcpyDeviceToDevice, s));
  }
}

}  // namespace pawfe
