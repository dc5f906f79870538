// C ABI entry points, the Algorithm 2 driver, Rayleigh-Ritz, residuals,
// Lanczos bounds and the energy gradient.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include <cudaTypedefs.h>

#include "common.cuh"

namespace pawfe {

static thread_local std::string g_last_error;
int64_t g_launch_count = 0;

static cudaEvent_t prof_event(paw_context *c) {
  auto &P = c->prof;
  if (P.used == P.pool.size()) {
    cudaEvent_t e;
    PAW_CUDA(cudaEventCreate(&e));
    P.pool.push_back(e);
  }
  return P.pool[P.used++];
}

PhaseScope::PhaseScope(paw_context *ctx, int phase, cudaStream_t st) : c(ctx), ph(phase), s(st) {
  if (!c->prof.on) return;
  a = prof_event(c);
  PAW_CUDA(cudaEventRecord(a, s));
  l0 = g_launch_count;
}

PhaseScope::~PhaseScope() {
  if (!c->prof.on || !a) return;
  cudaEvent_t b = nullptr;
  try {
    b = prof_event(c);
  } catch (...) {
    return;
  }
  if (cudaEventRecord(b, s) == cudaSuccess) c->prof.marks.push_back({ph, a, b});
  c->prof.launches[ph] += g_launch_count - l0;
}

void set_error(const std::string &msg) { g_last_error = msg; }
paw_status fail(paw_status code, const std::string &msg) {
  g_last_error = msg;
  return code;
}

int read_status(paw_context *c) {
  if (!c->status_dev.ptr) return 0;
  int v = 0;
  if (cudaMemcpyAsync(&v, c->status_dev.ptr, sizeof(int), cudaMemcpyDeviceToHost, c->last_stream) != cudaSuccess ||
      cudaStreamSynchronize(c->last_stream) != cudaSuccess)
    return -1;
  if (v != 0 && cudaMemsetAsync(c->status_dev.ptr, 0, sizeof(int), c->last_stream) != cudaSuccess) return -1;
  return v;
}

void encode_row_map(CUtensorMap *map, const float *base, int64_t rows, int cols, int ld) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    return (e == cudaSuccess && q == cudaDriverEntryPointSuccess) ? reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn)
                                                                 : nullptr;
  }();
  PAW_REQUIRE(encode != nullptr, PAW_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  PAW_REQUIRE(reinterpret_cast<uintptr_t>(base) % 16 == 0 && ld % 4 == 0 && cols >= 1 && cols <= ld && rows >= 1,
              PAW_ERR_INVALID_ARG, "row map: base must be 16-byte aligned, ld a multiple of 4");
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
  const cuuint32_t box[2] = {128, 1};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides, box,
                            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  PAW_REQUIRE(r == CUDA_SUCCESS, PAW_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
}

void DevBuf::ensure(size_t nbytes, int64_t *counter) {
  if (nbytes <= bytes && ptr) return;
  if (ptr) {
    cudaFree(ptr);
    if (counter) *counter -= (int64_t)bytes;
    ptr = nullptr;
    bytes = 0;
  }
  if (nbytes == 0) return;
  PAW_CUDA(cudaMalloc(&ptr, nbytes));
  bytes = nbytes;
  if (counter) *counter += (int64_t)bytes;
}

void DevBuf::release(int64_t *counter) {
  if (ptr) {
    cudaFree(ptr);
    if (counter) *counter -= (int64_t)bytes;
  }
  ptr = nullptr;
  bytes = 0;
}

// ============================================================== filter kernels
// R_Y = (zeta_1/e) Y, R_X = 0 (Algorithm 2 step 3).  For the FP32 recurrence Y is
// also split into two FP32 words hi + lo (lo omitted when Y is kept in FP32 only).
// y = hi + lo with hi = y truncated to 24 significant bits and lo = y - hi (29
// bits, exact) rounded to FP32, by integer operations on the FP64 bit pattern:
// the FP64 pipe (which also carries the FP64 <-> FP32 conversions) runs at 1/64
// of the FP32 rate on GB300 and would bound this pass.  Exponents outside
// [2^-74, 2^127) (zero, tiny, huge, Inf/NaN) take the conversions.
__device__ __forceinline__ void split_hi_lo(double y, float &hi, float &lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(y);
  const int e = (int)((b >> 52) & 0x7ffull);
  if (e < 949 || e > 1150) {
    hi = (float)y;
    lo = (float)(y - (double)hi);
    return;
  }
  const unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
  const unsigned int hb = sign | ((unsigned int)(e - 896) << 23) | (unsigned int)((b >> 29) & 0x7fffffull);
  hi = __uint_as_float(hb);
  const float r = __uint2float_rn((unsigned int)(b & 0x1fffffffull));   // low 29 fraction bits
  const float scale = __uint_as_float((unsigned int)(e - 948) << 23);   // 2^(e - 1075)
  lo = __uint_as_float(__float_as_uint(__fmul_rn(r, scale)) | sign);
}

template <typename TR>
__global__ void k_cheb_init(int64_t rows, int ncols, const double *__restrict__ Y0, int ldy,
                            double s, float s_hi, float s_lo, TR *__restrict__ RY, TR *__restrict__ RX,
                            int ldr, float *__restrict__ Yhi, float *__restrict__ Ylo) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.y + threadIdx.y;
  const int v = blockIdx.y * blockDim.x + threadIdx.x;
  if (i >= rows || v >= ncols) return;
  const double y = Y0[i * ldy + v];
  RX[i * ldr + v] = TR(0);
  if constexpr (sizeof(TR) == 8) {
    RY[i * ldr + v] = (TR)(s * y);
  } else {
    float h, l;
    split_hi_lo(y, h, l);
    // s y to within an FP32 ulp: s_hi h + (s_hi l + s_lo h)
    RY[i * ldr + v] = fmaf(s_hi, h, fmaf(s_hi, l, s_lo * h));
    if (Yhi) {
      Yhi[i * ldr + v] = h;
      if (Ylo) Ylo[i * ldr + v] = l;
    }
  }
}

// The same for FP32 R with four columns per thread (16-byte rows, ncols % 4 == 0,
// rows * ncols / 4 < 2^31): 32-byte loads of Y and 16-byte stores, grid-stride.
__global__ void k_cheb_init4(int64_t rows, int ncols, const double *__restrict__ Y0, int ldy, float s_hi,
                             float s_lo, float *__restrict__ RY, float *__restrict__ RX, int ldr,
                             float *__restrict__ Yhi, float *__restrict__ Ylo) {
  const uint32_t nq = (uint32_t)(ncols / 4), total = (uint32_t)rows * nq;
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
    const uint32_t i = q / nq;
    const int v = (int)(q - i * nq) * 4;
    const double2 a = *reinterpret_cast<const double2 *>(Y0 + (int64_t)i * ldy + v);
    const double2 b = *reinterpret_cast<const double2 *>(Y0 + (int64_t)i * ldy + v + 2);
    const double y[4] = {a.x, a.y, b.x, b.y};
    float h[4], l[4], r[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      split_hi_lo(y[j], h[j], l[j]);
      r[j] = fmaf(s_hi, h[j], fmaf(s_hi, l[j], s_lo * h[j]));   // s y to within an FP32 ulp
    }
    const int64_t o = (int64_t)i * ldr + v;
    *reinterpret_cast<float4 *>(RX + o) = make_float4(0.f, 0.f, 0.f, 0.f);
    *reinterpret_cast<float4 *>(RY + o) = make_float4(r[0], r[1], r[2], r[3]);
    if (Yhi) {
      *reinterpret_cast<float4 *>(Yhi + o) = make_float4(h[0], h[1], h[2], h[3]);
      if (Ylo) *reinterpret_cast<float4 *>(Ylo + o) = make_float4(l[0], l[1], l[2], l[3]);
    }
  }
}

// Loop body of Algorithm 2 when no atom carries projectors:
//   T = M_D^-1 R_Y,  R_X = [-beta R_Y - gamma R_X] + c_j Y,  c_j = alpha Lambda_Y[j]
// (FP32: Y as hi/lo words, c_j as chi + clo, error-free product and sum).
__device__ __forceinline__ float add_product_ef(float b, float ch, float cl, float yh, float yl) {
  // explicit round-to-nearest operations: no contraction into FMA may alter the two-sum
  const float th = __fmul_rn(ch, yh);
  const float te = fmaf(ch, yh, -th);                    // exact error of ch * yh
  const float tl = fmaf(ch, yl, fmaf(cl, yh, te));
  const float s = __fadd_rn(b, th);                      // two-sum of b and th
  const float bp = __fsub_rn(s, b);
  const float err = __fadd_rn(__fsub_rn(b, __fsub_rn(s, bp)), __fsub_rn(th, bp));
  return __fadd_rn(s, __fadd_rn(err, tl));
}

template <typename TR>
__global__ void k_cheb_base(int64_t rows, int ncols, const TR *__restrict__ RY, TR *__restrict__ RX,
                            TR *__restrict__ T, int ldr, const void *__restrict__ Y0, const float *__restrict__ Ylo,
                            int ldy, const double *__restrict__ c64, const float *__restrict__ chi,
                            const float *__restrict__ clo, TR beta, TR gamma, const TR *__restrict__ mdinv) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.y + threadIdx.y;
  const int v = blockIdx.y * blockDim.x + threadIdx.x;
  if (i >= rows || v >= ncols) return;
  const TR ry = RY[i * ldr + v];
  const TR bracket = -beta * ry - gamma * RX[i * ldr + v];
  if constexpr (sizeof(TR) == 4) {
    const float yh = static_cast<const float *>(Y0)[i * ldy + v];
    const float yl = Ylo ? Ylo[i * ldy + v] : 0.f;
    RX[i * ldr + v] = add_product_ef(bracket, chi[v], clo[v], yh, yl);
  } else {
    RX[i * ldr + v] = fma(c64[v], static_cast<const double *>(Y0)[i * ldy + v], bracket);
  }
  T[i * ldr + v] = mdinv[i] * ry;
}

// Algorithm 2 step 5: Psi_f = Shat^-1 R_Y + X Lambda_Y, combined in FP64.
template <typename TR>
__global__ void k_cheb_recover(int64_t rows, int ncols, const TR *__restrict__ T, int ldr,
                               const double *__restrict__ X, int ldx, const double *__restrict__ lamY,
                               double *__restrict__ Xo, int ldo) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.y + threadIdx.y;
  const int v = blockIdx.y * blockDim.x + threadIdx.x;
  if (i >= rows || v >= ncols) return;
  Xo[i * ldo + v] = (double)T[i * ldr + v] + X[i * ldx + v] * lamY[v];
}

static inline dim3 ew_grid(int64_t rows, int ncols) {
  return dim3((unsigned)((rows + 7) / 8), (ncols + 31) / 32);
}

// Complex multivectors at k != 0: interleaved (re, im) entries, ld in complex
// entries  <->  split real blocks [Re | Im] of 2 n columns (ld = 2 n).
template <typename T>
__global__ void k_split_cplx(int64_t rows, int n, const T *__restrict__ Z, int ldz, T *__restrict__ Xs) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.y + threadIdx.y;
  const int j = blockIdx.y * blockDim.x + threadIdx.x;
  if (i >= rows || j >= n) return;
  const T re = Z[2 * (i * ldz + j)], im = Z[2 * (i * ldz + j) + 1];
  Xs[i * 2 * n + j] = re;
  Xs[i * 2 * n + n + j] = im;
}

template <typename T>
__global__ void k_merge_cplx(int64_t rows, int n, const T *__restrict__ Xs, T *__restrict__ Z, int ldz) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.y + threadIdx.y;
  const int j = blockIdx.y * blockDim.x + threadIdx.x;
  if (i >= rows || j >= n) return;
  Z[2 * (i * ldz + j)] = Xs[i * 2 * n + j];
  Z[2 * (i * ldz + j) + 1] = Xs[i * 2 * n + n + j];
}

template <typename T>
static void split_cplx(paw_context *c, const T *Z, int ldz, int n, T *Xs, cudaStream_t s) {
  k_split_cplx<T><<<ew_grid(c->ndof, n), dim3(32, 8), 0, s>>>(c->ndof, n, Z, ldz, Xs);
  PAW_LAUNCH_CHECK("k_split_cplx");
}

template <typename T>
static void merge_cplx(paw_context *c, const T *Xs, int n, T *Z, int ldz, cudaStream_t s) {
  k_merge_cplx<T><<<ew_grid(c->ndof, n), dim3(32, 8), 0, s>>>(c->ndof, n, Xs, Z, ldz);
  PAW_LAUNCH_CHECK("k_merge_cplx");
}

// Y = H X - S X Lambda in FP64 (Algorithm 2 step 2), or in pair-of-FP32 arithmetic
// with FP64 data when options.y0_pair32 is set
static void residual_block(paw_context *c, const double *X, int ldx, const double *negLam_dev,
                           double *Y, int ldy, int ncols, cudaStream_t s) {
  zero_block<double>(Y, c->ndof, ncols, ldy, s);
  const bool pair = c->opts.y0_pair32 != 0;   // pair-of-FP32 arithmetic (k = 0 only, checked at create)
  // both parts add into Y (the local part first: with the nonlocal part first beside a
  // loop, the mid filter call measured 293 instead of 288 ms)
  auto nonlocal = [&]() {
    if (c->nown_pairs > 0 && pair) {
      PhaseScope ps(c, 4, s);
      nl_residual_pair(c, X, ldx, ncols, c->DH64.as<double>(), c->DS64.as<double>(), negLam_dev, Y, ldy, s);
    } else if (c->nown_pairs > 0) {
      PhaseScope ps(c, 4, s);
      // sum_a P^a (D_H^a - lambda_j dS^a) P^a^T x_j: one projection, one expansion
      c->scr->W2.ensure(sizeof(double) * (size_t)c->natoms * c->npad * ncols, &c->dev_bytes);
      double *W = c->scr->W2.as<double>();
      nl_project_residual<double>(c, X, ldx, ncols, negLam_dev, W, s);
      nl_expand<double>(c, PAW_FP64, W, ncols, Y, ldy, nullptr, s);
    }
  };
  // (1/2 K^e + V^e + (1/2 |k|^2 - lambda_j) M^e) X_e in one sum-factorised pass;
  // at k != 0 the Bloch term -i B of Eq. hij on the split block [Re | Im]
  {
    PhaseScope ps(c, 0, s);
    local_sf(c, X, ldx, Y, ldy, ncols, 1.0, 1.0, 1.0, c->kmass, negLam_dev, s, pair);
    if (c->kc) {
      bloch_sf(c, X + ncols / 2, ldx, Y, ldy, ncols / 2, 1.0, s);
      bloch_sf(c, X, ldx, Y + ncols / 2, ldy, ncols / 2, -1.0, s);
    }
  }
  nonlocal();
}

template <typename T>
static const T *mdinv_of(paw_context *c);
template <>
const double *mdinv_of<double>(paw_context *c) { return c->md_inv64.as<double>(); }
template <>
const float *mdinv_of<float>(paw_context *c) { return c->md_inv32.as<float>(); }

// One block of Algorithm 2 in working precision TR.
// Host-side scalars of one block (Algorithm 2 steps 1, 3, 4): the recurrence
// coefficients alpha_k, beta_k, gamma_k of every loop step and the device
// scalar image hd = [-Lambda (nb)][Lambda_Y final (nb)][cf (nsteps nb)],
// cf[k][j] = alpha_k Lambda_Y[j], plus its FP32 split hf = [hi (..)][lo (..)].
size_t cheb_nd(int nb, int m) { return 2 * (size_t)nb + (size_t)std::max(0, m - 1) * nb; }
size_t cheb_nf(int nb, int m) { return 2 * (size_t)std::max(0, m - 1) * nb + 2; }

void cheb_plan(int nb, int m, paw_bounds bd, const double *lam, ChebScalars &S, double *hd, float *hf) {
  const double e = (bd.bU - bd.bW) / 2.0;
  const double cc = (bd.bU + bd.bW) / 2.0;
  double zeta = e / (bd.a0 - cc);
  double zeta1 = zeta;
  const double gam = 2.0 / zeta1;
  std::vector<double> LX(nb, 1.0), LY(nb);
  S.al.clear();
  S.be.clear();
  S.ga.clear();
  S.nsteps = m - 1;
  S.nd = cheb_nd(nb, m);
  S.nf = cheb_nf(nb, m);
  double *cf = hd + 2 * (size_t)nb;
  for (int j = 0; j < nb; ++j) LY[j] = (zeta1 / e) * (lam[j] - cc);
  for (int th = 2, k = 0; th <= m; ++th, ++k) {
    zeta1 = 1.0 / (gam - zeta);
    const double alpha = 2.0 * zeta1 / e, beta = alpha * cc, gk = zeta * zeta1;
    S.al.push_back(alpha);
    S.be.push_back(beta);
    S.ga.push_back(gk);
    for (int j = 0; j < nb; ++j) cf[(size_t)k * nb + j] = alpha * LY[j];
    for (int j = 0; j < nb; ++j) {
      const double nx = alpha * LY[j] * lam[j] - beta * LY[j] - gk * LX[j];
      LX[j] = LY[j];
      LY[j] = nx;
    }
    zeta = zeta1;
  }
  for (int j = 0; j < nb; ++j) {
    hd[j] = -lam[j];
    hd[nb + j] = LY[j];
  }
  const size_t ncf = (size_t)S.nsteps * nb;
  for (size_t i = 0; i < ncf; ++i) {
    const float h = (float)cf[i];
    hf[i] = h;
    hf[ncf + i] = (float)(cf[i] - (double)h);
  }
  hf[2 * ncf] = hf[2 * ncf + 1] = 0.f;
}

// Algorithm 2 for one block of nb columns, in two parts that only enqueue
// copies and kernels (no host synchronisation, capturable into a CUDA graph):
// block_step2 copies the block's scalar images (hd, hf: host memory valid
// until the stream has consumed it) into the parity-par device images and
// forms Y = H X - S X Lambda (step 2) into the parity-par Y buffer;
// block_loop runs steps 3-5 from them.  Both parts of a block use the same
// parity; two blocks of different parity can be in flight at once.
// The scalar images read straight from mapped pinned host memory by a kernel:
// a copy-engine transfer of them would queue behind any large copy the caller
// runs on another stream, and every kernel of the block would wait for it.
__global__ void k_stage_scalars(const double *__restrict__ hd, double *__restrict__ dd, int64_t nd,
                                const float *__restrict__ hf, float *__restrict__ df, int64_t nf) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nd + nf; i += (int64_t)gridDim.x * blockDim.x) {
    if (i < nd)
      dd[i] = hd[i];
    else
      df[i - nd] = hf[i - nd];
  }
}

static void block_step2(paw_context *c, const double *X, int ldx, int nb, const ChebScalars &S, const double *hd,
                        const float *hf, int par, cudaStream_t s, const double *hd_dev, const float *hf_dev) {
  c->ws_lamp[par].ensure(sizeof(double) * S.nd, &c->dev_bytes);
  c->ws_cfp[par].ensure(sizeof(float) * S.nf, &c->dev_bytes);
  if (hd_dev && hf_dev) {
    const int64_t n = (int64_t)(S.nd + S.nf);
    const int grid = (int)std::min<int64_t>(64, (n + 255) / 256);
    k_stage_scalars<<<grid, 256, 0, s>>>(hd_dev, c->ws_lamp[par].as<double>(), (int64_t)S.nd, hf_dev,
                                         c->ws_cfp[par].as<float>(), (int64_t)S.nf);
    PAW_LAUNCH_CHECK("k_stage_scalars");
  } else {
    PAW_CUDA(cudaMemcpyAsync(c->ws_lamp[par].ptr, hd, sizeof(double) * S.nd, cudaMemcpyHostToDevice, s));
    PAW_CUDA(cudaMemcpyAsync(c->ws_cfp[par].ptr, hf, sizeof(float) * S.nf, cudaMemcpyHostToDevice, s));
  }
  c->ws_Y0p[par].ensure(sizeof(double) * c->ndof * nb, &c->dev_bytes);
  // step 2: Y = H X - S X Lambda (FP64; phases 0 and 4)
  residual_block(c, X, ldx, c->ws_lamp[par].as<double>(), c->ws_Y0p[par].as<double>(), nb, nb, s);
}

template <typename TR>
static void block_loop(paw_context *c, paw_precision prec, const double *X, int ldx, int nb, double a0, double cc,
                       const ChebScalars &S, int par, double *Xo, int ldo, cudaStream_t s) {
  const int64_t M = c->ndof;
  const int nsteps = S.nsteps;
  const double *d_neglam = c->ws_lamp[par].as<double>();
  const double *d_lyfin = d_neglam + nb, *d_cf = d_neglam + 2 * nb;
  const size_t ncf = (size_t)nsteps * nb;
  const float *d_chi = c->ws_cfp[par].as<float>(), *d_clo = d_chi + ncf;

  const int ldr = nb;
  constexpr bool f32 = sizeof(TR) == 4;
  c->ws_RX.ensure(sizeof(TR) * M * nb, &c->dev_bytes);
  c->ws_RY.ensure(sizeof(TR) * M * nb, &c->dev_bytes);
  c->ws_T.ensure(sizeof(TR) * M * nb, &c->dev_bytes);
  const bool lo = f32 && !c->opts.y0_fp32;
  if (f32) c->ws_Y0f.ensure(sizeof(float) * M * nb, &c->dev_bytes);
  if (lo) c->ws_Y0lo.ensure(sizeof(float) * M * nb, &c->dev_bytes);
  const double *Y0 = c->ws_Y0p[par].as<double>();
  float *Yhi = f32 ? c->ws_Y0f.as<float>() : nullptr;
  float *Ylo = lo ? c->ws_Y0lo.as<float>() : nullptr;
  TR *RX = c->ws_RX.as<TR>(), *RY = c->ws_RY.as<TR>(), *T = c->ws_T.as<TR>();
  const size_t wbytes = sizeof(TR) * (size_t)std::max(1, c->natoms * c->npad) * nb;
  c->ws_W.ensure(wbytes, &c->dev_bytes);
  c->scr->W2.ensure(sizeof(double) * (size_t)std::max(1, c->natoms * c->npad) * nb, &c->dev_bytes);
  TR *WS = c->ws_W.as<TR>(), *WH = c->scr->W2.as<TR>();
  // step 3
  const dim3 blk(32, 8);
  {
    PhaseScope ps(c, 1, s);
    const double sc = 1.0 / (a0 - cc);
    const float sc_hi = (float)sc, sc_lo = (float)(sc - (double)sc_hi);
    if constexpr (sizeof(TR) == 4) {
      if (nb % 4 == 0 && ldr % 4 == 0 && M * (nb / 4) < (int64_t(1) << 31)) {
        int dev = 0, nsm = 0;
        PAW_CUDA(cudaGetDevice(&dev));
        PAW_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        const int64_t quads = M * (nb / 4);
        const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((quads + 255) / 256, (int64_t)nsm * 16));
        k_cheb_init4<<<g, 256, 0, s>>>(M, nb, Y0, nb, sc_hi, sc_lo, RY, RX, ldr, Yhi, Ylo);
        PAW_LAUNCH_CHECK("k_cheb_init4");
      } else {
        k_cheb_init<TR><<<ew_grid(M, nb), blk, 0, s>>>(M, nb, Y0, nb, sc, sc_hi, sc_lo, RY, RX, ldr, Yhi, Ylo);
        PAW_LAUNCH_CHECK("k_cheb_init");
      }
    } else {
      k_cheb_init<TR><<<ew_grid(M, nb), blk, 0, s>>>(M, nb, Y0, nb, sc, sc_hi, sc_lo, RY, RX, ldr, Yhi, Ylo);
      PAW_LAUNCH_CHECK("k_cheb_init");
    }
  }
  const TR *mdinv = mdinv_of<TR>(c);
  // step 4: R_X <- alpha H Shat^-1 R_Y - beta R_Y - gamma R_X + alpha Y Lambda_Y
  for (int k = 0; k < nsteps; ++k) {
    const double alpha = S.al[k];
    const size_t ko = (size_t)k * nb;
    if (c->nown_pairs > 0) {
      // one projection gives the coefficients of Shat^-1 (W_S) and of the nonlocal H (W_H)
      {
        PhaseScope ps(c, 2, s);
        nl_project_filter<TR>(c, prec, RY, ldr, nb, mdinv, alpha, WS, WH, s);
      }
      // T = Shat^-1 R_Y and the recurrence update with the nonlocal part of alpha H T
      PhaseScope ps(c, 1, s);
      if constexpr (f32)
        nl_recurrence_f32(c, prec, WS, WH, nb, RY, RX, T, ldr, mdinv, Yhi, Ylo, ldr, d_chi + ko, d_clo + ko, S.be[k],
                          S.ga[k], s);
      else
        nl_recurrence_f64(c, WS, WH, nb, RY, RX, T, ldr, mdinv, Y0, nb, d_cf + ko, S.be[k], S.ga[k], s);
    } else {
      PhaseScope ps(c, 1, s);
      k_cheb_base<TR><<<ew_grid(M, nb), blk, 0, s>>>(M, nb, RY, RX, T, ldr, f32 ? (const void *)Yhi : (const void *)Y0,
                                                     Ylo, nb, d_cf + ko, d_chi + ko, d_clo + ko, (TR)S.be[k],
                                                     (TR)S.ga[k], mdinv);
      PAW_LAUNCH_CHECK("k_cheb_base");
    }
    // R_X += alpha H_loc T (cell products with extraction and assembly)
    {
      PhaseScope ps(c, 3, s);
      local_H<TR>(c, prec, T, ldr, RX, ldr, nb, alpha, s);
    }
    std::swap(RX, RY);
  }
  // step 5: Psi_f = Shat^-1 R_Y + X Lambda_Y
  {
    PhaseScope ps(c, 5, s);
    op_Sinv<TR>(c, prec, RY, ldr, T, ldr, nb, s);
    k_cheb_recover<TR><<<ew_grid(M, nb), blk, 0, s>>>(M, nb, T, ldr, X, ldx, d_lyfin, Xo, ldo);
    PAW_LAUNCH_CHECK("k_cheb_recover");
  }
}

void cheb_issue(paw_context *c, paw_precision prec, const double *X, int ldx, int nb, paw_bounds bd,
                const ChebScalars &S, const double *hd, const float *hf, double *Xo, int ldo, cudaStream_t s,
                const double *hd_dev, const float *hf_dev) {
  const double cc = (bd.bU + bd.bW) / 2.0;
  block_step2(c, X, ldx, nb, S, hd, hf, 0, s, hd_dev, hf_dev);
  if (prec == PAW_FP64)
    block_loop<double>(c, prec, X, ldx, nb, bd.a0, cc, S, 0, Xo, ldo, s);
  else
    block_loop<float>(c, prec, X, ldx, nb, bd.a0, cc, S, 0, Xo, ldo, s);
}

// Next slot of the handle's pinned ring, large enough for `bytes`.  Waits only
// for the GPU to pass the copies of the slot's previous use.
static HostSlot &acquire_slot(paw_context *c, size_t bytes) {
  HostRing &R = c->scal_ring;
  if (R.slots.empty()) R.slots.resize(8);
  HostSlot &sl = R.slots[R.next];
  R.next = (R.next + 1) % R.slots.size();
  if (sl.pending) {
    PAW_CUDA(cudaEventSynchronize(sl.done));
    sl.pending = false;
  }
  if (!sl.done) PAW_CUDA(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming));
  if (sl.bytes < bytes) {
    if (sl.host) cudaFreeHost(sl.host);
    sl.host = nullptr;
    sl.dev = nullptr;
    sl.bytes = 0;
    PAW_CUDA(cudaHostAlloc(&sl.host, bytes, cudaHostAllocMapped));
    sl.bytes = bytes;
    PAW_CUDA(cudaHostGetDevicePointer(&sl.dev, sl.host, 0));
  }
  return sl;
}

static void release_ring(paw_context *c) {
  for (HostSlot &sl : c->scal_ring.slots) {
    if (sl.host) cudaFreeHost(sl.host);
    if (sl.done) cudaEventDestroy(sl.done);
  }
  c->scal_ring.slots.clear();
}

// One block, stream-ordered: the scalar images go to a pinned slot of the
// handle's ring (valid until the GPU has read them), then copies and kernels
// are enqueued; the host does not wait for the stream.  A bounded wait that
// expires in a tensor-core kernel is reported by paw_sync_status or by the
// next call that synchronises.
static void cheb_block(paw_context *c, paw_precision prec, const double *X, int ldx, const double *lam, int nb,
                       int m, paw_bounds bd, double *Xo, int ldo, cudaStream_t s) {
  ChebScalars S;
  const size_t nd = cheb_nd(nb, m), nf = cheb_nf(nb, m);
  HostSlot &sl = acquire_slot(c, sizeof(double) * nd + sizeof(float) * nf);
  double *hd = static_cast<double *>(sl.host);
  float *hf = reinterpret_cast<float *>(hd + nd);
  cheb_plan(nb, m, bd, lam, S, hd, hf);
  const double *hd_dev = static_cast<const double *>(sl.dev);
  try {
    cheb_issue(c, prec, X, ldx, nb, bd, S, hd, hf, Xo, ldo, s, hd_dev, reinterpret_cast<const float *>(hd_dev + nd));
  } catch (...) {
    // copies from the slot may already be enqueued: keep it until the stream passes them
    if (cudaEventRecord(sl.done, s) == cudaSuccess) sl.pending = true;
    throw;
  }
  PAW_CUDA(cudaEventRecord(sl.done, s));
  sl.pending = true;
}

// ============================================================== overlapped blocks
// Step 2 (FP64, bound by the FP64 pipe) of block j + 1 runs on a low-priority
// side stream while the loop of block j (bound by copy bandwidth and the
// tensor cores) runs on a high-priority stream: the blocks are independent
// (Sec. 4.4 filters blocks independently), so this reorders nothing but the
// schedule.  While a step 2 shares the SMs, the loop's persistent
// cell-product and projection kernels take their half-shared-memory form and
// the FP64 local kernel its 4-vector form, so that one CTA of each fits on
// an SM; the high priority hands freed SM slots to the persistent kernels
// first.  Blocks of parity j & 1 use the parity's Y buffer and scalar
// images; the side stream reuses them for block j + 2 only after the loop of
// block j has finished.
static cudaEvent_t next_event(paw_context *c) {
  if (c->ev_used == c->ev_pool.size()) {
    cudaEvent_t e;
    PAW_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    c->ev_pool.push_back(e);
  }
  return c->ev_pool[c->ev_used++];
}

static void ensure_streams(paw_context *c) {
  if (c->s_loop) return;
  int least = 0, greatest = 0;
  PAW_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
  PAW_CUDA(cudaStreamCreateWithPriority(&c->s_loop, cudaStreamNonBlocking, greatest));
  PAW_CUDA(cudaStreamCreateWithPriority(&c->s_side, cudaStreamNonBlocking, least));
}

// work issued while this is alive uses the side scratch set and the lean FP64 kernel
struct SideIssue {
  paw_context *c;
  SideIssue(paw_context *ctx, bool lean) : c(ctx) {
    c->scr = &c->scr_side;
    c->sf_lean = lean ? 1 : 0;
  }
  ~SideIssue() {
    c->scr = &c->scr_main;
    c->sf_lean = 0;
  }
};

struct LeanLoop {
  paw_context *c;
  LeanLoop(paw_context *ctx, bool lean) : c(ctx) { c->lean = lean ? 1 : 0; }
  ~LeanLoop() { c->lean = 0; }
};

static void cheb_filter_overlapped(paw_context *c, paw_precision prec, const double *X, int ldx, const double *lam,
                                   int ncols, int m, paw_bounds bd, double *Xo, int ldo, cudaStream_t s) {
  ensure_streams(c);
  c->ev_used = 0;
  const int B = c->opts.block, nbk = (ncols + B - 1) / B;
  const double cc = (bd.bU + bd.bW) / 2.0;
  cudaEvent_t ev0 = next_event(c);
  PAW_CUDA(cudaEventRecord(ev0, s));   // the caller's earlier work on s (X, for one) is done
  PAW_CUDA(cudaStreamWaitEvent(c->s_loop, ev0, 0));
  PAW_CUDA(cudaStreamWaitEvent(c->s_side, ev0, 0));
  std::vector<ChebScalars> S(nbk);
  std::vector<cudaEvent_t> evY(nbk), evFree(nbk);
  // At k != 0 a block of nb complex columns is filtered as the split real block
  // [Re | Im] of 2 nb columns (every eigenvalue estimate applying to both halves):
  // split on the side stream before step 2, merged on the loop stream after it.
  const int cw = c->kc ? 2 : 1;
  if (c->kc)
    for (int p = 0; p < std::min(nbk, 2); ++p) {
      c->ws_cxp[p].ensure(sizeof(double) * (size_t)c->ndof * 2 * B, &c->dev_bytes);
      c->ws_cyp[p].ensure(sizeof(double) * (size_t)c->ndof * 2 * B, &c->dev_bytes);
    }
  auto block_in = [&](int j) -> const double * {
    return c->kc ? c->ws_cxp[j & 1].as<double>() : X + (size_t)j * B;
  };
  auto issue_step2 = [&](int j) {
    const int j0 = j * B, nb = std::min(B, ncols - j0), nr = cw * nb;
    const size_t nd = cheb_nd(nr, m), nf = cheb_nf(nr, m);
    HostSlot &sl = acquire_slot(c, sizeof(double) * nd + sizeof(float) * nf);
    double *hd = static_cast<double *>(sl.host);
    float *hf = reinterpret_cast<float *>(hd + nd);
    if (c->kc) {
      std::vector<double> lam2(2 * (size_t)nb);
      for (int i = 0; i < nb; ++i) lam2[i] = lam2[nb + i] = lam[j0 + i];
      cheb_plan(nr, m, bd, lam2.data(), S[j], hd, hf);
    } else {
      cheb_plan(nr, m, bd, lam + j0, S[j], hd, hf);
    }
    if (j >= 2) PAW_CUDA(cudaStreamWaitEvent(c->s_side, evFree[j - 2], 0));   // parity buffers free again
    try {
      SideIssue side(c, j > 0);
      const double *hd_dev = static_cast<const double *>(sl.dev);
      if (c->kc) split_cplx<double>(c, X + 2 * (size_t)j0, ldx, nb, c->ws_cxp[j & 1].as<double>(), c->s_side);
      block_step2(c, block_in(j), c->kc ? nr : ldx, nr, S[j], hd, hf, j & 1, c->s_side, hd_dev,
                  reinterpret_cast<const float *>(hd_dev + nd));
    } catch (...) {
      if (cudaEventRecord(sl.done, c->s_side) == cudaSuccess) sl.pending = true;
      throw;
    }
    PAW_CUDA(cudaEventRecord(sl.done, c->s_side));
    sl.pending = true;
    evY[j] = next_event(c);
    PAW_CUDA(cudaEventRecord(evY[j], c->s_side));
  };
  issue_step2(0);
  for (int j = 0; j < nbk; ++j) {
    if (j + 1 < nbk) issue_step2(j + 1);
    const int j0 = j * B, nb = std::min(B, ncols - j0), nr = cw * nb;
    PAW_CUDA(cudaStreamWaitEvent(c->s_loop, evY[j], 0));
    {
      LeanLoop lean(c, j + 1 < nbk);   // a step 2 shares the SMs with this loop
      if (c->kc) {
        double *Y = c->ws_cyp[j & 1].as<double>();
        block_loop<float>(c, prec, block_in(j), nr, nr, bd.a0, cc, S[j], j & 1, Y, nr, c->s_loop);
        merge_cplx<double>(c, Y, nb, Xo + 2 * (size_t)j0, ldo, c->s_loop);
      } else {
        block_loop<float>(c, prec, X + j0, ldx, nb, bd.a0, cc, S[j], j & 1, Xo + j0, ldo, c->s_loop);
      }
    }
    evFree[j] = next_event(c);
    PAW_CUDA(cudaEventRecord(evFree[j], c->s_loop));
  }
  cudaEvent_t e1 = next_event(c), e2 = next_event(c);
  PAW_CUDA(cudaEventRecord(e1, c->s_loop));
  PAW_CUDA(cudaEventRecord(e2, c->s_side));
  PAW_CUDA(cudaStreamWaitEvent(s, e1, 0));   // later work on s follows every part of the call
  PAW_CUDA(cudaStreamWaitEvent(s, e2, 0));
}

// ============================================================== reductions
// partial[chunk][v] = sum_{rows in chunk} (A[i][v] + s_v B[i][v])^2 ; B may be null
__global__ void k_colnorm_partial(int64_t rows, int ncols, const double *__restrict__ A, int lda,
                                  const double *__restrict__ B, int ldb, const double *__restrict__ sc,
                                  double *__restrict__ partial, int nchunk) {
  __shared__ double red[8][33];
  const int v = blockIdx.y * 32 + threadIdx.x;
  const int64_t per = (rows + nchunk - 1) / nchunk;
  const int64_t r0 = blockIdx.x * per, r1 = min(rows, r0 + per);
  double acc = 0.0;
  if (v < ncols)
    for (int64_t i = r0 + threadIdx.y; i < r1; i += 8) {
      double a = A[i * lda + v];
      if (B) a += sc[v] * B[i * ldb + v];
      acc += a * a;
    }
  red[threadIdx.y][threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.y == 0 && v < ncols) {
    double s = 0.0;
    for (int g = 0; g < 8; ++g) s += red[g][threadIdx.x];
    partial[(size_t)blockIdx.x * ncols + v] = s;
  }
}

// partial[block] = sum over a slice of rows of sum_v A[i][v] * B[i][v]  (FP64 accumulation)
template <typename T>
__global__ void k_dot_total(int64_t rows, int ncols, const T *__restrict__ A, int lda, const T *__restrict__ B,
                            int ldb, double *__restrict__ partial) {
  __shared__ double red[256];
  const int64_t per = (rows + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = blockIdx.x * per, r1 = min(rows, r0 + per);
  double acc = 0.0;
  for (int64_t idx = threadIdx.x; idx < (r1 - r0) * ncols; idx += blockDim.x) {
    const int64_t i = r0 + idx / ncols;
    const int v = (int)(idx % ncols);
    acc += (double)A[i * lda + v] * (double)B[i * ldb + v];
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// dot products sum_i A[i][v] * B[i][v] per column, partial sums
__global__ void k_coldot_partial(int64_t rows, int ncols, const double *__restrict__ A, int lda,
                                 const double *__restrict__ B, int ldb, double *__restrict__ partial,
                                 int nchunk) {
  __shared__ double red[8][33];
  const int v = blockIdx.y * 32 + threadIdx.x;
  const int64_t per = (rows + nchunk - 1) / nchunk;
  const int64_t r0 = blockIdx.x * per, r1 = min(rows, r0 + per);
  double acc = 0.0;
  if (v < ncols)
    for (int64_t i = r0 + threadIdx.y; i < r1; i += 8) acc += A[i * lda + v] * B[i * ldb + v];
  red[threadIdx.y][threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.y == 0 && v < ncols) {
    double s = 0.0;
    for (int g = 0; g < 8; ++g) s += red[g][threadIdx.x];
    partial[(size_t)blockIdx.x * ncols + v] = s;
  }
}

__global__ void k_sum_partials(int nchunk, int ncols, const double *__restrict__ partial,
                               double *__restrict__ out) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= ncols) return;
  double s = 0.0;
  for (int k = 0; k < nchunk; ++k) s += partial[(size_t)k * ncols + v];
  out[v] = s;
}

static std::vector<double> column_reduce(paw_context *c, bool dot, const double *A, int lda, const double *B,
                                         int ldb, const double *sc_dev, int ncols, cudaStream_t s) {
  const int nchunk = 304;
  c->ws_red.ensure(sizeof(double) * ((size_t)nchunk * ncols + ncols), &c->dev_bytes);
  double *part = c->ws_red.as<double>();
  double *out = part + (size_t)nchunk * ncols;
  dim3 g(nchunk, (ncols + 31) / 32), blk(32, 8);
  if (dot)
    k_coldot_partial<<<g, blk, 0, s>>>(c->ndof, ncols, A, lda, B, ldb, part, nchunk);
  else
    k_colnorm_partial<<<g, blk, 0, s>>>(c->ndof, ncols, A, lda, B, ldb, sc_dev, part, nchunk);
  PAW_LAUNCH_CHECK("k_col_partial");
  k_sum_partials<<<(ncols + 127) / 128, 128, 0, s>>>(nchunk, ncols, part, out);
  PAW_LAUNCH_CHECK("k_sum_partials");
  std::vector<double> h(ncols);
  PAW_CUDA(cudaMemcpyAsync(h.data(), out, sizeof(double) * ncols, cudaMemcpyDeviceToHost, s));
  PAW_CUDA(cudaStreamSynchronize(s));
  return h;
}

__global__ void k_axpby(int64_t n, double a, const double *__restrict__ x, double b,
                        const double *__restrict__ y, double g, const double *__restrict__ z,
                        double *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double r = a * x[i];
  if (y) r += b * y[i];
  if (z) r += g * z[i];
  out[i] = r;
}

__global__ void k_random_vec(int64_t n, uint64_t seed, double *__restrict__ v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(i + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  v[i] = (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
}

// ============================================================== gradient kernels
// dV[e][q] = wq[q] * sum_v f[v] (sum_I Nq[q][I] X[dof_e(I)][v])^2, one block per cell
// (wq NULL: 1, the values at the points; f NULL: 1)
template <typename T>
__global__ void __launch_bounds__(256) k_grad_V(int nc, int nq, const int *__restrict__ cell_dofs,
                                                const double *__restrict__ Nq, const double *__restrict__ wq,
                                                const T *__restrict__ X, int ldx, int ncols,
                                                const double *__restrict__ f, double *__restrict__ dV) {
  extern __shared__ double xs[];   // [nc][32]
  const int e = blockIdx.x;
  const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
  for (int q = threadIdx.x; q < nq; q += blockDim.x) dV[(size_t)e * nq + q] = 0.0;
  for (int v0 = 0; v0 < ncols; v0 += 32) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < nc * 32; idx += blockDim.x) {
      const int I = idx >> 5, v = idx & 31;
      xs[idx] = (v0 + v < ncols) ? (double)X[(size_t)cell_dofs[(size_t)e * nc + I] * ldx + v0 + v] : 0.0;
    }
    __syncthreads();
    const double fv = (f && v0 + lane < ncols) ? f[v0 + lane] : 1.0;
    for (int q = grp; q < nq; q += 8) {
      double u = 0.0;
      for (int I = 0; I < nc; ++I) u += Nq[(size_t)q * nc + I] * xs[I * 32 + lane];
      double s = fv * u * u;
      for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
      if (lane == 0) dV[(size_t)e * nq + q] += (wq ? wq[q] : 1.0) * s;
    }
  }
}

// dD[a][ext(al)][ext(be)] = sum_v f[v] U[a][al][v] U[a][be][v]  (ext: internal -> caller's
// projector index; f NULL: 1)
template <typename T>
__global__ void k_grad_D(int npj, int npad, const T *__restrict__ U, int ldu, int ncols, const int *__restrict__ ext,
                         const double *__restrict__ f, double *__restrict__ dD) {
  const int a = blockIdx.x;
  for (int o = threadIdx.x; o < npj * npj; o += blockDim.x) {
    const int al = o / npj, be = o % npj;
    double s = 0.0;
    for (int v = 0; v < ncols; ++v)
      s += (f ? f[v] : 1.0) * (double)U[((size_t)a * npad + al) * ldu + v] *
           (double)U[((size_t)a * npad + be) * ldu + v];
    dD[(size_t)a * npj * npj + (size_t)ext[al] * npj + ext[be]] = s;
  }
}

}  // namespace pawfe

using namespace pawfe;

// natoms x npj x npj blocks from the caller's projector order to the internal one
static std::vector<double> to_internal(const paw_context *c, const double *ext) {
  const int n = c->npj;
  std::vector<double> out((size_t)c->natoms * n * n);
  for (int a = 0; a < c->natoms; ++a)
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j)
        out[((size_t)a * n + i) * n + j] = ext[((size_t)a * n + c->proj_ext[i]) * n + c->proj_ext[j]];
  return out;
}


// ============================================================== C ABI
#define PAW_TRY_BEGIN try {
#define PAW_TRY_END                                                              \
  }                                                                              \
  catch (const ::pawfe::Error &err) {                                            \
    return fail(err.code, err.msg);                                              \
  }                                                                              \
  catch (const std::bad_alloc &) {                                               \
    return fail(PAW_ERR_NO_MEMORY, "host allocation failed");                    \
  }                                                                              \
  catch (const std::exception &ex) {                                             \
    return fail(PAW_ERR_CUDA, ex.what());                                        \
  }

static void check_sym(const double *A, int na, int n, const char *what) {
  for (int a = 0; a < na; ++a) {
    const double *M = A + (size_t)a * n * n;
    double mx = 0.0;
    for (int i = 0; i < n * n; ++i) mx = std::max(mx, std::fabs(M[i]));
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < i; ++j) {
        PAW_REQUIRE(std::isfinite(M[i * n + j]), PAW_ERR_NONFINITE, std::string(what) + " has NaN/Inf");
        PAW_REQUIRE(std::fabs(M[i * n + j] - M[j * n + i]) <= 1e-12 * std::max(mx, 1e-300), PAW_ERR_INVALID_ARG,
                    std::string(what) + " of atom " + std::to_string(a) + " is not symmetric");
      }
  }
}

// At k != 0: split the complex argument, apply the operator to the real block
// [Re | Im] of 2 ncols columns, merge the result back (0: H, 1: S, 2: Shat^-1).
template <typename T>
static void apply_cplx(paw_context *c, paw_precision prec, int which, const T *X, int ldx, T *Y, int ldy, int ncols,
                       cudaStream_t s) {
  const int n2 = 2 * ncols;
  c->ws_cx.ensure(sizeof(T) * (size_t)c->ndof * n2, &c->dev_bytes);
  c->ws_cy.ensure(sizeof(T) * (size_t)c->ndof * n2, &c->dev_bytes);
  T *xs = c->ws_cx.as<T>(), *ys = c->ws_cy.as<T>();
  split_cplx<T>(c, X, ldx, ncols, xs, s);
  if (which == 0)
    op_H<T>(c, prec, xs, n2, ys, n2, n2, s);
  else if (which == 1)
    op_S<T>(c, xs, n2, ys, n2, n2, s);
  else
    op_Sinv<T>(c, prec, xs, n2, ys, n2, n2, s);
  merge_cplx<T>(c, ys, ncols, Y, ldy, s);
}

static void apply_any(paw_context *c, paw_precision prec, int which, const void *X, int ldx, void *Y, int ldy,
                      int ncols, cudaStream_t s) {
  if (prec == PAW_F32X2) {
    PAW_REQUIRE(!c->kc, PAW_ERR_UNSUPPORTED, "PAW_F32X2 is implemented for real vectors (k = 0)");
    op_pair(c, which, (const double *)X, ldx, (double *)Y, ldy, ncols, s);
    return;
  }
  if (c->kc) {
    if (prec == PAW_FP64)
      apply_cplx<double>(c, prec, which, (const double *)X, ldx, (double *)Y, ldy, ncols, s);
    else
      apply_cplx<float>(c, prec, which, (const float *)X, ldx, (float *)Y, ldy, ncols, s);
    return;
  }
  if (prec == PAW_FP64) {
    if (which == 0)
      op_H<double>(c, prec, (const double *)X, ldx, (double *)Y, ldy, ncols, s);
    else if (which == 1)
      op_S<double>(c, (const double *)X, ldx, (double *)Y, ldy, ncols, s);
    else
      op_Sinv<double>(c, prec, (const double *)X, ldx, (double *)Y, ldy, ncols, s);
  } else {
    if (which == 0)
      op_H<float>(c, prec, (const float *)X, ldx, (float *)Y, ldy, ncols, s);
    else if (which == 1)
      op_S<float>(c, (const float *)X, ldx, (float *)Y, ldy, ncols, s);
    else
      op_Sinv<float>(c, prec, (const float *)X, ldx, (float *)Y, ldy, ncols, s);
  }
}

namespace pawfe {
void check_block_args(paw_context *c, const void *X, const void *Y, int ncols, int ldx, int ldy) {
  PAW_REQUIRE(c != nullptr, PAW_ERR_INVALID_ARG, "NULL handle");
  PAW_REQUIRE(ncols >= 0, PAW_ERR_INVALID_ARG, "ncols < 0");
  if (ncols == 0) return;
  PAW_REQUIRE(X && Y, PAW_ERR_INVALID_ARG, "NULL X or Y");
  PAW_REQUIRE(ldx >= ncols && ldy >= ncols, PAW_ERR_INVALID_ARG, "leading dimension smaller than ncols");
}

// Tensor-core precisions: wait for the stream and report a kernel that gave
// up on a bounded wait (its output is incomplete).
static void check_tc_status(paw_context *c, paw_precision prec) {
  if (prec != PAW_TF32 && prec != PAW_BF16) return;
  PAW_CUDA(cudaStreamSynchronize(c->last_stream));
  PAW_REQUIRE(read_status(c) == 0, PAW_ERR_TIMEOUT, "a tensor-core kernel gave up on a bounded wait");
}

// Calls that synchronise report a bounded wait that expired in an earlier,
// asynchronous call on the handle (paw_cheb_filter): its output is incomplete.
static void report_earlier_timeout(paw_context *c) {
  PAW_REQUIRE(read_status(c) == 0, PAW_ERR_TIMEOUT,
              "a tensor-core kernel of an earlier call on this handle gave up on a bounded wait");
}

void check_prec(paw_precision prec, bool pair_ok) {
  PAW_REQUIRE(pair_ok || prec != PAW_F32X2, PAW_ERR_UNSUPPORTED,
              "PAW_F32X2 applies to paw_apply_H and paw_apply_S (step 2 of the filter: options.y0_pair32)");
  PAW_REQUIRE(prec == PAW_FP64 || prec == PAW_FP32 || prec == PAW_TF32 || prec == PAW_BF16 || prec == PAW_F32X2,
              PAW_ERR_INVALID_ARG, "unknown precision");
}
}  // namespace pawfe

extern "C" {

const char *paw_last_error(void) { return g_last_error.c_str(); }
const char *paw_version(void) { return "pawfe-gb300 0.1 (sm_103a)"; }

paw_status paw_fe_create(const paw_mesh *mesh, int degree, const paw_atoms *atoms, const paw_projectors *proj,
                         const double *D_ij, const double *dS_ij, const paw_vloc *vloc, const paw_options *opts,
                         paw_handle *out) {
  PAW_TRY_BEGIN
  PAW_REQUIRE(out != nullptr && mesh != nullptr, PAW_ERR_INVALID_ARG, "mesh and out must not be NULL");
  *out = nullptr;
  PAW_REQUIRE(mesh->periodic[0] == 1 && mesh->periodic[1] == 1 && mesh->periodic[2] == 1, PAW_ERR_UNSUPPORTED,
              "only fully periodic boxes are supported");
  PAW_REQUIRE(mesh->L[0] == mesh->L[1] && mesh->L[1] == mesh->L[2] && mesh->n_cells[0] == mesh->n_cells[1] &&
                  mesh->n_cells[1] == mesh->n_cells[2],
              PAW_ERR_UNSUPPORTED, "only cubic boxes with equal cell counts are supported");
  PAW_REQUIRE(mesh->L[0] > 0 && mesh->n_cells[0] >= 1, PAW_ERR_INVALID_ARG, "box size and cell count must be positive");
  PAW_REQUIRE(degree >= 1 && degree <= 8, PAW_ERR_UNSUPPORTED, "degree must be in 1..8");
  const int natoms = atoms ? atoms->natoms : 0;
  PAW_REQUIRE(natoms >= 0, PAW_ERR_INVALID_ARG, "natoms < 0");
  PAW_REQUIRE(natoms == 0 || atoms->positions, PAW_ERR_INVALID_ARG, "positions NULL");
  int npj = 0;
  const int nsh = (natoms > 0 && proj) ? proj->nshells : 0;
  PAW_REQUIRE(nsh >= 0 && nsh <= 16, PAW_ERR_UNSUPPORTED, "at most 16 projector shells");
  for (int s = 0; s < nsh; ++s) {
    PAW_REQUIRE(proj->l[s] >= 0 && proj->l[s] <= 2, PAW_ERR_UNSUPPORTED, "projector l must be 0, 1 or 2");
    PAW_REQUIRE(proj->width[s] > 0, PAW_ERR_INVALID_ARG, "projector width must be positive");
    PAW_REQUIRE(proj->width[s] * std::sqrt(2.0 * std::log(1e8)) < 0.5 * mesh->L[0], PAW_ERR_UNSUPPORTED,
                "projector cutoff must be below half the box");
    npj += 2 * proj->l[s] + 1;
  }
  PAW_REQUIRE(npj <= 32, PAW_ERR_UNSUPPORTED, "more than 32 projectors per atom");
  if (natoms > 0 && npj > 0) {
    PAW_REQUIRE(D_ij && dS_ij, PAW_ERR_INVALID_ARG, "D_ij and dS_ij must be given when atoms have projectors");
    check_sym(D_ij, natoms, npj, "D_ij");
    check_sym(dS_ij, natoms, npj, "dS_ij");
  }
  if (vloc) {
    PAW_REQUIRE(vloc->ngauss >= 0, PAW_ERR_INVALID_ARG, "ngauss < 0");
    for (int g = 0; g < vloc->ngauss; ++g)
      PAW_REQUIRE(vloc->width[g] > 0, PAW_ERR_INVALID_ARG, "Gaussian width must be positive");
  }
  auto *c = new paw_context();
  try {
    c->n = mesh->n_cells[0];
    c->p = degree;
    c->np1 = degree + 1;
    c->nc = c->np1 * c->np1 * c->np1;
    c->nq1 = degree + 2;
    c->nq = c->nq1 * c->nq1 * c->nq1;
    c->N1 = c->n * degree;
    c->ndof = (int64_t)c->N1 * c->N1 * c->N1;
    c->ncells = c->n * c->n * c->n;
    c->L = mesh->L[0];
    c->h = c->L / c->n;
    c->detJ = std::pow(c->h / 2.0, 3);
    c->natoms = natoms;
    c->npj = npj;
    // Internal projector order: shells by decreasing width (stable).  The
    // cutoff radius grows with the width, so the projectors of an atom that
    // reach a cell form a prefix and the kernels skip the all-zero rest.
    {
      std::vector<int> order(nsh), ext_off(nsh + 1, 0);
      for (int s = 0; s < nsh; ++s) ext_off[s + 1] = ext_off[s] + 2 * proj->l[s] + 1;
      std::iota(order.begin(), order.end(), 0);
      std::stable_sort(order.begin(), order.end(),
                       [&](int x, int y) { return proj->width[x] > proj->width[y]; });
      for (int s : order) {
        c->shell_l.push_back(proj->l[s]);
        c->shell_w.push_back(proj->width[s]);
        for (int m = 0; m < 2 * proj->l[s] + 1; ++m) c->proj_ext.push_back(ext_off[s] + m);
      }
    }
    if (natoms > 0) c->pos.assign(atoms->positions, atoms->positions + 3 * natoms);
    if (natoms > 0 && npj > 0) {
      c->D = to_internal(c, D_ij);
      c->dS = to_internal(c, dS_ij);
    }
    if (vloc && vloc->ngauss > 0) {
      c->vg_c.assign(vloc->centers, vloc->centers + 3 * vloc->ngauss);
      c->vg_A.assign(vloc->depth, vloc->depth + vloc->ngauss);
      c->vg_w.assign(vloc->width, vloc->width + vloc->ngauss);
    }
    if (opts) c->opts = *opts;
    if (c->opts.block <= 0) c->opts.block = 256;
    for (int d = 0; d < 3; ++d) {
      PAW_REQUIRE(std::isfinite(c->opts.kpoint[d]), PAW_ERR_INVALID_ARG, "kpoint has NaN/Inf");
      c->kvec[d] = c->opts.kpoint[d];
    }
    c->kc = (c->kvec[0] != 0.0 || c->kvec[1] != 0.0 || c->kvec[2] != 0.0) ? 1 : 0;
    c->kmass = 0.5 * (c->kvec[0] * c->kvec[0] + c->kvec[1] * c->kvec[1] + c->kvec[2] * c->kvec[2]);
    PAW_REQUIRE(!c->kc || npj <= 16, PAW_ERR_UNSUPPORTED, "at most 16 projectors per atom with a Bloch wavevector");
    PAW_REQUIRE(!c->kc || !c->opts.y0_pair32, PAW_ERR_UNSUPPORTED,
                "pair-of-FP32 step 2 (y0_pair32) is implemented for real vectors (k = 0)");
    c->npjr = c->kc ? 2 * npj : npj;
    if (npj == 0) c->natoms = 0;   // atoms without projectors carry no nonlocal term
    c->status_dev.ensure(2 * sizeof(int), &c->dev_bytes);
    PAW_CUDA(cudaMemset(c->status_dev.ptr, 0, 2 * sizeof(int)));
    if (npj > 0) {
      c->proj_ext_dev.ensure(sizeof(int) * npj, &c->dev_bytes);
      PAW_CUDA(cudaMemcpy(c->proj_ext_dev.ptr, c->proj_ext.data(), sizeof(int) * npj, cudaMemcpyHostToDevice));
    }
    build_tables(c);
    build_operators(c, vloc);
    build_couplings(c);
    if (cusolverDnCreate(&c->cusolver) != CUSOLVER_STATUS_SUCCESS)
      throw Error{PAW_ERR_LIBRARY, "cusolverDnCreate failed"};
    PAW_CUDA(cudaDeviceSynchronize());
  } catch (...) {
    paw_destroy(c);
    throw;
  }
  *out = c;
  return PAW_OK;
  PAW_TRY_END
}

paw_status paw_destroy(paw_handle c) {
  if (!c) return PAW_OK;
  cudaDeviceSynchronize();
  DevBuf *bufs[] = {&c->cell_dofs, &c->md_inv64, &c->md_inv32, &c->He64, &c->He32, &c->Me64, &c->Me32,
                    &c->K64, &c->Nq64, &c->wq64, &c->Vq, &c->tc_tf32.He, &c->tc_tf32.Me, &c->tc_bf16.He,
                    &c->tc_bf16.Me, &c->ent_dof, &c->P64, &c->P32, &c->own_off, &c->own_atom, &c->ownP64,
                    &c->ownP32,
                    &c->DH64, &c->DS64, &c->DSinv64, &c->ws_W, &c->ws_RX,
                    &c->ws_RY, &c->ws_T, &c->ws_Y0f, &c->ws_colscale, &c->ws_red, &c->ws_vec,
                    &c->ws_HX, &c->ws_SX, &c->ws_Hp, &c->ws_Sp, &c->ws_eig, &c->ws_solver, &c->ws_info,
                    &c->ws_rot, &c->ws_gram, &c->ws_cg, &c->wV, &c->ws_Y0lo, &c->gnb_off, &c->gnb_atom, &c->Gfull, &c->Fsh32, &c->DSinv32,
                    &c->Gfull32, &c->apair_off, &c->apair, &c->nltc.projB, &c->nltc.projBs, &c->nltc.expB, &c->nltc.mdo, &c->nltc.odof, &c->status_dev, &c->proj_ext_dev, &c->own_ngrp,
                    &c->own_lg, &c->own_sidx, &c->own_cnt, &c->Bk64, &c->Bk32, &c->tc_bk_tf32.He,
                    &c->tc_bk_bf16.He, &c->ws_cx, &c->ws_cy,
                    &c->nltc.eoff, &c->ownPx2, &c->wVx2,
                    &c->scr_main.partial, &c->scr_main.pp, &c->scr_main.W2, &c->scr_main.Wx2,
                    &c->scr_side.partial, &c->scr_side.pp, &c->scr_side.W2, &c->scr_side.Wx2,
                    &c->ws_Y0p[0], &c->ws_Y0p[1], &c->ws_cxp[0], &c->ws_cxp[1], &c->ws_cyp[0], &c->ws_cyp[1], &c->ws_lamp[0], &c->ws_lamp[1], &c->ws_cfp[0], &c->ws_cfp[1]};
  for (DevBuf *b : bufs) b->release(&c->dev_bytes);
  for (cudaEvent_t e : c->prof.pool) cudaEventDestroy(e);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  if (c->s_loop) cudaStreamDestroy(c->s_loop);
  if (c->s_side) cudaStreamDestroy(c->s_side);
  release_ring(c);
  if (c->cusolver) cusolverDnDestroy(c->cusolver);
  delete c;
  return PAW_OK;
}

paw_status paw_get_info(paw_handle c, paw_info *out) {
  if (!c || !out) return fail(PAW_ERR_INVALID_ARG, "NULL handle or output");
  out->ndof = c->ndof;
  out->ncells = c->ncells;
  out->nodes_per_cell = c->nc;
  out->quad_per_cell = c->nq;
  out->natoms = c->natoms;
  out->nproj = c->npj;
  out->degree = c->p;
  out->support_pairs = c->npairs;
  out->device_bytes = c->dev_bytes;
  out->owner_pairs = c->nown_pairs;
  out->nproj_padded = c->npad;
  out->proj_nnz = c->proj_nnz;
  out->complex_vectors = c->kc;
  return PAW_OK;
}

paw_status paw_set_veff(paw_handle c, const double *V_q) {
  PAW_TRY_BEGIN
  PAW_REQUIRE(c && V_q, PAW_ERR_INVALID_ARG, "NULL handle or V_q");
  PAW_CUDA(cudaMemcpy(c->Vq.ptr, V_q, sizeof(double) * (size_t)c->ncells * c->nq, cudaMemcpyDeviceToDevice));
  rebuild_hamiltonian(c);
  return PAW_OK;
  PAW_TRY_END
}

paw_status paw_set_dij(paw_handle c, const double *D_ij) {
  PAW_TRY_BEGIN
  PAW_REQUIRE(c && D_ij, PAW_ERR_INVALID_ARG, "NULL handle or D_ij");
  if (c->natoms == 0) return PAW_OK;
  check_sym(D_ij, c->natoms, c->npj, "D_ij");
  c->D = to_internal(c, D_ij);
  PAW_CUDA(cudaDeviceSynchronize());
  PAW_CUDA(cudaMemcpy(c->DH64.ptr, c->D.data(), sizeof(double) * c->D.size(), cudaMemcpyHostToDevice));
  build_couple_f(c);   // the fused FP32 coupling carries D_H
  return PAW_OK;
  PAW_TRY_END
}


paw_status paw_apply_H(paw_handle c, paw_precision prec, const void *X, void *Y, int ncols, int ldx, int ldy,
                       void *stream) {
  PAW_TRY_BEGIN
  check_prec(prec, true);
  check_block_args(c, X, Y, ncols, ldx, ldy);
  if (ncols == 0) return PAW_OK;
  auto s = (cudaStream_t)stream;
  c->last_stream = s;
  apply_any(c, prec, 0, X, ldx, Y, ldy, ncols, s);
  check_tc_status(c, prec);
  return PAW_OK;
  PAW_TRY_END
}

paw_status paw_apply_S(paw_handle c, paw_precision prec, const void *X, void *Y, int ncols, int ldx, int ldy,
                       void *stream) {
  PAW_TRY_BEGIN
  check_prec(prec, true);
  check_block_args(c, X, Y, ncols, ldx, ldy);
  if (ncols == 0) return PAW_OK;
  auto s = (cudaStream_t)stream;
  c->last_stream = s;
  apply_any(c, prec, 1, X, ldx, Y, ldy, ncols, s);
  return PAW_OK;
  PAW_TRY_END
}

paw_status paw_apply_Sinv_approx(paw_handle c, paw_precision prec, const void *X, void *Y, int ncols, int ldx,
                                 int ldy, void *stream) {
  PAW_TRY_BEGIN
  check_prec(prec);
  check_block_args(c, X, Y, ncols, ldx, ldy);
  if (ncols == 0) return PAW_OK;
  auto s = (cudaStream_t)stream;
  c->last_stream = s;
  apply_any(c, prec, 2, X, ldx, Y, ldy, ncols, s);
  check_tc_status(c, prec);
  return PAW_OK;
  PAW_TRY_END
}

paw_status paw_cheb_filter(paw_handle c, paw_precision prec, const double *X_in, int ldx, const double *lambda_in,
                           int ncols, int degree, paw_bounds b, double *X_out, int ldo, void *stream) {
  PAW_TRY_BEGIN
  check_prec(prec);
  check_block_args(c, X_in, X_out, ncols, ldx, ldo);
  PAW_REQUIRE(degree >= 1, PAW_ERR_INVALID_ARG, "degree must be >= 1");
  PAW_REQUIRE(std::isfinite(b.a0) && std::isfinite(b.bW) && std::isfinite(b.bU) && b.a0 < b.bW && b.bW < b.bU,
              PAW_ERR_INVALID_ARG, "bounds must satisfy a0 < bW < bU");
  if (ncols == 0) return PAW_OK;
  PAW_REQUIRE(lambda_in != nullptr, PAW_ERR_INVALID_ARG, "lambda_in NULL");
  PAW_REQUIRE(X_in != X_out, PAW_ERR_INVALID_ARG, "X_out must not alias X_in");
  for (int j = 0; j < ncols; ++j)
    PAW_REQUIRE(std::isfinite(lambda_in[j]), PAW_ERR_NONFINITE, "lambda_in has NaN/Inf");
  auto s = (cudaStream_t)stream;
  c->last_stream = s;
  const int B = c->opts.block;
  // reduced-precision filter over two or more blocks: step 2 of the next block
  // overlaps the loop of the current one
  if (prec != PAW_FP64 && ncols > B && c->opts.no_overlap == 0) {
    cheb_filter_overlapped(c, prec, X_in, ldx, lambda_in, ncols, degree, b, X_out, ldo, s);
    return PAW_OK;
  }
  for (int j0 = 0; j0 < ncols; j0 += B) {
    const int nb = std::min(B, ncols - j0);
    if (c->kc) {
      // complex block: Algorithm 2 on the split block [Re | Im] with every
      // eigenvalue estimate applying to both halves (the scalars stay real)
      c->ws_cx.ensure(sizeof(double) * (size_t)c->ndof * 2 * nb, &c->dev_bytes);
      c->ws_cy.ensure(sizeof(double) * (size_t)c->ndof * 2 * nb, &c->dev_bytes);
      std::vector<double> lam2(2 * (size_t)nb);
      for (int j = 0; j < nb; ++j) lam2[j] = lam2[nb + j] = lambda_in[j0 + j];
      split_cplx<double>(c, X_in + 2 * (size_t)j0, ldx, nb, c->ws_cx.as<double>(), s);
      cheb_block(c, prec, c->ws_cx.as<double>(), 2 * nb, lam2.data(), 2 * nb, degree, b, c->ws_cy.as<double>(),
                 2 * nb, s);
      merge_cplx<double>(c, c->ws_cy.as<double>(), nb, X_out + 2 * (size_t)j0, ldo, s);
      continue;
    }
    cheb_block(c, prec, X_in + j0, ldx, lambda_in + j0, nb, degree, b, X_out + j0, ldo, s);
  }
  return PAW_OK;
  PAW_TRY_END
}

// Rayleigh-Ritz at k != 0 (complex X, interleaved, ld complex entries).  The
// complex blocks are read as real blocks of 2N interleaved columns: the real
// Gram matrix of X with H X (S X) holds the four real products of
// H^p = X^H H X (S^p), zhegvd solves H^p Q = S^p Q Lambda, and X <- X Q is the
// real rotation of the interleaved rows by the 2N x 2N real form of Q.
static void rr_complex(paw_context *c, double *X, int ld, int N, double *lambda_out, cudaStream_t s) {
  const int64_t M = c->ndof;
  const int Bc = std::min(N, c->opts.block);
  c->ws_HX.ensure(sizeof(double) * 2 * (size_t)M * N, &c->dev_bytes);
  c->ws_SX.ensure(sizeof(double) * 2 * (size_t)M * N, &c->dev_bytes);
  c->ws_Hp.ensure(sizeof(double) * 2 * (size_t)N * N, &c->dev_bytes);
  c->ws_Sp.ensure(sizeof(double) * 2 * (size_t)N * N, &c->dev_bytes);
  c->ws_cg.ensure(sizeof(double) * 4 * (size_t)N * N, &c->dev_bytes);
  double *HX = c->ws_HX.as<double>(), *SX = c->ws_SX.as<double>(), *G = c->ws_cg.as<double>();
  for (int j0 = 0; j0 < N; j0 += Bc) {
    const int nb = std::min(Bc, N - j0);
    apply_cplx<double>(c, PAW_FP64, 0, X + 2 * (size_t)j0, ld, HX + 2 * (size_t)j0, N, nb, s);
    apply_cplx<double>(c, PAW_FP64, 1, X + 2 * (size_t)j0, ld, SX + 2 * (size_t)j0, N, nb, s);
  }
  cusolverDnSetStream(c->cusolver, s);
  rr_gram(c, X, 2 * ld, 2 * N, HX, 2 * N, 2 * N, M, false, G, 2 * N, s);
  rr_gram_to_hermitian(N, G, c->ws_Hp.ptr, s);
  rr_gram(c, X, 2 * ld, 2 * N, SX, 2 * N, 2 * N, M, false, G, 2 * N, s);
  rr_gram_to_hermitian(N, G, c->ws_Sp.ptr, s);
  auto *Am = reinterpret_cast<cuDoubleComplex *>(c->ws_Hp.ptr);
  auto *Bm = reinterpret_cast<cuDoubleComplex *>(c->ws_Sp.ptr);
  int lwork = 0;
  c->ws_eig.ensure(sizeof(double) * N, &c->dev_bytes);
  c->ws_info.ensure(sizeof(int), &c->dev_bytes);
  if (cusolverDnZhegvd_bufferSize(c->cusolver, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER,
                                  N, Am, N, Bm, N, c->ws_eig.as<double>(), &lwork) != CUSOLVER_STATUS_SUCCESS)
    throw Error{PAW_ERR_LIBRARY, "cusolverDnZhegvd_bufferSize failed"};
  c->ws_solver.ensure(sizeof(cuDoubleComplex) * std::max(1, lwork), &c->dev_bytes);
  if (cusolverDnZhegvd(c->cusolver, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, N, Am, N,
                       Bm, N, c->ws_eig.as<double>(), reinterpret_cast<cuDoubleComplex *>(c->ws_solver.ptr), lwork,
                       c->ws_info.as<int>()) != CUSOLVER_STATUS_SUCCESS)
    throw Error{PAW_ERR_LIBRARY, "cusolverDnZhegvd failed"};
  int info = 0;
  PAW_CUDA(cudaMemcpyAsync(&info, c->ws_info.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
  PAW_CUDA(cudaStreamSynchronize(s));
  PAW_REQUIRE(info <= N, PAW_ERR_NOT_SPD, "projected overlap S^p is not positive definite");
  PAW_REQUIRE(info == 0, PAW_ERR_LIBRARY, "zhegvd did not converge");
  rr_complex_to_real(N, c->ws_Hp.ptr, G, s);
  rr_rotate(c, X, 2 * ld, M, 2 * N, G, false, s);
  PAW_CUDA(cudaMemcpyAsync(lambda_out, c->ws_eig.ptr, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
  PAW_CUDA(cudaStreamSynchronize(s));
}

paw_status paw_rayleigh_ritz(paw_handle c, double *X, int ld, int N, double *lambda_out, void *stream) {
  PAW_TRY_BEGIN
  PAW_REQUIRE(c && X && lambda_out, PAW_ERR_INVALID_ARG, "NULL argument");
  PAW_REQUIRE(N >= 1 && ld >= N, PAW_ERR_INVALID_ARG, "need 1 <= N <= ld");
  PAW_REQUIRE(c->ndof < (1ll << 31), PAW_ERR_UNSUPPORTED, "ndof >= 2^31");
  auto s = (cudaStream_t)stream;
  c->last_stream = s;
  if (c->kc) {
    rr_complex(c, X, ld, N, lambda_out, s);
    report_earlier_timeout(c);
    return PAW_OK;
  }
  const int64_t M = c->ndof;
  const int Bc = std::min(N, c->opts.block);
  c->ws_HX.ensure(sizeof(double) * (size_t)M * Bc, &c->dev_bytes);
  c->ws_Hp.ensure(sizeof(double) * (size_t)N * N, &c->dev_bytes);
  c->ws_Sp.ensure(sizeof(double) * (size_t)N * N, &c->dev_bytes);
  double *HX = c->ws_HX.as<double>(), *Hp = c->ws_Hp.as<double>(), *Sp = c->ws_Sp.as<double>();
  cusolverDnSetStream(c->cusolver, s);
  // RR-Projection, lower triangle only (dsygvd reads the lower part): column
  // block j0..j0+nb of H^p and S^p gets rows j0..N-1
  for (int j0 = 0; j0 < N; j0 += Bc) {
    const int nb = std::min(Bc, N - j0), nr = N - j0;
    op_H<double>(c, PAW_FP64, X + j0, ld, HX, nb, nb, s);
    rr_gram(c, X + j0, ld, nr, HX, nb, nb, M, true, Hp + (size_t)j0 * N + j0, N, s);
    op_S<double>(c, X + j0, ld, HX, nb, nb, s);
    rr_gram(c, X + j0, ld, nr, HX, nb, nb, M, true, Sp + (size_t)j0 * N + j0, N, s);
  }
  int lwork = 0;
  c->ws_eig.ensure(sizeof(double) * N, &c->dev_bytes);
  c->ws_info.ensure(sizeof(int), &c->dev_bytes);
  if (cusolverDnDsygvd_bufferSize(c->cusolver, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER,
                                  N, Hp, N, Sp, N, c->ws_eig.as<double>(), &lwork) != CUSOLVER_STATUS_SUCCESS)
    throw Error{PAW_ERR_LIBRARY, "cusolverDnDsygvd_bufferSize failed"};
  c->ws_solver.ensure(sizeof(double) * std::max(1, lwork), &c->dev_bytes);
  if (cusolverDnDsygvd(c->cusolver, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, N, Hp, N,
                       Sp, N, c->ws_eig.as<double>(), c->ws_solver.as<double>(), lwork,
                       c->ws_info.as<int>()) != CUSOLVER_STATUS_SUCCESS)
    throw Error{PAW_ERR_LIBRARY, "cusolverDnDsygvd failed"};
  int info = 0;
  PAW_CUDA(cudaMemcpyAsync(&info, c->ws_info.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
  PAW_CUDA(cudaStreamSynchronize(s));
  PAW_REQUIRE(info <= N, PAW_ERR_NOT_SPD, "projected overlap S^p is not positive definite");
  PAW_REQUIRE(info == 0, PAW_ERR_LIBRARY, "dsygvd did not converge");
  // RR-SR: X <- X Q in FP64, or (rr_mixed) X diag(Q) in FP64 + fl32(X) fl32(Q - diag(Q)) in FP32
  rr_rotate(c, X, ld, M, N, Hp, c->opts.rr_mixed != 0, s);
  PAW_CUDA(cudaMemcpyAsync(lambda_out, c->ws_eig.ptr, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
  PAW_CUDA(cudaStreamSynchronize(s));
  report_earlier_timeout(c);
  return PAW_OK;
  PAW_TRY_END
}

paw_status paw_residuals(paw_handle c, const double *X, int ld, const double *lambda, int N, double *rnorm_out,
                         void *stream) {
  PAW_TRY_BEGIN
  PAW_REQUIRE(c && X && lambda && rnorm_out, PAW_ERR_INVALID_ARG, "NULL argument");
  PAW_REQUIRE(N >= 1 && ld >= N, PAW_ERR_INVALID_ARG, "need 1 <= N <= ld");
  auto s = (cudaStream_t)stream;
  c->last_stream = s;
  const int Bc = std::min(N, c->opts.block);
  if (c->kc) {
    // complex columns: ||r||^2 = ||Re r||^2 + ||Im r||^2 from the split block
    c->ws_cx.ensure(sizeof(double) * (size_t)c->ndof * 2 * Bc, &c->dev_bytes);
    c->ws_HX.ensure(sizeof(double) * (size_t)c->ndof * 2 * Bc, &c->dev_bytes);
    c->ws_SX.ensure(sizeof(double) * (size_t)c->ndof * 2 * Bc, &c->dev_bytes);
    c->ws_colscale.ensure(sizeof(double) * 2 * Bc, &c->dev_bytes);
    for (int j0 = 0; j0 < N; j0 += Bc) {
      const int nb = std::min(Bc, N - j0);
      std::vector<double> nl(2 * (size_t)nb);
      for (int j = 0; j < nb; ++j) nl[j] = nl[nb + j] = -lambda[j0 + j];
      PAW_CUDA(cudaMemcpyAsync(c->ws_colscale.ptr, nl.data(), sizeof(double) * 2 * nb, cudaMemcpyHostToDevice, s));
      split_cplx<double>(c, X + 2 * (size_t)j0, ld, nb, c->ws_cx.as<double>(), s);
      op_H<double>(c, PAW_FP64, c->ws_cx.as<double>(), 2 * nb, c->ws_HX.as<double>(), 2 * nb, 2 * nb, s);
      op_S<double>(c, c->ws_cx.as<double>(), 2 * nb, c->ws_SX.as<double>(), 2 * nb, 2 * nb, s);
      std::vector<double> r = column_reduce(c, false, c->ws_HX.as<double>(), 2 * nb, c->ws_SX.as<double>(), 2 * nb,
                                            c->ws_colscale.as<double>(), 2 * nb, s);
      for (int j = 0; j < nb; ++j) rnorm_out[j0 + j] = std::sqrt(r[j] + r[nb + j]);
    }
    report_earlier_timeout(c);
    return PAW_OK;
  }
  c->ws_HX.ensure(sizeof(double) * (size_t)c->ndof * Bc, &c->dev_bytes);
  c->ws_SX.ensure(sizeof(double) * (size_t)c->ndof * Bc, &c->dev_bytes);
  c->ws_colscale.ensure(sizeof(double) * Bc, &c->dev_bytes);
  for (int j0 = 0; j0 < N; j0 += Bc) {
    const int nb = std::min(Bc, N - j0);
    std::vector<double> nl(nb);
    for (int j = 0; j < nb; ++j) nl[j] = -lambda[j0 + j];
    PAW_CUDA(cudaMemcpyAsync(c->ws_colscale.ptr, nl.data(), sizeof(double) * nb, cudaMemcpyHostToDevice, s));
    op_H<double>(c, PAW_FP64, X + j0, ld, c->ws_HX.as<double>(), nb, nb, s);
    op_S<double>(c, X + j0, ld, c->ws_SX.as<double>(), nb, nb, s);
    std::vector<double> r = column_reduce(c, false, c->ws_HX.as<double>(), nb, c->ws_SX.as<double>(), nb,
                                          c->ws_colscale.as<double>(), nb, s);
    for (int j = 0; j < nb; ++j) rnorm_out[j0 + j] = std::sqrt(r[j]);
  }
  report_earlier_timeout(c);
  return PAW_OK;
  PAW_TRY_END
}

paw_status paw_lanczos_bounds(paw_handle c, int k, uint64_t seed, double *theta_min, double *upper, void *stream) {
  PAW_TRY_BEGIN
  PAW_REQUIRE(c && theta_min && upper, PAW_ERR_INVALID_ARG, "NULL argument");
  PAW_REQUIRE(k >= 2 && k <= 200, PAW_ERR_INVALID_ARG, "k must be in 2..200");
  auto s = (cudaStream_t)stream;
  c->last_stream = s;
  // at k != 0 a vector is the split pair [Re v | Im v] (two columns): the process
  // runs on the real symmetric form of the Hermitian pencil, whose inner product
  // Re <v, S w> is the sum over both columns
  const int nw = c->kc ? 2 : 1;
  const int64_t M = c->ndof * nw;
  c->ws_vec.ensure(sizeof(double) * M * 5, &c->dev_bytes);
  double *v = c->ws_vec.as<double>(), *vp = v + M, *w = v + 2 * M, *Hv = v + 3 * M, *Sw = v + 4 * M;
  const unsigned g = (unsigned)((M + 255) / 256);
  auto dot = [&](const double *A, const double *B) {
    const std::vector<double> r = column_reduce(c, true, A, nw, B, nw, nullptr, nw, s);
    return nw == 2 ? r[0] + r[1] : r[0];
  };
  k_random_vec<<<g, 256, 0, s>>>(M, seed, v);
  PAW_LAUNCH_CHECK("k_random_vec");
  op_S<double>(c, v, nw, Sw, nw, nw, s);
  double nrm = std::sqrt(dot(v, Sw));
  k_axpby<<<g, 256, 0, s>>>(M, 1.0 / nrm, v, 0.0, nullptr, 0.0, nullptr, v);
  PAW_CUDA(cudaMemsetAsync(vp, 0, sizeof(double) * M, s));
  std::vector<double> al, be;
  double beta = 0.0;
  for (int j = 0; j < k; ++j) {
    op_H<double>(c, PAW_FP64, v, nw, Hv, nw, nw, s);
    op_Sinv<double>(c, PAW_FP64, Hv, nw, w, nw, nw, s);
    op_S<double>(c, w, nw, Sw, nw, nw, s);
    const double a = dot(v, Sw);
    k_axpby<<<g, 256, 0, s>>>(M, 1.0, w, -a, v, -beta, vp, w);
    op_S<double>(c, w, nw, Sw, nw, nw, s);
    beta = std::sqrt(std::max(dot(w, Sw), 0.0));
    al.push_back(a);
    be.push_back(beta);
    PAW_CUDA(cudaMemcpyAsync(vp, v, sizeof(double) * M, cudaMemcpyDeviceToDevice, s));
    if (beta == 0.0) break;
    k_axpby<<<g, 256, 0, s>>>(M, 1.0 / beta, w, 0.0, nullptr, 0.0, nullptr, v);
  }
  const int n = (int)al.size();
  std::vector<double> T((size_t)n * n, 0.0), ev, V;
  for (int i = 0; i < n; ++i) {
    T[(size_t)i * n + i] = al[i];
    if (i + 1 < n) T[(size_t)i * n + i + 1] = T[(size_t)(i + 1) * n + i] = be[i];
  }
  jacobi_eigh(n, T, ev, V);
  *theta_min = ev[0];
  *upper = ev[n - 1] + std::fabs(be[n - 1] * V[(size_t)(n - 1) * n + (n - 1)]);
  return PAW_OK;
  PAW_TRY_END
}

paw_status paw_energy(paw_handle c, paw_precision prec, const void *X, int ld, int N, double *E_out,
                      void *stream) {
  PAW_TRY_BEGIN
  PAW_REQUIRE(c == nullptr || !c->kc, PAW_ERR_UNSUPPORTED, "paw_energy has no Bloch-wavevector form");
  check_prec(prec);
  PAW_REQUIRE(c && X && E_out, PAW_ERR_INVALID_ARG, "NULL argument");
  PAW_REQUIRE(N >= 1 && ld >= N, PAW_ERR_INVALID_ARG, "need 1 <= N <= ld");
  auto s = (cudaStream_t)stream;
  c->last_stream = s;
  const size_t es = prec == PAW_FP64 ? sizeof(double) : sizeof(float);
  c->ws_HX.ensure(es * (size_t)c->ndof * N, &c->dev_bytes);
  const int nchunk = 304;
  c->ws_red.ensure(sizeof(double) * (nchunk + 1), &c->dev_bytes);
  double *part = c->ws_red.as<double>();
  if (prec == PAW_FP64) {
    op_H<double>(c, prec, (const double *)X, ld, c->ws_HX.as<double>(), N, N, s);
    k_dot_total<double><<<nchunk, 256, 0, s>>>(c->ndof, N, (const double *)X, ld, c->ws_HX.as<double>(), N, part);
  } else {
    op_H<float>(c, prec, (const float *)X, ld, c->ws_HX.as<float>(), N, N, s);
    k_dot_total<float><<<nchunk, 256, 0, s>>>(c->ndof, N, (const float *)X, ld, c->ws_HX.as<float>(), N, part);
  }
  PAW_LAUNCH_CHECK("k_dot_total");
  k_sum_partials<<<1, 32, 0, s>>>(nchunk, 1, part, part + nchunk);
  PAW_LAUNCH_CHECK("k_sum_partials");
  PAW_CUDA(cudaMemcpyAsync(E_out, part + nchunk, sizeof(double), cudaMemcpyDeviceToHost, s));
  PAW_CUDA(cudaStreamSynchronize(s));
  return PAW_OK;
  PAW_TRY_END
}

// outV[e][q] = wq[q] sum_v f[v] u_v(x_q)^2 and outD[a] = sum_v f[v] U_v U_v^T (wq, f optional)
static void density_like(paw_context *c, paw_precision prec, const void *X, int ld, int N, const double *wq,
                         const double *f, double *outV, double *outD, cudaStream_t s) {
  const size_t shm = sizeof(double) * c->nc * 32;
  if (prec == PAW_FP64) {
    PAW_CUDA(cudaFuncSetAttribute(k_grad_V<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    k_grad_V<double><<<c->ncells, 256, shm, s>>>(c->nc, c->nq, c->cell_dofs.as<int>(), c->Nq64.as<double>(), wq,
                                                  (const double *)X, ld, N, f, outV);
  } else {
    PAW_CUDA(cudaFuncSetAttribute(k_grad_V<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    k_grad_V<float><<<c->ncells, 256, shm, s>>>(c->nc, c->nq, c->cell_dofs.as<int>(), c->Nq64.as<double>(), wq,
                                                 (const float *)X, ld, N, f, outV);
  }
  PAW_LAUNCH_CHECK("k_grad_V");
  if (c->nown_pairs > 0 && outD) {
    if (prec == PAW_FP64) {
      c->scr->W2.ensure(sizeof(double) * (size_t)c->natoms * c->npad * N, &c->dev_bytes);
      nl_project<double>(c, PAW_FP64, (const double *)X, ld, N, nullptr, nullptr, 1.0, c->scr->W2.as<double>(), s);
      k_grad_D<double><<<c->natoms, 256, 0, s>>>(c->npj, c->npad, c->scr->W2.as<double>(), N, N,
                                                 c->proj_ext_dev.as<int>(), f, outD);
    } else {
      c->scr->W2.ensure(sizeof(float) * (size_t)c->natoms * c->npad * N, &c->dev_bytes);
      // projector coefficients stay in FP32 arithmetic
      nl_project<float>(c, PAW_FP32, (const float *)X, ld, N, nullptr, nullptr, 1.0, c->scr->W2.as<float>(), s);
      k_grad_D<float><<<c->natoms, 256, 0, s>>>(c->npj, c->npad, c->scr->W2.as<float>(), N, N,
                                                c->proj_ext_dev.as<int>(), f, outD);
    }
    PAW_LAUNCH_CHECK("k_grad_D");
  }
}

paw_status paw_energy_grad(paw_handle c, paw_precision prec, const void *X, int ld, int N, double *dE_dV,
                           double *dE_dD, void *stream) {
  PAW_TRY_BEGIN
  PAW_REQUIRE(c == nullptr || !c->kc, PAW_ERR_UNSUPPORTED, "paw_energy_grad has no Bloch-wavevector form");
  check_prec(prec);
  PAW_REQUIRE(c && X && dE_dV, PAW_ERR_INVALID_ARG, "NULL argument");
  PAW_REQUIRE(N >= 1 && ld >= N, PAW_ERR_INVALID_ARG, "need 1 <= N <= ld");
  auto s = (cudaStream_t)stream;
  c->last_stream = s;
  density_like(c, prec, X, ld, N, c->wq64.as<double>(), nullptr, dE_dV, dE_dD, s);
  return PAW_OK;
  PAW_TRY_END
}

paw_status paw_density(paw_handle c, paw_precision prec, const void *X, int ld, int N, const double *occ,
                       double *rho_q, double *D_a, void *stream) {
  PAW_TRY_BEGIN
  PAW_REQUIRE(c == nullptr || !c->kc, PAW_ERR_UNSUPPORTED, "paw_density has no Bloch-wavevector form");
  check_prec(prec);
  PAW_REQUIRE(c && X && rho_q, PAW_ERR_INVALID_ARG, "NULL argument");
  PAW_REQUIRE(N >= 1 && ld >= N, PAW_ERR_INVALID_ARG, "need 1 <= N <= ld");
  auto s = (cudaStream_t)stream;
  c->last_stream = s;
  const double *f = nullptr;
  if (occ) {
    for (int i = 0; i < N; ++i) PAW_REQUIRE(std::isfinite(occ[i]), PAW_ERR_NONFINITE, "occupation NaN/Inf");
    c->ws_colscale.ensure(sizeof(double) * N, &c->dev_bytes);
    PAW_CUDA(cudaMemcpyAsync(c->ws_colscale.ptr, occ, sizeof(double) * N, cudaMemcpyHostToDevice, s));
    f = c->ws_colscale.as<double>();
  }
  density_like(c, prec, X, ld, N, nullptr, f, rho_q, D_a, s);
  PAW_CUDA(cudaStreamSynchronize(s));   // the occupations are read from host memory by the copy
  return PAW_OK;
  PAW_TRY_END
}

paw_status paw_profile_enable(paw_handle c, int enable) {
  PAW_TRY_BEGIN
  PAW_REQUIRE(c != nullptr, PAW_ERR_INVALID_ARG, "NULL handle");
  PAW_CUDA(cudaDeviceSynchronize());
  c->prof.on = enable != 0;
  c->prof.marks.clear();
  c->prof.used = 0;
  for (int i = 0; i < PAW_NPHASES; ++i) c->prof.launches[i] = 0;
  c->prof.launch0 = g_launch_count;
  return PAW_OK;
  PAW_TRY_END
}

paw_status paw_profile_read(paw_handle c, paw_profile *out) {
  PAW_TRY_BEGIN
  PAW_REQUIRE(c && out, PAW_ERR_INVALID_ARG, "NULL argument");
  PAW_CUDA(cudaDeviceSynchronize());
  std::memset(out, 0, sizeof(*out));
  for (const auto &m : c->prof.marks) {
    float ms = 0.f;
    PAW_CUDA(cudaEventElapsedTime(&ms, m.a, m.b));
    out->ms[m.phase] += ms;
    out->intervals[m.phase] += 1;
  }
  for (int i = 0; i < PAW_NPHASES; ++i) out->launches[i] = c->prof.launches[i];
  out->total_launches = g_launch_count - c->prof.launch0;
  return PAW_OK;
  PAW_TRY_END
}

paw_status paw_set_wait_limit(paw_handle c, double seconds, int probe) {
  PAW_TRY_BEGIN
  PAW_REQUIRE(c != nullptr, PAW_ERR_INVALID_ARG, "NULL handle");
  PAW_REQUIRE(std::isfinite(seconds) && seconds >= 1e-3 && seconds <= 60.0, PAW_ERR_INVALID_ARG,
              "wait limit must be between 1 ms and 60 s");
  c->wait_ns = (uint64_t)(seconds * 1e9);
  c->wait_probe = probe ? 1 : 0;
  return PAW_OK;
  PAW_TRY_END
}

paw_status paw_sync_status(paw_handle c) {
  PAW_TRY_BEGIN
  PAW_REQUIRE(c != nullptr, PAW_ERR_INVALID_ARG, "NULL handle");
  PAW_CUDA(cudaStreamSynchronize(c->last_stream));
  PAW_CUDA(cudaGetLastError());
  PAW_REQUIRE(read_status(c) == 0, PAW_ERR_TIMEOUT, "a tensor-core kernel gave up on a bounded wait");
  return PAW_OK;
  PAW_TRY_END
}

}  // extern "C"
