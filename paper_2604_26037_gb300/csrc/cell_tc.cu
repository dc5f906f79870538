// Cell products on the 5th-generation tensor cores (tcgen05) of sm_103a.
//
//   Y[dof_e(n)][v] += alpha * sum_k H^e[n][k] T[dof_e(k)][v]       (Sec. 4.3 steps i, iii, iv)
//
// One CTA computes D[v][n] = sum_k T_e[k][v] H^e[n][k] for one cell e, one tile
// of output nodes n (MMA N) and 128 vectors v (MMA M):
//   A operand  T_e^T  (M = 128 vectors x K nodes): gathered from the global
//              DoF-major block by all threads (one vector row per thread,
//              coalesced across the warp), written transposed into a K-major
//              128-byte-swizzled shared-memory tile.
//   B operand  H^e    (N nodes x K nodes, K-major): pre-arranged once in global
//              memory in exactly the swizzled shared-memory image, copied with
//              one cp.async.bulk per K-chunk (mbarrier transaction count).
//   D          FP32 accumulators in tensor memory (128 lanes x N columns).
// K advances in 128-byte chunks (32 TF32 or 64 BF16 nodes), double-buffered.
// The epilogue reads TMEM with tcgen05.ld (lane = vector) and scatter-adds each
// output node row with coalesced FP32 reductions: node rows of the DoF-major
// block are contiguous in the vector index.
//
// Every mbarrier wait is bounded (2 s of %globaltimer); on expiry the CTA
// records a status word, skips its epilogue, frees its tensor memory and exits.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "tc_ptx.cuh"
#include "tc_stream.cuh"

namespace pawfe {

namespace {

constexpr int MT = 128;            // vectors per CTA = MMA M
constexpr int THREADS = 256;           // two gather threads per A row
constexpr int STAGES = 2;
constexpr uint32_t A_BYTES = MT * 128;
constexpr uint32_t TMEM_COLS = 256;
using namespace tcp;

struct TcArgs {
  const uint8_t *Ht;       // tiled cell matrices
  size_t cell_bytes;       // bytes of one cell in Ht (0: shared matrix)
  int nc, ntile, ntiles, kchunks, vtiles;
  const int *cell_dofs;
  const float *X;
  int ldx;
  float *Y;
  int ldy, ncols;
  float alpha;
  int *status;             // set to 1 when a bounded wait expires
};

template <bool BF16>
__global__ void __launch_bounds__(THREADS, 1) k_cell_tc(TcArgs a) {
  constexpr int EPR = BF16 ? 64 : 32;   // K elements per 128-byte row
  constexpr int GPT = EPR / 2;           // elements gathered per thread and K-chunk (half a row)
  constexpr int EPC = EPR / 8;           // elements per 16-byte chunk
  extern __shared__ uint8_t smem_raw[];
  uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t B_BYTES = (uint32_t)a.ntile * 128u;
  const uint32_t STAGE_BYTES = A_BYTES + B_BYTES;
  uint64_t *bars = reinterpret_cast<uint64_t *>(base + STAGES * STAGE_BYTES);   // full[2], done[2], acc
  uint32_t *taddr_smem = reinterpret_cast<uint32_t *>(bars + 5);
  int *dofs = reinterpret_cast<int *>(taddr_smem + 4);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int bid = blockIdx.x;
  const int vt = bid % a.vtiles;
  const int t = (bid / a.vtiles) % a.ntiles;
  const int e = bid / (a.vtiles * a.ntiles);
  const int kpad = a.kchunks * EPR;

  for (int i = tid; i < kpad; i += THREADS) dofs[i] = (i < a.nc) ? a.cell_dofs[(size_t)e * a.nc + i] : -1;
  const uint32_t full0 = smem_u32(&bars[0]), done0 = smem_u32(&bars[2]), accb = smem_u32(&bars[4]);
  if (tid == 0) {
    mbar_init(full0, THREADS + 1);
    mbar_init(full0 + 8, THREADS + 1);
    mbar_init(done0, 1);
    mbar_init(done0 + 8, 1);
    mbar_init(accb, 1);
    fence_barrier_init();
    fence_proxy_async();
  }
  if (warp == 0) {
    __syncwarp();
    tmem_alloc(smem_u32(taddr_smem), TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *taddr_smem;

  // gather role: row r of the A tile (vector v), half `hf` of its 128 bytes
  const int r = tid & (MT - 1), hf = tid >> 7;
  const int v = vt * MT + r;
  const bool vok = v < a.ncols;
  const uint8_t *Hsrc = a.Ht + (size_t)e * a.cell_bytes + (size_t)t * a.kchunks * B_BYTES;
  const uint32_t idesc = make_idesc(BF16, MT, a.ntile);
  bool ok = true;

  float cur[GPT], nxt[GPT];
  auto load_chunk = [&](int kc, float(&f)[GPT]) {
    const int k0 = kc * EPR + hf * GPT;
#pragma unroll
    for (int u = 0; u < GPT; ++u) {
      const int d = dofs[k0 + u];
      f[u] = (vok && d >= 0) ? __ldg(a.X + (size_t)d * a.ldx + v) : 0.f;
    }
  };
  load_chunk(0, nxt);

  for (int kc = 0; kc < a.kchunks; ++kc) {
    const int s = kc & 1;
    const uint32_t use = (uint32_t)(kc >> 1);
    uint8_t *sA = base + s * STAGE_BYTES;
    uint8_t *sB = sA + A_BYTES;
    const uint32_t full = full0 + 8u * s, done = done0 + 8u * s;
#pragma unroll
    for (int u = 0; u < GPT; ++u) cur[u] = nxt[u];
    if (kc + 1 < a.kchunks) load_chunk(kc + 1, nxt);   // in flight while this chunk is stored and multiplied
    if (kc >= STAGES && !mbar_wait(done, (use - 1) & 1u)) {
      ok = false;
      break;
    }
    if (tid == 0) {
      mbar_arrive_tx(full, B_BYTES);
      bulk_g2s(smem_u32(sB), Hsrc + (size_t)kc * B_BYTES, B_BYTES, full);
    }
    uint8_t *row = sA + r * 128;
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      const int c = hf * 4 + cc;
      uint4 q;
      if constexpr (BF16) {
        __nv_bfloat162 p0 = __floats2bfloat162_rn(cur[cc * EPC + 0], cur[cc * EPC + 1]);
        __nv_bfloat162 p1 = __floats2bfloat162_rn(cur[cc * EPC + 2], cur[cc * EPC + 3]);
        __nv_bfloat162 p2 = __floats2bfloat162_rn(cur[cc * EPC + 4], cur[cc * EPC + 5]);
        __nv_bfloat162 p3 = __floats2bfloat162_rn(cur[cc * EPC + 6], cur[cc * EPC + 7]);
        q.x = *reinterpret_cast<uint32_t *>(&p0);
        q.y = *reinterpret_cast<uint32_t *>(&p1);
        q.z = *reinterpret_cast<uint32_t *>(&p2);
        q.w = *reinterpret_cast<uint32_t *>(&p3);
      } else {
        q = make_uint4(__float_as_uint(cur[cc * 4 + 0]), __float_as_uint(cur[cc * 4 + 1]),
                       __float_as_uint(cur[cc * 4 + 2]), __float_as_uint(cur[cc * 4 + 3]));
      }
      *reinterpret_cast<uint4 *>(row + ((c ^ (r & 7)) << 4)) = q;
    }
    fence_proxy_async();
    mbar_arrive(full);
    if (tid == 0) {
      if (!mbar_wait(full, use & 1u)) {
        mbar_wait(full, use & 1u);   // second bounded wait: let the bulk copy in flight land
        ok = false;
        break;
      }
      tc_fence_after();
      const uint64_t ad = sw128_desc(smem_u32(sA));
      const uint64_t bd = sw128_desc(smem_u32(sB));
#pragma unroll
      for (int j = 0; j < 4; ++j)   // 4 MMAs of 32 bytes of K each
        mma<BF16>(tmem, ad + (uint64_t)(2 * j), bd + (uint64_t)(2 * j), idesc, (kc | j) != 0);
      mma_commit(done);
    }
  }
  if (tid == 0 && ok) mma_commit(accb);
  if (!mbar_wait(accb, 0)) ok = false;
  tc_fence_after();

  if (ok) {
    // warp w reads TMEM lane quarter (w & 3) = vectors 32 (w & 3) .. +31; the two warp
    // groups split the columns (output nodes) of the tile
    const int q = warp & 3, ch = warp >> 2;
    const int nch = (a.ntile + 31) / 32;
    const int per = (nch + 1) / 2;
    const int c_beg = ch * per * 32, c_end = min(a.ntile, (ch + 1) * per * 32);
    const int vout = vt * MT + q * 32 + lane;
    const bool wok = vout < a.ncols;
    const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16);
    for (int c0 = c_beg; c0 < c_end; c0 += 32) {
      uint32_t rr[32];
      tmem_ld32(tl + (uint32_t)c0, rr);
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int nl = c0 + j;
        const int n = t * a.ntile + nl;
        if (wok && nl < c_end && n < a.nc)
          atomicAdd(&a.Y[(size_t)dofs[n] * a.ldy + vout], a.alpha * __uint_as_float(rr[j]));
      }
    }
  } else if (lane == 0) {
    atomicExch(a.status, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

// H^e (FP32, row-major per cell) -> swizzled K-major tiles, TF32-rounded or BF16.
template <bool BF16>
__global__ void k_tile_mats(const float *__restrict__ He, long long stride, int ncells, int nc, int ntile,
                            int ntiles, int kchunks, uint8_t *__restrict__ out) {
  constexpr int EPR = BF16 ? 64 : 32;
  const int64_t total = (int64_t)ncells * ntiles * kchunks * ntile * 8;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int c = (int)(idx & 7);
  int64_t r1 = idx >> 3;
  const int r = (int)(r1 % ntile);
  r1 /= ntile;
  const int kc = (int)(r1 % kchunks);
  r1 /= kchunks;
  const int t = (int)(r1 % ntiles);
  const int e = (int)(r1 / ntiles);
  const int n = t * ntile + r;
  const float *H = He + (long long)e * stride;
  uint4 q;
  if constexpr (BF16) {
    float f[8];
    for (int u = 0; u < 8; ++u) {
      const int k = kc * EPR + 8 * c + u;
      f[u] = (n < nc && k < nc) ? H[(size_t)n * nc + k] : 0.f;
    }
    __nv_bfloat162 p0 = __floats2bfloat162_rn(f[0], f[1]);
    __nv_bfloat162 p1 = __floats2bfloat162_rn(f[2], f[3]);
    __nv_bfloat162 p2 = __floats2bfloat162_rn(f[4], f[5]);
    __nv_bfloat162 p3 = __floats2bfloat162_rn(f[6], f[7]);
    q.x = *reinterpret_cast<uint32_t *>(&p0);
    q.y = *reinterpret_cast<uint32_t *>(&p1);
    q.z = *reinterpret_cast<uint32_t *>(&p2);
    q.w = *reinterpret_cast<uint32_t *>(&p3);
  } else {
    uint32_t w[4];
    for (int u = 0; u < 4; ++u) {
      const int k = kc * EPR + 4 * c + u;
      const float f = (n < nc && k < nc) ? H[(size_t)n * nc + k] : 0.f;
      uint32_t o;
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(o) : "f"(f));
      w[u] = o;
    }
    q = make_uint4(w[0], w[1], w[2], w[3]);
  }
  const size_t chunk = (size_t)ntile * 128;
  uint8_t *dst = out + ((((size_t)e * ntiles + t) * kchunks + kc) * chunk) + (size_t)r * 128 + ((c ^ (r & 7)) << 4);
  *reinterpret_cast<uint4 *>(dst) = q;
}

// Persistent warp-specialised form (tc_stream.cuh) for 16-byte-aligned rows:
// tile = (cell, 128 vectors), one accumulation round per N tile of H^e.
// SMALL: N tiles of at most 176 rows (degree <= 6), which leaves room for one
// more pipeline stage.  LEAN: two stages (about half the shared memory), the
// form used while an FP64 step 2 shares the SMs (paw_cheb_filter).
template <bool BF, bool SMALL, bool LEAN = false>
struct CellStream {
  static constexpr int NW = 1, NEPI = 8;
  static constexpr int S = LEAN ? 2 : (BF ? 2 : 3) + (SMALL ? 1 : 0);
  static constexpr bool BF16 = BF;
  static constexpr uint32_t B_MAX = (SMALL ? 176u : 256u) * 128u;
  static constexpr int KR = BF ? 64 : 32;
  CUtensorMap tm[NW];   // rows of X (gathered with TMA)
  int ntiles, ncols, vtiles, nc, ntile, ntiles_n, kchunks, ldx, ldy;
  size_t cell_bytes;
  const uint8_t *Ht;
  const int *cell_dofs;
  const float *X;
  float *Y;
  float alpha;
  struct Tile {
    int e, vt;
  };
  __device__ Tile tile(int t) const {
    Tile T;
    T.e = t / vtiles;
    T.vt = t - T.e * vtiles;
    return T;
  }
  __device__ int vt(const Tile &T) const { return T.vt; }
  __device__ int nsub(const Tile &) const { return ntiles_n; }
  __device__ int nchunks(const Tile &, int) const { return kchunks; }
  __device__ int ncol(const Tile &, int) const { return ntile; }
  __device__ int xcol(const Tile &T) const { return T.vt * MT; }
  __device__ int row_id(const Tile &T, int, int kc, int j, int) const {
    const int k = kc * KR + j;
    return k < nc ? cell_dofs[(size_t)T.e * nc + k] : -1;
  }
  __device__ const uint8_t *bsrc(const Tile &T, int sub, int kc) const {
    return Ht + (size_t)T.e * cell_bytes + ((size_t)sub * kchunks + kc) * ntile * 128;
  }
  __device__ uint32_t dcol(int) const { return 0; }
  // Y[dof(n)][v] += alpha D[v][n]: coalesced FP32 reductions, one node row per warp instruction
  __device__ void epilogue(const Tile &T, int sub, uint32_t tl, int q, int part, int lane, bool) const {
    const int ng = ntile / 16, per = (ng + 1) / 2;
    const int g_beg = part * per, g_end = min(ng, (part + 1) * per);
    const int v = T.vt * MT + q * 32 + lane;
    const int *dofs = cell_dofs + (size_t)T.e * nc + (size_t)sub * ntile;
    const int nrem = nc - sub * ntile;   // nodes of this N tile that exist
    for (int gi = g_beg; gi < g_end; ++gi) {
      const int c0 = gi * 16;
      int dd[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) dd[j] = (c0 + j < nrem) ? dofs[c0 + j] : -1;
      uint32_t rr[16];
      tmem_ld16_nowait(tl + (uint32_t)c0, rr);
      tmem_ld_wait();
      if (v < ncols) {
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (dd[j] >= 0) atomicAdd(Y + (size_t)dd[j] * ldy + v, alpha * __uint_as_float(rr[j]));
      }
    }
  }
};

}  // namespace

static void tile_geometry(int nc, bool bf16, int &ntile, int &ntiles, int &kchunks) {
  const int epr = bf16 ? 64 : 32;
  ntiles = (nc + 255) / 256;
  const int per = (nc + ntiles - 1) / ntiles;
  ntile = ((per + 15) / 16) * 16;
  kchunks = (nc + epr - 1) / epr;
}

// Tiled tcgen05 image of nmat FP32 cell matrices (nc x nc, row-major, stride
// nc^2) into T (TF32-rounded or BF16), built once.
static void tc_prepare_mats(paw_context *c, paw_precision prec, TcMats &T, const float *src, int nmat,
                            cudaStream_t s) {
  if (T.valid) return;
  const bool bf16 = prec == PAW_BF16;
  tile_geometry(c->nc, bf16, T.ntile, T.ntiles, T.kchunks);
  T.chunk_bytes = (size_t)T.ntile * 128;
  T.cell_bytes = T.chunk_bytes * T.kchunks * T.ntiles;
  T.He.ensure(T.cell_bytes * nmat, &c->dev_bytes);
  const int64_t total = (int64_t)nmat * T.ntiles * T.kchunks * T.ntile * 8;
  const unsigned grid = (unsigned)((total + 255) / 256);
  if (bf16)
    k_tile_mats<true><<<grid, 256, 0, s>>>(src, (long long)c->nc * c->nc, nmat, c->nc, T.ntile, T.ntiles,
                                           T.kchunks, T.He.as<uint8_t>());
  else
    k_tile_mats<false><<<grid, 256, 0, s>>>(src, (long long)c->nc * c->nc, nmat, c->nc, T.ntile, T.ntiles,
                                            T.kchunks, T.He.as<uint8_t>());
  PAW_LAUNCH_CHECK("k_tile_mats");
  T.valid = 1;
}

void tc_prepare(paw_context *c, paw_precision prec, cudaStream_t s) {
  tc_prepare_mats(c, prec, prec == PAW_BF16 ? c->tc_bf16 : c->tc_tf32, c->He32.as<float>(), c->ncells, s);
}

size_t tc_smem_bytes(int ntile, int kchunks, bool bf16) {
  const int epr = bf16 ? 64 : 32;
  const size_t stage = A_BYTES + (size_t)ntile * 128;
  size_t b = 1024 + STAGES * stage + 5 * 8 + 16 + sizeof(int) * (size_t)kchunks * epr;
  // at most two CTAs per SM so that their tensor-memory allocations (2 x 256 columns) always fit
  return b < 80 * 1024 ? 80 * 1024 : b;
}

template <bool BF, bool SMALL, bool LEAN>
static void cell_stream(paw_context *c, const TcMats &T, const float *X, int ldx, float *Y, int ldy, int ncols,
                        float alpha, cudaStream_t s) {
  CellStream<BF, SMALL, LEAN> p;
  p.vtiles = (ncols + MT - 1) / MT;
  const int64_t nt = (int64_t)c->ncells * p.vtiles;
  PAW_REQUIRE(nt < (1ll << 31), PAW_ERR_UNSUPPORTED, "too many cell tiles");
  p.ntiles = (int)nt;
  p.ncols = ncols;
  p.nc = c->nc;
  p.ntile = T.ntile;
  p.ntiles_n = T.ntiles;
  p.kchunks = T.kchunks;
  p.ldx = ldx;
  p.ldy = ldy;
  p.cell_bytes = T.cell_bytes;
  p.Ht = T.He.as<uint8_t>();
  p.cell_dofs = c->cell_dofs.as<int>();
  p.X = X;
  p.Y = Y;
  p.alpha = alpha;
  encode_row_map(&p.tm[0], X, c->ndof, ncols, ldx);
  using P = CellStream<BF, SMALL, LEAN>;
  const size_t shm = tcs::Geo<P>::SMEM;
  PAW_CUDA(cudaFuncSetAttribute(tcs::k_tc_stream<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  if (LEAN)   // the whole shared memory configured, so that an FP64 CTA fits beside this one
    PAW_CUDA(cudaFuncSetAttribute(tcs::k_tc_stream<P>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  cudaSharedmemCarveoutMaxShared));
  int dev = 0, nsm = 0;
  PAW_CUDA(cudaGetDevice(&dev));
  PAW_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int cap = c->grid_cap > 0 ? std::min(c->grid_cap, nsm) : nsm;
  const int grid = std::max(1, std::min(p.ntiles, cap));
  tcs::k_tc_stream<P><<<grid, tcs::threads_for(P::NEPI), shm, s>>>(p, c->status_dev.as<int>(), c->wait_ns,
                                                                     c->wait_probe);
  PAW_LAUNCH_CHECK("k_tc_stream<cell>");
}

// Y += alpha A_e X_e cell by cell with the tiled matrices of T (cell_bytes = 0:
// one matrix shared by every cell)
static void cell_apply_tc_mats(paw_context *c, paw_precision prec, const TcMats &T, size_t cell_bytes,
                               const float *X, int ldx, float *Y, int ldy, int ncols, float alpha, cudaStream_t s) {
  const bool bf16 = prec == PAW_BF16;
  TcMats Tm = T;
  Tm.cell_bytes = cell_bytes;
  // rows of X gathered with TMA: aligned base, pitch and vector range
  if (c->tc_variant == 0 && reinterpret_cast<uintptr_t>(X) % 16 == 0 && ldx % 4 == 0 && ncols % 4 == 0 &&
      Tm.ntile <= 256) {
    const bool small = Tm.ntile <= 176;
    if (c->lean) {   // an FP64 step 2 shares the SMs: half the shared memory
      if (bf16)
        small ? cell_stream<true, true, true>(c, Tm, X, ldx, Y, ldy, ncols, alpha, s)
              : cell_stream<true, false, true>(c, Tm, X, ldx, Y, ldy, ncols, alpha, s);
      else
        small ? cell_stream<false, true, true>(c, Tm, X, ldx, Y, ldy, ncols, alpha, s)
              : cell_stream<false, false, true>(c, Tm, X, ldx, Y, ldy, ncols, alpha, s);
      return;
    }
    if (bf16) {
      if (small)
        cell_stream<true, true, false>(c, Tm, X, ldx, Y, ldy, ncols, alpha, s);
      else
        cell_stream<true, false, false>(c, Tm, X, ldx, Y, ldy, ncols, alpha, s);
    } else {
      if (small)
        cell_stream<false, true, false>(c, Tm, X, ldx, Y, ldy, ncols, alpha, s);
      else
        cell_stream<false, false, false>(c, Tm, X, ldx, Y, ldy, ncols, alpha, s);
    }
    return;
  }
  TcArgs a;
  a.Ht = Tm.He.as<uint8_t>();
  a.cell_bytes = cell_bytes;
  a.nc = c->nc;
  a.ntile = Tm.ntile;
  a.ntiles = Tm.ntiles;
  a.kchunks = Tm.kchunks;
  a.vtiles = (ncols + MT - 1) / MT;
  a.cell_dofs = c->cell_dofs.as<int>();
  a.X = X;
  a.ldx = ldx;
  a.Y = Y;
  a.ldy = ldy;
  a.ncols = ncols;
  a.alpha = alpha;
  a.status = c->status_dev.as<int>();
  const size_t shm = tc_smem_bytes(Tm.ntile, Tm.kchunks, bf16);
  const int64_t blocks = (int64_t)c->ncells * Tm.ntiles * a.vtiles;
  PAW_REQUIRE(blocks < (1ll << 31), PAW_ERR_UNSUPPORTED, "too many cell tiles");
  if (bf16) {
    PAW_CUDA(cudaFuncSetAttribute(k_cell_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    k_cell_tc<true><<<(unsigned)blocks, THREADS, shm, s>>>(a);
  } else {
    PAW_CUDA(cudaFuncSetAttribute(k_cell_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    k_cell_tc<false><<<(unsigned)blocks, THREADS, shm, s>>>(a);
  }
  PAW_LAUNCH_CHECK("k_cell_tc");
}

void cell_apply_tc(paw_context *c, paw_precision prec, const float *X, int ldx, float *Y, int ldy, int ncols,
                   float alpha, cudaStream_t s) {
  if (ncols <= 0) return;
  tc_prepare(c, prec, s);
  const TcMats &T = prec == PAW_BF16 ? c->tc_bf16 : c->tc_tf32;
  cell_apply_tc_mats(c, prec, T, T.cell_bytes, X, ldx, Y, ldy, ncols, alpha, s);
}

void bloch_apply_tc(paw_context *c, paw_precision prec, const float *X, int ldx, float *Y, int ldy, int ncols,
                    float alpha, cudaStream_t s) {
  if (ncols <= 0 || !c->kc) return;
  TcMats &T = prec == PAW_BF16 ? c->tc_bk_bf16 : c->tc_bk_tf32;
  tc_prepare_mats(c, prec, T, c->Bk32.as<float>(), 1, s);
  cell_apply_tc_mats(c, prec, T, 0, X, ldx, Y, ldy, ncols, alpha, s);
}

}  // namespace pawfe
