// Nonlocal PAW terms on the 5th-generation tensor cores (tcgen05, TF32
// operands, FP32 accumulation in tensor memory), owner-cell formulation of
// Eq. FE nonlocal contribution and Eqs. Sinvapprox / Delta Sinv.
//
// Projection, one CTA per (cell e, 128 vectors), for each N tile of up to
// 256 / npad (cell, atom) pairs k of the cell:
//   D[v][k al] = sum_o (s(o) X[o][v]) P[k][o][al]        (o: the p^3 owned nodes)
//   A  owned rows of X scaled by s = M_D^-1 (or 1), gathered by all threads
//      (coalesced over vectors) into a K-major 128-byte-swizzled tile, K = nodes;
//   B  the pairs' projector values, pre-arranged in global memory as the
//      swizzled N x K image and copied with one cp.async.bulk per K-chunk.
// The accumulators leave TMEM as per-pair partials [k][al][v] (plain coalesced
// stores); the fixed-order per-atom sum of the SIMT path follows.
//
// Expansion, one CTA per (cell e, tile of owned nodes, 128 vectors):
//   D1[v][o] = sum_{k, al} W1[a_k][al][v] P[k][o][al]      (D2 likewise with W2)
//   A  the W rows of the cell's atoms (K = pair x projector, 32 per chunk),
//   B  projector values as node rows (N) x (pair, projector) (K).
// The epilogue reads D1, D2 (lane = vector) and applies the output stage of
// the SIMT kernel to every owned node row, coalesced over the vectors.
//
// Every mbarrier wait is bounded (2 s); on expiry the CTA records a status
// word, skips its epilogue, drains its MMAs, frees its tensor memory and exits.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "nonlocal_common.cuh"
#include "tc_ptx.cuh"
#include "tc_stream.cuh"

namespace pawfe {

namespace {

using namespace tcp;

constexpr int MT = 128;                  // vectors per CTA = MMA M
constexpr int THREADS = 256;             // two gather threads per A row
constexpr uint32_t A_BYTES = MT * 128;   // one K-chunk of A (128 rows x 32 TF32)
constexpr uint32_t TMEM_COLS = 256;
constexpr int OWN_MAX_TC = 512;          // p <= 8
constexpr int PAIR_MAX = PAIRS_PER_CELL_MAX;   // pairs of one cell (checked at set-up)
constexpr uint32_t PROJ_STAGE = A_BYTES + 256u * 128u;

__host__ __device__ constexpr uint32_t exp_stage_bytes(int nw) { return (uint32_t)nw * A_BYTES + 128u * 128u; }

__device__ __forceinline__ uint8_t *align1024(uint8_t *p) {
  return reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

// 16 values -> the 16-byte chunks 4 hf .. 4 hf + 3 of row r of a swizzled tile, TF32-rounded
__device__ __forceinline__ void store_row_half(uint8_t *tile, int r, int hf, const float (&f)[16]) {
#pragma unroll
  for (int cc = 0; cc < 4; ++cc) {
    const uint4 q = make_uint4(to_tf32(f[cc * 4 + 0]), to_tf32(f[cc * 4 + 1]), to_tf32(f[cc * 4 + 2]),
                               to_tf32(f[cc * 4 + 3]));
    *reinterpret_cast<uint4 *>(tile + sw128_off(r, hf * 4 + cc)) = q;
  }
}

__device__ __forceinline__ void init_barriers(uint32_t full0, uint32_t done0, uint32_t accb) {
  mbar_init(full0, THREADS + 1);
  mbar_init(full0 + 8, THREADS + 1);
  mbar_init(done0, 1);
  mbar_init(done0 + 8, 1);
  mbar_init(accb, 1);
  fence_barrier_init();
  fence_proxy_async();
}

// ------------------------------------------------------------------ projection
struct ProjTcArgs {
  int n, p, N1, own, npad, kc_own, ppt, vtiles, ncols, ldx;
  const int *own_off;
  const uint8_t *B;
  const float *X;
  const float *rowscale;
  float *PP;
  int *status;   // set to 1 when a bounded wait expires
};

__global__ void __launch_bounds__(THREADS, 2) k_nl_project_tc(ProjTcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *base = align1024(smem_raw);
  uint64_t *bars = reinterpret_cast<uint64_t *>(base + 2 * PROJ_STAGE);   // full[2], done[2], acc
  uint32_t *taddr_smem = reinterpret_cast<uint32_t *>(bars + 5);
  int *ooff = reinterpret_cast<int *>(taddr_smem + 4);   // [OWN_MAX_TC]
  float *rs = reinterpret_cast<float *>(ooff + OWN_MAX_TC);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int vt = blockIdx.x % a.vtiles;
  const int e = blockIdx.x / a.vtiles;   // vector tiles of one cell are adjacent: B reused from L2
  const int k0 = a.own_off[e], k1 = a.own_off[e + 1];
  // uniform over the CTA, before any barrier or TMEM use: no pairs, or an
  // earlier CTA gave up on a bounded wait (the launch is reported as failed)
  if (k0 == k1 || *reinterpret_cast<volatile int *>(a.status) != 0) return;
  const int64_t cb = owned_base(e, a.n, a.p, a.N1);
  for (int o = tid; o < a.own; o += THREADS) {
    const int off = owned_offset(o, a.p, a.N1);
    ooff[o] = off;
    rs[o] = a.rowscale ? a.rowscale[cb + off] : 1.f;
  }
  const uint32_t full0 = smem_u32(&bars[0]), done0 = smem_u32(&bars[2]), accb = smem_u32(&bars[4]);
  if (tid == 0) init_barriers(full0, done0, accb);
  if (warp == 0) {
    __syncwarp();
    tmem_alloc(smem_u32(taddr_smem), TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *taddr_smem;

  // gather role: row r of the A tile (vector v), half hf of each 128-byte row
  const int r = tid & (MT - 1), hf = tid >> 7;
  const int v = vt * MT + r;
  const bool vok = v < a.ncols;
  const int KC = a.kc_own;
  const int np = k1 - k0, ntl = (np + a.ppt - 1) / a.ppt;
  bool ok = true;
  float cur[16], nxt[16];
  auto load_chunk = [&](int kc, float(&f)[16]) {
    const int o0 = kc * 32 + hf * 16;
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int o = o0 + u;
      f[u] = (vok && o < a.own) ? __ldg(a.X + (cb + ooff[o]) * a.ldx + v) * rs[o] : 0.f;
    }
  };
  load_chunk(0, nxt);

  int g = 0;   // K-chunks issued so far: stage g & 1, its use number g >> 1
  for (int t = 0; t < ntl; ++t) {
    const int ncol = min(a.ppt, np - t * a.ppt) * a.npad;
    const uint32_t bbytes = (uint32_t)ncol * 128u;
    const uint8_t *Bt = a.B + (size_t)(k0 + t * a.ppt) * a.npad * 128 * KC;
    const uint32_t idesc = make_idesc(false, MT, ncol);
    for (int kc = 0; kc < KC; ++kc, ++g) {
      const int s = g & 1;
      const uint32_t use = (uint32_t)(g >> 1);
      uint8_t *sA = base + s * PROJ_STAGE;
      uint8_t *sB = sA + A_BYTES;
      const uint32_t full = full0 + 8u * s, done = done0 + 8u * s;
#pragma unroll
      for (int u = 0; u < 16; ++u) cur[u] = nxt[u];
      if (!(t == ntl - 1 && kc == KC - 1)) load_chunk(kc + 1 < KC ? kc + 1 : 0, nxt);   // A is the same for every tile
      if (!ok) continue;
      if (g >= 2 && !mbar_wait(done, (use - 1) & 1u)) {
        ok = false;
        continue;
      }
      if (tid == 0) {
        mbar_arrive_tx(full, bbytes);
        bulk_g2s(smem_u32(sB), Bt + (size_t)kc * bbytes, bbytes, full);
      }
      store_row_half(sA, r, hf, cur);
      fence_proxy_async();
      mbar_arrive(full);
      if (tid == 0) {
        if (!mbar_wait(full, use & 1u)) {
          mbar_wait(full, use & 1u);   // second bounded wait: let the bulk copy in flight land
          ok = false;
          continue;
        }
        tc_fence_after();
        const uint64_t ad = sw128_desc(smem_u32(sA)), bd = sw128_desc(smem_u32(sB));
#pragma unroll
        for (int j = 0; j < 4; ++j) mma<false>(tmem, ad + (uint64_t)(2 * j), bd + (uint64_t)(2 * j), idesc, (kc | j) != 0);
        mma_commit(done);
      }
    }
    if (tid == 0) mma_commit(accb);   // also after a failure: drains the MMAs in flight
    const bool got = mbar_wait(accb, (uint32_t)(t & 1)) && ok;
    ok = __syncthreads_and(got) != 0;
    tc_fence_after();
    if (ok) {
      // warp w reads TMEM lane quarter (w & 3); the two warp groups split the columns
      const int q = warp & 3, ch = warp >> 2;
      const int nch = (ncol + 31) / 32, per = (nch + 1) / 2;
      const int c_beg = ch * per * 32, c_end = min(ncol, (ch + 1) * per * 32);
      const int vout = vt * MT + q * 32 + lane;
      float *dst = a.PP + (size_t)(k0 + t * a.ppt) * a.npad * a.ncols + vout;
      for (int c0 = c_beg; c0 < c_end; c0 += 32) {
        uint32_t rr[32];
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, rr);
        if (vout < a.ncols) {
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (c0 + j < c_end) dst[(size_t)(c0 + j) * a.ncols] = __uint_as_float(rr[j]);
        }
      }
    }
    tc_fence_before();
    __syncthreads();   // every TMEM read of this tile precedes the next tile's MMAs
    tc_fence_after();
    if (!ok) break;
  }
  if (!ok && lane == 0) atomicExch(a.status, 1);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

// ------------------------------------------------------------------ expansion
struct ExpTcArgs {
  int npad, ppc, ntile, nh, vtiles, own;
  const uint8_t *B;
  const int *eoff;
  int *status;
};

template <int MODE>
__global__ void __launch_bounds__(THREADS, 2) k_nl_expand_tc(ExpArgs A, ExpTcArgs a, const float *__restrict__ W1,
                                                            const float *__restrict__ W2) {
  constexpr int NW = (MODE == EXP_RECURRENCE) ? 2 : 1;
  constexpr uint32_t STAGE = exp_stage_bytes(NW);
  extern __shared__ uint8_t smem_raw[];
  uint8_t *base = align1024(smem_raw);
  uint64_t *bars = reinterpret_cast<uint64_t *>(base + 2 * STAGE);
  uint32_t *taddr_smem = reinterpret_cast<uint32_t *>(bars + 5);
  int *ooff = reinterpret_cast<int *>(taddr_smem + 4);   // [128] owned offsets of this node tile
  int *patom = ooff + 128;                               // [PAIR_MAX] atoms of the cell's pairs

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int bid = blockIdx.x;
  const int vt = bid % a.vtiles;
  const int h = (bid / a.vtiles) % a.nh;
  const int e = bid / (a.vtiles * a.nh);
  const int k0 = A.own_off[e], k1 = A.own_off[e + 1];
  const int np = k1 - k0;
  if (MODE == EXP_ADD && np == 0) return;   // nothing to add (uniform, before any barrier)
  if (*reinterpret_cast<volatile int *>(a.status) != 0) return;   // an earlier CTA gave up
  const int KC = a.eoff[e + 1] - a.eoff[e];
  const int ncols = A.ncols;
  const int o_beg = h * a.ntile;
  const int64_t cb = owned_base(e, A.n, A.p, A.N1);
  for (int i = tid; i < a.ntile; i += THREADS)
    ooff[i] = (o_beg + i < a.own) ? owned_offset(o_beg + i, A.p, A.N1) : 0;
  for (int i = tid; i < np; i += THREADS) patom[i] = A.own_atom[k0 + i];
  const uint32_t full0 = smem_u32(&bars[0]), done0 = smem_u32(&bars[2]), accb = smem_u32(&bars[4]);
  if (tid == 0) init_barriers(full0, done0, accb);
  if (warp == 0) {
    __syncwarp();
    tmem_alloc(smem_u32(taddr_smem), TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *taddr_smem;

  const int r = tid & (MT - 1), hf = tid >> 7;
  const int v = vt * MT + r;
  const bool vok = v < ncols;
  const uint32_t bbytes = (uint32_t)a.ntile * 128u;
  const uint8_t *Bc = a.B + ((size_t)a.eoff[e] * a.nh + (size_t)h * KC) * bbytes;
  const uint32_t idesc = make_idesc(false, MT, a.ntile);
  bool ok = true;
  float cur[NW][16], nxt[NW][16];
  // K elements 16 hf .. 16 hf + 15 of chunk kc: pair kk, projectors al0 ..
  auto load_chunk = [&](int kc, float(&f)[NW][16]) {
    const int j0 = hf * 16;
    const int kk = kc * a.ppc + j0 / a.npad;
    const int al0 = j0 % a.npad;
    const bool live = vok && kk < np;
    const size_t rowb = ((size_t)(live ? patom[kk] : 0) * a.npad + al0) * ncols + v;
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      f[0][u] = live ? __ldg(W1 + rowb + (size_t)u * ncols) : 0.f;
      if constexpr (NW == 2) f[NW - 1][u] = live ? __ldg(W2 + rowb + (size_t)u * ncols) : 0.f;
    }
  };
  if (KC > 0) load_chunk(0, nxt);
  for (int kc = 0; kc < KC; ++kc) {
    const int s = kc & 1;
    const uint32_t use = (uint32_t)(kc >> 1);
    uint8_t *sA = base + s * STAGE;
    uint8_t *sB = sA + NW * A_BYTES;
    const uint32_t full = full0 + 8u * s, done = done0 + 8u * s;
#pragma unroll
    for (int w = 0; w < NW; ++w)
#pragma unroll
      for (int u = 0; u < 16; ++u) cur[w][u] = nxt[w][u];
    if (kc + 1 < KC) load_chunk(kc + 1, nxt);
    if (!ok) continue;
    if (kc >= 2 && !mbar_wait(done, (use - 1) & 1u)) {
      ok = false;
      continue;
    }
    if (tid == 0) {
      mbar_arrive_tx(full, bbytes);
      bulk_g2s(smem_u32(sB), Bc + (size_t)kc * bbytes, bbytes, full);
    }
#pragma unroll
    for (int w = 0; w < NW; ++w) store_row_half(sA + w * A_BYTES, r, hf, cur[w]);
    fence_proxy_async();
    mbar_arrive(full);
    if (tid == 0) {
      if (!mbar_wait(full, use & 1u)) {
        mbar_wait(full, use & 1u);
        ok = false;
        continue;
      }
      tc_fence_after();
      const uint64_t bd = sw128_desc(smem_u32(sB));
#pragma unroll
      for (int w = 0; w < NW; ++w) {
        const uint64_t ad = sw128_desc(smem_u32(sA + w * A_BYTES));
#pragma unroll
        for (int j = 0; j < 4; ++j)
          mma<false>(tmem + (uint32_t)(w * 128), ad + (uint64_t)(2 * j), bd + (uint64_t)(2 * j), idesc,
                     (kc | j) != 0);
      }
      mma_commit(done);
    }
  }
  if (tid == 0) mma_commit(accb);
  const bool got = mbar_wait(accb, 0) && ok;
  ok = __syncthreads_and(got) != 0;
  tc_fence_after();

  if (ok) {
    const int q = warp & 3, ch = warp >> 2;
    const int ng = a.ntile / 16, per = (ng + 1) / 2;
    const int g_beg = ch * per, g_end = min(ng, (ch + 1) * per);
    const int vout = vt * MT + q * 32 + lane;
    const bool wok = vout < ncols;
    const int vj = min(vout, ncols - 1);
    const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16);
    float chi = 0.f, clo = 0.f, csv = 1.f;
    if (MODE == EXP_RECURRENCE) {
      chi = A.chi[vj];
      clo = A.clo[vj];
    }
    if (MODE == EXP_ADD && A.cs) csv = (float)A.cs[vj];
    const float *mdinv = static_cast<const float *>(A.mdinv);
    const float *Xin = static_cast<const float *>(A.Xin);
    float *Y = static_cast<float *>(A.Y);
    float *RX = static_cast<float *>(A.RX);
    const float *Yh = static_cast<const float *>(A.Y0);
    const float *Yl = static_cast<const float *>(A.Y0lo);
    const float be = (float)A.beta, ga = (float)A.gamma;
    for (int gi = g_beg; gi < g_end; ++gi) {
      const int c0 = gi * 16;
      uint32_t s1[16], s2[16];
      if (KC > 0) {
        tmem_ld16_nowait(tl + (uint32_t)c0, s1);
        if (NW == 2) tmem_ld16_nowait(tl + 128u + (uint32_t)c0, s2);
        tmem_ld_wait();
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) s1[j] = s2[j] = 0u;
      }
      if (!wok) continue;
      const int nrow = min(16, a.own - (o_beg + c0));   // warp-uniform
      // two batches of 8 node rows: all loads of a batch in flight before its stores
#pragma unroll
      for (int jb = 0; jb < 16; jb += 8) {
        if (MODE == EXP_ADD) {
          float y[8];
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (jb + j < nrow) y[j] = Y[(cb + ooff[c0 + jb + j]) * A.ldy + vout];
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (jb + j < nrow)
              Y[(cb + ooff[c0 + jb + j]) * A.ldy + vout] = fmaf(csv, __uint_as_float(s1[jb + j]), y[j]);
        } else if (MODE == EXP_SINV) {
          float x[8], m[8];
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (jb + j < nrow) {
              const int64_t d = cb + ooff[c0 + jb + j];
              x[j] = Xin[d * A.ldx + vout];
              m[j] = mdinv[d];
            }
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (jb + j < nrow)
              Y[(cb + ooff[c0 + jb + j]) * A.ldy + vout] = m[j] * (x[j] - __uint_as_float(s1[jb + j]));
        } else {
          float ry[8], rx[8], yh[8], yl[8], m[8];
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (jb + j < nrow) {
              const int64_t d = cb + ooff[c0 + jb + j];
              m[j] = mdinv[d];
              ry[j] = Xin[d * A.ldx + vout];
              rx[j] = RX[d * A.ldx + vout];
              yh[j] = Yh[d * A.ldy0 + vout];
              yl[j] = Yl ? Yl[d * A.ldy0 + vout] : 0.f;
            }
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (jb + j < nrow) {
              const int64_t d = cb + ooff[c0 + jb + j];
              const float t = m[j] * (ry[j] - __uint_as_float(s1[jb + j]));
              const float bracket = -be * ry[j] - ga * rx[j] + __uint_as_float(s2[jb + j]);
              Y[d * A.ldy + vout] = t;
              RX[d * A.ldx + vout] = add_product_df(bracket, chi, clo, yh[j], yl[j]);
            }
        }
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

// ------------------------------------------------------------------ operand images
// projection B: pair tile starting at pair ks (ntp pairs, ncol = ntp npad rows),
// K-chunk kc of 32 owned nodes: rows (pair, projector), TF32
__global__ void k_build_projB(const float *__restrict__ oP, const int *__restrict__ own_off,
                              const int *__restrict__ pcell, int64_t npairs, int own, int npad, int kc_own, int ppt,
                              int n, int p, int N1, const float *__restrict__ rowscale, uint8_t *__restrict__ out) {
  const int64_t total = npairs * npad * kc_own * 8;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int c16 = (int)(idx & 7);
  int64_t r1 = idx >> 3;
  const int rr = (int)(r1 % npad);
  r1 /= npad;
  const int kc = (int)(r1 % kc_own);
  const int64_t k = r1 / kc_own;
  const int e = pcell[k];
  const int k0 = own_off[e], k1 = own_off[e + 1];
  const int64_t ks = k0 + (int64_t)(((int)(k - k0)) / ppt) * ppt;
  const int ncol = min(ppt, (int)(k1 - ks)) * npad;
  const int r = (int)(k - ks) * npad + rr;
  const int64_t cb = owned_base(e, n, p, N1);
  uint32_t w[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int o = kc * 32 + c16 * 4 + u;
    float f = o < own ? oP[((size_t)k * own + o) * npad + rr] : 0.f;
    if (rowscale && o < own) f *= rowscale[cb + owned_offset(o, p, N1)];
    w[u] = to_tf32(f);
  }
  uint8_t *dst = out + (size_t)ks * npad * 128 * kc_own + (size_t)kc * ncol * 128 + sw128_off(r, c16);
  *reinterpret_cast<uint4 *>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
}

// expansion B: chunk gch = eoff[e] nh + h KC_e + kc; rows = owned nodes h ntile + r,
// K = (pair kc ppc + j / npad, projector j % npad), TF32
__global__ void k_build_expB(const float *__restrict__ oP, const int *__restrict__ own_off,
                             const int *__restrict__ eoff, int ncells, int own, int npad, int ppc, int ntile, int nh,
                             int64_t nchunks, uint8_t *__restrict__ out) {
  const int64_t total = nchunks * ntile * 8;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int c16 = (int)(idx & 7);
  const int r = (int)((idx >> 3) % ntile);
  const int64_t gch = (idx >> 3) / ntile;
  int lo = 0, hi = ncells;   // largest e with eoff[e] nh <= gch
  while (hi - lo > 1) {
    const int mid = (lo + hi) / 2;
    if ((int64_t)eoff[mid] * nh <= gch)
      lo = mid;
    else
      hi = mid;
  }
  const int e = lo;
  const int KCe = eoff[e + 1] - eoff[e];
  const int64_t local = gch - (int64_t)eoff[e] * nh;
  const int h = (int)(local / KCe), kc = (int)(local % KCe);
  const int k0 = own_off[e], np = own_off[e + 1] - k0;
  const int o = h * ntile + r;
  uint32_t w[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int j = c16 * 4 + u;
    const int kk = kc * ppc + j / npad, al = j % npad;
    w[u] = to_tf32((o < own && kk < np) ? oP[((size_t)(k0 + kk) * own + o) * npad + al] : 0.f);
  }
  uint8_t *dst = out + (size_t)gch * ntile * 128 + sw128_off(r, c16);
  *reinterpret_cast<uint4 *>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
}

// ------------------------------------------------------------------ streaming forms
// Persistent warp-specialised forms (tc_stream.cuh) for 16-byte-aligned rows.
// LEAN: two stages, the form used while an FP64 step 2 shares the SMs.
template <bool LEAN = false>
struct ProjStream {
  static constexpr int NW = 1, S = LEAN ? 2 : 4, NEPI = 4;
  static constexpr bool BF16 = false;
  static constexpr uint32_t B_MAX = 192u * 128u;
  CUtensorMap tm[NW];   // rows of X (gathered with TMA)
  int ntiles, ncols, n, p, N1, own, npad, kc_own, ppt, vtiles, ldx;
  const int *own_off, *own_atom;
  const uint8_t *B;
  const float *X;
  float *U;             // per-atom sums (zeroed before the launch)
  struct Tile {
    int e, vt, k0, np;
    int64_t cb;
  };
  __device__ Tile tile(int t) const {
    Tile T;
    T.e = t / vtiles;
    T.vt = t - T.e * vtiles;
    T.k0 = own_off[T.e];
    T.np = own_off[T.e + 1] - T.k0;
    T.cb = owned_base(T.e, n, p, N1);
    return T;
  }
  __device__ int vt(const Tile &T) const { return T.vt; }
  __device__ int nsub(const Tile &T) const { return (T.np + ppt - 1) / ppt; }
  __device__ int nchunks(const Tile &, int) const { return kc_own; }
  __device__ int ncol(const Tile &T, int sub) const { return min(ppt, T.np - sub * ppt) * npad; }
  __device__ int xcol(const Tile &T) const { return T.vt * MT; }
  __device__ int row_id(const Tile &T, int, int kc, int j, int) const {
    const int o = kc * 32 + j;
    return o < own ? (int)(T.cb + owned_offset(o, p, N1)) : -1;
  }
  __device__ const uint8_t *bsrc(const Tile &T, int sub, int kc) const {
    return B + (size_t)(T.k0 + sub * ppt) * npad * 128 * kc_own + (size_t)kc * ncol(T, sub) * 128;
  }
  __device__ uint32_t dcol(int) const { return 0; }
  // U[atom of pair][al][v] += column (pair, al) of the tile: FP32 reductions into
  // the per-atom sums (no per-pair partials); four warps, one per lane quarter.
  // Columns come in whole pairs of npad (a multiple of 16), so a 16-column
  // group belongs to one pair.
  __device__ void epilogue(const Tile &T, int sub, uint32_t tl, int q, int, int lane, bool) const {
    const int nc = ncol(T, sub);
    const int v = T.vt * MT + q * 32 + lane;
    const int kb = T.k0 + sub * ppt;
    for (int c0 = 0; c0 < nc; c0 += 16) {
      uint32_t rr[16];
      tmem_ld16_nowait(tl + (uint32_t)c0, rr);
      tmem_ld_wait();
      const int kk = c0 / npad, al0 = c0 - kk * npad;
      float *dst = U + ((size_t)own_atom[kb + kk] * npad + al0) * ncols + v;
      if (v < ncols) {
#pragma unroll
        for (int j = 0; j < 16; ++j) atomicAdd(dst + (size_t)j * ncols, __uint_as_float(rr[j]));
      }
    }
  }
};

// Persistent expansion.  The A operands (W rows, small and L2-resident) are
// gathered by the transposer threads straight from global memory; the node
// rows the output stage reads (R_Y, R_X, Y hi/lo, or X, or Y) are prefetched
// 16 rows at a time into a four-deep staging ring with TMA row gathers
// (tile::gather4 from one tensor map per array); the epilogue warps read the
// rows' M_D^-1 and DoF indices (owner order) from global memory before they
// wait for a group, then read shared memory and store.
//   warp 0      B loader (one bulk copy per K-chunk)
//   warp 1      MMA (lane 0), TMEM allocation
//   warps 2..5  A gather (thread = vector row)
//   warp 6      output-stage loader: lane 4 k + q gathers rows 4 q .. 4 q + 3
//               of array k (the epilogue reads M_D^-1 and the DoF indices itself)
//   warp 7      idle
//   warps 8..15 epilogue: lane quarter warp % 4, half (warp - 8) / 4 of each 16-row group
namespace xs {
constexpr int SMAX = 3, NBUF = 4;   // A/B stages (at most), staged row groups
constexpr int WARP_B = 0, WARP_MMA = 1, WARP_G0 = 2, WARP_SL = 6, NSL = 2, WARP_E0 = 8, NEPI = 8;
constexpr int THREADS = 32 * (WARP_E0 + NEPI);
constexpr uint32_t ROWB = 512;   // one staged node row: 128 vectors

template <int MODE>
struct Geo {
  static constexpr int NW = (MODE == EXP_RECURRENCE) ? 2 : 1;
  static constexpr int S = (MODE == EXP_RECURRENCE) ? 2 : 3;    // A/B stages
  static constexpr int NA = (MODE == EXP_RECURRENCE) ? 4 : 1;   // staged arrays
  static constexpr uint32_t STAGE = NW * A_BYTES + 128u * 128u;
  static constexpr uint32_t GROUP = NA * 16u * ROWB;              // 16 staged rows of each array
};

struct Shared {
  uint64_t full[SMAX], afull[SMAX], empty[SMAX], accf[2], acce[2], sfull[NBUF], sempty[NBUF], drain;
  uint32_t taddr;
  int abort;
};

// at least 120 KB: one CTA per SM, so that its 512 TMEM columns are always free
template <int MODE>
constexpr size_t smem_bytes() {
  const size_t b =
      1024 + (size_t)Geo<MODE>::S * Geo<MODE>::STAGE + NBUF * (size_t)Geo<MODE>::GROUP + sizeof(Shared);
  return b < 120 * 1024 ? 120 * 1024 : b;
}

struct Args {
  CUtensorMap tm[4];   // staged arrays (R_Y, R_X, Y hi, Y lo; or X; or Y), rows gathered with TMA
  int amask;           // bit k: array k is staged
  ExpArgs A;
  int ntiles, npad, ppc, ntile, nh, vtiles, own;
  const uint8_t *B;
  const int *eoff;
  const float *W1, *W2;
  const float *mdo;   // M_D^-1 in owner order, nh * ntile per cell
  const int *odof;    // DoF indices in owner order, same layout
};

struct Tile {
  int e, h, vt, k0, np, kc, eo, o_beg, nrows, ngroups;
  int64_t cb;
};

__device__ __forceinline__ Tile tile_of(const Args &a, int t) {
  Tile T;
  T.vt = t % a.vtiles;
  T.h = (t / a.vtiles) % a.nh;
  T.e = t / (a.vtiles * a.nh);
  T.k0 = a.A.own_off[T.e];
  T.np = a.A.own_off[T.e + 1] - T.k0;
  T.eo = a.eoff[T.e];
  T.kc = a.eoff[T.e + 1] - T.eo;
  T.cb = owned_base(T.e, a.A.n, a.A.p, a.A.N1);
  T.o_beg = T.h * a.ntile;
  T.nrows = min(a.ntile, a.own - T.o_beg);
  T.ngroups = (T.nrows + 15) / 16;
  return T;
}

template <int MODE>
__device__ __forceinline__ bool skip_tile(const Tile &T) {
  return MODE == EXP_ADD && T.np == 0;   // nothing to add
}

template <int MODE>
__global__ void __launch_bounds__(THREADS, 1) k_exp_stream(const __grid_constant__ Args a, int *status) {
  using G = Geo<MODE>;
  constexpr int S = G::S;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *base = tcs::align1024(smem_raw);
  uint8_t *stg = base + (size_t)S * G::STAGE;   // [NBUF] x ([NA][16][128] floats, M_D^-1[16])
  Shared *sh = reinterpret_cast<Shared *>(stg + NBUF * (size_t)G::GROUP);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ncols = a.A.ncols;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(smem_u32(&sh->full[s]), 1);
      mbar_init(smem_u32(&sh->afull[s]), 128);
      mbar_init(smem_u32(&sh->empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&sh->accf[b]), 1);
      mbar_init(smem_u32(&sh->acce[b]), NEPI);
    }
    for (int b = 0; b < NBUF; ++b) {
      mbar_init(smem_u32(&sh->sfull[b]), 1);   // one arrival carrying the byte count
      mbar_init(smem_u32(&sh->sempty[b]), NEPI);
    }
    mbar_init(smem_u32(&sh->drain), 1);
    sh->abort = (*reinterpret_cast<volatile int *>(status) != 0) ? 1 : 0;
    fence_barrier_init();
    fence_proxy_async();
  }
  if (warp == WARP_MMA) {
    __syncwarp();
    tmem_alloc(smem_u32(&sh->taddr), 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sh->taddr;
  volatile int *abort = &sh->abort;
  const uint32_t bbytes = (uint32_t)a.ntile * 128u;

  if (warp == WARP_B) {
    // ---------------------------------------------------------------- B loader
    if (lane == 0) {
      uint32_t g = 0;
      bool run = !*abort;
      for (int t = blockIdx.x; run && t < a.ntiles; t += gridDim.x) {
        const Tile T = tile_of(a, t);
        if (skip_tile<MODE>(T)) continue;
        for (int kc = 0; kc < T.kc; ++kc, ++g) {
          const int s = (int)(g % S);
          const uint32_t u = g / S;
          if (g >= (uint32_t)S && !tcs::wait_or_abort(smem_u32(&sh->empty[s]), (u - 1) & 1u, abort)) {
            run = false;
            break;
          }
          const uint32_t full = smem_u32(&sh->full[s]);
          mbar_arrive_tx(full, bbytes);
          bulk_g2s(smem_u32(base + (size_t)s * G::STAGE + G::NW * A_BYTES),
                   a.B + ((size_t)T.eo * a.nh + (size_t)T.h * T.kc + kc) * bbytes, bbytes, full);
        }
      }
      for (int s = 0; s < S && (uint32_t)s < g; ++s) {   // let the copies in flight land
        const uint32_t last = ((g - 1 - (uint32_t)s) / S) * S + (uint32_t)s;
        mbar_wait(smem_u32(&sh->full[s]), (last / S) & 1u);
      }
    }
    __syncwarp();
  } else if (warp == WARP_MMA) {
    // ---------------------------------------------------------------- MMA
    if (lane == 0) {
      const uint32_t idesc = make_idesc(false, MT, a.ntile);
      uint32_t g = 0, tc = 0;
      bool run = !*abort;
      for (int t = blockIdx.x; run && t < a.ntiles; t += gridDim.x) {
        const Tile T = tile_of(a, t);
        if (skip_tile<MODE>(T)) continue;
        const int b = (int)(tc & 1u);
        if (tc >= 2 && !tcs::wait_or_abort(smem_u32(&sh->acce[b]), ((tc >> 1) - 1) & 1u, abort)) break;
        tc_fence_after();
        for (int kc = 0; kc < T.kc; ++kc, ++g) {
          const int s = (int)(g % S);
          const uint32_t u = g / S;
          if (!tcs::wait_or_abort(smem_u32(&sh->full[s]), u & 1u, abort) ||
              !tcs::wait_or_abort(smem_u32(&sh->afull[s]), u & 1u, abort)) {
            run = false;
            break;
          }
          tc_fence_after();
          uint8_t *st = base + (size_t)s * G::STAGE;
          const uint64_t bd = sw128_desc(smem_u32(st + G::NW * A_BYTES));
#pragma unroll
          for (int w = 0; w < G::NW; ++w) {
            const uint64_t ad = sw128_desc(smem_u32(st + w * A_BYTES));
#pragma unroll
            for (int j = 0; j < 4; ++j)
              mma<false>(tmem + (uint32_t)(b * 256 + w * 128), ad + (uint64_t)(2 * j), bd + (uint64_t)(2 * j),
                         idesc, (kc | j) != 0);
          }
          mma_commit(smem_u32(&sh->empty[s]));
        }
        if (!run) break;
        mma_commit(smem_u32(&sh->accf[b]));
        ++tc;
      }
      mma_commit(smem_u32(&sh->drain));   // nothing may still write TMEM when it is freed
      mbar_wait(smem_u32(&sh->drain), 0);
    }
    __syncwarp();
  } else if (warp < WARP_SL) {
    // ---------------------------------------------------------------- A gather
    const int r = threadIdx.x - 32 * WARP_G0;
    uint32_t g = 0;
    bool run = !*abort;
    for (int t = blockIdx.x; run && t < a.ntiles; t += gridDim.x) {
      const Tile T = tile_of(a, t);
      if (skip_tile<MODE>(T)) continue;
      const int v = T.vt * MT + r;
      const bool vok = v < ncols;
      for (int kc = 0; kc < T.kc; ++kc, ++g) {
        const int s = (int)(g % S);
        const uint32_t u = g / S;
        // K element j of this chunk: pair kc ppc + j / npad, projector j % npad
        float f[G::NW][32];
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          const int kk = kc * a.ppc + (hh * 16) / a.npad;
          const int al0 = (hh * 16) % a.npad;
          const bool live = vok && kk < T.np;
          const size_t rowb = ((size_t)(live ? a.A.own_atom[T.k0 + kk] : 0) * a.npad + al0) * ncols + v;
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            f[0][hh * 16 + i] = live ? __ldg(a.W1 + rowb + (size_t)i * ncols) : 0.f;
            if constexpr (G::NW == 2) f[G::NW - 1][hh * 16 + i] = live ? __ldg(a.W2 + rowb + (size_t)i * ncols) : 0.f;
          }
        }
        if (g >= (uint32_t)S && !tcs::wait_or_abort(smem_u32(&sh->empty[s]), (u - 1) & 1u, abort)) {
          run = false;
          break;
        }
        uint8_t *st = base + (size_t)s * G::STAGE;
#pragma unroll
        for (int w = 0; w < G::NW; ++w)
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const uint4 q = make_uint4(to_tf32(f[w][4 * c]), to_tf32(f[w][4 * c + 1]), to_tf32(f[w][4 * c + 2]),
                                       to_tf32(f[w][4 * c + 3]));
            *reinterpret_cast<uint4 *>(st + w * A_BYTES + sw128_off(r, c)) = q;
          }
        fence_proxy_async();
        mbar_arrive(smem_u32(&sh->afull[s]));
      }
    }
  } else if (warp == WARP_SL) {
    // ---------------------------------------------------------------- output-stage loader
    int na = 0;
#pragma unroll
    for (int k = 0; k < G::NA; ++k) na += (a.amask >> k) & 1;
    const uint32_t gbytes = (uint32_t)na * 16u * ROWB;   // row gathers
    const int k = lane >> 2, q = lane & 3;
    const bool mine = k < G::NA && ((a.amask >> k) & 1);
    uint32_t gc = 0;
    bool run = __shfl_sync(0xffffffffu, *abort, 0) == 0;
    for (int t = blockIdx.x; run && t < a.ntiles; t += gridDim.x) {
      const Tile T = tile_of(a, t);
      if (skip_tile<MODE>(T)) continue;
      const int x = T.vt * MT;
      for (int gi = 0; gi < T.ngroups; ++gi, ++gc) {
        const int gb = (int)(gc % NBUF);
        const uint32_t ug = gc / NBUF;
        if (gc >= NBUF && !tcs::warp_wait(smem_u32(&sh->sempty[gb]), (ug - 1) & 1u, abort, lane)) {
          run = false;
          break;
        }
        // row j of the group (lanes 0..15); rows past the tile repeat its first row (never read back)
        const int nrow = min(16, T.nrows - gi * 16);
        const int jr = (lane & 15) < nrow ? (lane & 15) : 0;
        const int d = (int)(T.cb + owned_offset(T.o_beg + gi * 16 + jr, a.A.p, a.A.N1));
        int r4[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) r4[i] = __shfl_sync(0xffffffffu, d, 4 * q + i);
        uint8_t *grp = stg + (size_t)gb * G::GROUP;
        const uint32_t full = smem_u32(&sh->sfull[gb]);
        if (lane == 0) mbar_arrive_tx(full, gbytes);
        __syncwarp();
        if (mine)
          tma_gather4(smem_u32(grp) + (uint32_t)(k * 16 + 4 * q) * ROWB, &a.tm[k], x, r4[0], r4[1], r4[2], r4[3],
                      full);
      }
    }
    if (lane == 0)
      for (int gb = 0; gb < NBUF && (uint32_t)gb < gc; ++gb) {   // let the copies in flight land
        const uint32_t last = ((gc - 1 - (uint32_t)gb) / NBUF) * NBUF + (uint32_t)gb;
        mbar_wait(smem_u32(&sh->sfull[gb]), (last / NBUF) & 1u);
      }
    __syncwarp();
  } else if (warp < WARP_E0) {
    // idle
  } else {
    // ---------------------------------------------------------------- epilogue
    const int q = warp & 3, part = (warp - WARP_E0) >> 2;
    const float be = (float)a.A.beta, ga = (float)a.A.gamma;
    float *Y = static_cast<float *>(a.A.Y);
    float *RX = static_cast<float *>(a.A.RX);
    const bool has_lo = a.A.Y0lo != nullptr;
    uint32_t tc = 0, gc = 0;
    bool run = __shfl_sync(0xffffffffu, *abort, 0) == 0;
    for (int t = blockIdx.x; run && t < a.ntiles; t += gridDim.x) {
      const Tile T = tile_of(a, t);
      if (skip_tile<MODE>(T)) continue;
      const int b = (int)(tc & 1u);
      if (!tcs::warp_wait(smem_u32(&sh->accf[b]), (tc >> 1) & 1u, abort, lane)) break;
      tc_fence_after();
      const int vl = q * 32 + lane;
      const int v = T.vt * MT + vl;
      const bool vok = v < ncols;
      const int vj = min(v, ncols - 1);
      float chi = 0.f, clo = 0.f, csv = 1.f;
      if (MODE == EXP_RECURRENCE) {
        chi = a.A.chi[vj];
        clo = a.A.clo[vj];
      }
      if (MODE == EXP_ADD && a.A.cs) csv = (float)a.A.cs[vj];
      const uint32_t tl = tmem + (uint32_t)(b * 256) + ((uint32_t)(q * 32) << 16);
      for (int gi = 0; gi < T.ngroups; ++gi, ++gc) {
        const int gb = (int)(gc % NBUF);
        // M_D^-1 and DoF index of the warp's 8 rows (owner order, padded to whole
        // groups), read before the wait so that the loads overlap it
        const size_t oo = ((size_t)T.e * a.nh + T.h) * a.ntile + gi * 16 + part * 8;
        float mj[8];
        int dj[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          mj[j] = (MODE != EXP_ADD) ? __ldg(a.mdo + oo + j) : 0.f;
          dj[j] = __ldg(a.odof + oo + j);
        }
        if (!tcs::warp_wait(smem_u32(&sh->sfull[gb]), (gc / NBUF) & 1u, abort, lane)) {
          run = false;
          break;
        }
        const int c0 = gi * 16 + part * 8;   // first tile column (node row) of this warp
        uint32_t s1[8], s2[8];
        if (T.kc > 0) {
          tmem_ld8_nowait(tl + (uint32_t)c0, s1);
          if (G::NW == 2) tmem_ld8_nowait(tl + 128u + (uint32_t)c0, s2);
          tmem_ld_wait();
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j) s1[j] = s2[j] = 0u;
        }
        const float *sg = reinterpret_cast<const float *>(stg + (size_t)gb * G::GROUP);
        const int nv = min(8, T.nrows - (gi * 16 + part * 8));   // rows of this warp in the group
        if (vok) {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int jr = part * 8 + j;   // staged row
            if (j >= nv) break;
            const int64_t d = dj[j];
            if (MODE == EXP_RECURRENCE) {
              const float ry = sg[(0 * 16 + jr) * MT + vl], rx = sg[(1 * 16 + jr) * MT + vl];
              const float yh = sg[(2 * 16 + jr) * MT + vl];
              const float yl = has_lo ? sg[(3 * 16 + jr) * MT + vl] : 0.f;
              const float m = mj[j];
              Y[d * a.A.ldy + v] = m * (ry - __uint_as_float(s1[j]));
              const float bracket = -be * ry - ga * rx + __uint_as_float(s2[j]);
              RX[d * a.A.ldx + v] = add_product_df(bracket, chi, clo, yh, yl);
            } else if (MODE == EXP_SINV) {
              Y[d * a.A.ldy + v] = mj[j] * (sg[jr * MT + vl] - __uint_as_float(s1[j]));
            } else {
              Y[d * a.A.ldy + v] = fmaf(csv, __uint_as_float(s1[j]), sg[jr * MT + vl]);
            }
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&sh->sempty[gb]));
      }
      if (!run) break;
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&sh->acce[b]));
      ++tc;
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == WARP_MMA) {
    __syncwarp();
    tmem_dealloc(tmem, 512);
  }
  if (threadIdx.x == 0 && sh->abort) atomicExch(status, 1);
}
}  // namespace xs

size_t proj_smem() {
  const size_t b = 1024 + 2 * (size_t)PROJ_STAGE + 64 + 2 * sizeof(int) * OWN_MAX_TC;
  return std::max<size_t>(b, 80 * 1024);   // at most two CTAs (2 x 256 TMEM columns) per SM
}

size_t exp_smem(int nw) {
  const size_t b = 1024 + 2 * (size_t)exp_stage_bytes(nw) + 64 + sizeof(int) * (128 + PAIR_MAX);
  return std::max<size_t>(b, 80 * 1024);
}

}  // namespace

bool nltc_supported(const paw_context *c) {
  return c->nown_pairs > 0 && c->own <= OWN_MAX_TC && (c->npad == 16 || c->npad == 32) &&
         c->max_own_pairs <= PAIR_MAX;
}

void nltc_prepare(paw_context *c, cudaStream_t s) {
  NlTcMats &N = c->nltc;
  if (N.valid) return;
  PAW_REQUIRE(nltc_supported(c), PAW_ERR_UNSUPPORTED, "tensor-core nonlocal kernels: unsupported projector layout");
  N.kc_own = (c->own + 31) / 32;
  N.ppt = 192 / c->npad;   // N tile <= 192 columns: four 56 KB stages fit the persistent kernel
  N.ppc = 32 / c->npad;
  N.nh = (c->own + 127) / 128;
  N.ntile = (((c->own + N.nh - 1) / N.nh) + 15) / 16 * 16;
  std::vector<int> off(c->ncells + 1);
  PAW_CUDA(cudaMemcpy(off.data(), c->own_off.ptr, sizeof(int) * off.size(), cudaMemcpyDeviceToHost));
  std::vector<int> eoff(c->ncells + 1, 0), pcell((size_t)c->nown_pairs);
  for (int e = 0; e < c->ncells; ++e) {
    const int np = off[e + 1] - off[e];
    eoff[e + 1] = eoff[e] + (np + N.ppc - 1) / N.ppc;
    for (int k = off[e]; k < off[e + 1]; ++k) pcell[k] = e;
  }
  N.exp_chunks = eoff[c->ncells];
  N.eoff.ensure(sizeof(int) * eoff.size(), &c->dev_bytes);
  PAW_CUDA(cudaMemcpy(N.eoff.ptr, eoff.data(), sizeof(int) * eoff.size(), cudaMemcpyHostToDevice));
  int64_t tmp = 0;
  DevBuf d_pcell;
  d_pcell.ensure(sizeof(int) * pcell.size(), &tmp);
  PAW_CUDA(cudaMemcpy(d_pcell.ptr, pcell.data(), sizeof(int) * pcell.size(), cudaMemcpyHostToDevice));
  const size_t pbytes = (size_t)c->nown_pairs * c->npad * 128 * N.kc_own;
  const size_t ebytes = (size_t)N.exp_chunks * N.nh * N.ntile * 128;
  N.projB.ensure(pbytes, &c->dev_bytes);
  N.projBs.ensure(pbytes, &c->dev_bytes);
  N.expB.ensure(std::max<size_t>(ebytes, 16), &c->dev_bytes);
  {
    const int64_t total = c->nown_pairs * c->npad * N.kc_own * 8;
    const unsigned grid = (unsigned)((total + 255) / 256);
    k_build_projB<<<grid, 256, 0, s>>>(c->ownP32.as<float>(), c->own_off.as<int>(), d_pcell.as<int>(),
                                       c->nown_pairs, c->own, c->npad, N.kc_own, N.ppt, c->n, c->p, c->N1, nullptr,
                                       N.projB.as<uint8_t>());
    PAW_LAUNCH_CHECK("k_build_projB");
    // the same blocks with M_D^-1 of each node folded in (projection of M_D^-1 X)
    k_build_projB<<<grid, 256, 0, s>>>(c->ownP32.as<float>(), c->own_off.as<int>(), d_pcell.as<int>(),
                                       c->nown_pairs, c->own, c->npad, N.kc_own, N.ppt, c->n, c->p, c->N1,
                                       c->md_inv32.as<float>(), N.projBs.as<uint8_t>());
    PAW_LAUNCH_CHECK("k_build_projB");
  }
  if (N.exp_chunks > 0) {
    const int64_t total = N.exp_chunks * N.nh * N.ntile * 8;
    k_build_expB<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(
        c->ownP32.as<float>(), c->own_off.as<int>(), N.eoff.as<int>(), c->ncells, c->own, c->npad, N.ppc, N.ntile,
        N.nh, N.exp_chunks * N.nh, N.expB.as<uint8_t>());
    PAW_LAUNCH_CHECK("k_build_expB");
  }
  // M_D^-1 and DoF indices in owner order (cell, owned node), nh * ntile entries per cell
  {
    const size_t ostride = (size_t)N.nh * N.ntile;
    std::vector<float> mdo((size_t)c->ncells * ostride, 0.f);
    std::vector<int> odof((size_t)c->ncells * ostride, -1);
    for (int e = 0; e < c->ncells; ++e) {
      const int64_t cb = owned_base(e, c->n, c->p, c->N1);
      for (int o = 0; o < c->own; ++o) {
        const int64_t d = cb + owned_offset(o, c->p, c->N1);
        mdo[(size_t)e * ostride + o] = (float)c->mdinv_h[d];
        odof[(size_t)e * ostride + o] = (int)d;
      }
    }
    N.mdo.ensure(sizeof(float) * mdo.size(), &c->dev_bytes);
    N.odof.ensure(sizeof(int) * odof.size(), &c->dev_bytes);
    PAW_CUDA(cudaMemcpy(N.mdo.ptr, mdo.data(), sizeof(float) * mdo.size(), cudaMemcpyHostToDevice));
    PAW_CUDA(cudaMemcpy(N.odof.ptr, odof.data(), sizeof(int) * odof.size(), cudaMemcpyHostToDevice));
  }
  PAW_CUDA(cudaStreamSynchronize(s));
  d_pcell.release(&tmp);
  N.valid = 1;
}

// CTAs of a persistent launch: the SM count of the current device, capped by
// the instance's grid limit (set when instances share the GPU)
static int persistent_grid(const paw_context *c) {
  int dev = 0, n = 0;
  PAW_CUDA(cudaGetDevice(&dev));
  PAW_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
  return c->grid_cap > 0 ? std::min(c->grid_cap, n) : n;
}

template <class P>
static void launch_stream(const paw_context *c, const P &p, cudaStream_t s, const char *what) {
  const size_t shm = tcs::Geo<P>::SMEM;
  PAW_CUDA(cudaFuncSetAttribute(tcs::k_tc_stream<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  if (c->lean)   // the whole shared memory configured, so that an FP64 CTA fits beside this one
    PAW_CUDA(cudaFuncSetAttribute(tcs::k_tc_stream<P>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  cudaSharedmemCarveoutMaxShared));
  const int grid = std::max(1, std::min(p.ntiles, persistent_grid(c)));
  tcs::k_tc_stream<P><<<grid, tcs::threads_for(P::NEPI), shm, s>>>(p, c->status_dev.as<int>(), c->wait_ns,
                                                                     c->wait_probe);
  PAW_LAUNCH_CHECK(what);
}

static bool rows16(const void *p, int ld) {
  return reinterpret_cast<uintptr_t>(p) % 16 == 0 && ld % 4 == 0;
}

template <bool LEAN>
static void proj_stream(paw_context *c, const float *X, int ldx, int ncols, bool scaled, float *U, int vtiles,
                        cudaStream_t s) {
  const NlTcMats &N = c->nltc;
  ProjStream<LEAN> p;
  p.ntiles = c->ncells * vtiles;
  p.ncols = ncols;
  p.n = c->n;
  p.p = c->p;
  p.N1 = c->N1;
  p.own = c->own;
  p.npad = c->npad;
  p.kc_own = N.kc_own;
  p.ppt = N.ppt;
  p.vtiles = vtiles;
  p.ldx = ldx;
  p.own_off = c->own_off.as<int>();
  p.own_atom = c->own_atom.as<int>();
  p.B = scaled ? N.projBs.as<uint8_t>() : N.projB.as<uint8_t>();
  p.X = X;
  p.U = U;
  PAW_CUDA(cudaMemsetAsync(U, 0, sizeof(float) * (size_t)c->natoms * c->npad * ncols, s));
  encode_row_map(&p.tm[0], X, c->ndof, ncols, ldx);
  launch_stream(c, p, s, LEAN ? "k_tc_stream<projection, lean>" : "k_tc_stream<projection>");
}

bool nltc_project(paw_context *c, const float *X, int ldx, int ncols, const float *rowscale, float *PP,
                  float *U, cudaStream_t s) {
  if (ncols <= 0) return false;
  nltc_prepare(c, s);
  const NlTcMats &N = c->nltc;
  const int vtiles = (ncols + MT - 1) / MT;
  const bool scaled = rowscale != nullptr && rowscale == c->md_inv32.as<float>();
  if (c->tc_variant == 0 && (rowscale == nullptr || scaled) && rows16(X, ldx) && ncols % 4 == 0) {
    if (c->lean)
      proj_stream<true>(c, X, ldx, ncols, scaled, U, vtiles, s);
    else
      proj_stream<false>(c, X, ldx, ncols, scaled, U, vtiles, s);
    return true;   // U holds the per-atom sums
  }
  ProjTcArgs a;
  a.n = c->n;
  a.p = c->p;
  a.N1 = c->N1;
  a.own = c->own;
  a.npad = c->npad;
  a.kc_own = N.kc_own;
  a.ppt = N.ppt;
  a.vtiles = vtiles;
  a.ncols = ncols;
  a.ldx = ldx;
  a.own_off = c->own_off.as<int>();
  a.B = N.projB.as<uint8_t>();
  a.X = X;
  a.rowscale = rowscale;
  a.PP = PP;
  a.status = c->status_dev.as<int>();
  const int64_t blocks = (int64_t)c->ncells * a.vtiles;
  PAW_REQUIRE(blocks < (1ll << 31), PAW_ERR_UNSUPPORTED, "too many projection tiles");
  const size_t shm = proj_smem();
  PAW_CUDA(cudaFuncSetAttribute(k_nl_project_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  k_nl_project_tc<<<(unsigned)blocks, THREADS, shm, s>>>(a);
  PAW_LAUNCH_CHECK("k_nl_project_tc");
  return false;   // per-pair partials in PP
}

template <int MODE>
static void expand_stream(paw_context *c, const ExpArgs &A, const float *W1, const float *W2, cudaStream_t s) {
  const NlTcMats &N = c->nltc;
  xs::Args p;
  p.A = A;
  p.vtiles = (A.ncols + MT - 1) / MT;
  const int64_t nt = (int64_t)c->ncells * N.nh * p.vtiles;
  PAW_REQUIRE(nt < (1ll << 31), PAW_ERR_UNSUPPORTED, "too many expansion tiles");
  p.ntiles = (int)nt;
  p.npad = c->npad;
  p.ppc = N.ppc;
  p.ntile = N.ntile;
  p.nh = N.nh;
  p.own = c->own;
  p.B = N.expB.as<uint8_t>();
  p.eoff = N.eoff.as<int>();
  p.W1 = W1;
  p.W2 = W2;
  p.mdo = N.mdo.as<float>();
  p.odof = N.odof.as<int>();
  // staged arrays: R_Y, R_X, Y hi, Y lo (recurrence); X (Shat^-1); Y (add)
  const void *arr[4] = {nullptr, nullptr, nullptr, nullptr};
  int ld[4] = {0, 0, 0, 0};
  if (MODE == EXP_RECURRENCE) {
    arr[0] = A.Xin, ld[0] = A.ldx;
    arr[1] = A.RX, ld[1] = A.ldx;
    arr[2] = A.Y0, ld[2] = A.ldy0;
    arr[3] = A.Y0lo, ld[3] = A.ldy0;
  } else if (MODE == EXP_SINV) {
    arr[0] = A.Xin, ld[0] = A.ldx;
  } else {
    arr[0] = A.Y, ld[0] = A.ldy;
  }
  p.amask = 0;
  for (int k = 0; k < 4; ++k)
    if (arr[k]) {
      encode_row_map(&p.tm[k], static_cast<const float *>(arr[k]), c->ndof, A.ncols, ld[k]);
      p.amask |= 1 << k;
    }
  // (the expansion keeps its four staged groups while a step 2 shares the SMs: a two-group
  // form, 160 KB, still leaves too little room for the FP64 kernel and slowed the loop)
  const size_t shm = xs::smem_bytes<MODE>();
  PAW_CUDA(cudaFuncSetAttribute(xs::k_exp_stream<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  const int grid = std::max(1, std::min(p.ntiles, persistent_grid(c)));
  xs::k_exp_stream<MODE><<<grid, xs::THREADS, shm, s>>>(p, c->status_dev.as<int>());
  PAW_LAUNCH_CHECK("k_exp_stream");
}

void nltc_expand(paw_context *c, int mode, const ExpArgs &A, const float *W1, const float *W2, cudaStream_t s) {
  if (A.ncols <= 0) return;
  nltc_prepare(c, s);
  const NlTcMats &N = c->nltc;
  // bulk-copied rows (output-stage operands) must start on 16-byte boundaries
  bool rows_ok = c->tc_variant == 0 && A.ncols % 4 == 0;
  if (mode == EXP_RECURRENCE)
    rows_ok = rows_ok && rows16(A.Xin, A.ldx) && rows16(A.RX, A.ldx) && rows16(A.Y0, A.ldy0) &&
              (A.Y0lo == nullptr || rows16(A.Y0lo, A.ldy0));
  else if (mode == EXP_SINV)
    rows_ok = rows_ok && rows16(A.Xin, A.ldx);
  else
    rows_ok = rows_ok && rows16(A.Y, A.ldy);
  if (rows_ok) {
    if (mode == EXP_ADD)
      expand_stream<EXP_ADD>(c, A, W1, W2, s);
    else if (mode == EXP_SINV)
      expand_stream<EXP_SINV>(c, A, W1, W2, s);
    else
      expand_stream<EXP_RECURRENCE>(c, A, W1, W2, s);
    return;
  }
  ExpTcArgs a;
  a.npad = c->npad;
  a.ppc = N.ppc;
  a.ntile = N.ntile;
  a.nh = N.nh;
  a.vtiles = (A.ncols + MT - 1) / MT;
  a.own = c->own;
  a.B = N.expB.as<uint8_t>();
  a.eoff = N.eoff.as<int>();
  a.status = c->status_dev.as<int>();
  const int64_t blocks = (int64_t)c->ncells * N.nh * a.vtiles;
  PAW_REQUIRE(blocks < (1ll << 31), PAW_ERR_UNSUPPORTED, "too many expansion tiles");
  const size_t shm = exp_smem(mode == EXP_RECURRENCE ? 2 : 1);
  switch (mode) {
    case EXP_ADD:
      PAW_CUDA(cudaFuncSetAttribute(k_nl_expand_tc<EXP_ADD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
      k_nl_expand_tc<EXP_ADD><<<(unsigned)blocks, THREADS, shm, s>>>(A, a, W1, W2);
      break;
    case EXP_SINV:
      PAW_CUDA(
          cudaFuncSetAttribute(k_nl_expand_tc<EXP_SINV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
      k_nl_expand_tc<EXP_SINV><<<(unsigned)blocks, THREADS, shm, s>>>(A, a, W1, W2);
      break;
    default:
      PAW_CUDA(cudaFuncSetAttribute(k_nl_expand_tc<EXP_RECURRENCE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)shm));
      k_nl_expand_tc<EXP_RECURRENCE><<<(unsigned)blocks, THREADS, shm, s>>>(A, a, W1, W2);
      break;
  }
  PAW_LAUNCH_CHECK("k_nl_expand_tc");
}

}  // namespace pawfe
