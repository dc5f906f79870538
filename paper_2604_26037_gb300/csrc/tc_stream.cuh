// Persistent, warp-specialised tcgen05 pipeline for the dense contractions of
// the filter (projector blocks, cell matrices).
//
// One CTA per SM walks a static list of tiles (tile t, t + gridDim.x, ...).
// A tile is one or more accumulation rounds
//     D (128 vectors x N) = A (128 vectors x K) . B (N x K)^T
// into a double-buffered FP32 accumulator in tensor memory (2 x 256 columns),
// so the epilogue of one round overlaps the MMAs of the next.
//
// The rows of A are contiguous 128-vector slices of a row-major block (a node
// row of a DoF-major multivector, or a projector row of the atom-major
// coefficients), so a chunk arrives vector-contiguous (MN-major); four
// transposer warps turn it into the K-major operand.  The landed rows cannot
// serve as an MN-major operand as they are: each is 512 bytes of 128 vectors at
// a 512-byte pitch, while the MN-major shared-memory layouts of tcgen05 hold
// MN-contiguous runs of at most 128 bytes per K row (the 128-, 64- and 32-byte
// swizzle atoms, 8 K rows of one run each; without swizzle, core matrices of
// 8 K rows by 16 bytes, 16 bytes apart).  Landing the rows in such a layout
// takes one TMA copy per 32 vectors of a row, four times the row copies, and
// the loader's copy issue already sets these kernels' rate.
// Roles:
//   warp 0        loader: the K rows of a chunk with TMA row gathers
//                 (tile::gather4, four 512-byte rows per instruction, issued by
//                 lanes 0 .. K/4 - 1 from the operand's tensor map) into a raw
//                 [K][128] FP32 stage, and the pre-arranged B chunk as one
//                 cp.async.bulk; rows that do not exist repeat the chunk's
//                 first row (the B operand is zero there).  The TMA unit keeps
//                 far more bytes in flight per SM than warp-wide 16-byte
//                 cp.async, whose issue stalled the loaders.  The row indices
//                 of the next chunk are looked up before the wait for a free
//                 stage
//   warp 6        idle
//   warp 1        MMA: lane 0 issues tcgen05.mma (4 per 128-byte K-chunk);
//                 the warp allocates and frees the tensor memory
//   warps 2..5    transposers: thread = vector row; raw FP32 -> K-major
//                 128-byte-swizzled A operand (TF32 or BF16)
//   warps 7..     epilogue: warp w reads TMEM lane quarter w % 4
// Barriers per stage s: full[s] (copies landed: one arrival with the byte
// count of the row gathers and the B chunk), afull[s] (A written by the 128
// transposer threads), empty[s] (MMAs done, tcgen05.commit); per
// accumulator b: accf[b] (commit) and acce[b] (one arrival per epilogue warp).
//
// Every pipeline wait is bounded (wait_ns, 2 s unless paw_set_wait_limit
// changed it) and gives up early once another role has given up (a shared
// abort word).  The CTA then lets its bulk copies land and drains its MMAs
// (those two waits keep the fixed 2 s bound: they end as soon as the copies
// and MMAs already issued complete), frees the tensor memory and records the
// failure in status[0].  With probe set, thread 0 first waits on status[1], a
// word nothing writes, so the launch gives up before it issues any copy or MMA:
// the failure path, exercised without a fault.
#pragma once

#include <cuda_bf16.h>

#include "tc_ptx.cuh"

namespace pawfe {
namespace tcs {

using namespace tcp;

constexpr int MT = 128;                       // vectors per tile = MMA M
constexpr uint32_t ROW_BYTES = MT * 4;        // one raw A row
constexpr uint32_t A_BYTES = MT * 128;        // one swizzled A chunk
constexpr uint32_t TMEM_COLS = 512;           // two accumulators of 256 columns
constexpr int WARP_LOAD = 0, WARP_MMA = 1, WARP_XP0 = 2, NXP = 4, WARP_IDLE = 6, WARP_EPI0 = 7;

__host__ __device__ constexpr int threads_for(int nepi) { return 32 * (WARP_EPI0 + nepi); }

constexpr int SMAX = 6;                       // stages at most

struct Shared {
  uint64_t full[SMAX], afull[SMAX], empty[SMAX], accf[2], acce[2], drain;
  uint64_t wait_ns;                           // give-up bound of the pipeline waits of this launch
  uint32_t taddr;
  int abort;
};

template <class P>
struct Geo {
  static constexpr int KR = P::BF16 ? 64 : 32;                  // A rows (K elements) per chunk
  static constexpr uint32_t RAW = KR * ROW_BYTES;               // raw rows of one operand
  static constexpr uint32_t STAGE = P::NW * (RAW + A_BYTES) + P::B_MAX;
  // at least 120 KB: one CTA per SM, so that its 512 TMEM columns are always free
  static constexpr size_t SMEM0 = 1024 + (size_t)P::S * STAGE + sizeof(Shared);
  static constexpr size_t SMEM = SMEM0 < 120 * 1024 ? 120 * 1024 : SMEM0;
  static_assert(P::B_MAX % 1024 == 0, "B stage must keep 1024-byte alignment");
  static_assert(P::S >= 2 && P::S <= SMAX && P::NW >= 1 && P::NW <= 2, "stage / operand counts");
  static_assert(P::NEPI % 4 == 0, "epilogue warps come in lane-quarter groups");
};

__device__ __forceinline__ uint8_t *align1024(uint8_t *p) {
  return reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

// Bounded wait that also returns false as soon as another role has given up.
// Warps that go on to warp-collective instructions call warp_wait instead,
// so that all 32 lanes take the same decision.
__device__ __forceinline__ bool wait_or_abort(uint32_t bar, uint32_t parity, volatile int *abort,
                                              uint64_t limit = WAIT_NS) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort) return false;
    if (gtimer() - t0 > limit) {
      *abort = 1;
      return false;
    }
  }
  return true;
}

// lane 0 waits, the warp follows its result
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, volatile int *abort, int lane,
                                          uint64_t limit = WAIT_NS) {
  int ok = 0;
  if (lane == 0) ok = wait_or_abort(bar, parity, abort, limit) ? 1 : 0;
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

template <class P>
__device__ __forceinline__ uint8_t *stage_raw(uint8_t *base, int s, int w) {
  return base + (size_t)s * Geo<P>::STAGE + (size_t)w * Geo<P>::RAW;
}
template <class P>
__device__ __forceinline__ uint8_t *stage_A(uint8_t *base, int s, int w) {
  return base + (size_t)s * Geo<P>::STAGE + (size_t)P::NW * Geo<P>::RAW + (size_t)w * A_BYTES;
}
template <class P>
__device__ __forceinline__ uint8_t *stage_B(uint8_t *base, int s) {
  return base + (size_t)s * Geo<P>::STAGE + (size_t)P::NW * (Geo<P>::RAW + A_BYTES);
}

// ------------------------------------------------------------------ roles
// The chunk sequence of one CTA: tiles t = blockIdx.x, t + gridDim.x, ...,
// their accumulation rounds, and the K-chunks of each round, in the order
// every role consumes them.
template <class P>
struct Walk {
  typename P::Tile T;
  int t, ns, sub, nk, kc;
  __device__ bool start(const P &p) {
    t = (int)blockIdx.x - (int)gridDim.x;
    ns = nk = kc = sub = 0;
    return settle(p);
  }
  __device__ bool next(const P &p) {
    ++kc;
    return settle(p);
  }
  // first chunk at or after the current position; false past the last tile
  __device__ bool settle(const P &p) {
    while (kc >= nk) {
      kc = 0;
      if (++sub >= ns) {
        t += gridDim.x;
        if (t >= p.ntiles) return false;
        T = p.tile(t);
        ns = p.nsub(T);
        sub = 0;
        if (ns == 0) {
          nk = 0;
          continue;
        }
      }
      nk = p.nchunks(T, sub);
    }
    return true;
  }
};

// row indices of the current chunk: lane l holds rows l, 32 + l, ... (-1: no row)
template <class P>
__device__ __forceinline__ void chunk_ids(const P &p, const Walk<P> &w, int lane, int (&rid)[P::NW][Geo<P>::KR / 32]) {
#pragma unroll
  for (int o = 0; o < P::NW; ++o)
#pragma unroll
    for (int jj = 0; jj < Geo<P>::KR / 32; ++jj) rid[o][jj] = p.row_id(w.T, w.sub, w.kc, jj * 32 + lane, o);
}

template <class P>
__device__ void role_loader(const P &p, uint8_t *base, Shared *sh, int lane) {
  constexpr int KR = Geo<P>::KR, S = P::S, RPL = KR / 32;
  volatile int *abort = &sh->abort;
  uint32_t g = 0;
  bool run = __shfl_sync(0xffffffffu, *abort, 0) == 0;   // warp-uniform
  Walk<P> w;
  bool have = w.start(p);
  int rid[P::NW][RPL];
  if (have) chunk_ids<P>(p, w, lane, rid);
  for (; run && have; ++g) {
    const int s = (int)(g % S);
    const uint32_t u = g / S;
    if (g >= (uint32_t)S && !warp_wait(smem_u32(&sh->empty[s]), (u - 1) & 1u, abort, lane, sh->wait_ns)) {
      run = false;
      break;
    }
    const uint32_t full = smem_u32(&sh->full[s]);
    const uint32_t bbytes = (uint32_t)p.ncol(w.T, w.sub) * 128u;
    if (lane == 0) mbar_arrive_tx(full, bbytes + (uint32_t)(P::NW * KR) * ROW_BYTES);
    __syncwarp();
    if (lane == 0) bulk_g2s(smem_u32(stage_B<P>(base, s)), p.bsrc(w.T, w.sub, w.kc), bbytes, full);
    const int x = p.xcol(w.T);
#pragma unroll
    for (int o = 0; o < P::NW; ++o) {
      // rows that do not exist repeat the chunk's first row (always present)
      const int first = __shfl_sync(0xffffffffu, rid[o][0], 0);
      // lane l < KR / 4 gathers rows 4 l .. 4 l + 3, held by lanes (4 l + i) % 32, slot (4 l + i) / 32
      int r4[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int row = 4 * lane + i;
        int val = 0;
#pragma unroll
        for (int jj = 0; jj < RPL; ++jj) {
          const int t = __shfl_sync(0xffffffffu, rid[o][jj], row & 31);
          if ((row >> 5) == jj) val = t;
        }
        r4[i] = val >= 0 ? val : first;
      }
      if (lane < KR / 4)
        tma_gather4(smem_u32(stage_raw<P>(base, s, o)) + (uint32_t)lane * 4u * ROW_BYTES, &p.tm[o], x, r4[0], r4[1],
                    r4[2], r4[3], full);
    }
    have = w.next(p);
    if (have) chunk_ids<P>(p, w, lane, rid);   // consumed after the next stage wait
  }
  // let every copy in flight land before the CTA can exit
  if (lane == 0) {
    const uint32_t issued = g;
    for (int s = 0; s < S; ++s) {
      if ((uint32_t)s >= issued) break;
      const uint32_t last = ((issued - 1 - (uint32_t)s) / S) * S + (uint32_t)s;   // last chunk on stage s
      mbar_wait(smem_u32(&sh->full[s]), (last / S) & 1u);
    }
  }
  __syncwarp();
}

template <class P>
__device__ void role_transpose(const P &p, uint8_t *base, Shared *sh, int r) {
  constexpr int S = P::S;
  volatile int *abort = &sh->abort;
  uint32_t g = 0;
  bool run = !*abort;
  for (int t = blockIdx.x; run && t < p.ntiles; t += gridDim.x) {
    const auto T = p.tile(t);
    const int ns = p.nsub(T);
    for (int sub = 0; run && sub < ns; ++sub) {
      const int nk = p.nchunks(T, sub);
      for (int kc = 0; kc < nk; ++kc, ++g) {
        const int s = (int)(g % S);
        const uint32_t u = g / S;
        if (!wait_or_abort(smem_u32(&sh->full[s]), u & 1u, abort, sh->wait_ns)) {
          run = false;
          break;
        }
#pragma unroll
        for (int w = 0; w < P::NW; ++w) {
          const float *raw = reinterpret_cast<const float *>(stage_raw<P>(base, s, w));
          uint8_t *A = stage_A<P>(base, s, w);
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            uint4 q;
            if constexpr (P::BF16) {
              uint32_t h[4];
#pragma unroll
              for (int i = 0; i < 4; ++i) {
                const int j = c * 8 + 2 * i;
                __nv_bfloat162 b2 = __floats2bfloat162_rn(raw[j * MT + r], raw[(j + 1) * MT + r]);
                h[i] = *reinterpret_cast<uint32_t *>(&b2);
              }
              q = make_uint4(h[0], h[1], h[2], h[3]);
            } else {
              uint32_t h[4];
#pragma unroll
              for (int i = 0; i < 4; ++i) {
                const int j = c * 4 + i;
                h[i] = to_tf32(raw[j * MT + r]);
              }
              q = make_uint4(h[0], h[1], h[2], h[3]);
            }
            *reinterpret_cast<uint4 *>(A + sw128_off(r, c)) = q;
          }
        }
        fence_proxy_async();
        mbar_arrive(smem_u32(&sh->afull[s]));
      }
    }
  }
}

template <class P>
__device__ void role_mma(const P &p, uint8_t *base, Shared *sh, uint32_t tmem) {
  constexpr int S = P::S;
  volatile int *abort = &sh->abort;
  uint32_t g = 0, tc = 0;
  bool run = !*abort;
  for (int t = blockIdx.x; run && t < p.ntiles; t += gridDim.x) {
    const auto T = p.tile(t);
    const int ns = p.nsub(T);
    for (int sub = 0; run && sub < ns; ++sub, ++tc) {
      const int b = (int)(tc & 1u);
      const uint32_t ub = tc >> 1;
      if (tc >= 2 && !wait_or_abort(smem_u32(&sh->acce[b]), (ub - 1) & 1u, abort, sh->wait_ns)) {
        run = false;
        break;
      }
      tc_fence_after();
      const int nk = p.nchunks(T, sub);
      const uint32_t idesc = make_idesc(P::BF16, MT, p.ncol(T, sub));
      for (int kc = 0; kc < nk; ++kc, ++g) {
        const int s = (int)(g % S);
        const uint32_t u = g / S;
        if (!wait_or_abort(smem_u32(&sh->afull[s]), u & 1u, abort, sh->wait_ns)) {
          run = false;
          break;
        }
        tc_fence_after();
        const uint64_t bd = sw128_desc(smem_u32(stage_B<P>(base, s)));
#pragma unroll
        for (int w = 0; w < P::NW; ++w) {
          const uint64_t ad = sw128_desc(smem_u32(stage_A<P>(base, s, w)));
#pragma unroll
          for (int j = 0; j < 4; ++j)   // K-step j: 32 bytes of every K-major row
            mma<P::BF16>(tmem + (uint32_t)(b * 256) + p.dcol(w), ad + (uint64_t)(2 * j), bd + (uint64_t)(2 * j),
                         idesc, (kc | j) != 0);
        }
        mma_commit(smem_u32(&sh->empty[s]));
      }
      if (!run) break;
      mma_commit(smem_u32(&sh->accf[b]));
    }
  }
  // no MMA may still be writing the tensor memory when it is freed
  mma_commit(smem_u32(&sh->drain));
  mbar_wait(smem_u32(&sh->drain), 0);
}

template <class P>
__device__ void role_epilogue(const P &p, Shared *sh, uint32_t tmem, int warp, int lane) {
  volatile int *abort = &sh->abort;
  const int q = warp & 3, part = (warp - WARP_EPI0) >> 2;
  uint32_t tc = 0;
  bool run = __shfl_sync(0xffffffffu, *abort, 0) == 0;   // warp-uniform
  for (int t = blockIdx.x; run && t < p.ntiles; t += gridDim.x) {
    const auto T = p.tile(t);
    const int ns = p.nsub(T);
    for (int sub = 0; sub < ns; ++sub, ++tc) {
      const int b = (int)(tc & 1u);
      const uint32_t ub = tc >> 1;
      if (!warp_wait(smem_u32(&sh->accf[b]), ub & 1u, abort, lane, sh->wait_ns)) {
        run = false;
        break;
      }
      tc_fence_after();
      p.epilogue(T, sub, tmem + (uint32_t)(b * 256) + ((uint32_t)(q * 32) << 16), q, part, lane,
                 p.nchunks(T, sub) > 0);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&sh->acce[b]));
    }
  }
}

template <class P>
__global__ void __launch_bounds__(threads_for(P::NEPI), 1) k_tc_stream(const __grid_constant__ P p, int *status, uint64_t wait_ns,
                                                                     int probe) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *base = align1024(smem_raw);
  Shared *sh = reinterpret_cast<Shared *>(base + (size_t)P::S * Geo<P>::STAGE);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < P::S; ++s) {
      mbar_init(smem_u32(&sh->full[s]), 1);   // one arrival carrying the byte count
      mbar_init(smem_u32(&sh->afull[s]), NXP * 32);
      mbar_init(smem_u32(&sh->empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&sh->accf[b]), 1);
      mbar_init(smem_u32(&sh->acce[b]), P::NEPI);
    }
    mbar_init(smem_u32(&sh->drain), 1);
    sh->wait_ns = wait_ns;
    sh->abort = (*reinterpret_cast<volatile int *>(status) != 0) ? 1 : 0;   // an earlier CTA gave up
    if (probe && !sh->abort) {
      // failure-path probe: wait on status[1], a word nothing sets, before any copy or
      // MMA is issued; the bounded wait runs out and every role of the CTA gives up
      const volatile int *gate = status + 1;
      const uint64_t t0 = gtimer();
      while (*gate == 0) {
        if (gtimer() - t0 > wait_ns) {
          sh->abort = 1;
          break;
        }
      }
    }
    fence_barrier_init();
    fence_proxy_async();
  }
  if (warp == WARP_MMA) {
    __syncwarp();
    tmem_alloc(smem_u32(&sh->taddr), TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sh->taddr;

  if (warp == WARP_LOAD) {
    role_loader<P>(p, base, sh, lane);
  } else if (warp == WARP_IDLE) {
  } else if (warp == WARP_MMA) {
    if (lane == 0) role_mma<P>(p, base, sh, tmem);
    __syncwarp();
  } else if (warp < WARP_XP0 + NXP) {
    role_transpose<P>(p, base, sh, threadIdx.x - 32 * WARP_XP0);
  } else {
    role_epilogue<P>(p, sh, tmem, warp, lane);
  }

  tc_fence_before();
  __syncthreads();
  if (warp == WARP_MMA) {
    __syncwarp();
    tmem_dealloc(tmem, TMEM_COLS);
  }
  if (threadIdx.x == 0 && sh->abort) atomicExch(status, 1);
}

}  // namespace tcs
}  // namespace pawfe
