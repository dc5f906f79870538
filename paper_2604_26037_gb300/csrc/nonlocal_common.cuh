// Definitions shared by the SIMT (nonlocal.cu) and tensor-core (nonlocal_tc.cu)
// forms of the owner-cell nonlocal expansion.
#pragma once

#include <cstdint>

namespace pawfe {

// fl32(b + c y) for c = ch + cl, y = yh + yl, with error-free FP32 steps.
__device__ __forceinline__ float add_product_df(float b, float ch, float cl, float yh, float yl) {
  // explicit round-to-nearest operations: no contraction into FMA may alter the two-sum
  const float th = __fmul_rn(ch, yh);
  const float te = fmaf(ch, yh, -th);                    // exact error of ch * yh
  const float tl = fmaf(ch, yl, fmaf(cl, yh, te));
  const float s = __fadd_rn(b, th);                      // two-sum of b and th
  const float bp = __fsub_rn(s, b);
  const float err = __fadd_rn(__fsub_rn(b, __fsub_rn(s, bp)), __fsub_rn(th, bp));
  return __fadd_rn(s, __fadd_rn(err, tl));
}

constexpr int EXP_ADD = 0, EXP_SINV = 1, EXP_RECURRENCE = 2;

struct ExpArgs {
  int n, p, N1;
  const int *own_off, *own_atom;
  const int *own_ngrp;           // per pair: groups of 4 projectors with nonzero values
  int ncols;
  const double *cs;              // ADD: per-column factor (may be NULL)
  const void *Xin;               // SINV: X; RECURRENCE: R_Y
  int ldx;
  void *Y;                       // ADD/SINV output; RECURRENCE: T
  int ldy;
  const void *mdinv;
  void *RX;                      // RECURRENCE: R_X (ld = ldx)
  const void *Y0, *Y0lo;         // RECURRENCE: Y (FP64) or its FP32 hi/lo split
  int ldy0;
  const double *c64;             // FP64 path: alpha * Lambda_Y per column
  const float *chi, *clo;        // FP32 path: the same, split in two FP32 words
  double beta, gamma;
  int vec_ok;                    // every row pointer above 16-byte aligned (set by own_expand)
};


// Offsets of the p^3 owned nodes of a cell relative to its first owned DoF
// (owned: local indices a, b, c < p on the (n p)^3 periodic lattice of pitch N1).
__host__ __device__ __forceinline__ int owned_offset(int o, int p, int N1) {
  const int a = o % p, b = (o / p) % p, cc = o / (p * p);
  return a + N1 * (b + N1 * cc);
}
__host__ __device__ __forceinline__ int64_t owned_base(int e, int n, int p, int N1) {
  const int cx = e % n, cy = (e / n) % n, cz = e / (n * n);
  return (int64_t)cx * p + (int64_t)N1 * ((int64_t)cy * p + (int64_t)N1 * ((int64_t)cz * p));
}

}  // namespace pawfe
