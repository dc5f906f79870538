// Operator application on the GPU (Sec. 4.3, Fig. computing AX):
//   extraction (gather of cell blocks) -> cell-local dense product ->
//   assembly (scatter-add), plus the atom-centred nonlocal parts
//   P^a D^a P^a^T X (Eq. FE nonlocal contribution) and the approximate
//   inverse overlap (Eq. Sinvapprox).
//
// Layout: multivectors are DoF-major with the vector index fastest
// (X[dof * ld + j]), so a cell gather reads, for each of the cell's nodes, one
// contiguous run of vector values: fully coalesced, and the scatter-add of a
// node row is a coalesced run of atomics.
#include <algorithm>

#include "common.cuh"

namespace pawfe {

// ============================================================== cell product (SIMT)
// One block per (cell, vector tile).  The gathered block X_e (nc x VT) stays in
// shared memory; the cell matrix streams through in NT x KT tiles; every
// thread owns a TM x TN register tile of the output; the output tile is
// scatter-added to the global rows of the cell's nodes.
template <typename T, int NT, int VT, int TM, int TN, int KT>
__global__ void __launch_bounds__((NT / TM) * (VT / TN))
k_cell_simt(const T *__restrict__ mats, long long stride, int nc, const int *__restrict__ cell_dofs,
            const T *__restrict__ X, int ldx, T *__restrict__ Y, int ldy, int ncols, T alpha,
            const double *__restrict__ colscale) {
  constexpr int NTHR = (NT / TM) * (VT / TN);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *Xs = reinterpret_cast<T *>(smem_raw);             // [nc][VT]
  T *Hs = Xs + (size_t)nc * VT;                        // [KT][NT + 1]
  int *dofs = reinterpret_cast<int *>(Hs + KT * (NT + 1));
  const int tid = threadIdx.x;
  const int e = blockIdx.x;
  const int v0 = blockIdx.y * VT;
  const T *A = mats + (long long)e * stride;
  for (int i = tid; i < nc; i += NTHR) dofs[i] = cell_dofs[(size_t)e * nc + i];
  __syncthreads();
  for (int idx = tid; idx < nc * VT; idx += NTHR) {
    const int k = idx / VT, v = idx - k * VT;
    Xs[idx] = (v0 + v < ncols) ? X[(size_t)dofs[k] * ldx + v0 + v] : T(0);
  }
  const int tx = tid % (VT / TN), ty = tid / (VT / TN);
  for (int n0 = 0; n0 < nc; n0 += NT) {
    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
    for (int k0 = 0; k0 < nc; k0 += KT) {
      __syncthreads();
      for (int idx = tid; idx < NT * KT; idx += NTHR) {
        const int nn = idx / KT, kk = idx - nn * KT;
        const int n = n0 + nn, k = k0 + kk;
        Hs[kk * (NT + 1) + nn] = (n < nc && k < nc) ? A[(size_t)n * nc + k] : T(0);
      }
      __syncthreads();
      const int kmax = min(KT, nc - k0);
      for (int kk = 0; kk < kmax; ++kk) {
        T a[TM], b[TN];
#pragma unroll
        for (int i = 0; i < TM; ++i) a[i] = Hs[kk * (NT + 1) + ty * TM + i];
#pragma unroll
        for (int j = 0; j < TN; ++j) b[j] = Xs[(size_t)(k0 + kk) * VT + tx * TN + j];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int n = n0 + ty * TM + i;
      if (n >= nc) continue;
      const size_t base = (size_t)dofs[n] * ldy;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int v = v0 + tx * TN + j;
        if (v < ncols) {
          const T s = colscale ? T(colscale[v]) * alpha : alpha;
          atomicAdd(&Y[base + v], s * acc[i][j]);
        }
      }
    }
  }
}

template <typename T>
struct CellCfg;
template <>
struct CellCfg<double> {
  static constexpr int NT = 64, VT = 32, TM = 4, TN = 2, KT = 16;
};
template <>
struct CellCfg<float> {
  static constexpr int NT = 64, VT = 64, TM = 4, TN = 4, KT = 16;
};

template <typename T>
void cell_apply_simt(paw_context *c, const T *mats, long long stride, const T *X, int ldx, T *Y,
                     int ldy, int ncols, double alpha, const double *colscale, cudaStream_t s) {
  if (ncols <= 0) return;
  using C = CellCfg<T>;
  constexpr int NTHR = (C::NT / C::TM) * (C::VT / C::TN);
  auto kern = k_cell_simt<T, C::NT, C::VT, C::TM, C::TN, C::KT>;
  const size_t shm = sizeof(T) * ((size_t)c->nc * C::VT + C::KT * (C::NT + 1)) + sizeof(int) * c->nc;
  static size_t configured = 0;
  if (shm > configured) {
    PAW_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    configured = shm;
  }
  dim3 grid(c->ncells, (ncols + C::VT - 1) / C::VT);
  kern<<<grid, NTHR, shm, s>>>(mats, stride, c->nc, c->cell_dofs.as<int>(), X, ldx, Y, ldy, ncols,
                               (T)alpha, colscale);
  PAW_LAUNCH_CHECK("k_cell_simt");
}

template void cell_apply_simt<double>(paw_context *, const double *, long long, const double *, int,
                                      double *, int, int, double, const double *, cudaStream_t);
template void cell_apply_simt<float>(paw_context *, const float *, long long, const float *, int,
                                     float *, int, int, double, const double *, cudaStream_t);

// ============================================================== elementwise
template <typename T>
__global__ void k_zero_block(T *Y, int64_t rows, int ncols, int ld) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.y + threadIdx.y;
  const int v = blockIdx.y * blockDim.x + threadIdx.x;
  if (i < rows && v < ncols) Y[i * ld + v] = T(0);
}

template <typename T>
void zero_block(T *Y, int64_t rows, int ncols, int ld, cudaStream_t s) {
  if (ncols <= 0 || rows <= 0) return;
  if (ld == ncols) {
    PAW_CUDA(cudaMemsetAsync(Y, 0, sizeof(T) * rows * ncols, s));
    return;
  }
  dim3 blk(32, 8);
  dim3 g((unsigned)((rows + 7) / 8), (ncols + 31) / 32);
  k_zero_block<T><<<g, blk, 0, s>>>(Y, rows, ncols, ld);
  PAW_LAUNCH_CHECK("k_zero_block");
}
template void zero_block<double>(double *, int64_t, int, int, cudaStream_t);
template void zero_block<float>(float *, int64_t, int, int, cudaStream_t);

template <typename T>
__global__ void k_scale_rows(const T *X, int ldx, T *Y, int ldy, int64_t rows, int ncols, const T *rs) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.y + threadIdx.y;
  const int v = blockIdx.y * blockDim.x + threadIdx.x;
  if (i < rows && v < ncols) Y[i * ldy + v] = rs[i] * X[i * ldx + v];
}

template <typename T>
void scale_rows(const T *X, int ldx, T *Y, int ldy, int64_t rows, int ncols, const T *rowscale,
                cudaStream_t s) {
  if (ncols <= 0 || rows <= 0) return;
  dim3 blk(32, 8);
  dim3 g((unsigned)((rows + 7) / 8), (ncols + 31) / 32);
  k_scale_rows<T><<<g, blk, 0, s>>>(X, ldx, Y, ldy, rows, ncols, rowscale);
  PAW_LAUNCH_CHECK("k_scale_rows");
}
template void scale_rows<double>(const double *, int, double *, int, int64_t, int, const double *,
                                 cudaStream_t);
template void scale_rows<float>(const float *, int, float *, int, int64_t, int, const float *,
                                cudaStream_t);

// ============================================================== composed operators
template <typename T>
static const T *HeMats(paw_context *c) { return c->He32.as<T>(); }
template <typename T>
static const T *MeMats(paw_context *c) { return c->Me32.as<T>(); }
template <typename T>
static const T *MdInv(paw_context *c);
template <>
const double *MdInv<double>(paw_context *c) { return c->md_inv64.as<double>(); }
template <>
const float *MdInv<float>(paw_context *c) { return c->md_inv32.as<float>(); }

// Local part H_loc X (Eq. FEM Ham entries) accumulated into Y with factor alpha:
// FP64 through the sum-factorised cell kernel, FP32 through the SIMT or
// tensor-core cell-matrix kernels.
template <typename T>
void local_H(paw_context *c, paw_precision prec, const T *X, int ldx, T *Y, int ldy, int ncols, double alpha,
             cudaStream_t s) {
  // A = 1/2 K + V + 1/2 |k|^2 M on every column (the |k|^2 term is in H^e and in cM)
  if constexpr (sizeof(T) == 8) {
    local_sf(c, X, ldx, Y, ldy, ncols, alpha, 1.0, 1.0, c->kmass, nullptr, s);
  } else {
    if (prec == PAW_TF32 || prec == PAW_BF16)
      cell_apply_tc(c, prec, X, ldx, Y, ldy, ncols, (float)alpha, s);
    else
      cell_apply_simt<T>(c, HeMats<T>(c), (long long)c->nc * c->nc, X, ldx, Y, ldy, ncols, alpha, nullptr, s);
  }
  if (!c->kc) return;
  // Bloch term of H_loc(k) = A - i B on the split block [Re | Im]:
  // Y_re += alpha B X_im, Y_im -= alpha B X_re
  const int nb = ncols / 2;
  if constexpr (sizeof(T) == 8) {
    bloch_sf(c, X + nb, ldx, Y, ldy, nb, alpha, s);
    bloch_sf(c, X, ldx, Y + nb, ldy, nb, -alpha, s);
  } else {
    if (prec == PAW_TF32 || prec == PAW_BF16) {
      bloch_apply_tc(c, prec, X + nb, ldx, Y, ldy, nb, (float)alpha, s);
      bloch_apply_tc(c, prec, X, ldx, Y + nb, ldy, nb, -(float)alpha, s);
    } else {
      cell_apply_simt<T>(c, c->Bk32.as<T>(), 0, X + nb, ldx, Y, ldy, nb, alpha, nullptr, s);
      cell_apply_simt<T>(c, c->Bk32.as<T>(), 0, X, ldx, Y + nb, ldy, nb, -alpha, nullptr, s);
    }
  }
}

template <typename T>
void op_H(paw_context *c, paw_precision prec, const T *X, int ldx, T *Y, int ldy, int ncols,
          cudaStream_t s) {
  zero_block<T>(Y, c->ndof, ncols, ldy, s);
  local_H<T>(c, prec, X, ldx, Y, ldy, ncols, 1.0, s);
  if (c->nown_pairs > 0) {
    c->ws_W.ensure(sizeof(T) * (size_t)c->natoms * c->npad * ncols, &c->dev_bytes);
    nl_project<T>(c, prec, X, ldx, ncols, nullptr, c->DH64.as<double>(), 1.0, c->ws_W.as<T>(), s);
    nl_expand<T>(c, prec, c->ws_W.as<T>(), ncols, Y, ldy, nullptr, s);
  }
}

template <typename T>
void op_S(paw_context *c, const T *X, int ldx, T *Y, int ldy, int ncols, cudaStream_t s) {
  zero_block<T>(Y, c->ndof, ncols, ldy, s);
  if constexpr (sizeof(T) == 8)
    local_sf(c, X, ldx, Y, ldy, ncols, 1.0, 0.0, 0.0, 1.0, nullptr, s);
  else
    cell_apply_simt<T>(c, MeMats<T>(c), 0, X, ldx, Y, ldy, ncols, 1.0, nullptr, s);
  if (c->nown_pairs > 0) {
    c->ws_W.ensure(sizeof(T) * (size_t)c->natoms * c->npad * ncols, &c->dev_bytes);
    const paw_precision prec = sizeof(T) == 8 ? PAW_FP64 : PAW_FP32;
    nl_project<T>(c, prec, X, ldx, ncols, nullptr, c->DS64.as<double>(), 1.0, c->ws_W.as<T>(), s);
    nl_expand<T>(c, prec, c->ws_W.as<T>(), ncols, Y, ldy, nullptr, s);
  }
}

void op_pair(paw_context *c, int which, const double *X, int ldx, double *Y, int ldy, int ncols, cudaStream_t s) {
  PAW_REQUIRE(!c->kc && (which == 0 || which == 1), PAW_ERR_UNSUPPORTED,
              "pair-of-FP32 arithmetic covers H and S of real vectors");
  zero_block<double>(Y, c->ndof, ncols, ldy, s);
  if (which == 0)
    local_sf(c, X, ldx, Y, ldy, ncols, 1.0, 1.0, 1.0, c->kmass, nullptr, s, true);
  else
    local_sf(c, X, ldx, Y, ldy, ncols, 1.0, 0.0, 0.0, 1.0, nullptr, s, true);
  const double *C = (which == 0) ? c->DH64.as<double>() : c->DS64.as<double>();
  nl_residual_pair(c, X, ldx, ncols, C, nullptr, nullptr, Y, ldy, s);
}

template <typename T>
void op_Sinv(paw_context *c, paw_precision prec, const T *X, int ldx, T *Y, int ldy, int ncols, cudaStream_t s) {
  if (c->nown_pairs == 0) {
    scale_rows<T>(X, ldx, Y, ldy, c->ndof, ncols, MdInv<T>(c), s);
    return;
  }
  c->ws_W.ensure(sizeof(T) * (size_t)c->natoms * c->npad * ncols, &c->dev_bytes);
  nl_project<T>(c, prec, X, ldx, ncols, MdInv<T>(c), c->DSinv64.as<double>(), 1.0, c->ws_W.as<T>(), s);
  nl_sinv_out<T>(c, prec, c->ws_W.as<T>(), ncols, X, ldx, Y, ldy, MdInv<T>(c), s);
}

template void local_H<double>(paw_context *, paw_precision, const double *, int, double *, int, int, double,
                              cudaStream_t);
template void local_H<float>(paw_context *, paw_precision, const float *, int, float *, int, int, double,
                             cudaStream_t);
template void op_H<double>(paw_context *, paw_precision, const double *, int, double *, int, int, cudaStream_t);
template void op_H<float>(paw_context *, paw_precision, const float *, int, float *, int, int, cudaStream_t);
template void op_S<double>(paw_context *, const double *, int, double *, int, int, cudaStream_t);
template void op_S<float>(paw_context *, const float *, int, float *, int, int, cudaStream_t);
template void op_Sinv<double>(paw_context *, paw_precision, const double *, int, double *, int, int,
                              cudaStream_t);
template void op_Sinv<float>(paw_context *, paw_precision, const float *, int, float *, int, int, cudaStream_t);

}  // namespace pawfe
