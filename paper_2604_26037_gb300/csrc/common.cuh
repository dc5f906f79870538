// Internal declarations shared by the translation units of libpawfe.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <cstdint>
#include <string>
#include <vector>

#include "paw_fe.h"

namespace pawfe {

// Atoms whose projectors reach the owned nodes of one cell: the owner-cell
// kernels stage the atom list of a cell in shared memory (checked at set-up).
constexpr int PAIRS_PER_CELL_MAX = 192;
// Projectors per group of the FP64 / pair-of-FP32 owner-cell nonlocal kernels: a
// node's projectors (stored by decreasing width) are multiplied group by group up
// to the last group with a nonzero value on the node (own_lg, own_cnt).
constexpr int OWN_GROUP = 2;

// ---------------------------------------------------------------- errors
struct Error {
  paw_status code;
  std::string msg;
};

void set_error(const std::string &msg);
paw_status fail(paw_status code, const std::string &msg);

#define PAW_CUDA(call)                                                        \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) {                                                  \
      throw ::pawfe::Error{e_ == cudaErrorMemoryAllocation ? PAW_ERR_NO_MEMORY \
                                                           : PAW_ERR_CUDA,     \
                           std::string(#call) + ": " + cudaGetErrorString(e_)}; \
    }                                                                         \
  } while (0)

// every kernel launch is followed by PAW_LAUNCH_CHECK, which also counts it
extern int64_t g_launch_count;

#define PAW_LAUNCH_CHECK(what)                                                \
  do {                                                                        \
    ++::pawfe::g_launch_count;                                                \
    cudaError_t e_ = cudaGetLastError();                                      \
    if (e_ != cudaSuccess)                                                    \
      throw ::pawfe::Error{PAW_ERR_CUDA,                                      \
                           std::string("launch ") + (what) + ": " +           \
                               cudaGetErrorString(e_)};                       \
  } while (0)

#define PAW_REQUIRE(cond, code, msg)                                          \
  do {                                                                        \
    if (!(cond)) throw ::pawfe::Error{(code), (msg)};                         \
  } while (0)

// ---------------------------------------------------------------- TMA
// Tensor map of a row-major FP32 block (rows x cols, row pitch ld elements,
// 16-byte aligned base, ld a multiple of 4) read by the row-gather copies of
// the persistent tcgen05 kernels: box = 128 columns x 1 row (tile::gather4
// fetches four such rows per instruction); columns past cols read as zero.
void encode_row_map(CUtensorMap *map, const float *base, int64_t rows, int cols, int ld);

// ---------------------------------------------------------------- memory
// Device buffer owned by a context.  Grows, never shrinks.
struct DevBuf {
  void *ptr = nullptr;
  size_t bytes = 0;
  void ensure(size_t nbytes, int64_t *counter);
  void release(int64_t *counter);
  template <typename T> T *as() const { return static_cast<T *>(ptr); }
};

// Per-precision cell-matrix storage used by the tensor-core kernels.
struct TcMats {
  DevBuf He;        // per-cell H^e, pre-tiled for the tcgen05 operand layout
  DevBuf Me;        // shared mass matrix, same layout
  int valid = 0;
  int kchunks = 0;  // K-chunks of 128 bytes
  int ntile = 0;    // rows of one N tile (multiple of 16)
  int ntiles = 0;   // N tiles per cell
  size_t chunk_bytes = 0;   // bytes of one (ntile x 128 B) chunk
  size_t cell_bytes = 0;    // bytes of one cell (ntiles * kchunks chunks)
};

// Projector blocks pre-arranged for the tcgen05 nonlocal kernels (TF32,
// 128-byte-swizzled K-major tiles, built once from the owner-cell values).
struct NlTcMats {
  DevBuf projB;     // projection B operand: per pair tile [K-chunk of owned nodes][pair x projector rows]
  DevBuf projBs;    // the same with M_D^-1 of each node folded in
  DevBuf expB;      // expansion B operand: per cell [node tile][K-chunk of pairs x projectors][node rows]
  DevBuf eoff;      // int32 ncells+1: prefix of the expansion K-chunks of each cell
  DevBuf mdo;       // M_D^-1 in owner order: nh * ntile floats per cell
  DevBuf odof;      // DoF indices in owner order (int32, same layout)
  int valid = 0;
  int kc_own = 0;   // K-chunks (32 nodes) over the owned nodes
  int ppt = 0;      // pairs per projection N tile (256 / npad)
  int ppc = 0;      // pairs per expansion K-chunk (32 / npad)
  int ntile = 0;    // owned nodes per expansion N tile (multiple of 16, <= 128)
  int nh = 0;       // expansion N tiles per cell
  int64_t exp_chunks = 0;
};

// Scratch of the nonlocal helpers (per-atom sums, per-pair partials,
// coefficients).  A context has two sets: step 2 of the next block, issued on
// a side stream while the current block's loop runs, uses the second.
struct NlScratch {
  DevBuf partial, pp, W2, Wx2;
};

// Pinned host slots for the scalar images of paw_cheb_filter's blocks.  A
// slot is rewritten only once the GPU has passed the copies that read it
// (its event), so the filter enqueues block after block without waiting for
// the stream; the host blocks only when it runs a whole ring ahead.
struct HostSlot {
  void *host = nullptr;
  void *dev = nullptr;   // the same memory as the device reads it (mapped)
  size_t bytes = 0;
  cudaEvent_t done = nullptr;
  bool pending = false;
};
struct HostRing {
  std::vector<HostSlot> slots;
  size_t next = 0;
};

// Phase timing (paw_profile_enable / paw_profile_read)
struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  struct Mark {
    int phase;
    cudaEvent_t a, b;
  };
  std::vector<Mark> marks;
  int64_t launches[PAW_NPHASES] = {0};
  int64_t launch0 = 0;
};

}  // namespace pawfe

// ---------------------------------------------------------------- context
struct paw_context {
  // mesh and discretisation
  int n = 0, p = 0, np1 = 0, nc = 0, nq1 = 0, nq = 0, N1 = 0, ncells = 0;
  int64_t ndof = 0;
  double L = 0, h = 0, detJ = 0;
  int natoms = 0, npj = 0;
  // Bloch wavevector: kc = 1 when k != 0.  Complex multivectors are then
  // processed as real blocks of 2 ncols columns [Re | Im]; the projectors
  // C^{a,k} are stored as npjr = 2 npj real projectors [Re C | Im C]
  // (npjr = npj at k = 0) and the per-atom couplings act on complex
  // coefficients.
  int kc = 0, npjr = 0;
  double kvec[3] = {0.0, 0.0, 0.0};
  double kmass = 0.0;                         // 1/2 |k|^2
  std::vector<double> C1s;                    // 1D skew matrix (C1 - C1^T)/2, C1[a][b] = int l_a l_b' dxi
  pawfe::DevBuf Bk64, Bk32;                   // Bloch cell matrix B^e = sum_d k_d G^e_d (nc x nc, all cells)
  std::vector<int> shell_l;                   // shells in internal order (decreasing width)
  std::vector<double> shell_w;
  std::vector<int> proj_ext;                  // internal projector -> caller's projector index
  pawfe::DevBuf proj_ext_dev;
  std::vector<double> pos, D, dS, G, Dsinv;   // host copies
  std::vector<double> vg_c, vg_A, vg_w;       // local potential Gaussians
  paw_options opts{};
  int64_t dev_bytes = 0;

  // host tables (built by the library's own FE code)
  std::vector<double> K_ref, M_ref, Nq, wq;   // nc*nc, nc*nc, nq*nc, nq
  std::vector<double> gq;                     // (p+2) Gauss nodes on [-1,1]
  std::vector<double> M1, D1, phiq;           // 1D mass, stiffness ((p+1) Gauss), Lagrange at (p+2) Gauss

  // device operator data
  pawfe::DevBuf cell_dofs;   // int32 ncells*nc
  pawfe::DevBuf md_inv64, md_inv32;           // 1 / M_D
  pawfe::DevBuf He64, He32;                   // ncells*nc*nc
  pawfe::DevBuf Me64, Me32, K64;              // nc*nc
  pawfe::DevBuf Nq64, wq64;                   // nq*nc, nq
  pawfe::DevBuf Vq;                           // ncells*nq
  pawfe::DevBuf wV;                           // ncells*nq: w_q detJ V_q (sum-factorised V^e)
  int wV_valid = 0;
  int wVx2_valid = 0;                          // wVx2 = wV as pairs of FP32 numbers
  pawfe::DevBuf wVx2;
  pawfe::TcMats tc_tf32, tc_bf16;
  pawfe::TcMats tc_bk_tf32, tc_bk_bf16;       // tcgen05 images of B^e (one shared matrix)
  pawfe::NlTcMats nltc;

  // projectors: atom-major support entries
  int64_t nent = 0;                           // sum_a |supp_a| (node entries)
  int64_t npairs = 0;                         // (cell, atom) support pairs
  std::vector<int64_t> ent_off;               // natoms+1
  pawfe::DevBuf ent_dof;                      // int32 nent
  pawfe::DevBuf P64, P32;                     // nent * npj
  // owner-cell view: every DoF is owned by exactly one cell (its local indices
  // a, b, c < p); pair k = (cell, atom) lists the atoms whose P^a is nonzero on
  // an owned node of the cell, with the assembled values P^a at those nodes.
  int npad = 16;                              // npj rounded up to 16
  int own = 0;                                // owned nodes per cell = p^3
  int64_t nown_pairs = 0;
  int max_own_pairs = 0;                      // largest pair count of one cell
  pawfe::DevBuf own_off;                      // int32 ncells+1
  pawfe::DevBuf own_atom;                     // int32 nown_pairs
  pawfe::DevBuf ownP64, ownP32;               // nown_pairs * own * npad
  pawfe::DevBuf ownPx2;                       // the same as pairs of FP32 numbers (built on first use)
  pawfe::DevBuf own_ngrp;                     // int32 per pair: projector groups of 4 with a nonzero value
  // per pair and owned node o: index of the last projector group of 4 with a
  // nonzero value at o (-1: none); the owned nodes sorted by that index
  // (descending) and, per group g, the number of nodes whose index is >= g.
  // The FP64 kernels multiply only groups that can be nonzero on a node.
  pawfe::DevBuf own_lg;                       // int8  nown_pairs * own
  pawfe::DevBuf own_sidx;                     // int16 nown_pairs * own
  pawfe::DevBuf own_cnt;                      // int32 nown_pairs * npad/OWN_GROUP
  int64_t proj_nnz = 0;                       // nonzero (owned node, projector) entries over all pairs
  pawfe::DevBuf apair_off, apair;             // atom-major list of the pairs (int32)
  // atom-pair Gram blocks G_ab = P^a^T M_D^-1 P^b for atoms with common support
  // nodes (CSR over atoms, a included); lets P^T Shat^-1 R follow from P^T M_D^-1 R
  pawfe::DevBuf gnb_off, gnb_atom;            // int32 natoms+1, ngpairs
  pawfe::DevBuf Gfull, Gfull32;               // FP64 / FP32 ngpairs * npad * npad
  // FP32 coupling of the filter loop (k = 0): per Gram slot s (atoms a, b) the block
  // F_s = D_H,a (delta_ab I - G_ab DeltaSinv_b), and DeltaSinv per atom, npad x npad each
  pawfe::DevBuf Fsh32, DSinv32;
  int64_t ngpairs = 0;
  std::vector<double> mdinv_h;                // 1 / M_D on the host
  // couplings (FP64, natoms*npj*npj)
  pawfe::DevBuf DH64, DS64, DSinv64;

  // workspaces
  pawfe::DevBuf ws_W, ws_RX, ws_RY, ws_T, ws_Y0f, ws_Y0lo;
  pawfe::DevBuf ws_colscale, ws_red, ws_vec;
  pawfe::NlScratch scr_main, scr_side;       // nonlocal scratch sets (partial = U, pp, W2, Wx2)
  pawfe::NlScratch *scr = &scr_main;         // the set the helpers use while work is issued
  // per-block buffers, by block parity (two blocks in flight when step 2 of the
  // next block overlaps the loop of the current one): Y = HX - SX Lambda (FP64)
  // and the scalar images of the block (FP64 -Lambda, Lambda_Y, alpha Lambda_Y;
  // FP32 hi/lo words)
  pawfe::DevBuf ws_Y0p[2], ws_lamp[2], ws_cfp[2];
  int lean = 0;      // 1: persistent cell/projection kernels in their half-shared-memory form
  int sf_lean = 0;   // 1: FP64 sum-factorised kernel in its 4-vector form
  cudaStream_t s_loop = nullptr, s_side = nullptr;   // internal streams of the overlapped filter
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  pawfe::DevBuf ws_HX, ws_SX, ws_Hp, ws_Sp, ws_eig, ws_solver, ws_info, ws_rot;
  pawfe::DevBuf ws_gram;                      // split partial tiles of the RR projection
  pawfe::DevBuf ws_cg;                        // real 2N x 2N Gram / rotation matrix (k != 0)
  pawfe::DevBuf ws_cx, ws_cy;                 // split [Re | Im] copies of complex arguments (k != 0)
  pawfe::DevBuf ws_cxp[2], ws_cyp[2];         // the same per block parity (overlapped filter at k != 0)

  // tensor-core kernel family: 0 persistent warp-specialised where the layout
  // allows it, 1 one-CTA-per-tile kernels; grid_cap > 0 limits the CTAs of a
  // persistent launch (instances sharing the GPU)
  int tc_variant = 0, grid_cap = 0;
  pawfe::DevBuf status_dev;                   // int[2]: [0] set by a kernel whose bounded wait expired,
                                              // [1] a word nothing sets (wait probe, paw_set_wait_limit)
  uint64_t wait_ns = 2000000000ull;           // give-up bound of the pipeline waits of tensor-core kernels
  int wait_probe = 0;                         // 1: persistent tensor-core launches first wait on status[1]
  pawfe::HostRing scal_ring;                  // pinned scalar images of paw_cheb_filter blocks

  cusolverDnHandle_t cusolver = nullptr;
  cudaStream_t last_stream = nullptr;
  pawfe::Profiler prof;
};

namespace pawfe {

// ---------------------------------------------------------------- setup.cu
void build_tables(paw_context *c);
void build_operators(paw_context *c, const paw_vloc *vloc);
void rebuild_hamiltonian(paw_context *c);
void build_couplings(paw_context *c);
// F_s and DeltaSinv in FP32 for the fused coupling of the filter loop (after
// build_couplings and after every change of D_H); synchronises the device
void build_couple_f(paw_context *c);

// ---------------------------------------------------------------- ops.cu
// Y += alpha * colscale[j] * (sum_e Q_e^T A_e Q_e X)  with A_e = mats + e*stride
template <typename T>
void cell_apply_simt(paw_context *c, const T *mats, long long stride, const T *X, int ldx,
                     T *Y, int ldy, int ncols, double alpha, const double *colscale,
                     cudaStream_t s);
// W[a] = coup_scale * coup[a] * P^a^T (rowscale .* X); W is natoms x npad x ncols
// prec PAW_TF32 / PAW_BF16 with T = float: tensor-core (tcgen05, TF32 operands)
// projection and expansion; otherwise SIMT in the arithmetic of T.
template <typename T>
void nl_project(paw_context *c, paw_precision prec, const T *X, int ldx, int ncols, const T *rowscale,
                const double *coup, double coup_scale, T *W, cudaStream_t s);
// Y[dof] += colscale[j] * sum_a P^a W[a]   (owner-cell expansion, no atomics)
template <typename T>
void nl_expand(paw_context *c, paw_precision prec, const T *W, int ncols, T *Y, int ldy,
               const double *colscale, cudaStream_t s);
// Y = M_D^-1 (X - sum_a P^a W[a])
template <typename T>
void nl_sinv_out(paw_context *c, paw_precision prec, const T *W, int ncols, const T *X, int ldx, T *Y,
                 int ldy, const T *mdinv, cudaStream_t s);
// W[a] = (D_H[a] + cs[j] dS[a]) P^a^T X  (nonlocal part of H X - S X Lambda, cs = -Lambda)
template <typename T>
void nl_project_residual(paw_context *c, const T *X, int ldx, int ncols, const double *cs, T *W,
                         cudaStream_t s);
// One projection per filter step: U = P^T M_D^-1 R_Y, W_S = Dsinv U and
// W_H = alpha D_H (U - G W_S) = alpha D_H P^T Shat^-1 R_Y (G: atom-pair Gram blocks)
template <typename T>
void nl_project_filter(paw_context *c, paw_precision prec, const T *RY, int ldr, int ncols, const T *mdinv,
                       double alpha, T *WS, T *WH, cudaStream_t s);
// T = M_D^-1 (R_Y - sum_a P^a W_S[a]);
// R_X = [-beta R_Y - gamma R_X + sum_a P^a W_H[a]] + c_j Y   with c_j = alpha Lambda_Y[j]
// FP32: Y given as hi/lo FP32 words (lo may be NULL), c_j as chi + clo, exact-product sum.
void nl_recurrence_f32(paw_context *c, paw_precision prec, const float *WS, const float *WH, int ncols,
                       const float *RY, float *RX, float *Tout, int ldr, const float *mdinv,
                       const float *Y0hi, const float *Y0lo, int ldy0, const float *chi, const float *clo,
                       double beta, double gamma, cudaStream_t s);
void nl_recurrence_f64(paw_context *c, const double *WS, const double *WH, int ncols,
                       const double *RY, double *RX, double *Tout, int ldr, const double *mdinv,
                       const double *Y0, int ldy0, const double *c64, double beta, double gamma,
                       cudaStream_t s);
// tensor-core owner-cell kernels (nonlocal_tc.cu), T = float, TF32 operands
bool nltc_supported(const paw_context *c);
void nltc_prepare(paw_context *c, cudaStream_t s);
// U[a][al][v] = sum over the pairs k of atom a of sum_o P[k][o][al] rowscale[o] X[o][v]:
// the persistent kernel reduces into U directly (FP32 reductions, returns true);
// the one-CTA-per-tile form writes per-pair partials PP[k][al][v] (returns false)
bool nltc_project(paw_context *c, const float *X, int ldx, int ncols, const float *rowscale, float *PP,
                  float *U, cudaStream_t s);
// nonlocal part of step 2 in pair-of-FP32 arithmetic (k = 0):
// Y += sum_a P^a (C^a + cs_j C2^a) P^a^T x_j (C2, cs may be NULL), X and Y FP64
void nl_residual_pair(paw_context *c, const double *X, int ldx, int ncols, const double *C, const double *C2,
                      const double *cs, double *Y, int ldy, cudaStream_t s);
// expansion with the output stage of mode (EXP_ADD / EXP_SINV / EXP_RECURRENCE)
struct ExpArgs;
void nltc_expand(paw_context *c, int mode, const ExpArgs &A, const float *W1, const float *W2, cudaStream_t s);
// FP64 sum-factorised local operator (sumfac.cu):
// Y += alpha * (cK K^e + cV V^e + (cM + cMcol[j]) M^e) X, cell by cell with assembly;
// pair32: the contractions in pair-of-FP32 arithmetic (f32x2.cuh), X and Y FP64
void local_sf(paw_context *c, const double *X, int ldx, double *Y, int ldy, int ncols, double alpha,
              double cK, double cV, double cM, const double *cMcol, cudaStream_t s, bool pair32 = false);
// FP64 sum-factorised Bloch term: Y += alpha * B X, B = sum_d k_d G_d cell by cell
// (G_d the skew cell form of int N_I dN_J/dx_d, Eq. hij), with assembly
void bloch_sf(paw_context *c, const double *X, int ldx, double *Y, int ldy, int ncols, double alpha,
              cudaStream_t s);
// local part of H, accumulated with factor alpha.  With k != 0, ncols is even
// and X, Y are split complex blocks [Re | Im] of ncols / 2 columns each:
// H_loc(k) = A - i B adds Y_re += alpha B X_im and Y_im -= alpha B X_re.
template <typename T>
void local_H(paw_context *c, paw_precision prec, const T *X, int ldx, T *Y, int ldy, int ncols,
             double alpha, cudaStream_t s);
template <typename T>
void zero_block(T *Y, int64_t rows, int ncols, int ld, cudaStream_t s);
template <typename T>
void scale_rows(const T *X, int ldx, T *Y, int ldy, int64_t rows, int ncols,
                const T *rowscale, cudaStream_t s);

// full operators into Y (overwrite); the element type is T
template <typename T>
void op_H(paw_context *c, paw_precision prec, const T *X, int ldx, T *Y, int ldy,
          int ncols, cudaStream_t s);
template <typename T>
void op_S(paw_context *c, const T *X, int ldx, T *Y, int ldy, int ncols,
          cudaStream_t s);
template <typename T>
void op_Sinv(paw_context *c, paw_precision prec, const T *X, int ldx, T *Y, int ldy, int ncols,
             cudaStream_t s);
// H X (which = 0) or S X (which = 1) in pair-of-FP32 arithmetic, FP64 data, k = 0
void op_pair(paw_context *c, int which, const double *X, int ldx, double *Y, int ldy, int ncols, cudaStream_t s);

// tensor-core cell products (cell_tc.cu)
void tc_prepare(paw_context *c, paw_precision prec, cudaStream_t s);
void cell_apply_tc(paw_context *c, paw_precision prec, const float *X, int ldx,
                   float *Y, int ldy, int ncols, float alpha, cudaStream_t s);
// the same with the one Bloch cell matrix B^e shared by every cell (k != 0)
void bloch_apply_tc(paw_context *c, paw_precision prec, const float *X, int ldx,
                    float *Y, int ldy, int ncols, float alpha, cudaStream_t s);
// argument checks shared by the entry points (api.cu).  pair_ok: the call
// takes PAW_F32X2 (paw_apply_H, paw_apply_S)
void check_prec(paw_precision prec, bool pair_ok = false);
void check_block_args(paw_context *c, const void *X, const void *Y, int ncols, int ldx, int ldy);
// device status word of the instance: 0 when no bounded wait of a tensor-core
// kernel expired since the last read, 1 when one did (read on the last stream,
// then cleared); -1 when it cannot be read
int read_status(paw_context *c);

// Algorithm 2 for one block of nb columns (api.cu).  cheb_plan fills the host
// scalar images hd (cheb_nd entries) and hf (cheb_nf entries); cheb_issue
// enqueues the transfer of those images and all kernels on stream s without
// any host synchronisation (capturable into a CUDA graph; hd and hf must stay
// valid until the stream has consumed them).  With hd_dev / hf_dev (the same
// memory, mapped pinned, as the device addresses it) a kernel reads the images;
// otherwise two cudaMemcpyAsync copy them.
struct ChebScalars {
  std::vector<double> al, be, ga;
  int nsteps = 0;
  size_t nd = 0, nf = 0;
};
size_t cheb_nd(int nb, int m);
size_t cheb_nf(int nb, int m);
void cheb_plan(int nb, int m, paw_bounds bd, const double *lam, ChebScalars &S, double *hd, float *hf);
void cheb_issue(paw_context *c, paw_precision prec, const double *X, int ldx, int nb, paw_bounds bd,
                const ChebScalars &S, const double *hd, const float *hf, double *Xo, int ldo, cudaStream_t s,
                const double *hd_dev = nullptr, const float *hf_dev = nullptr);

// RAII bracket of one phase of the filter (records events only when enabled)
struct PhaseScope {
  paw_context *c;
  int ph;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  int64_t l0 = 0;
  PhaseScope(paw_context *ctx, int phase, cudaStream_t st);
  ~PhaseScope();
};

// Rayleigh-Ritz contractions (rr.cu).  rr_gram: G[c * ldg + r] =
// sum_{i < K} A[i][r] B[i][c] for r < R, c < C (column-major G; lower: only
// tiles that reach the lower triangle, r >= c, are computed and written).
// rr_rotate: X <- X Q for M rows of N columns (Q column-major N x N), in FP64
// or mixed (diagonal of Q in FP64, the rest in FP32).  At k != 0:
// rr_gram_to_hermitian turns the real Gram matrix (2N x 2N) of interleaved
// complex columns into X^H Y (complex column-major), rr_complex_to_real the
// complex Q into its real 2N x 2N form.
void rr_gram(paw_context *c, const double *A, int lda, int R, const double *B, int ldb, int C, int64_t K, bool lower,
             double *G, int ldg, cudaStream_t s);
void rr_rotate(paw_context *c, double *X, int ld, int64_t M, int N, const double *Q, bool mixed, cudaStream_t s);
void rr_gram_to_hermitian(int N, const double *G, void *Ap, cudaStream_t s);
void rr_complex_to_real(int N, const void *Q, double *Qr, cudaStream_t s);

// small host linear algebra (setup.cu)
void jacobi_eigh(int n, std::vector<double> &A, std::vector<double> &evals,
                 std::vector<double> &evecs);
bool invert_small(int n, std::vector<double> &A);

}  // namespace pawfe
