/*
 * paw_fe.h -- C ABI of the GB300 (sm_103a) PAW finite-element Chebyshev filter.
 *
 * The library implements the Chebyshev-filtering step of the residual-based
 * Chebyshev filtered subspace iteration (R-ChFSI) for the PAW generalised
 * eigenproblem H X = S X Lambda discretised with finite elements
 * (Algorithm 2 of the paper; Sec. 3.1 and Sec. 4.3-4.4), together with the
 * operators it is built from and the FP64 Rayleigh-Ritz step around it
 * (Algorithm 1, steps 4-6).
 *
 * Conventions
 * -----------
 * - Every call returns a paw_status; nothing throws or aborts across the ABI.
 *   paw_last_error() returns a message for the last failing call made by the
 *   calling thread (valid until that thread's next call).
 * - Multivectors are caller-owned DEVICE arrays, DoF-major with the vector
 *   index fastest: element (dof, j) of X is X[dof * ld + j], ld >= ncols.
 *   (A column block of a wider array is addressed by offsetting the pointer
 *   by the first column and passing the full row length as ld.)
 * - Element type follows the precision argument: double for PAW_FP64,
 *   float for PAW_FP32 / PAW_TF32 / PAW_BF16.
 * - Small descriptor arrays (positions, shells, coupling matrices,
 *   eigenvalues, bounds) are HOST arrays, copied or read during the call.
 * - Work is enqueued on the caller's CUDA stream (cudaStream_t passed as
 *   void*; NULL = legacy default stream).  Calls that return host results
 *   (eigenvalues, norms, bounds) synchronise that stream.  paw_cheb_filter
 *   returns as soon as its work is enqueued.  Consecutive calls on one
 *   handle share its workspaces: issue them on one stream (or order the
 *   streams yourself).
 * - Device-detected failures (a bounded wait of a tensor-core kernel that
 *   expired: its output is incomplete) are reported as PAW_ERR_TIMEOUT by
 *   paw_sync_status and by the next call on the handle that synchronises:
 *   paw_apply_H / paw_apply_Sinv_approx in PAW_TF32 or PAW_BF16,
 *   paw_rayleigh_ritz, paw_residuals.
 * - The library owns the device memory behind a handle (operator data and
 *   workspaces); it is freed by paw_destroy().  Workspaces grow on demand,
 *   so the first call at a new block width may allocate.
 * - One handle must not be used from two host threads at the same time.
 *
 * Discretisation (Sec. 2.2, Sec. 4.1): periodic cube [0, L)^3 split into n^3
 * equal cells; C0 Lagrange elements of degree p on Gauss-Lobatto-Legendre
 * nodes; global DoF of lattice point (i, j, k) is i + N1 (j + N1 k) with
 * N1 = n p.  Kinetic and mass cell matrices use (p+1)^3 Gauss points, the
 * potential and projector integrals use (p+2)^3 Gauss points; quadrature
 * point q = i + (p+2) (j + (p+2) k) of cell e = cx + n (cy + n cz).
 *
 * Bloch wavevector (Eq. FE PAW governing equations, k in the Brillouin zone):
 * paw_options.kpoint = k (Cartesian, 1/bohr).  With k != 0 the handle solves
 * H(k) u = eps S(k) u for the periodic factor u of psi = e^{i k.x} u, with the
 * 1/2 |k|^2 mass term and the -i k . N_I grad N_J term of Eq. hij and the
 * Bloch phases e^{-i k.(x - L_r)} of C^{a,k} (Eqs. FE nonlocal contribution,
 * FEM Cmatrix), and every multivector argument of paw_apply_H / _S /
 * _Sinv_approx, paw_cheb_filter, paw_rayleigh_ritz and paw_residuals is
 * COMPLEX, interleaved (real, imaginary) per entry: element (dof, j) is the
 * pair X[2 (dof * ld + j)], X[2 (dof * ld + j) + 1] (cuDoubleComplex for
 * FP64 arguments, cuFloatComplex for FP32 ones), ld counted in complex
 * entries.  Eigenvalues, bounds and norms stay real.  paw_lanczos_bounds,
 * paw_energy, paw_energy_grad, paw_density, the batch calls and
 * paw_apply_Sinv_approx_noalloc return PAW_ERR_UNSUPPORTED for such handles.
 */
#ifndef PAW_FE_H
#define PAW_FE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct paw_context *paw_handle;

typedef enum {
  PAW_OK = 0,
  PAW_ERR_INVALID_ARG = 1,   /* bad size, pointer, ordering of bounds ...      */
  PAW_ERR_UNSUPPORTED = 2,   /* non-periodic mesh, k != 0, l > 2, degree > 8  */
  PAW_ERR_NOT_SPD = 3,       /* overlap not positive definite (create / RR)   */
  PAW_ERR_CUDA = 4,          /* a CUDA runtime call or kernel launch failed   */
  PAW_ERR_NO_MEMORY = 5,     /* device allocation failed                       */
  PAW_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up             */
  PAW_ERR_NONFINITE = 7,     /* NaN/Inf detected in an input or a result       */
  PAW_ERR_LIBRARY = 8        /* cuBLAS / cuSOLVER reported an error            */
} paw_status;

typedef enum {
  PAW_FP64 = 0,  /* every step in FP64: the plain method                      */
  PAW_FP32 = 1,  /* filter bracket in FP32 storage and FP32 FMA arithmetic     */
  PAW_TF32 = 2,  /* FP32 storage; cell products and projector contractions   */
                 /* on tcgen05 tensor cores (TF32 operands, FP32 accumulation */
                 /* in tensor memory)                                          */
  PAW_BF16 = 3,  /* as PAW_TF32 with BF16 cell-matrix and vector operands of  */
                 /* the cell products (projector contractions stay TF32)       */
  PAW_F32X2 = 4  /* FP64 storage; every product and sum in pair-of-FP32      */
                 /* arithmetic (a value is hi + lo, two FP32 numbers: about   */
                 /* 48 significant bits, relative rounding about 2^-47) on    */
                 /* the FP32 pipes, which GB300 issues 64x faster than FP64.  */
                 /* Taken by paw_apply_H and paw_apply_S (k = 0); the filter's */
                 /* step 2 uses it through paw_options.y0_pair32.  Other calls */
                 /* return PAW_ERR_UNSUPPORTED.                               */
} paw_precision;

/* Periodic cubic box: L[0] = L[1] = L[2] and n_cells equal, periodic = 1. */
typedef struct {
  double L[3];
  int32_t n_cells[3];
  int32_t periodic[3];
} paw_mesh;

/* Atom positions (bohr), host array natoms x 3.  natoms may be 0. */
typedef struct {
  int32_t natoms;
  const double *positions;
} paw_atoms;

/* Projector shells shared by every atom: shell s is the Gaussian-radial
 * projector family N_l r^l exp(-r^2 / (2 w_s^2)) Y_lm(r^) (real harmonics,
 * m = -l..l, unit L2 norm, truncated at w_s sqrt(2 ln 1e8)), l_s in 0..2.
 * Projectors of an atom are numbered shell by shell, m ascending. */
typedef struct {
  int32_t nshells;
  const int32_t *l;
  const double *width;
} paw_projectors;

/* Synthetic local potential V(x) = -sum_g A_g exp(-|x - c_g|^2 / (2 w_g^2))
 * summed over periodic images within 8 w_g.  ngauss may be 0 (V = 0). */
typedef struct {
  int32_t ngauss;
  const double *centers; /* ngauss x 3 */
  const double *depth;   /* ngauss, A_g (Ha) */
  const double *width;   /* ngauss, w_g (bohr) */
} paw_vloc;

typedef struct {
  int32_t block;       /* vector block width B of paw_cheb_filter (0: 256)      */
  int32_t pp_overlap;  /* 1: use G_a = <p|p> (Sec. 3.1, third approximation)     */
  int32_t y0_fp32;     /* 1: store Y = H X - S X Lambda in FP32 in mixed modes   */
  int32_t rr_mixed;    /* 1: paw_rayleigh_ritz rotates with the diagonal of Q in
                          FP64 and its off-diagonal part in FP32 (Sec. 4.4,
                          mixed-precision subspace rotation)                    */
  double kpoint[3];    /* Bloch wavevector k (1/bohr); nonzero: complex vectors
                          (see the conventions at the top of this file)        */
  int32_t y0_pair32;   /* 1: form Y = H X - S X Lambda of paw_cheb_filter (step
                          2) in PAW_F32X2 arithmetic instead of FP64; Y keeps
                          FP64 storage.  k = 0 only (else paw_fe_create returns
                          PAW_ERR_UNSUPPORTED).  Default 0: FP64, as Algorithm 2 */
  int32_t no_overlap;  /* 1: paw_cheb_filter runs its blocks one after another.
                          Default 0: with two or more blocks (real, or complex
                          at k != 0) in PAW_FP32/TF32/BF16, step 2 of block j + 1 runs
                          on an internal stream while the loop of block j runs
                          on another (the results are the same up to the order
                          of FP32 additions)                                    */
} paw_options;

/* Filter bounds (Algorithm 2 inputs): a0 lower end of the wanted spectrum,
 * bW upper end of the wanted spectrum, bU upper bound of the whole spectrum.
 * Requires a0 < bW < bU. */
typedef struct {
  double a0, bW, bU;
} paw_bounds;

typedef struct {
  int64_t ndof;        /* M = (n p)^3                                        */
  int32_t ncells;      /* n^3                                                */
  int32_t nodes_per_cell;  /* (p+1)^3                                       */
  int32_t quad_per_cell;   /* (p+2)^3                                       */
  int32_t natoms;
  int32_t nproj;       /* projectors per atom                                */
  int32_t degree;      /* p                                                  */
  int64_t support_pairs;   /* number of (cell, atom) pairs in projector supports */
  int64_t device_bytes;    /* device memory currently held by the handle       */
  int64_t owner_pairs;     /* (cell, atom) pairs with P^a nonzero on a node the
                              cell owns (local indices < p): the work unit of the
                              projector contractions                          */
  int32_t nproj_padded;    /* projectors per atom as stored (16 or 32; with k != 0
                              the real and imaginary parts of C^{a,k} are stored
                              as 2 nproj real projectors)                      */
  int32_t complex_vectors; /* 1: k != 0, multivector arguments are complex     */
  int64_t proj_nnz;        /* nonzero entries of the assembled P^a on owned nodes,
                              summed over atoms: the algorithmic size of one
                              projector contraction (per vector)              */
} paw_info;

/* Build every operator of the problem (Sec. 4.1): cell matrices
 * H^e = 1/2 K^e + V^e (Eq. FEM Ham entries), the shared mass cell matrix M^e
 * (Eq. FEM S_loc entries), the lumped GLL mass M_D, projector cell matrices
 * C^{e,a} (Eq. FEM Cmatrix) and their assembly P^a, G_a = P^a^T M_D^-1 P^a
 * and Delta_Sinv^a = dS^a (I + G_a dS^a)^-1 (Eq. Delta Sinv).
 *   D_ij, dS_ij : host, natoms x nproj x nproj, symmetric (checked to 1e-12
 *                 relative); Delta_H^a and Delta_S^a of Eq. FE nonlocal
 *                 contribution.
 *   vloc        : may be NULL (V = 0); see also paw_set_veff.
 *   opts        : may be NULL (defaults).
 * Errors: INVALID_ARG (sizes, asymmetry, NULL out), UNSUPPORTED (non-cubic
 * or non-periodic box, degree outside 1..8, l > 2, a projector cutoff of
 * half the box or more), NOT_SPD (I + G_a dS^a singular or with a
 * non-positive eigenvalue for some atom), NO_MEMORY, CUDA. */
paw_status paw_fe_create(const paw_mesh *mesh, int degree, const paw_atoms *atoms,
                         const paw_projectors *proj, const double *D_ij,
                         const double *dS_ij, const paw_vloc *vloc,
                         const paw_options *opts, paw_handle *out);

/* Replace the potential: V_q is a DEVICE array ncells x (p+2)^3 (FP64) of the
 * potential at the quadrature points; rebuilds V^e and H^e (Eq. FEM Ham
 * entries).  Synchronous. */
paw_status paw_set_veff(paw_handle h, const double *V_q);

/* Replace Delta_H (host, natoms x nproj x nproj, symmetric).  Synchronous. */
paw_status paw_set_dij(paw_handle h, const double *D_ij);

paw_status paw_get_info(paw_handle h, paw_info *out);

/* Y = H X (Eq. FE nonlocal contribution: cell-matrix local part by
 * extraction, cell products and assembly, Sec. 4.3, plus sum_a P^a D^a P^a^T).
 * X, Y device, ncols >= 0 (0 is a no-op), ldx, ldy >= ncols; X and Y must
 * not overlap.  FP64 and FP32 calls are asynchronous on `stream`; PAW_TF32
 * and PAW_BF16 calls wait for the stream and return TIMEOUT when a
 * tensor-core kernel gave up on one of its bounded waits (Y is then
 * incomplete).  The same holds for paw_apply_Sinv_approx.  PAW_F32X2: X, Y
 * FP64 as for PAW_FP64, asynchronous, real vectors only (k = 0). */
paw_status paw_apply_H(paw_handle h, paw_precision prec, const void *X, void *Y,
                       int ncols, int ldx, int ldy, void *stream);

/* Y = S X with S = M + sum_a P^a dS^a P^a^T (consistent mass M). */
paw_status paw_apply_S(paw_handle h, paw_precision prec, const void *X, void *Y,
                       int ncols, int ldx, int ldy, void *stream);

/* Y = Shat^-1 X, the approximate inverse overlap of Eq. Sinvapprox:
 * M_D^-1 X - sum_a M_D^-1 P^a Delta_Sinv^a P^a^T M_D^-1 X. */
paw_status paw_apply_Sinv_approx(paw_handle h, paw_precision prec, const void *X,
                                 void *Y, int ncols, int ldx, int ldy, void *stream);

/* Same result as paw_apply_Sinv_approx, but this call never allocates device
 * memory.  It is meant for callers that cannot call cudaMalloc at the point of
 * use: real-time loops that must not block on the allocator, or hosts that
 * hand the library a fixed memory budget.
 * (Library-side engineering; the paper has no counterpart.)
 *
 * Its scratch (projector partial sums and coefficients) lives in one
 * statically sized device array of PAW_NOALLOC_SCRATCH_BYTES inside the
 * library, which every GPU that loads the library holds until the process
 * exits.  It needs elem * npad * ncols * (owner pairs + 2 natoms) bytes
 * (elem = 8 for PAW_FP64, 4 otherwise; npad = projectors per atom rounded up
 * to 16); a larger request returns PAW_ERR_INVALID_ARG before any device work.
 * The first call on a device looks the array up (cudaGetSymbolAddress, which
 * may load the library's device code), so make that first call on each device
 * before any stream capture begins.  All calls share the one array and leave their partial
 * sums in it; every value a call reads it has first written itself, so
 * nothing needs clearing, but calls whose GPU work overlaps (different
 * streams, or different handles on one device) race on the array and must be
 * serialised by the caller.  The lookup is repeated when the current context
 * of the device changes (after a device reset). */
#define PAW_NOALLOC_SCRATCH_BYTES (32u << 20)
paw_status paw_apply_Sinv_approx_noalloc(paw_handle h, paw_precision prec, const void *X,
                                         void *Y, int ncols, int ldx, int ldy, void *stream);

/* Algorithm 2: Psi_f = Shat^-1 R_m + Psi_in C_m(Lambda~) for one or more
 * blocks of columns (processed opts.block columns at a time).  Stream-ordered:
 * the call enqueues every kernel on `stream` and returns without waiting for
 * them (the per-block scalars sit in mapped pinned host memory owned by the
 * handle and a kernel reads them, so the call issues no copy that could queue
 * behind the caller's own transfers; the host only waits when it is eight
 * blocks ahead of the GPU).  Read failures with paw_sync_status.  With two or
 * more blocks in a reduced precision (and options.no_overlap = 0), the call
 * runs on two internal streams of the handle that wait for `stream` and that
 * `stream` waits for: step 2 of block j + 1 runs beside the loop of block j.
 *   X_in      : device FP64 ndof x ncols (ld ldx), the block Psi_in
 *   lambda_in : host FP64 ncols, the eigenvalue estimates Lambda
 *   degree    : m >= 1 (H applied m times, Shat^-1 applied m times)
 *   X_out     : device FP64 ndof x ncols (ld ldo); may not alias X_in
 * Y = H X - S X Lambda is formed in FP64 (step 2; in PAW_F32X2 arithmetic when
 * options.y0_pair32 is set); for PAW_FP32/TF32/BF16 the recurrence bracket
 * is evaluated in reduced precision and R is stored in FP32 (Sec. 4.4, mixed
 * precision computation).  The full-precision term (2 zeta/e) Y Lambda_Y is
 * added to the FP32 bracket by error-free FP32 arithmetic (an exact product
 * and a two-sum) on a hi + lo split of the FP64 Y (about 48 significant bits;
 * the lo word is dropped when options.y0_fp32 is set), then rounded once to
 * FP32; in PAW_FP64 it is an FP64 FMA.  Errors: INVALID_ARG (a0 < bW < bU violated,
 * degree < 1, sizes), NO_MEMORY, CUDA. */
paw_status paw_cheb_filter(paw_handle h, paw_precision prec, const double *X_in,
                           int ldx, const double *lambda_in, int ncols, int degree,
                           paw_bounds bounds, double *X_out, int ldo, void *stream);

/* ---------------------------------------------------------------- batches
 * Algorithm 2 for many independent instances at once (uneven meshes, FE
 * degrees, atom counts and block widths; the paper filters blocks of one
 * problem independently, Sec. 4.4 compute-communication overlap, and this
 * extends the same independence to separate problems).  Every launch of every
 * instance is captured once into a single CUDA graph: instances run on up to
 * `streams` concurrent branches of the graph, and each call replays the whole
 * batch with one cudaGraphLaunch.  The graph is recaptured when a problem's
 * pointers, sizes, degree, bounds or the precision change; eigenvalue
 * estimates (lambda_in) may change freely between calls.
 *
 * Autotuning (options.autotune = 1) happens on the first call and after a
 * recapture: for every instance the tensor-core kernel family (persistent
 * warp-specialised vs one CTA per tile) is timed on a short filter of its
 * first block; then the branch count (1, 2, 4, 8 up to `streams`) is timed on
 * the whole captured graph, the CTAs of persistent launches being capped at
 * SMs / branches.  The fastest combination is kept (paw_batch_tuning).
 *
 * The handles are not owned by the batch; they must stay valid until
 * paw_batch_destroy and must not be used concurrently by other calls. */
typedef struct paw_batch_s *paw_batch;

typedef struct {
  const double *X_in;       /* device FP64 ndof x ncols (ld ldx)                 */
  int32_t ldx;
  const double *lambda_in;  /* host FP64 ncols                                  */
  int32_t ncols;            /* 0: the instance is skipped                       */
  int32_t degree;           /* m >= 1                                           */
  paw_bounds bounds;        /* a0 < bW < bU                                     */
  double *X_out;            /* device FP64 ndof x ncols (ld ldo), no aliasing   */
  int32_t ldo;
} paw_batch_problem;

typedef struct {
  int32_t streams;      /* concurrent graph branches at most (0: 4)          */
  int32_t autotune;     /* 1: tune kernel family and branch count            */
  int32_t reserved[6];
} paw_batch_options;

typedef struct {
  int32_t tc_variant;   /* 0 persistent warp-specialised, 1 one CTA per tile */
  int32_t grid_cap;     /* CTAs of a persistent launch (0: all SMs)          */
  int32_t branch;       /* graph branch (stream) the instance runs on        */
  int32_t branches;     /* branches of the graph                             */
  int32_t graph_nodes;  /* nodes of the captured graph                       */
  int32_t kernel_nodes; /* of which kernel launches                          */
  int32_t captures;     /* graphs captured so far by this batch              */
  double tuned_ms[2];   /* timed short filter per kernel family (0: untimed) */
} paw_batch_tuning;

/* handles: count instance handles created by paw_fe_create (same device).
 * Errors: INVALID_ARG (count < 1, NULL handle, handle repeated), CUDA. */
paw_status paw_batch_create(const paw_handle *handles, int count, const paw_batch_options *options,
                            paw_batch *out);

/* problems: count entries (host).  status_out (host, count entries, may be
 * NULL) receives each instance's status: OK, INVALID_ARG / NONFINITE for a
 * rejected problem (that instance is skipped, the others run), TIMEOUT when a
 * tensor-core kernel of the instance gave up on a bounded wait.  The call
 * returns the first non-OK instance status, or a call-level error (CUDA,
 * NO_MEMORY).  Synchronises `stream` before returning. */
paw_status paw_batch_cheb_filter(paw_batch b, paw_precision prec, const paw_batch_problem *problems,
                                 paw_status *status_out, void *stream);

/* Tuning result and graph facts for instance i (after a filter call). */
paw_status paw_batch_tuning_get(paw_batch b, int i, paw_batch_tuning *out);

paw_status paw_batch_destroy(paw_batch b);

/* Rayleigh-Ritz (Algorithm 1 steps 4-6) in FP64:
 * H^p = X^T H X, S^p = X^T S X, H^p Q = S^p Q Lambda, X <- X Q.
 *   X          : device FP64 ndof x N (ld), overwritten by the S-orthonormal
 *                Ritz vectors in ascending order of Ritz value
 *   lambda_out : host FP64 N
 * H X and S X are formed block by block (opts.block columns) with the FP64
 * cell kernels; only the lower triangle of H^p and S^p is projected (column
 * block j0 gives rows j0..N-1; Sec. 4.5 RR-Projection), by the library's own
 * split-contraction FP64 kernels; the projected problem is solved by cuSOLVER
 * dsygvd (zhegvd at k != 0).  The rotation is an FP64 GEMM kernel of the
 * library over row chunks, or with opts.rr_mixed = 1: X <- X diag(Q) in FP64
 * plus fl32(X) (Q - diag(Q)) with FP32 products and sums (Sec. 4.5 RR-SR: the
 * off-diagonal part of Q is small near convergence).
 * Errors: NOT_SPD (S^p not positive definite), LIBRARY, NO_MEMORY, and
 * TIMEOUT for a failure left by an earlier asynchronous call. */
paw_status paw_rayleigh_ritz(paw_handle h, double *X, int ld, int N,
                             double *lambda_out, void *stream);

/* rnorm_out[i] = || H x_i - lambda_i S x_i ||_2 (FP64, unweighted), host out. */
paw_status paw_residuals(paw_handle h, const double *X, int ld, const double *lambda,
                         int N, double *rnorm_out, void *stream);

/* k-step generalised Lanczos on Shat^-1 H in the S inner product from a seeded
 * random start (FP64): theta_min, and upper = theta_max + |beta_k s_k| as the
 * estimate of b_U (Algorithm 1 step 1).  Host outputs. */
paw_status paw_lanczos_bounds(paw_handle h, int k, uint64_t seed, double *theta_min,
                              double *upper, void *stream);

/* E = tr(X^T H X) = sum_i x_i^T H x_i (host FP64 out), the subspace
 * Rayleigh-quotient energy whose gradient paw_energy_grad returns.  X is
 * FP64 (PAW_FP64) or FP32 (other precisions; H applied as by paw_apply_H). */
paw_status paw_energy(paw_handle h, paw_precision prec, const void *X, int ld, int N,
                      double *E_out, void *stream);

/* Gradient of E = tr(X^T H X) with X fixed (linear in V and Delta_H):
 *   dE_dV : device FP64 ncells x (p+2)^3, w_q detJ sum_i u_i(x_q)^2
 *   dE_dD : device FP64 natoms x nproj x nproj, sum_i U_i U_i^T, U = P^a^T X
 * (entries of Delta_H treated as independent).  X is FP64 or FP32 by prec. */
paw_status paw_energy_grad(paw_handle h, paw_precision prec, const void *X, int ld,
                           int N, double *dE_dV, double *dE_dD, void *stream);

/* Valence pseudo-density and PAW occupation matrices of a block of states
 * (Eq. FE PAW governing equations at the Gamma point, one spin channel; the
 * core density and the compensation charges are not included):
 *   rho_q : device FP64 ncells x (p+2)^3, sum_i f_i u_i(x_q)^2 at the Gauss
 *           points of every cell, u_i the FE function of column i
 *   D_a   : device FP64 natoms x nproj x nproj (may be NULL),
 *           sum_i f_i U_i U_i^T with U_i = P^a^T x_i (caller's projector order)
 *   occ   : host FP64 N occupations f_i (NULL: all 1)
 * X is FP64 (PAW_FP64) or FP32 (other precisions).  The same contractions as
 * paw_energy_grad, without the quadrature weights.  Synchronises `stream`. */
paw_status paw_density(paw_handle h, paw_precision prec, const void *X, int ld, int N,
                       const double *occ, double *rho_q, double *D_a, void *stream);

/* Phase timing of paw_cheb_filter (tracing, not part of the method).  When
 * enabled, every phase of Algorithm 2 is bracketed by CUDA events recorded on
 * the stream that runs it (the caller's stream, or the handle's internal
 * streams when paw_cheb_filter overlaps its blocks: a phase's time then
 * includes the SMs it shares with the other stream); paw_profile_read
 * synchronises and returns the summed device time per phase and the number of
 * kernels the library launched.
 * Phases: 0 local part of Y = H X - S X Lambda (step 2, FP64 cell kernel),
 * 1 recurrence update fused with T = Shat^-1 R_Y and the nonlocal part of
 * alpha H T, 2 projector contraction P^T M_D^-1 R_Y and couplings, 3 cell
 * products H^e T_e with extraction and assembly, 4 nonlocal part of
 * Y = H X - S X Lambda, 5 recovery (step 5). */
#define PAW_NPHASES 6
typedef struct {
  double ms[PAW_NPHASES];
  int64_t intervals[PAW_NPHASES];
  int64_t launches[PAW_NPHASES];
  int64_t total_launches;   /* all kernels launched by the library since enable */
} paw_profile;

/* enable = 1 resets the accumulators and starts recording; 0 stops. */
paw_status paw_profile_enable(paw_handle h, int enable);
paw_status paw_profile_read(paw_handle h, paw_profile *out);

/* Device-side status words (bounded waits, non-finite checks) since the last
 * call; PAW_OK if none was raised.  Synchronises the handle's last stream. */
paw_status paw_sync_status(paw_handle h);

/* Bounded device waits of the persistent tensor-core pipelines (cell products
 * and projector contractions of PAW_TF32 / PAW_BF16), for launches enqueued
 * after this call (library engineering; the paper has no counterpart).
 *   seconds : give-up bound of every pipeline wait, 1e-3 .. 60 (default 2)
 *   probe   : 1 makes every such launch first wait on a device word that
 *             nothing writes, before it issues any copy or MMA: the wait runs
 *             out after `seconds`, the launch gives up, and the call that
 *             reports device failures returns PAW_ERR_TIMEOUT.  This exercises
 *             the failure path without faulting anything; 0 (default) off.
 * The waits that let copies and MMAs already in flight finish before a CTA
 * exits keep their fixed 2 s bound.  Graphs captured by paw_batch_* keep the
 * setting they were captured with.  Errors: INVALID_ARG. */
paw_status paw_set_wait_limit(paw_handle h, double seconds, int probe);

paw_status paw_destroy(paw_handle h);

/* Message of the last failing call made by the calling thread (thread-local
 * rather than per handle: a handle is used by one thread at a time). */
const char *paw_last_error(void);

/* Library version string (static storage). */
const char *paw_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PAW_FE_H */
