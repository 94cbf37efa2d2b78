/*
 * gsyeig — a few eigenpairs of the dense symmetric-definite generalized
 * eigenproblem  A X = B X Lambda  on one NVIDIA GB300 (sm_103a).
 *
 * Paper: Aliaga, Bientinesi, Davidovic, Di Napoli, Igual, Quintana-Orti,
 * "Solving Dense Generalized Eigenproblems on Multi-threaded Architectures"
 * (arXiv 1111.6374).  The route is the paper's Krylov variant KE
 * (Section 2.3, Table 1):
 *
 *   gs1  B = U^T U                      Cholesky, U upper          (Eq. 2)
 *   gs2  C = U^-T A U^-1                explicit standard form     (Eq. 3)
 *   ke1  z = C w                        symmetric matrix-vector product
 *   ke2  Lanczos recurrence with full reorthogonalisation ("twice is
 *        enough") and implicit restarts (QR iteration on T_m)
 *   ke3  Ritz pairs of the tridiagonal T_m, Y = V_m S
 *   bt1  X = U^-1 Y                     back-transform              (Eq. 4)
 *
 * Conventions for every entry point below
 *  - Matrices are double precision, column-major, element (i, j) at
 *    M[i + j*ld], with ld >= n.  A symmetric matrix stored full is the same
 *    in row- and column-major order.
 *  - Unless stated otherwise pointers are DEVICE pointers owned by the
 *    caller; the library never frees them.  gsyeig_solve also accepts host
 *    pointers (see there).
 *  - Every call is synchronous on return.  Work is issued on the handle's
 *    own stream, ordered after the work already queued on the stream given
 *    to gsyeig_create (NULL = the legacy default stream).
 *  - Return value: GSYEIG_SUCCESS (0); -i when argument i (1-based) is
 *    invalid; or one of the positive status codes below.  Nothing is
 *    written to outputs when an argument is invalid.
 *  - A handle is not thread-safe: use one handle per host thread.
 */
#ifndef GSYEIG_H
#define GSYEIG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gsyeig_ctx *gsyeig_handle;

typedef enum { GSYEIG_SMALLEST = 0, GSYEIG_LARGEST = 1 } gsyeig_which;

enum {
  GSYEIG_SUCCESS = 0,
  GSYEIG_NOT_SPD = 1,        /* Cholesky of B met a non-positive pivot (Eq. 2); see info.potrf_index */
  GSYEIG_NO_CONVERGENCE = 2, /* max_restarts reached with fewer than s converged pairs; best pairs returned */
  GSYEIG_TIMEOUT = 3,        /* opts.timeout_ms ran out between restarts, or a bounded device-side wait
                                of the tensor-core GEMM expired (results then invalid) */
  GSYEIG_CUDA_ERROR = 4,     /* a CUDA runtime call failed; the handle should be destroyed */
  GSYEIG_OOM = 5,            /* device workspace could not be allocated */
  GSYEIG_NOT_SUPPORTED = 6,  /* option combination not available */
  GSYEIG_SCRATCH_TOO_SMALL = 7 /* gsyeig_tridiag_eig_noalloc: 5*m*cnt exceeds its fixed scratch */
};

/* Solver options (gsyeig_default_options fills the defaults). */
typedef struct {
  double tol;           /* accept Ritz pair i when |beta_m s_{m,i}| <= tol * ||T|| (running estimate; default 1e-12) */
  int64_t krylov_dim;   /* m, Lanczos basis size, s < m <= n; 0 = min(n, max(3s, s + 16)) */
  int64_t keep;         /* k, vectors kept at a restart, s <= k < m; 0 = min(s + max(2, s/4), m - 1) */
  int64_t max_restarts; /* default 2000 */
  uint64_t seed;        /* seed of the counter-based start vector (default 0) */
  const double *v0;     /* optional device start vector of length n (NULL = random) */
  double timeout_ms;    /* 0 = none; checked between restarts only */
  int32_t block;        /* panel width nb of the blocked factorisations (and order of the diagonal
                           blocks factored on one SM), 16..160; 0 = default (128).  The trailing
                           matrix gets rank-512 updates when nb divides 512, else rank-4nb ones */
  int32_t profile;      /* 1 = time every GEMM-engine and symv launch with CUDA events on the
                           library stream and report them in gsyeig_info (small overhead) */
  int32_t fp64_gemm;    /* 0 (default): the GEMMs of gsyeig_solve (the O(n^3) ones of gs1/gs2/bt1 and the
                           Lanczos basis products) run on the bf16 tensor cores (tcgen05) by
                           error-free slicing (FP64-accurate, normwise), K in slabs of up to 512;
                           1: plain FP64 FMA; 2: the same slicing on the legacy mma.sync path */
  int32_t fp64_symv;    /* 0 (default): ke1 streams C's lower triangle as fp32 hi/lo tiles built once per
                           solve (C_hi + C_lo = C to ~2^-48) with compensated fp32 products, HBM-bound;
                           1: plain FP64 product over the full square of C */
  int32_t qr_restart;   /* 0 (default): thick restart -- keep the k wanted Ritz vectors and continue from
                           the last Lanczos vector (the same subspace and projection as an exact-shift
                           implicit restart, computed in parallel); 1: implicit restart by p = m - k
                           exact-shift QR steps on T_m (Givens bulge chase), as ARPACK does */
  int32_t inverse;      /* 0 (default): the route as stated for `which`.  1, with which = SMALLEST: when A
                           is positive definite too, solve the inverse problem B X = A X M (M = Lambda^-1,
                           Section 3.1) for its s LARGEST eigenvalues, which Lanczos finds in far fewer
                           steps when the wanted lambda lie at the bottom of a wide spectrum; A is then
                           the matrix factored and B the one transformed.  If A's Cholesky meets a
                           non-positive pivot, A is restored and the direct route runs.  Ignored for
                           which = LARGEST. */
  int32_t preserve_inputs; /* 1: device A and B are left as they were (the solve runs on copies held by
                           the handle, 2 n^2 doubles); host inputs are never modified */
  int32_t verify;       /* 1: after the solve, check the result against the original pencil in FP64
                           on the device and report info.max_eta and info.orth_err (two more n^2
                           copies; not part of the stage times) */
  int32_t implicit;     /* 0 (default): variant KE, C = U^-T G U^-1 formed explicitly (gs2) and applied
                           by ke1.  1: variant KI (Section 2.3, Table 1): C is never formed; each
                           Lanczos step applies z = U^-T (G (U^-1 w)) with the untouched G (A, or B on
                           the inverse route) and the triangular factor, 4n^2 flops per step.  The
                           two triangular solves are applied through the explicit inverse U^-1,
                           computed once after gs1 on the tensor-core engine (see gsyeig_solve).
                           On exit G is left as it was (its lower triangle mirrored into the
                           upper) instead of holding C. */
  int32_t wait_limit;   /* testing hook, 0 (default) = off.  > 0: the device-side waits inside the main
                           loops of the tensor-core GEMM and of the ke1 kernel give up after this many
                           polls instead of after about a second, so that a test can make them run
                           out and check that the call returns GSYEIG_TIMEOUT and that the next call
                           with wait_limit = 0 succeeds.  Results of a call that timed out are
                           invalid. */
  /* Warm start for a sequence of related problems (the paper's Section 3 motivates it with the
   * dozens of related problems of a DFT self-consistency cycle).  With start_block != NULL the
   * Lanczos start vector is F (X0 w): X0 (n x start_cols, leading dimension ld_start, device) holds
   * eigenvector approximations of the pencil (e.g. a previous solve's X), w (start_weights, device,
   * start_cols entries; NULL = all ones) mixes them, and F is the upper-triangular factor of gs1
   * that maps them into the operator's space.  start_block takes precedence over v0. */
  const double *start_block;
  const double *start_weights;
  int64_t start_cols, ld_start;
  /* filter_degree > 0: before the first Lanczos step the start vector goes through the Chebyshev
   * polynomial of that degree (at most 64) that is bounded by 1 on the interval between
   * filter_cut and filter_edge (the unwanted end of the operator's spectrum: [cut, edge] with
   * edge above the cut for the smallest pairs, below it for the largest) and grows fast outside
   * it (Zhou and Saad's Chebyshev filter); each degree costs one operator application, counted
   * in info.matvecs and info.filter_matvecs. */
  double filter_cut, filter_edge;
  int32_t filter_degree;
  /* check_every > 0: besides the end of every cycle, test the wanted Ritz pairs after every
   * check_every Lanczos steps (once the projected matrix holds the kept pairs), so that a good
   * start can stop before the Krylov dimension is reached; 0 (default): at the end of a cycle only. */
  int32_t check_every;
  /* Mixed precision for the Lanczos stage (the paper's operator is the per-iteration cost, Section
   * 2.3).  Both forms start with block Lanczos (block size 16) with C streamed as fp32 tiles and
   * fp32 accumulation, FP64 reorthogonalisation (CGS2) and projected matrix, giving the k = s +
   * max(16, s/8) Ritz vectors of the band matrix (krylov_dim is the block Krylov dimension, default
   * max(3s, s + 64) for mixed = 1 and max(5s, s + 64) for mixed = 2, rounded up to 16).  Then:
   * 1: the FP64-accurate Lanczos (ke1 on the double-float operator) started from the sum of the k
   *    fp32 Ritz vectors, with Ritz tests every check_every steps (32 if 0), so that it stops once
   *    the s pairs meet the tolerance;
   * 2: an FP64 block refinement (LOBPCG on the k vectors, Rayleigh-Ritz on an orthonormal [X, P, W]
   *    with the products by C on the FP64-accurate tensor-core engine) until the s wanted residuals
   *    meet tol ||C||; if it cannot, the FP64 Lanczos stage runs from a random start (info
   *    refine_fallback).
   * gs1, gs2 and bt1 are unchanged.  Not with implicit = 1. */
  int32_t mixed;
  /* 1: each Lanczos cycle (without check_every) is captured once into a CUDA graph and replayed
   * while the handle's buffers and the operator stay the same: one host launch per cycle instead of
   * about 8 per step, for the many small problems of a batch.  Ignored while profile = 1. */
  int32_t graph;
  /* > 0: at most this many CTAs (SMs) for the persistent tensor-core GEMM, so that the problems of a
   * batch solved concurrently on several streams share the GPU; 0 = one CTA per SM. */
  int32_t max_ctas;
  /* 1, with start_block (start_cols >= s columns): start from the whole block instead of one vector:
   * the FP64 block refinement of the mixed route (LOBPCG, products on the tensor-core engine) runs
   * directly from the block F X0 plus max(8, s/4) random guard columns, with no Lanczos stage; for a
   * sequence of related problems whose eigenvectors move little from one problem to the next. */
  int32_t block_start;
  /* With inverse = 1 and which = SMALLEST: solve the shifted pencil (A - shift B, B) on the inverse
   * route, A - shift B = L^T L, and return lambda = shift + 1/mu.  A shift below the smallest
   * eigenvalue makes A - shift B positive definite when A itself is not (Section 3.1's route then
   * applies to any pencil whose smallest eigenvalue is known to lie above the shift).  The shift is
   * applied to the upper triangle only (the part the Cholesky reads): if A - shift B is not positive
   * definite, A's diagonal is restored and the unshifted direct route runs, reading A's untouched
   * lower triangle.  0 (default): no shift. */
  double shift;
} gsyeig_opts;

/* Per-solve report.  Stage times are CUDA-event milliseconds per paper key
 * (Table 2 / Table 6: gs1, gs2, ke1+ke2, ke3, bt1). */
typedef struct {
  int64_t n, s;
  int64_t nconv;        /* wanted pairs whose Ritz estimate met tol */
  int64_t restarts;     /* implicit restarts performed */
  int64_t matvecs;      /* applications of C (ke1) */
  int64_t krylov_dim, keep;
  int64_t potrf_index;  /* 1-based failing pivot when GSYEIG_NOT_SPD, else 0 */
  int64_t breakdowns;   /* Lanczos breakdowns recovered by a fresh random vector */
  int64_t kernel_launches; /* kernels launched by this call (graph nodes included) */
  double ms_gs1, ms_gs2, ms_ke, ms_ke3, ms_bt1, ms_total;
  double max_ritz_estimate; /* max over wanted pairs of |beta_m s_{m,i}| / max|theta| */
  /* opts.profile = 1: per kernel class (GEMM engine of gs1/gs2/bt1/restarts; symv of ke1)
   * the launches, summed CUDA-event time, and the algorithmic flops and bytes of those launches */
  int64_t gemm_launches, symv_launches;
  double gemm_ms, gemm_flops, gemm_bytes;
  double symv_ms, symv_flops, symv_bytes;
  /* opts.profile = 1: event time of the Lanczos bookkeeping (ke2): reorthogonalisation and
   * normalisation, restarts (QR iteration on T_m and V_m Q), Ritz problems on T_m */
  double orth_ms, restart_ms, ritz_ms;
  int64_t inverse;      /* 1 when the inverse problem (opts.inverse) was solved, else 0 */
  /* opts.verify = 1: max over the pairs of the normwise backward error
   * ||A x - lambda B x|| / ((||A|| + |lambda| ||B||) ||x||) (2-norms, the matrix norms by power
   * iteration) and max |X^T B X - I|, both in FP64 against the original A and B; else 0 */
  double max_eta, orth_err;
  /* opts.profile = 1: the tensor-core kernel of the GEMM engine alone (gemm_ms above also covers
   * the kernels that slice the FP64 operands into bf16 digit planes), with the FP64-equivalent
   * flops of those launches */
  int64_t gemm_core_launches;
  double gemm_core_ms, gemm_core_flops;
  /* opts.profile = 1: the kernels that factor and invert the nb x nb diagonal blocks of gs1 (one
   * group of launches per block: its Cholesky over sub-panels of 32 rows, then its inverse) and
   * their summed event time */
  int64_t diag_launches;
  double diag_ms;
  double tnorm;           /* the recurrence's running estimate of ||T|| (bounds the operator's spectrum
                             from the Krylov space: a filter_edge for a following solve) */
  int64_t filter_matvecs; /* operator applications of the start vector's Chebyshev filter */
  double slice_ms;        /* opts.profile = 1: event time of the kernels slicing GEMM operands into digits */
  /* opts.mixed: fp32 block steps, FP64 block-refinement iterations (mixed = 2) and the event time of
   * the fp32 stage and of the FP64 stage that follows it */
  int64_t block_steps, refine_iters;
  double ms_block_lanczos, ms_refine;
  int64_t refine_stop;     /* 1: the block refinement stopped on numerically dependent residuals; 2: its
                              observed rate did not reach the tolerance within 60 steps */
  int64_t refine_fallback; /* 1: the block refinement did not converge and the FP64 Lanczos stage ran */
  /* opts.profile = 1: launches and event time of the fp32 block operator of the mixed stage */
  int64_t symm32_launches;
  double symm32_ms;
  /* host inputs: event time from the start of the call to the end of the first matrix's transfer
   * (the other overlaps the Cholesky factorisation), and the host time the two copy requests took
   * to return (near zero for page-locked buffers; a pageable buffer is copied through staging
   * memory before the request returns) */
  double ms_h2d_first, host_ms_h2d_enqueue;
} gsyeig_info;

/* Create a handle on CUDA device `device`; `cuda_stream` is a cudaStream_t
 * (NULL = legacy default stream) that all calls order themselves after. */
int gsyeig_create(gsyeig_handle *h, int device, void *cuda_stream);

/* Release the handle and its device workspace. */
int gsyeig_destroy(gsyeig_handle h);

/* Fill *o with the defaults. */
int gsyeig_default_options(gsyeig_opts *o);

/* Copy *o into the handle (validated: tol > 0, keep < krylov_dim, ...). */
int gsyeig_set_options(gsyeig_handle h, const gsyeig_opts *o);

/* Human-readable text for a status code. */
const char *gsyeig_strerror(int status);

/*
 * The whole KE route (Section 2.3) for the s smallest (which = SMALLEST) or
 * largest eigenpairs of (A, B), 1 <= s < n.
 *  dA (n x n, lda): on entry the symmetric A, lower triangle read; on exit
 *      C = U^-T A U^-1 stored full, written over A (Section 2.1, Eq. 3).
 *  dB (n x n, ldb): on entry the SPD B, upper triangle read; on exit U in
 *      the upper triangle (Eq. 2); the strictly lower triangle is not touched.
 *  w  (s): eigenvalues in ascending order.  Host or device pointer.
 *  dX (n x s, ldx): B-orthonormal eigenvectors, column i for w[i].
 *  info: may be NULL.
 * With opts.inverse = 1, which = SMALLEST and A positive definite
 * (info.inverse = 1) the roles swap: A = L^T L is factored (L written over
 * A's upper triangle, A's strictly lower triangle kept), B is overwritten by
 * C' = L^-T B L^-1 (full), the s largest eigenpairs (mu, y) of C' are found,
 * and lambda = 1/mu, x = L^-1 y / sqrt(mu) are returned in the same order
 * and normalisation (X^T B X = I) as the direct route.  B is not factored
 * on this route: its positive definiteness is assumed, and only a wanted
 * mu <= 0 is reported (GSYEIG_NOT_SPD with info.potrf_index = 0).
 * If dA and dB are HOST pointers the library copies them to its own device
 * workspace, leaves the host arrays unchanged, and dX must then be a host
 * pointer too (the result is copied back).  Page-locked contiguous host
 * matrices (ld = n, 16-byte aligned) are read by the library's own copy
 * kernel through their device mapping, so each must hold n*n doubles;
 * others go through cudaMemcpy(2D)Async.  Returns GSYEIG_NOT_SPD,
 * GSYEIG_NO_CONVERGENCE (best pairs still written), GSYEIG_TIMEOUT, ...
 */
int gsyeig_solve(gsyeig_handle h, double *dA, int64_t lda, double *dB, int64_t ldb, int64_t n, int64_t s,
                 int which, double *w, double *dX, int64_t ldx, gsyeig_info *info);

/* ---- single steps of the route, device pointers only ------------------ */

/* gs1 (Eq. 2): B = U^T U, U written over the upper triangle of dB; strictly
 * lower triangle untouched.  *potrf_index (host, may be NULL) gets 0 or the
 * 1-based index of the first non-positive pivot (then GSYEIG_NOT_SPD). */
int gsyeig_potrf(gsyeig_handle h, double *dB, int64_t ldb, int64_t n, int64_t *potrf_index);

/* gs2 (Eq. 3): C = U^-T A U^-1 over dA (lower triangle of A read, C written
 * full), U the upper triangle of dU. */
int gsyeig_sygst(gsyeig_handle h, double *dA, int64_t lda, const double *dU, int64_t ldu, int64_t n);

/* ke1: z = C w for the full symmetric n x n dC (both triangles read). */
int gsyeig_symv(gsyeig_handle h, const double *dC, int64_t ldc, int64_t n, const double *dw, double *dz);

/* bt1 (Eq. 4): Y <- U^-1 Y in place on the n x s block dY. */
int gsyeig_trsm_back(gsyeig_handle h, const double *dU, int64_t ldu, int64_t n, double *dY, int64_t ldy, int64_t s);

/* Stage (2) of KE alone: s eigenpairs of the full symmetric dC by
 * implicitly restarted Lanczos.  w (host or device, ascending), dY (n x s,
 * orthonormal columns).  dC is read only. */
int gsyeig_syev_lanczos(gsyeig_handle h, const double *dC, int64_t ldc, int64_t n, int64_t s, int which,
                        double *w, double *dY, int64_t ldy, gsyeig_info *info);

/* ke3 building block: eigenvalues lam[0..cnt-1] with indices first..first+cnt-1
 * (ascending order, 0-based) of the symmetric tridiagonal (d[0..m-1],
 * e[0..m-2]) by Sturm-count bisection, and, if dZ != NULL, unit eigenvectors
 * by inverse iteration (m x cnt, ldz).  All pointers device. */
int gsyeig_tridiag_eig(gsyeig_handle h, const double *d, const double *e, int64_t m, int64_t first, int64_t cnt,
                       double *lam, double *dZ, int64_t ldz);

/* Allocation-free form of gsyeig_tridiag_eig (same results).  The paper has
 * no counterpart; it is here for callers that cannot allocate device memory
 * when they need this solve: code whose device memory belongs entirely to
 * another allocator or a fixed budget, and latency-critical loops in which a
 * cudaMalloc/cudaFree would synchronise the device.  No handle and no
 * allocation: the inverse-iteration scratch is a fixed 8 MiB array inside
 * the library (held on every GPU that loads it until the process exits), so
 * with dZ != NULL the call requires 5 * m * cnt <= 1048576 and otherwise
 * returns GSYEIG_SCRATCH_TOO_SMALL without touching the outputs.  Runs on
 * the calling thread's current device, on `cuda_stream` (cudaStream_t, NULL =
 * legacy default stream), synchronous on return.  The call looks up the
 * scratch address on the current device (a lookup allocates nothing), so
 * the address stays right after a device reset; the first call on a device
 * does this set-up for that device: make it before any stream capture.
 * All calls share the one scratch array: calls whose
 * work overlaps on the GPU (other streams, other host threads) race and must
 * be serialised by the caller.  Argument codes: -1 d, -2 e, -3 m, -4 first,
 * -5 cnt, -6 lam, -8 ldz. */
int gsyeig_tridiag_eig_noalloc(const double *d, const double *e, int64_t m, int64_t first, int64_t cnt, double *lam,
                               double *dZ, int64_t ldz, void *cuda_stream);

/* C = alpha op(A) op(B) + beta C (op = transpose when transA / transB is
 * nonzero) with the GEMM engine the handle's options select (by default the
 * FP64-accurate sliced bf16 tensor-core engine; opts.fp64_gemm = 1: FP64 FMA).
 * op(A) is M x K, op(B) K x N, C M x N, all column-major device arrays.  The
 * paper's route needs only its own products; this is the same engine for
 * callers' products (e.g. the overlaps X(t+1)^T B X(t) of a warm-started
 * sequence). */
int gsyeig_gemm(gsyeig_handle h, int transA, int transB, int64_t M, int64_t N, int64_t K, double alpha, const double *A,
                int64_t lda, const double *B, int64_t ldb, double beta, double *C, int64_t ldc);

/* ---- learned warm start (NEXT to the paper's route) ---------------------
 * Sequences of related problems (Section 3: the related eigenproblems of a
 * DFT self-consistency cycle) let a small network propose the start of the
 * next solve.  The MLP maps n_in features -> n_hidden -> n_hidden -> n_out
 * (ReLU after the two hidden layers); n_in <= 256, n_hidden a multiple of 16
 * up to 256, n_out <= 256.  Its parameters are fp32, packed as W1
 * (n_hidden x n_in, row-major), b1, W2 (n_hidden x n_hidden), b2, W3 (n_out x
 * n_hidden), b3; every product of the forward and backward pass runs on the
 * bf16 tensor cores (operands rounded to bf16 to nearest even, fp32
 * accumulation).  Matrices X (batch x n_in), Y, T (batch x n_out) are
 * row-major fp32.  All pointers are device pointers; the caller provides a
 * workspace of gsyeig_mlp_workspace_floats() floats, and the calls allocate
 * nothing.  Calls run on `stream` (cudaStream_t, NULL = legacy default) and
 * are synchronous on return except gsyeig_mlp_adam and the gsyeig_ws_*
 * calls, which are only enqueued.  Negative returns name the bad argument
 * (1-based); GSYEIG_TIMEOUT if a bounded wait for the tensor core ran out. */
int64_t gsyeig_mlp_param_count(int32_t n_in, int32_t n_hidden, int32_t n_out);           /* -1: bad sizes */
int64_t gsyeig_mlp_workspace_floats(int32_t n_in, int32_t n_hidden, int32_t n_out, int64_t batch);
/* weights uniform in +-sqrt(6 / fan_in) from a counter-based generator of seed, biases 0 */
int gsyeig_mlp_init(float *params, int32_t n_in, int32_t n_hidden, int32_t n_out, uint64_t seed, void *stream);
/* Y = net(X), batch rows */
int gsyeig_mlp_forward(const float *params, int32_t n_in, int32_t n_hidden, int32_t n_out, const float *X,
                       int64_t batch, float *Y, float *ws, void *stream);
/* Gradient (packed like the parameters) of the weighted mean squared error
 * loss = sum_{b,o} w_o (Y - T)^2 / (2 batch) (out_weights: n_out entries, NULL
 * = all ones), batch <= 256; *loss (device float, may be NULL) gets the loss. */
int gsyeig_mlp_grad(const float *params, int32_t n_in, int32_t n_hidden, int32_t n_out, const float *X,
                    const float *T, const float *out_weights, int64_t batch, float *grad, float *loss, float *ws,
                    void *stream);
/* One Adam step (Kingma and Ba 2015, bias-corrected; step counts from 1) on
 * `count` parameters with moments m, v (zero before the first step). */
int gsyeig_mlp_adam(float *params, float *m, float *v, const float *grad, int64_t count, int64_t step, float lr,
                    float beta1, float beta2, float eps, void *stream);
/* Features of a solved problem for its successor, from its s ascending
 * eigenvalues theta and those of the problem before (theta_prev): with g the
 * mean spacing of theta, f[j] = (theta[j] - theta[s-1]) / g, f[s+j] =
 * (theta[j] - theta_prev[j]) / g, f[2s] = dt_rel (2s + 1 features);
 * scal[0..1] (device doubles) = theta[s-1], g for decoding. */
int gsyeig_ws_features(int64_t s, const double *theta, const double *theta_prev, double dt_rel, float *features,
                       double *scal, void *stream);
/* Block warm start (opts.block_start): the network proposes, for each
 * eigenvector of the last solved problem, how far to extrapolate it along
 * the sequence.  gsyeig_ws_align: out_j = sgn_j Y[:, pi_j] - X[:, j], where
 * pi_j is the column of Y with the largest |P[j, i]| (P = X^T B Y, s x s, ld
 * ldp) and sgn_j that overlap's sign; columns whose best |overlap| is below
 * 1/2 (eigenvalue crossings) get 0; match (s floats, may be NULL) gets the
 * best |overlap| of every column.  gsyeig_ws_coef_targets: the B-optimal
 * extrapolation coefficients t_j = clamp(-(D_j^T BE_j) / (D_j^T BD_j), lo,
 * hi) of training data (D = align(X(t), X(t-1)), E = align(X(t), X(t+1)),
 * BD = B D, BE = B E).  gsyeig_ws_extrapolate: out_j = X_j - clamp(c_j, lo,
 * hi) D_j, the start block proposed for the next problem.  All device
 * pointers, column-major, enqueued on `stream`. */
int gsyeig_ws_align(int64_t n, int64_t s, const double *X, int64_t ldx, const double *Y, int64_t ldy, const double *P,
                    int64_t ldp, double *out, int64_t ldo, float *match, void *stream);
int gsyeig_ws_coef_targets(int64_t n, int64_t s, const double *D, int64_t ldd, const double *BD, int64_t ldbd,
                           const double *BE, int64_t ldbe, double lo, double hi, float *targets, void *stream);
int gsyeig_ws_extrapolate(int64_t n, int64_t s, const double *X, int64_t ldx, const double *D, int64_t ldd,
                          const float *coef, double lo, double hi, double *out, int64_t ldo, void *stream);
/* The shift of the next solve (gsyeig_opts.shift, Section 3.1's inverse route on A - shift B): with
 * the eigenvalues w_prev (ascending, s) and w_prev2 of the previous two problems,
 * gsyeig_ws_shift writes shift[0] = w_prev[0] + clamp(coef[0], lo, hi) (w_prev[0] - w_prev2[0])
 * - frac (w_prev[s-1] - w_prev[0]) / s, a margin of frac mean spacings below the extrapolated
 * smallest eigenvalue (coef NULL: no extrapolation, w_prev2 may then be NULL).
 * gsyeig_ws_shift_target writes the coefficient that would have extrapolated to w[0] exactly,
 * clamped to [lo, hi] (0 when w_prev[0] = w_prev2[0]): the training target.  Device pointers. */
int gsyeig_ws_shift(int64_t s, const double *w_prev2, const double *w_prev, const float *coef, double lo, double hi,
                    double frac, double *shift, void *stream);
int gsyeig_ws_shift_target(const double *w_prev2, const double *w_prev, const double *w, double lo, double hi,
                           float *target, void *stream);

/* ---- batches of independent problems ---------------------------------- */
/* One problem of a batch: the arguments of gsyeig_solve (device pointers). */
typedef struct {
  double *A;
  int64_t lda;
  double *B;
  int64_t ldb;
  int64_t n, s;
  int32_t which, reserved;
  double *w;
  double *X;
  int64_t ldx;
} gsyeig_problem;

/* Solve `count` independent problems (device pointers; each as
 * gsyeig_solve with the options of h) concurrently: `nstreams` (1..16)
 * internal handles, each on its own stream and host thread, take the
 * problems largest first from a shared queue; the tensor-core GEMM of each
 * is capped at ceil(SMs / nstreams) CTAs (unless opts.max_ctas is set) and
 * every Lanczos cycle is replayed from a CUDA graph (opts.graph).  The
 * panel width of each problem comes from a built-in autotuner (when
 * opts.block = 0): for each size class (n rounded up to a multiple of 512)
 * it times the factorisation steps of a synthetic SPD matrix of that order
 * for each candidate width once per handle and keeps the fastest
 * (gsyeig_autotuned_block reports the choice).  statuses[i] and infos[i]
 * (both may be NULL) receive each problem's outcome; the call returns
 * GSYEIG_SUCCESS when every problem succeeded, else the first failing
 * problem's status.  Synchronous on return. */
int gsyeig_solve_batched(gsyeig_handle h, int64_t count, const gsyeig_problem *probs, int32_t nstreams,
                         int32_t *statuses, gsyeig_info *infos);

/* The panel width the autotuner of gsyeig_solve_batched chose for order n
 * on this handle (tuning it now if needed); 0 on failure. */
int32_t gsyeig_autotuned_block(gsyeig_handle h, int64_t n);

/* Number of kernels this library has launched in the calling process. */
int64_t gsyeig_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* GSYEIG_H */
