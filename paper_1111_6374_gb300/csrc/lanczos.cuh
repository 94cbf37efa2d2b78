// Device-side pieces of the Lanczos stage (ke2, ke3): recurrence helpers
// (lanczos.cu) and the small tridiagonal problems on T_m (tridiag.cu).
#pragma once

#include "common.cuh"

namespace gs {

// Scalars the recurrence keeps on the device between kernels.
struct LanczosState {
  double tnorm;          // running estimate of ||T|| (max |alpha_j| + beta_j + beta_{j-1})
  double inv_beta;       // 1 / beta_j for the next scaling (0 after a breakdown)
  int64_t breakdown_at;  // first step j of this pass with beta_j ~ 0, or -1
  int64_t nconv;         // converged wanted Ritz pairs (written by the convergence test)
  double max_est;        // max over wanted pairs of |beta_m s_{m,i}| / max|theta|
  double scratch;
};

// --- lanczos.cu -------------------------------------------------------------
int lz_nparts(int64_t n);
int lz_dots(cudaStream_t st, int64_t n, int64_t ncols, const double *V, int64_t ldv, const double *z, double *h);
int lz_sub(cudaStream_t st, int64_t n, int64_t ncols, const double *V, int64_t ldv, const double *h, double *z,
           double *sq);
// CGS2 of z against V[:, 0:ncols]; coefficients in h1, h2; per-slice sums of
// squares of the result in sq (lz_nparts(n) entries).
int lz_cgs2(cudaStream_t st, int64_t n, int64_t ncols, const double *V, int64_t ldv, double *z, double *h1,
            double *h2, double *sq);
int lz_finalize(cudaStream_t st, int64_t j, int64_t m, const double *h1, const double *h2, const double *sq,
                int nparts, double *alpha, double *beta, LanczosState *state);
int lz_scale_into(cudaStream_t st, int64_t n, const double *z, double *out, const LanczosState *state);
int lz_norm_finish(cudaStream_t st, const double *sq, int nparts, LanczosState *state, double *norm_out);
int lz_random(cudaStream_t st, int64_t n, uint64_t seed, uint64_t stream, double *v);
// Thick restart bookkeeping: d[i] = theta[i], arrow b[i] = beta[m-1] S[m-1, i]
// and e[i] = 0 for i < k (S is m x k, ld m).
int lz_thick_restart(cudaStream_t st, int64_t m, int64_t k, const double *theta, const double *S, double *d, double *e,
                     double *b);
// Inverse problem (B x = mu (A - shift B) x, theta = its s largest mu,
// ascending) back to (A, B): X column i <- X column s-1-i /
// sqrt(theta[s-1-i]) and theta[i] <- shift + 1 / theta[s-1-i], so lambda
// ascends and X^T B X = I.
int lz_invert_pairs(cudaStream_t st, int64_t n, int64_t s, double *theta, double *X, int64_t ldx, double shift = 0.0);
// A(i, j) -= shift B(i, j) over the upper triangles (i <= j)
int lz_shift_upper(cudaStream_t st, int64_t n, double *A, int64_t lda, const double *B, int64_t ldb, double shift);
// out = X w (X n x k, ld ldx; w device, k entries, NULL = all ones).
int lz_weighted_sum(cudaStream_t st, int64_t n, int64_t k, const double *X, int64_t ldx, const double *w,
                    double *out);
// out = U v for the upper triangle of U (n x n, ld ldu); the strictly lower
// triangle of U is not read.
int lz_trmv_upper(cudaStream_t st, int64_t n, const double *U, int64_t ldu, const double *v, double *out);
// One step of the Chebyshev recurrence on [c - e, c + e]: out = (Cy - c y) / e
// when first, else out = 2 (Cy - c y) / e - yprev (out may alias yprev).
int lz_cheb_step(cudaStream_t st, int64_t n, const double *Cy, const double *y, const double *yprev, double c,
                 double e, bool first, double *out);
int lz_restart_residual(cudaStream_t st, int64_t n, int64_t k, int64_t m, const double *Vq, int64_t ldvq,
                        const double *vm, const double *betaP, const double *beta, const double *Q, int64_t ldq,
                        double *f);

// --- tridiag.cu -------------------------------------------------------------
// The small symmetric matrices M of the Lanczos stage: diagonal d[0..m-1];
// rows i < ka couple only to row ka, through b[i] (the "arrow" left by a
// thick restart; ka = 0, b = NULL for a plain tridiagonal); rows i >= ka are
// tridiagonal with e[i] coupling rows i and i+1.
// Eigenvalues with ascending indices first..first+cnt-1 of M by bisection.
int tri_bisect(cudaStream_t st, int64_t m, const double *d, const double *e, int64_t ka, const double *b, int64_t first,
               int64_t cnt, double *lam);
// Unit eigenvectors (m x cnt, ldz) of M for ascending eigenvalues lam by
// inverse iteration; eigenvalues closer than 1e-10 ||M|| are orthogonalised
// as a cluster.  work: cnt * 5m doubles.
int tri_invit(cudaStream_t st, int64_t m, const double *d, const double *e, int64_t ka, const double *b, int64_t cnt,
              const double *lam, double *Z, int64_t ldz, double *work);
// p = m - k exact-shift implicit QR steps on T_m (alpha, beta); shift i is
// shifts[i] (dir > 0) or shifts[p - 1 - i] (dir < 0).  Writes the
// transformed T into (alphaP, betaP) and the accumulated orthogonal Q
// (m x m, ldq).  rot: 2 p (m - 1) doubles of rotation scratch.
int tri_qr_shifts(cudaStream_t st, int64_t m, int64_t p, const double *alpha, const double *beta,
                  const double *shifts, int dir, double *alphaP, double *betaP, double *Q, int64_t ldq, double *rot);
// Convergence test of the wanted Ritz pairs: estimate_i = |beta[m-1] Z[m-1, i]|
// relative to the running ||T|| estimate state->tnorm.
int tri_converged(cudaStream_t st, int64_t m, int64_t cnt, const double *theta_all, const double *beta,
                  const double *Z, int64_t ldz, double tol, LanczosState *state);

}  // namespace gs
