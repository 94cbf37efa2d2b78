/*
 * Plain CPU FP64 oracle for the symmetric-definite generalized eigenproblem
 * A X = B X Lambda (Eq. 1), following the transformation route of Section 2:
 *
 *   Cholesky B = U^T U (Eq. 2), C = U^{-T} A U^{-1} by two triangular solves
 *   (Eq. 3, the 2 n^3 form chosen in Section 4.1), Householder reduction of C
 *   to tridiagonal T (variant TD, Section 2.2), implicit QL on T for the
 *   eigenvalues, eigenvectors of T by QL accumulation or inverse iteration,
 *   back-application of the reflectors (Y = Q Z) and X = U^{-1} Y (Eq. 4).
 *   A cyclic Jacobi eigensolver is kept as an independent brute-force check.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is slow on purpose: loops are written
 * the way the definitions read, with OpenMP only over independent rows or
 * columns, and no blocking.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load it; the GPU library never does, and
 * the two share no code.
 *
 * Storage: column-major, element (i, j) of a matrix with leading dimension
 * ld is M[i + j*ld].  All arithmetic is IEEE double.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define IDX(i, j, ld) ((size_t)(i) + (size_t)(j) * (size_t)(ld))

/* ------------------------------------------------------------------------ */
/* Eq. 2: B = U^T U with U upper triangular, written over the upper triangle */
/* of B.  Column j of U:                                                     */
/*   U[j][j] = sqrt(B[j][j] - sum_{k<j} U[k][j]^2)                           */
/*   U[j][i] = (B[j][i] - sum_{k<j} U[k][j] U[k][i]) / U[j][j],  i > j       */
/* Returns 0, or the 1-based index of the first non-positive pivot.  The     */
/* strictly lower triangle of B is not referenced.                           */
/* ------------------------------------------------------------------------ */
int oracle_potrf(int64_t n, double *B, int64_t ldb) {
  for (int64_t j = 0; j < n; j++) {
    double s = B[IDX(j, j, ldb)];
    for (int64_t k = 0; k < j; k++) s -= B[IDX(k, j, ldb)] * B[IDX(k, j, ldb)];
    if (!(s > 0.0)) return (int)(j + 1);
    double ujj = sqrt(s);
    B[IDX(j, j, ldb)] = ujj;
#pragma omp parallel for schedule(static)
    for (int64_t i = j + 1; i < n; i++) {
      double t = B[IDX(j, i, ldb)];
      for (int64_t k = 0; k < j; k++) t -= B[IDX(k, j, ldb)] * B[IDX(k, i, ldb)];
      B[IDX(j, i, ldb)] = t / ujj;
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Eq. 3: C = U^{-T} A U^{-1}.  A is symmetric; its lower triangle (i >= j)  */
/* is read.  Step 1 solves U^T W = A column by column (forward substitution */
/* with the lower-triangular U^T); step 2 solves C U = W row by row.  C is   */
/* then made exactly symmetric, C <- (C + C^T)/2, and written in full over A.*/
/* U is the upper triangle of a matrix with leading dimension ldu.           */
/* ------------------------------------------------------------------------ */
void oracle_sygst(int64_t n, double *A, int64_t lda, const double *U, int64_t ldu) {
  /* full symmetric A from its lower triangle */
  for (int64_t j = 0; j < n; j++)
    for (int64_t i = 0; i < j; i++) A[IDX(i, j, lda)] = A[IDX(j, i, lda)];
  /* W = U^{-T} A: for each column c, w_i = (a_i - sum_{k<i} U[k][i] w_k) / U[i][i] */
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t c = 0; c < n; c++) {
    double *w = &A[IDX(0, c, lda)];
    for (int64_t i = 0; i < n; i++) {
      double t = w[i];
      for (int64_t k = 0; k < i; k++) t -= U[IDX(k, i, ldu)] * w[k];
      w[i] = t / U[IDX(i, i, ldu)];
    }
  }
  /* C = W U^{-1}: for each row r, x_j = (w_j - sum_{k<j} x_k U[k][j]) / U[j][j] */
#pragma omp parallel
  {
    double *x = (double *)malloc((size_t)n * sizeof(double));
#pragma omp for schedule(dynamic, 8)
    for (int64_t r = 0; r < n; r++) {
      for (int64_t j = 0; j < n; j++) {
        double t = A[IDX(r, j, lda)];
        for (int64_t k = 0; k < j; k++) t -= x[k] * U[IDX(k, j, ldu)];
        x[j] = t / U[IDX(j, j, ldu)];
      }
      for (int64_t j = 0; j < n; j++) A[IDX(r, j, lda)] = x[j];
    }
    free(x);
  }
  for (int64_t j = 0; j < n; j++)
    for (int64_t i = j + 1; i < n; i++) {
      double s = 0.5 * (A[IDX(i, j, lda)] + A[IDX(j, i, lda)]);
      A[IDX(i, j, lda)] = s;
      A[IDX(j, i, lda)] = s;
    }
}

/* ------------------------------------------------------------------------ */
/* Eq. 4: X = U^{-1} Y, in place on the n-by-s block Y (leading dim ldy).    */
/* Back substitution by columns of U: x_j = y_j / U[j][j], then              */
/* y[0:j] -= x_j U[0:j][j].                                                  */
/* ------------------------------------------------------------------------ */
void oracle_backsolve(int64_t n, int64_t s, const double *U, int64_t ldu, double *Y, int64_t ldy) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t c = 0; c < s; c++) {
    double *y = &Y[IDX(0, c, ldy)];
    for (int64_t j = n - 1; j >= 0; j--) {
      double xj = y[j] / U[IDX(j, j, ldu)];
      y[j] = xj;
      for (int64_t i = 0; i < j; i++) y[i] -= xj * U[IDX(i, j, ldu)];
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Variant TD, first stage (Section 2.2): Q^T C Q = T by Householder          */
/* reflectors H_k = I - tau_k v_k v_k^T, k = 0..n-3, each annihilating       */
/* C[k+2:n, k].  v_k has v_k[k+1] = 1 and its tail is stored in C[k+2:n, k]  */
/* (the annihilated entries).  On return d[0..n-1] is the diagonal of T and  */
/* e[0..n-2] its off-diagonal; C must be full symmetric on entry and only    */
/* the part on and below the subdiagonal is meaningful afterwards.           */
/* The trailing update is the symmetric rank-2 form:                          */
/*   p = tau C v,  w = p - (tau/2)(p^T v) v,  C <- C - v w^T - w v^T.         */
/* ------------------------------------------------------------------------ */
void oracle_tridiag(int64_t n, double *C, int64_t ldc, double *d, double *e, double *tau) {
  double *v = (double *)malloc((size_t)n * sizeof(double));
  double *p = (double *)malloc((size_t)n * sizeof(double));
  for (int64_t k = 0; k + 2 < n; k++) {
    int64_t m = n - k - 1; /* length of x = C[k+1:n, k] */
    double *x = &C[IDX(k + 1, k, ldc)];
    double sigma = 0.0;
    for (int64_t i = 1; i < m; i++) sigma += x[i] * x[i];
    double alpha = x[0];
    double t = 0.0;
    if (sigma == 0.0) {
      /* already in tridiagonal form in this column: H_k = I */
      e[k] = alpha;
      tau[k] = 0.0;
      for (int64_t i = 1; i < m; i++) x[i] = 0.0;
      continue;
    }
    double nrm = sqrt(alpha * alpha + sigma);
    /* beta = -sign(alpha) ||x||; v = x - beta e1, scaled so v[0] = 1 */
    double beta = (alpha >= 0.0) ? -nrm : nrm;
    double v0 = alpha - beta;
    t = (beta - alpha) / beta; /* tau = 2 v0^2 / (sigma + v0^2) */
    v[0] = 1.0;
    for (int64_t i = 1; i < m; i++) v[i] = x[i] / v0;
    e[k] = beta;
    tau[k] = t;
    for (int64_t i = 1; i < m; i++) x[i] = v[i];
    x[0] = beta;
    /* p = tau * C[k+1:, k+1:] v  (full symmetric trailing block) */
    double *Ct = &C[IDX(k + 1, k + 1, ldc)];
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; i++) {
      double acc = 0.0;
      for (int64_t j = 0; j < m; j++) acc += Ct[IDX(j, i, ldc)] * v[j]; /* C symmetric: row i = column i */
      p[i] = t * acc;
    }
    double pv = 0.0;
    for (int64_t i = 0; i < m; i++) pv += p[i] * v[i];
    double half = 0.5 * t * pv;
    for (int64_t i = 0; i < m; i++) p[i] -= half * v[i]; /* p now holds w */
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < m; j++)
      for (int64_t i = 0; i < m; i++) Ct[IDX(i, j, ldc)] -= v[i] * p[j] + p[i] * v[j];
  }
  for (int64_t i = 0; i < n; i++) d[i] = C[IDX(i, i, ldc)];
  if (n >= 2) {
    e[n - 2] = C[IDX(n - 1, n - 2, ldc)];
    tau[n - 2] = 0.0;
  }
  free(v);
  free(p);
}

/* Y <- Q Y with Q = H_0 H_1 ... H_{n-3}, reflectors as left by oracle_tridiag. */
void oracle_apply_q(int64_t n, const double *C, int64_t ldc, const double *tau, int64_t s, double *Y, int64_t ldy) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t c = 0; c < s; c++) {
    double *y = &Y[IDX(0, c, ldy)];
    for (int64_t k = n - 3; k >= 0; k--) {
      if (tau[k] == 0.0) continue;
      /* v = [1, C[k+2:n, k]] acting on y[k+1:n] */
      double dot = y[k + 1];
      for (int64_t i = k + 2; i < n; i++) dot += C[IDX(i, k, ldc)] * y[i];
      dot *= tau[k];
      y[k + 1] -= dot;
      for (int64_t i = k + 2; i < n; i++) y[i] -= dot * C[IDX(i, k, ldc)];
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Number of eigenvalues of the symmetric tridiagonal T = (d, e) that are    */
/* strictly less than x: the count of negative pivots of the LDL^T           */
/* factorisation of T - x I (Sylvester's law of inertia).                    */
/* ------------------------------------------------------------------------ */
int64_t oracle_sturm_count(int64_t n, const double *d, const double *e, double x) {
  int64_t count = 0;
  double q = 1.0;
  for (int64_t i = 0; i < n; i++) {
    double off = (i > 0) ? e[i - 1] * e[i - 1] : 0.0;
    q = (d[i] - x) - ((i > 0) ? off / q : 0.0);
    if (q == 0.0) q = -1e-300; /* a zero pivot is nudged to the negative side */
    if (q < 0.0) count++;
  }
  return count;
}

/* ------------------------------------------------------------------------ */
/* Implicit QL with a Wilkinson-type shift on T = (d, e): every eigenvalue,  */
/* and, when Z is given, the rotations accumulated into the n-by-n Z (which */
/* should hold I, or Q from the tridiagonal reduction, on entry).            */
/* For the unreduced block [l, m], the shift is the eigenvalue of the        */
/* leading 2x2 block closest to d[l]; one QL sweep with that shift is then   */
/* applied as a chain of Givens rotations from the bottom of the block up.  */
/* e is destroyed.  Eigenvalues are returned sorted ascending (vectors      */
/* permuted alike).  Returns 0, or -1 if some block needed > 60 sweeps.     */
/* The method is the textbook implicit QL algorithm for symmetric           */
/* tridiagonal matrices (Bowdler, Martin, Reinsch and Wilkinson, "The QR    */
/* and QL algorithms for symmetric matrices", Numer. Math. 11 (1968), the   */
/* procedure tql2 of the Handbook for Automatic Computation, vol. II); it   */
/* was written from that published description.                            */
/* ------------------------------------------------------------------------ */
int oracle_tql(int64_t n, double *d, double *e, double *Z, int64_t ldz) {
  double *f = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  for (int64_t i = 0; i + 1 < n; i++) f[i] = e[i]; /* f[i] couples i and i+1 */
  int status = 0;
  for (int64_t l = 0; l < n; l++) {
    int sweeps = 0;
    for (;;) {
      int64_t m = l;
      while (m + 1 < n) {
        double dd = fabs(d[m]) + fabs(d[m + 1]);
        if (fabs(f[m]) <= 0x1p-53 * dd) break;
        m++;
      }
      if (m == l) break;
      if (++sweeps > 60) { status = -1; break; }
      /* shift from the 2x2 block at the top (index l) */
      double g = (d[l + 1] - d[l]) / (2.0 * f[l]);
      double r = hypot(g, 1.0);
      double mu = d[l] - f[l] / (g + (g >= 0.0 ? r : -r));
      /* QL sweep from the bottom of the block: chase the bulge upward */
      double x = d[m] - mu;
      double c = 1.0, s = 1.0, pcarry = 0.0;
      int64_t i;
      for (i = m - 1; i >= l; i--) {
        double fi = s * f[i];
        double bi = c * f[i];
        r = hypot(fi, x);
        if (i + 1 < m) f[i + 1] = r;
        if (r == 0.0) {
          d[i + 1] -= pcarry;
          f[m] = 0.0;
          break;
        }
        s = fi / r;
        c = x / r;
        double gi = d[i + 1] - pcarry;
        double t = (d[i] - gi) * s + 2.0 * c * bi;
        pcarry = s * t;
        d[i + 1] = gi + pcarry;
        x = c * t - bi;
        if (Z) {
          for (int64_t k = 0; k < n; k++) {
            double zk1 = Z[IDX(k, i + 1, ldz)];
            double zk0 = Z[IDX(k, i, ldz)];
            Z[IDX(k, i + 1, ldz)] = s * zk0 + c * zk1;
            Z[IDX(k, i, ldz)] = c * zk0 - s * zk1;
          }
        }
      }
      if (r == 0.0 && i >= l) continue;
      d[l] -= pcarry;
      f[l] = x;
      f[m] = 0.0;
    }
    if (status) break;
  }
  /* selection sort ascending, carrying vectors */
  for (int64_t i = 0; i + 1 < n; i++) {
    int64_t k = i;
    for (int64_t j = i + 1; j < n; j++)
      if (d[j] < d[k]) k = j;
    if (k != i) {
      double t = d[i]; d[i] = d[k]; d[k] = t;
      if (Z)
        for (int64_t r2 = 0; r2 < n; r2++) {
          double u = Z[IDX(r2, i, ldz)];
          Z[IDX(r2, i, ldz)] = Z[IDX(r2, k, ldz)];
          Z[IDX(r2, k, ldz)] = u;
        }
    }
  }
  for (int64_t i = 0; i + 1 < n; i++) e[i] = 0.0;
  free(f);
  return status;
}

/* ------------------------------------------------------------------------ */
/* Inverse iteration on T = (d, e) for the eigenvalues lam[0..s-1] (sorted   */
/* ascending).  Each vector solves (T - lam I) z_new = z_old by Gaussian     */
/* elimination with partial pivoting on the tridiagonal (three sweeps), and */
/* is orthogonalised against the earlier vectors of its cluster (eigenvalue */
/* gaps below 1e-3 ||T||), as in the classic treatment of close eigenvalues.*/
/* Z is n-by-s, unit columns.                                               */
/* ------------------------------------------------------------------------ */
void oracle_tri_invit(int64_t n, const double *d, const double *e, int64_t s, const double *lam, double *Z, int64_t ldz) {
  double tnorm = 0.0;
  for (int64_t i = 0; i < n; i++) {
    double r = fabs(d[i]) + (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < n ? fabs(e[i]) : 0.0);
    if (r > tnorm) tnorm = r;
  }
  if (tnorm == 0.0) tnorm = 1.0;
  double pert = 0x1p-52 * tnorm;
  double *u0 = (double *)malloc((size_t)n * sizeof(double)); /* pivot row diag */
  double *u1 = (double *)malloc((size_t)n * sizeof(double)); /* first super */
  double *u2 = (double *)malloc((size_t)n * sizeof(double)); /* second super */
  double *ml = (double *)malloc((size_t)n * sizeof(double)); /* multipliers */
  char *sw = (char *)malloc((size_t)n);
  int64_t cluster_start = 0;
  uint64_t rng = 0x9E3779B97F4A7C15ull;
  for (int64_t c = 0; c < s; c++) {
    if (c > 0 && lam[c] - lam[c - 1] > 1e-3 * tnorm) cluster_start = c;
    double sh = lam[c];
    /* LU of T - sh I with row interchanges */
    {
      double a = d[0] - sh, b = (n > 1) ? e[0] : 0.0, cc = 0.0;
      for (int64_t i = 0; i < n; i++) {
        /* current row i holds (a at col i, b at col i+1, cc at col i+2) */
        if (i == n - 1) {
          u0[i] = (a == 0.0) ? pert : a; u1[i] = 0.0; u2[i] = 0.0; sw[i] = 0; ml[i] = 0.0;
          break;
        }
        double sub = e[i];                    /* T[i+1][i] */
        double nd = d[i + 1] - sh, ns = (i + 2 < n) ? e[i + 1] : 0.0;
        if (fabs(a) >= fabs(sub)) {
          double piv = (a == 0.0) ? pert : a;
          double mlt = sub / piv;
          u0[i] = piv; u1[i] = b; u2[i] = cc; sw[i] = 0; ml[i] = mlt;
          a = nd - mlt * b; b = ns - mlt * cc; cc = 0.0;
        } else {
          double mlt = a / sub;
          u0[i] = sub; u1[i] = nd; u2[i] = ns; sw[i] = 1; ml[i] = mlt;
          double na = b - mlt * nd, nb = cc - mlt * ns;
          a = na; b = nb; cc = 0.0;
        }
      }
    }
    double *z = &Z[IDX(0, c, ldz)];
    for (int64_t i = 0; i < n; i++) {
      rng ^= rng << 13; rng ^= rng >> 7; rng ^= rng << 17;
      z[i] = ((double)(rng >> 11) * 0x1p-53) - 0.5;
    }
    for (int it = 0; it < 4; it++) {
      /* forward: apply the row interchanges and multipliers */
      for (int64_t i = 0; i + 1 < n; i++) {
        if (sw[i]) { double t = z[i]; z[i] = z[i + 1]; z[i + 1] = t; }
        z[i + 1] -= ml[i] * z[i];
      }
      /* back substitution with the upper factor (diag u0, supers u1, u2) */
      for (int64_t i = n - 1; i >= 0; i--) {
        double t = z[i];
        if (i + 1 < n) t -= u1[i] * z[i + 1];
        if (i + 2 < n) t -= u2[i] * z[i + 2];
        z[i] = t / u0[i];
      }
      /* orthogonalise against the cluster (twice), then normalise */
      for (int pass = 0; pass < 2; pass++)
        for (int64_t j = cluster_start; j < c; j++) {
          const double *q = &Z[IDX(0, j, ldz)];
          double dot = 0.0;
          for (int64_t i = 0; i < n; i++) dot += q[i] * z[i];
          for (int64_t i = 0; i < n; i++) z[i] -= dot * q[i];
        }
      double nrm = 0.0;
      for (int64_t i = 0; i < n; i++) nrm += z[i] * z[i];
      nrm = sqrt(nrm);
      if (nrm == 0.0) nrm = 1.0;
      for (int64_t i = 0; i < n; i++) z[i] /= nrm;
    }
  }
  free(u0); free(u1); free(u2); free(ml); free(sw);
}

/* ------------------------------------------------------------------------ */
/* Brute force: cyclic-by-row Jacobi on a full symmetric C (n-by-n, small). */
/* Each rotation zeroes C[p][q]; sweeps repeat until the off-diagonal mass  */
/* is below 1e-30 of the total.  Eigenvalues ascending in w, vectors in V.  */
/* Independent of the Householder/QL route above.                           */
/* ------------------------------------------------------------------------ */
int oracle_jacobi(int64_t n, double *C, int64_t ldc, double *w, double *V, int64_t ldv) {
  for (int64_t j = 0; j < n; j++)
    for (int64_t i = 0; i < n; i++) V[IDX(i, j, ldv)] = (i == j) ? 1.0 : 0.0;
  int sweep;
  for (sweep = 0; sweep < 100; sweep++) {
    double off = 0.0, tot = 0.0;
    for (int64_t j = 0; j < n; j++)
      for (int64_t i = 0; i < n; i++) {
        double a = C[IDX(i, j, ldc)];
        tot += a * a;
        if (i != j) off += a * a;
      }
    if (off <= 1e-30 * tot) break;
    for (int64_t p = 0; p < n - 1; p++)
      for (int64_t q = p + 1; q < n; q++) {
        double apq = C[IDX(p, q, ldc)];
        if (apq == 0.0) continue;
        double theta = (C[IDX(q, q, ldc)] - C[IDX(p, p, ldc)]) / (2.0 * apq);
        double t = ((theta >= 0.0) ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        /* C <- J^T C J with J the rotation in the (p, q) plane */
        for (int64_t k = 0; k < n; k++) {
          double ckp = C[IDX(k, p, ldc)], ckq = C[IDX(k, q, ldc)];
          C[IDX(k, p, ldc)] = c * ckp - s * ckq;
          C[IDX(k, q, ldc)] = s * ckp + c * ckq;
        }
        for (int64_t k = 0; k < n; k++) {
          double cpk = C[IDX(p, k, ldc)], cqk = C[IDX(q, k, ldc)];
          C[IDX(p, k, ldc)] = c * cpk - s * cqk;
          C[IDX(q, k, ldc)] = s * cpk + c * cqk;
        }
        for (int64_t k = 0; k < n; k++) {
          double vkp = V[IDX(k, p, ldv)], vkq = V[IDX(k, q, ldv)];
          V[IDX(k, p, ldv)] = c * vkp - s * vkq;
          V[IDX(k, q, ldv)] = s * vkp + c * vkq;
        }
      }
  }
  for (int64_t i = 0; i < n; i++) w[i] = C[IDX(i, i, ldc)];
  for (int64_t i = 0; i + 1 < n; i++) {
    int64_t k = i;
    for (int64_t j = i + 1; j < n; j++)
      if (w[j] < w[k]) k = j;
    if (k != i) {
      double t = w[i]; w[i] = w[k]; w[k] = t;
      for (int64_t r = 0; r < n; r++) {
        double u = V[IDX(r, i, ldv)];
        V[IDX(r, i, ldv)] = V[IDX(r, k, ldv)];
        V[IDX(r, k, ldv)] = u;
      }
    }
  }
  return sweep < 100 ? 0 : -1;
}

/* ------------------------------------------------------------------------ */
/* The whole route for the s smallest (which = 0) or largest (which = 1)    */
/* eigenpairs of (A, B).  A (lower triangle read) is overwritten by C and   */
/* then by the reflectors; B's upper triangle by U.  w gets the s values in */
/* ascending order, X (n-by-s) the B-orthonormal eigenvectors.               */
/* vec_mode 0: QL accumulation of all vectors (O(n^3), small n);            */
/* vec_mode 1: inverse iteration on T for the s wanted vectors only.        */
/* Returns 0, a positive Cholesky pivot index, or -1 on QL failure.         */
/* ------------------------------------------------------------------------ */
int oracle_gsyeig(int64_t n, double *A, int64_t lda, double *B, int64_t ldb, int64_t s, int which,
                  int vec_mode, double *w, double *X, int64_t ldx) {
  int info = oracle_potrf(n, B, ldb);
  if (info) return info;
  oracle_sygst(n, A, lda, B, ldb);
  double *d = (double *)malloc((size_t)n * sizeof(double));
  double *e = (double *)calloc((size_t)n, sizeof(double));
  double *tau = (double *)calloc((size_t)n, sizeof(double));
  oracle_tridiag(n, A, lda, d, e, tau);
  int64_t off = (which == 1) ? n - s : 0;
  if (vec_mode == 0) {
    double *Z = (double *)calloc((size_t)n * (size_t)n, sizeof(double));
    for (int64_t i = 0; i < n; i++) Z[IDX(i, i, n)] = 1.0;
    int st = oracle_tql(n, d, e, Z, n);
    if (st) { free(Z); free(d); free(e); free(tau); return -1; }
    for (int64_t c = 0; c < s; c++) {
      w[c] = d[off + c];
      memcpy(&X[IDX(0, c, ldx)], &Z[IDX(0, off + c, n)], (size_t)n * sizeof(double));
    }
    free(Z);
  } else {
    double *dd = (double *)malloc((size_t)n * sizeof(double));
    double *ee = (double *)calloc((size_t)n, sizeof(double));
    memcpy(dd, d, (size_t)n * sizeof(double));
    memcpy(ee, e, (size_t)n * sizeof(double));
    int st = oracle_tql(n, dd, ee, NULL, 0);
    if (st) { free(dd); free(ee); free(d); free(e); free(tau); return -1; }
    for (int64_t c = 0; c < s; c++) w[c] = dd[off + c];
    oracle_tri_invit(n, d, e, s, w, X, ldx);
    free(dd);
    free(ee);
  }
  oracle_apply_q(n, A, lda, tau, s, X, ldx);
  oracle_backsolve(n, s, B, ldb, X, ldx);
  free(d);
  free(e);
  free(tau);
  return 0;
}

/* Number of OpenMP threads the oracle runs on (1 without OpenMP). */
int oracle_num_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}
