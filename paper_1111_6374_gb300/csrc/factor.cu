// Blocked dense steps of the route (gs1, gs2, bt1 in Table 1 of the paper):
//   potrf  B = U^T U                    (Eq. 2)   n^3/3 flops
//   sygst  C = U^-T A U^-1              (Eq. 3)   4n^3/3 flops here
//   trsm   X = U^-1 Y                   (Eq. 4)   n^2 s flops
// All bulk work goes through the GEMM engine; the only other kernels are the
// nb x nb diagonal-block factor/inverse (one CTA each) and copies.
//
// sygst: the paper computes C with two triangular solves (2n^3, Section 4.1)
// or, exploiting symmetry, with n^3.  Here step 1 forms W = U^-T A in full
// (n^3) and step 2 forms only the lower triangle of C = W U^-1, which needs
// only the lower triangle of W at each stage (n^3/3), then mirrors it:
// 4n^3/3 flops with nothing but GEMM-shaped updates.
#include "common.cuh"

namespace gs {
namespace {

constexpr int DIAG_THREADS = 256;

// Shared-memory nb x nb block, column-major with leading dimension nb + 1.
struct SmemBlock {
  double *p;
  int ld;
  __device__ double &operator()(int i, int j) { return p[i + j * ld]; }
};

// Inverse of the upper-triangular kb x kb block S (in shared memory) into
// the global nb x nb block `out` (ld nb, zeros below the diagonal): each
// thread owns whole columns c and back-substitutes U x = e_c upwards, so no
// thread reads another thread's output.
__device__ void upper_inverse(SmemBlock S, double *out, int nb, int kb) {
  for (int c = threadIdx.x; c < nb; c += blockDim.x) {
    double *x = out + (size_t)c * nb;
    for (int i = nb - 1; i > c || (c >= kb && i >= 0); i--) x[i] = 0.0;
    if (c >= kb) continue;
    x[c] = 1.0 / S(c, c);
    for (int i = c - 1; i >= 0; i--) {
      double t = 0.0;
      for (int k = i + 1; k <= c; k++) t = fma(S(i, k), x[k], t);
      x[i] = -t / S(i, i);
    }
  }
}

// Factor the diagonal block B[k0:k0+kb, k0:k0+kb] (upper triangle) in
// place, B_kk = U_kk^T U_kk, then store U_kk^-1 (kb x kb, ld nb, zeros below
// the diagonal) in Uinv.  A non-positive or NaN pivot records its global
// 1-based index in *flag and stops.
__global__ void __launch_bounds__(DIAG_THREADS) k_potrf_diag(double *B, int64_t ldb, int64_t k0, int kb, int nb,
                                                             double *Uinv, int *flag) {
  extern __shared__ double smem[];
  __shared__ int s_bad;
  if (*flag) return;
  SmemBlock S{smem, nb + 1};
  const int t = threadIdx.x;
  for (int idx = t; idx < kb * kb; idx += blockDim.x) {
    int i = idx % kb, j = idx / kb;
    S(i, j) = (i <= j) ? B[GS_IDX(k0 + i, k0 + j, ldb)] : 0.0;
  }
  if (t == 0) s_bad = 0;
  __syncthreads();
  for (int j = 0; j < kb; j++) {
    if (t == 0) {
      double d = S(j, j);
      if (!(d > 0.0)) {
        s_bad = (int)(k0 + j + 1);
      } else {
        S(j, j) = sqrt(d);
      }
    }
    __syncthreads();
    if (s_bad) break;
    double piv = S(j, j);
    for (int c = j + 1 + t; c < kb; c += blockDim.x) S(j, c) /= piv;
    __syncthreads();
    // trailing update of the upper triangle: S(r, c) -= S(j, r) S(j, c), j < r <= c
    int w = kb - j - 1;
    for (int idx = t; idx < w * w; idx += blockDim.x) {
      int r = j + 1 + idx % w, c = j + 1 + idx / w;
      if (r <= c) S(r, c) = fma(-S(j, r), S(j, c), S(r, c));
    }
    __syncthreads();
  }
  if (s_bad) {
    if (t == 0) atomicCAS(flag, 0, s_bad);
    return;
  }
  upper_inverse(S, Uinv, nb, kb);
  for (int idx = t; idx < kb * kb; idx += blockDim.x) {
    int i = idx % kb, j = idx / kb;
    if (i <= j) B[GS_IDX(k0 + i, k0 + j, ldb)] = S(i, j);
  }
}

// Inverse of every diagonal block of an upper-triangular U (one CTA each).
__global__ void __launch_bounds__(DIAG_THREADS) k_trtri_diag(int64_t n, const double *U, int64_t ldu, int nb,
                                                             double *Uinv) {
  extern __shared__ double smem[];
  SmemBlock S{smem, nb + 1};
  const int64_t k0 = (int64_t)blockIdx.x * nb;
  const int kb = (int)std::min<int64_t>(nb, n - k0);
  for (int idx = threadIdx.x; idx < kb * kb; idx += blockDim.x) {
    int i = idx % kb, j = idx / kb;
    S(i, j) = (i <= j) ? U[GS_IDX(k0 + i, k0 + j, ldu)] : 0.0;
  }
  __syncthreads();
  upper_inverse(S, Uinv + (size_t)blockIdx.x * nb * nb, nb, kb);
}

size_t diag_smem_bytes(int nb) { return (size_t)(nb + 1) * nb * sizeof(double); }

int set_smem(const void *fn, size_t bytes) {
  if (bytes > 48 * 1024) GS_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return GSYEIG_SUCCESS;
}

}  // namespace

int trtri_diag_blocks(cudaStream_t st, int64_t n, const double *U, int64_t ldu, int nb, double *Uinv) {
  size_t sm = diag_smem_bytes(nb);
  GS_TRY(set_smem((const void *)k_trtri_diag, sm));
  k_trtri_diag<<<(unsigned)ceil_div(n, nb), DIAG_THREADS, sm, st>>>(n, U, ldu, nb, Uinv);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

// Two-level blocking: inner steps of nb (the diagonal-block kernels and the
// panels) and outer blocks of NB = kOuter nb.  Within an outer block the
// inner rank-nb updates touch only the rest of the outer block; the trailing
// matrix beyond it receives one rank-NB update per outer block, so the
// GEMM engine's per-element epilogue is paid once per NB columns of K
// instead of once per nb.
constexpr int kOuter = 4;

int potrf_blocked(cudaStream_t st, int64_t n, double *B, int64_t ldb, int nb, FactorWork &w) {
  size_t sm = diag_smem_bytes(nb);
  GS_TRY(set_smem((const void *)k_potrf_diag, sm));
  GS_CUDA(cudaMemsetAsync(w.flag, 0, sizeof(int), st));
  const int64_t NB = (int64_t)kOuter * nb;
  for (int64_t J0 = 0; J0 < n; J0 += NB) {
    const int64_t J1 = std::min(n, J0 + NB);
    for (int64_t k0 = J0; k0 < J1; k0 += nb) {
      const int kb = (int)std::min<int64_t>(nb, J1 - k0);
      double *Uinv_k = w.Uinv + (size_t)(k0 / nb) * nb * nb;
      k_potrf_diag<<<1, DIAG_THREADS, sm, st>>>(B, ldb, k0, kb, nb, Uinv_k, w.flag);
      count_launch();
      GS_CHECK_LAUNCH();
      const int64_t rest = n - k0 - kb;
      if (rest <= 0) break;
      double *Bk = &B[GS_IDX(k0, k0 + kb, ldb)];
      // U_k,rest = U_kk^-T B_k,rest  (panel, kb x rest, staged)
      GS_TRY(dgemm(st, true, false, kb, rest, kb, 1.0, Uinv_k, nb, Bk, ldb, 0.0, w.panel, kb, TRI_ALL, 0, w.flag));
      GS_TRY(copy_block(st, kb, rest, w.panel, kb, Bk, ldb, w.flag));
      // rows of the outer block below this step: B (upper) -= U_k,.^T U_k,.
      const int64_t rin = J1 - k0 - kb;
      if (rin > 0)
        GS_TRY(dgemm(st, true, false, rin, rest, kb, -1.0, w.panel, kb, w.panel, kb, 1.0,
                     &B[GS_IDX(k0 + kb, k0 + kb, ldb)], ldb, TRI_UPPER, 0, w.flag));
    }
    // trailing matrix beyond the outer block (upper) -= U_J,rest^T U_J,rest
    const int64_t r2 = n - J1;
    if (r2 > 0)
      GS_TRY(dgemm(st, true, false, r2, r2, J1 - J0, -1.0, &B[GS_IDX(J0, J1, ldb)], ldb, &B[GS_IDX(J0, J1, ldb)], ldb,
                   1.0, &B[GS_IDX(J1, J1, ldb)], ldb, TRI_UPPER, 0, w.flag));
  }
  return GSYEIG_SUCCESS;
}

int sygst_blocked(cudaStream_t st, int64_t n, double *A, int64_t lda, const double *U, int64_t ldu, int nb,
                  FactorWork &w, bool have_uinv) {
  GS_TRY(symmetrize(st, n, A, lda, true));
  if (!have_uinv) GS_TRY(trtri_diag_blocks(st, n, U, ldu, nb, w.Uinv));
  const int64_t NB = (int64_t)kOuter * nb;
  // Step 1: W = U^-T A, block row by block row (forward substitution).
  for (int64_t J0 = 0; J0 < n; J0 += NB) {
    const int64_t J1 = std::min(n, J0 + NB);
    for (int64_t k0 = J0; k0 < J1; k0 += nb) {
      const int kb = (int)std::min<int64_t>(nb, J1 - k0);
      const double *Uinv_k = w.Uinv + (size_t)(k0 / nb) * nb * nb;
      double *Ak = &A[GS_IDX(k0, 0, lda)];
      GS_TRY(dgemm(st, true, false, kb, n, kb, 1.0, Uinv_k, nb, Ak, lda, 0.0, w.panel, kb));
      GS_TRY(copy_block(st, kb, n, w.panel, kb, Ak, lda));
      const int64_t rin = J1 - k0 - kb;  // rows of the outer block below this step
      if (rin > 0)
        GS_TRY(dgemm(st, true, false, rin, n, kb, -1.0, &U[GS_IDX(k0, k0 + kb, ldu)], ldu, w.panel, kb, 1.0,
                     &A[GS_IDX(k0 + kb, 0, lda)], lda));
    }
    const int64_t r2 = n - J1;  // rows beyond the outer block: one rank-NB update
    if (r2 > 0)
      GS_TRY(dgemm(st, true, false, r2, n, J1 - J0, -1.0, &U[GS_IDX(J0, J1, ldu)], ldu, &A[GS_IDX(J0, 0, lda)], lda,
                   1.0, &A[GS_IDX(J1, 0, lda)], lda));
  }
  // Step 2: lower triangle of C = W U^-1, block column by block column.
  for (int64_t J0 = 0; J0 < n; J0 += NB) {
    const int64_t J1 = std::min(n, J0 + NB);
    for (int64_t k0 = J0; k0 < J1; k0 += nb) {
      const int kb = (int)std::min<int64_t>(nb, J1 - k0);
      const int64_t rows = n - k0;
      const double *Uinv_k = w.Uinv + (size_t)(k0 / nb) * nb * nb;
      double *Ck = &A[GS_IDX(k0, k0, lda)];
      GS_TRY(dgemm(st, false, false, rows, kb, kb, 1.0, Ck, lda, Uinv_k, nb, 0.0, w.panel, rows));
      GS_TRY(copy_block(st, rows, kb, w.panel, rows, Ck, lda));
      const int64_t rest = n - k0 - kb;
      const int64_t cin = J1 - k0 - kb;  // columns of the outer block right of this step
      if (cin > 0)
        GS_TRY(dgemm(st, false, false, rest, cin, kb, -1.0, &w.panel[kb], rows, &U[GS_IDX(k0, k0 + kb, ldu)], ldu,
                     1.0, &A[GS_IDX(k0 + kb, k0 + kb, lda)], lda, TRI_LOWER, 0));
    }
    const int64_t r2 = n - J1;  // lower trailing matrix beyond the outer block: one rank-NB update
    if (r2 > 0)
      GS_TRY(dgemm(st, false, false, r2, r2, J1 - J0, -1.0, &A[GS_IDX(J1, J0, lda)], lda, &U[GS_IDX(J0, J1, ldu)],
                   ldu, 1.0, &A[GS_IDX(J1, J1, lda)], lda, TRI_LOWER, 0));
  }
  GS_TRY(symmetrize(st, n, A, lda, true));
  return GSYEIG_SUCCESS;
}

int trsm_back_blocked(cudaStream_t st, int64_t n, const double *U, int64_t ldu, double *Y, int64_t ldy, int64_t s,
                      int nb, FactorWork &w, bool have_uinv) {
  if (!have_uinv) GS_TRY(trtri_diag_blocks(st, n, U, ldu, nb, w.Uinv));
  const int64_t last = ((n - 1) / nb) * nb;
  for (int64_t k0 = last; k0 >= 0; k0 -= nb) {
    const int kb = (int)std::min<int64_t>(nb, n - k0);
    const double *Uinv_k = w.Uinv + (size_t)(k0 / nb) * nb * nb;
    double *Yk = &Y[GS_IDX(k0, 0, ldy)];
    GS_TRY(dgemm(st, false, false, kb, s, kb, 1.0, Uinv_k, nb, Yk, ldy, 0.0, w.panel, kb));
    GS_TRY(copy_block(st, kb, s, w.panel, kb, Yk, ldy));
    if (k0 > 0)
      GS_TRY(dgemm(st, false, false, k0, s, kb, -1.0, &U[GS_IDX(0, k0, ldu)], ldu, w.panel, kb, 1.0, Y, ldy));
  }
  return GSYEIG_SUCCESS;
}

}  // namespace gs
