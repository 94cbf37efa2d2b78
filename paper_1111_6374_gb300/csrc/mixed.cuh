// The mixed-precision Lanczos stage: an fp32 block operator (symm32.cu).
#pragma once

#include "common.cuh"

namespace gs {

// C's lower triangle as fp32 tiles (scaled by a power of two), with the
// fp32 staging blocks of one product.
struct F32Operator {
  int64_t n = 0, NT = 0, npad = 0;
  float *tiles = nullptr;              // f32_operator_bytes(n), scale word at its end
  float *W = nullptr, *Z = nullptr;    // f32_block_bytes(n) each
  unsigned long long *amax = nullptr;  // device: max |C| (bits)
};

size_t f32_operator_bytes(int64_t n);
size_t f32_block_bytes(int64_t n);
// Fill op.tiles from the full symmetric C (op.tiles, op.W, op.Z set by the caller).
int f32_operator_build(cudaStream_t st, int64_t n, const double *C, int64_t ldc, F32Operator &op);
// Z = C V for the n x 16 block V (column-major FP64, rounded to fp32), fp32
// products and sums, Z column-major FP64.
int f32_symm(cudaStream_t st, const F32Operator &op, const double *V, int64_t ldv, double *Z, int64_t ldz);

// ---- blocklz.cu: FP64 kernels of the block stage ---------------------------
// doubles of the slice partials of ts_dots for an n-row basis of w columns
size_t ts_part_doubles(int64_t n, int64_t w);
// H (w x b, ld ldh) = V^T Z for V n x w (ld ldv) and Z n x b (ld ldz), b <= 16
int ts_dots(cudaStream_t st, int64_t n, int64_t w, int b, const double *V, int64_t ldv, const double *Z, int64_t ldz,
            double *part, double *H, int64_t ldh);
// Z -= V H (w <= 1600)
int ts_update(cudaStream_t st, int64_t n, int64_t w, int b, const double *V, int64_t ldv, const double *H, int64_t ldh,
              double *Z, int64_t ldz);
int col_norms(cudaStream_t st, int64_t n, int64_t cols, const double *X, int64_t ldx, double *norms);
int scale_cols(cudaStream_t st, int64_t n, int64_t cols, double *X, int64_t ldx, const double *norms);
// R = CX - X diag(theta) (all n x k, leading dimension ld)
int block_resid(cudaStream_t st, int64_t n, int64_t k, const double *CX, const double *X, int64_t ld,
                const double *theta, double *R);
// T[r0.., c0..] = M (m x m), and its transpose at [c0.., r0..] with mirror
int put_block(cudaStream_t st, int m, const double *M, int64_t ldm, double *T, int64_t ldt, int64_t r0, int64_t c0,
              bool mirror);
// T <- (T + T^T) / 2
int sym_avg(cudaStream_t st, int64_t m, double *T, int64_t ldt);
// out[0] (device) = max_i sum_j |T(i, j)|
int inf_norm(cudaStream_t st, int64_t m, const double *T, int64_t ldt, double *out);
// out[c] = X(:, c) . Y(:, c) for c < cols
int column_dots(cudaStream_t st, int64_t n, int64_t cols, const double *X, int64_t ldx, const double *Y, int64_t ldy,
                double *out);
// M(i, j) *= theta_i^pa theta_j^pb (m x m; theta device, positive)
int scale_by_powers(cudaStream_t st, int64_t m, double *M, int64_t ldm, const double *theta, double pa, double pb);
// out[0] (device double) = the 1-norm of the n x n M
int mat_norm1(cudaStream_t st, int64_t n, const double *M, int64_t ldm, double *out);
// dst(:, c) = src(:, idx[c]) for c < cnt (idx device)
int gather_cols(cudaStream_t st, int64_t n, int64_t cnt, const int *idx, const double *src, int64_t lds, double *dst,
                int64_t ldd);
// dst = upper triangle of src, zeros below (b x b)
int copy_upper(cudaStream_t st, int64_t b, const double *src, int64_t lds, double *dst, int64_t ldd);
// T[r0.., r0..] = M1 + M2 (b x b, ld ldm)
int put_sum(cudaStream_t st, int b, const double *M1, const double *M2, int64_t ldm, double *T, int64_t ldt,
            int64_t r0);

}  // namespace gs
