// ke1 (Table 1): the Lanczos operator application z = C w, 2n^2 flops per
// product (Section 2.3, variant KE).  C is stored full and symmetric, so
// z_j = C[:, j] . w: one warp per column reads that column contiguously
// (16-byte loads), multiplies by w, and reduces with warp shuffles.  No
// workspace, no atomics; the result is bitwise reproducible.
//
// In FP64 this product is bound by the FP64 pipe on GB300 (n^2 FMAs at ~2
// per SM-clock), not by HBM: reading the full square (8n^2 bytes) at the
// measured 6.8 TB/s takes less time than the FMAs.
#include "common.cuh"

namespace gs {
namespace {

constexpr int SYMV_WARPS = 8;

__global__ void __launch_bounds__(SYMV_WARPS * 32) k_symv_cols_v2(int64_t n, const double *__restrict__ C, int64_t ldc,
                                                                  const double *__restrict__ w, double *__restrict__ z) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (int64_t)blockIdx.x * SYMV_WARPS + (threadIdx.x >> 5);
  const int64_t nwarps = (int64_t)gridDim.x * SYMV_WARPS;
  const int64_t n2 = n & ~(int64_t)1;
  const double2 *w2 = reinterpret_cast<const double2 *>(w);
  for (int64_t j = warp; j < n; j += nwarps) {
    const double2 *c2 = reinterpret_cast<const double2 *>(C + (size_t)j * ldc);
    double a0 = 0.0, a1 = 0.0;
    for (int64_t i = lane; i < n2 / 2; i += 32) {
      double2 c = __ldg(&c2[i]);
      double2 x = __ldg(&w2[i]);
      a0 = fma(c.x, x.x, a0);
      a1 = fma(c.y, x.y, a1);
    }
    double acc = a0 + a1;
    if ((n & 1) && lane == 0) acc = fma(C[(size_t)j * ldc + n - 1], w[n - 1], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) z[j] = acc;
  }
}

__global__ void __launch_bounds__(SYMV_WARPS * 32) k_symv_cols(int64_t n, const double *__restrict__ C, int64_t ldc,
                                                               const double *__restrict__ w, double *__restrict__ z) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (int64_t)blockIdx.x * SYMV_WARPS + (threadIdx.x >> 5);
  const int64_t nwarps = (int64_t)gridDim.x * SYMV_WARPS;
  for (int64_t j = warp; j < n; j += nwarps) {
    const double *c = C + (size_t)j * ldc;
    double acc = 0.0;
    for (int64_t i = lane; i < n; i += 32) acc = fma(__ldg(&c[i]), __ldg(&w[i]), acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) z[j] = acc;
  }
}

}  // namespace

int symv_f64(cudaStream_t st, int64_t n, const double *C, int64_t ldc, const double *w, double *z) {
  if (n <= 0) return GSYEIG_SUCCESS;
  const int64_t blocks = std::min<int64_t>(ceil_div(n, SYMV_WARPS), 152 * 16);
  const bool aligned = ((uintptr_t)C % 16 == 0) && (ldc % 2 == 0) && ((uintptr_t)w % 16 == 0);
  KernelProfiler *prof = current_profiler();
  size_t e0 = prof ? prof->start(st) : SIZE_MAX;
  if (aligned)
    k_symv_cols_v2<<<(unsigned)blocks, SYMV_WARPS * 32, 0, st>>>(n, C, ldc, w, z);
  else
    k_symv_cols<<<(unsigned)blocks, SYMV_WARPS * 32, 0, st>>>(n, C, ldc, w, z);
  count_launch();
  GS_CHECK_LAUNCH();
  // algorithmic: 2n^2 flops; the full square of C (8n^2 bytes) plus w and z
  if (prof) prof->stop(st, e0, PROF_SYMV, 2.0 * (double)n * n, 8.0 * ((double)n * n + 2.0 * n));
  return GSYEIG_SUCCESS;
}

}  // namespace gs
