// The mixed-precision operator (ke1 in FP32): Z = C W for a block W of 16
// vectors, with C stored once per solve as fp32 tiles of its lower triangle
// and every product accumulated in fp32.  Stored bytes are 4 n(n+1)/2, half
// of the double-float operator's; the block of 16 reuses each stored entry
// for 32 products.
//
// Layout: as the double-float operator (symv_df.cu), tile t = bi (bi + 1) /
// 2 + bj of 64 x 64 entries, element (r, c) at (r ^ (c & 31)) + 64 c, C
// scaled by the power of two 2^-e that brings max|C| into [1/2, 1) (exact;
// results scaled back).  W and Z are row-major n x 16 (the 16 values of a
// row contiguous).
//
// One CTA per block row i computes Z_i = sum_{j <= i} C_ij W_j +
// sum_{j > i} C_ji^T W_j: it reads the i + 1 tiles of its row and the
// NT - 1 - i tiles below the diagonal in its column, NT tiles for every CTA
// (balanced), and writes its 64 rows once: no atomics, no partial sums in
// memory, deterministic.  Each tile is read twice in all (8 n^2 bytes per
// product), through a two-deep ring of asynchronous 16-byte copies so that
// the next tile and W slice land while the current ones are used.
#include "mixed.cuh"

namespace gs {
namespace {

constexpr int TS = 64;
constexpr int NB = 16;          // vectors per block
constexpr int S32_THREADS = 256;  // thread (row r = t % 64, column quad q = t / 64)

__global__ void k_f32_absmax(int64_t n, const double *__restrict__ C, int64_t ldc, unsigned long long *amax) {
  const int64_t bi = blockIdx.y, bj = blockIdx.x;
  if (bj > bi) return;
  unsigned long long mx = 0;
  for (int idx = threadIdx.x; idx < TS * TS; idx += blockDim.x) {
    const int r = idx % TS, c = idx / TS;
    const int64_t i = bi * TS + r, j = bj * TS + c;
    if (i < n && j < n) {
      const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(C[i + j * ldc]));
      if (b < 0x7FF0000000000000ull && b > mx) mx = b;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = y > mx ? y : mx;
  }
  if ((threadIdx.x & 31) == 0 && mx) atomicMax(amax, mx);
}

__device__ __forceinline__ int scale_exp(const unsigned long long *amax) {
  const unsigned long long b = *amax;
  if (b == 0) return 0;
  int e;
  frexp(__longlong_as_double((long long)b), &e);
  return e;
}

__global__ void k_f32_build(int64_t n, const double *__restrict__ C, int64_t ldc, const unsigned long long *amax,
                            float *__restrict__ T) {
  const int64_t bi = blockIdx.y, bj = blockIdx.x;
  if (bj > bi) return;
  float *h = T + (bi * (bi + 1) / 2 + bj) * TS * TS;
  const int e = scale_exp(amax);
  for (int idx = threadIdx.x; idx < TS * TS; idx += blockDim.x) {
    const int r = idx % TS, c = idx / TS;
    const int64_t i = bi * TS + r, j = bj * TS + c;
    const double v = (i < n && j < n) ? ldexp(C[i + j * ldc], -e) : 0.0;
    h[(r ^ (c & 31)) + TS * c] = (float)v;
  }
}

// W32 (row-major npad x 16) = V (column-major n x 16, ld ldv), zero rows past n
__global__ void k_to_f32(int64_t n, int64_t npad, const double *__restrict__ V, int64_t ldv, float *__restrict__ W) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < npad * NB;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / NB;
    const int c = (int)(idx % NB);
    W[idx] = (i < n) ? (float)V[i + c * ldv] : 0.f;
  }
}

// Z (column-major n x 16, ld ldz, FP64) = 2^e Z32
__global__ void k_from_f32(int64_t n, const float *__restrict__ Z32, const unsigned long long *amax, double *__restrict__ Z,
                           int64_t ldz) {
  const int e = scale_exp(amax);
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n * NB;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / NB;
    const int c = (int)(idx % NB);
    Z[i + c * ldz] = ldexp((double)Z32[idx], e);
  }
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}

// The tile and W slice of step `step` of block row i into shared buffer b
// (asynchronous 16-byte copies, one commit group).
__device__ __forceinline__ void s32_prefetch(int i, int step, const float *__restrict__ T, const float *__restrict__ W,
                                             float *tile, float *wj) {
  const int j = step;
  const bool row = step <= i;
  const int bi = row ? i : j, bj = row ? j : i;
  const float *src = T + ((int64_t)bi * (bi + 1) / 2 + bj) * TS * TS;
  for (int idx = threadIdx.x; idx < TS * TS / 4; idx += S32_THREADS) cp_async16(tile + 4 * idx, src + 4 * idx);
  const float *ws = W + (int64_t)j * TS * NB;
  for (int idx = threadIdx.x; idx < TS * NB / 4; idx += S32_THREADS) cp_async16(wj + 4 * idx, ws + 4 * idx);
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

__global__ void __launch_bounds__(S32_THREADS) k_symm32(int NT, const float *__restrict__ T, const float *__restrict__ W,
                                                        float *__restrict__ Z) {
  // two buffers: the copies of step + 1 run while step is computed
  __shared__ __align__(16) float tile[2][TS * TS];
  __shared__ __align__(16) float wj[2][TS * NB];
  const int i = blockIdx.x;
  // thread (row r, quarter kq of the tile's 64 k): all 16 vectors of row r
  // over k = 16 kq .. 16 kq + 15; the W row of each k is one broadcast
  // 64-byte read per warp, so a warp does 16 FMAs per 5 shared-memory
  // wavefronts; the four quarters are summed once at the end
  const int t = threadIdx.x, r = t % TS, kq = t / TS;
  float acc[NB];
#pragma unroll
  for (int c = 0; c < NB; c++) acc[c] = 0.f;
  s32_prefetch(i, 0, T, W, tile[0], wj[0]);
  for (int step = 0; step < NT; step++) {
    const int b = step & 1;
    if (step + 1 < NT) {
      s32_prefetch(i, step + 1, T, W, tile[b ^ 1], wj[b ^ 1]);
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    }
    __syncthreads();  // every thread's copies of this step have landed
    const float *tl = tile[b];
    const float4 *wv = reinterpret_cast<const float4 *>(wj[b]);
    const bool row = step <= i;
#pragma unroll 4
    for (int kk = 0; kk < 16; kk++) {
      const int k = 16 * kq + kk;
      // row tiles: C_ij(r, k); column tiles: C_ji(k, r) (column r of the stored tile)
      const float c = row ? tl[(r ^ (k & 31)) + TS * k] : tl[(k ^ (r & 31)) + TS * r];
      const float4 w0 = wv[k * 4 + 0], w1 = wv[k * 4 + 1], w2 = wv[k * 4 + 2], w3 = wv[k * 4 + 3];
      acc[0] = fmaf(c, w0.x, acc[0]);
      acc[1] = fmaf(c, w0.y, acc[1]);
      acc[2] = fmaf(c, w0.z, acc[2]);
      acc[3] = fmaf(c, w0.w, acc[3]);
      acc[4] = fmaf(c, w1.x, acc[4]);
      acc[5] = fmaf(c, w1.y, acc[5]);
      acc[6] = fmaf(c, w1.z, acc[6]);
      acc[7] = fmaf(c, w1.w, acc[7]);
      acc[8] = fmaf(c, w2.x, acc[8]);
      acc[9] = fmaf(c, w2.y, acc[9]);
      acc[10] = fmaf(c, w2.z, acc[10]);
      acc[11] = fmaf(c, w2.w, acc[11]);
      acc[12] = fmaf(c, w3.x, acc[12]);
      acc[13] = fmaf(c, w3.y, acc[13]);
      acc[14] = fmaf(c, w3.z, acc[14]);
      acc[15] = fmaf(c, w3.w, acc[15]);
    }
    __syncthreads();  // buffer b is free for the copies of step + 2
  }
  // sum the four quarters (tile[0] as scratch: 4 x 64 x 16 floats)
  float *red = tile[0];
#pragma unroll
  for (int c = 0; c < NB; c++) red[(kq * TS + r) * NB + c] = acc[c];
  __syncthreads();
  for (int idx = t; idx < TS * NB; idx += S32_THREADS) {
    const int rr = idx / NB, c = idx % NB;
    Z[((int64_t)i * TS + rr) * NB + c] = ((red[(0 * TS + rr) * NB + c] + red[(1 * TS + rr) * NB + c]) +
                                          red[(2 * TS + rr) * NB + c]) + red[(3 * TS + rr) * NB + c];
  }
}

}  // namespace

size_t f32_operator_bytes(int64_t n) {
  const int64_t NT = ceil_div(n, TS);
  return (size_t)NT * (NT + 1) / 2 * TS * TS * sizeof(float) + 256;
}

size_t f32_block_bytes(int64_t n) { return (size_t)ceil_div(n, TS) * TS * NB * sizeof(float); }

int f32_operator_build(cudaStream_t st, int64_t n, const double *C, int64_t ldc, F32Operator &op) {
  const int64_t NT = ceil_div(n, TS);
  op.n = n;
  op.NT = NT;
  op.npad = NT * TS;
  op.amax = reinterpret_cast<unsigned long long *>(reinterpret_cast<char *>(op.tiles) + f32_operator_bytes(n) - 256);
  GS_CUDA(cudaMemsetAsync(op.amax, 0, sizeof(unsigned long long), st));
  k_f32_absmax<<<dim3((unsigned)NT, (unsigned)NT), 256, 0, st>>>(n, C, ldc, op.amax);
  k_f32_build<<<dim3((unsigned)NT, (unsigned)NT), 256, 0, st>>>(n, C, ldc, op.amax, op.tiles);
  count_launch(2);
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

int f32_symm(cudaStream_t st, const F32Operator &op, const double *V, int64_t ldv, double *Z, int64_t ldz) {
  KernelProfiler *prof = current_profiler();
  const size_t e0 = prof ? prof->start(st) : SIZE_MAX;
  const unsigned g = (unsigned)std::min<int64_t>(ceil_div(op.npad * NB, 256), 4096);
  k_to_f32<<<g, 256, 0, st>>>(op.n, op.npad, V, ldv, op.W);
  k_symm32<<<(unsigned)op.NT, S32_THREADS, 0, st>>>((int)op.NT, op.tiles, op.W, op.Z);
  k_from_f32<<<g, 256, 0, st>>>(op.n, op.Z, op.amax, Z, ldz);
  count_launch(3);
  GS_CHECK_LAUNCH();
  if (prof) {
    const double n = (double)op.n;
    // algorithmic: 2 n^2 x 16 flops; the stored triangle (4 bytes per entry) once, plus W and Z
    prof->stop(st, e0, PROF_SYMV32, 2.0 * n * n * NB, 4.0 * (n * (n + 1) / 2) + 2.0 * 4.0 * n * NB);
  }
  return GSYEIG_SUCCESS;
}

}  // namespace gs
