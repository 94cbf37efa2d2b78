// FP64 GEMM engine used by the blocked Cholesky, the explicit transform to
// standard form and the back-transform (Eqs. 2-4 of the paper: every O(n^3)
// flop of gs1/gs2 and the n^2 s flops of bt1 run here).
//
// GB300 has no fast FP64 path: a GB300 SM retires about two FP64 FMAs per
// clock, through DFMA or through the FP64 mma.sync forms alike (about
// 1.0 TFLOP/s for the chip, measured).  The kernel is therefore built to
// keep the FP64 pipe busy and nothing else: 64 x 64 output tile per CTA,
// 4 x 4 register block per thread, 16-deep K slices staged through shared
// memory.  At two FMAs per SM-clock a K slice takes ~32k cycles, so global
// load latency (~1k cycles) needs no multi-stage pipeline.
#include <mutex>

#include "common.cuh"

namespace gs {

std::atomic<int64_t> g_launches{0};

cudaError_t &last_cuda_error() {
  static thread_local cudaError_t e = cudaSuccess;
  return e;
}

int set_max_smem(const void *fn, int bytes) {
  struct Key {
    const void *fn;
    int dev, bytes;
  };
  static std::mutex mu;
  static std::vector<Key> done;
  int dev = 0;
  GS_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  for (const Key &k : done)
    if (k.fn == fn && k.dev == dev && k.bytes >= bytes) return GSYEIG_SUCCESS;
  GS_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  done.push_back({fn, dev, bytes});
  return GSYEIG_SUCCESS;
}

KernelProfiler *&current_profiler() {
  static thread_local KernelProfiler *p = nullptr;
  return p;
}

GemmContext *&current_gemm() {
  static thread_local GemmContext *g = nullptr;
  return g;
}

size_t KernelProfiler::start(cudaStream_t st) {
  if (used + 2 > pool.size()) {
    size_t grow = std::max<size_t>(256, pool.size());
    for (size_t i = 0; i < grow; i++) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return SIZE_MAX;
      }
      pool.push_back(e);
    }
  }
  size_t e0 = used;
  used += 2;
  cudaEventRecord(pool[e0], st);
  return e0;
}

void KernelProfiler::stop(cudaStream_t st, size_t e0, int cls, double flops, double bytes) {
  if (e0 == SIZE_MAX) return;
  cudaEventRecord(pool[e0 + 1], st);
  recs.push_back({cls, flops, bytes, e0});
}

void KernelProfiler::resolve(int64_t launches[PROF_NCLASS], double ms[PROF_NCLASS], double flops[PROF_NCLASS],
                             double bytes[PROF_NCLASS]) {
  for (int c = 0; c < PROF_NCLASS; c++) {
    launches[c] = 0;
    ms[c] = flops[c] = bytes[c] = 0.0;
  }
  for (const Rec &r : recs) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, pool[r.e0], pool[r.e0 + 1]) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    launches[r.cls]++;
    ms[r.cls] += t;
    flops[r.cls] += r.flops;
    bytes[r.cls] += r.bytes;
  }
  recs.clear();
  used = 0;
}

void KernelProfiler::release() {
  for (cudaEvent_t e : pool) cudaEventDestroy(e);
  pool.clear();
  recs.clear();
  used = 0;
}

namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

__global__ void __launch_bounds__(NT) k_dgemm(bool transA, bool transB, int64_t M, int64_t N, int64_t K,
                                              double alpha, const double *__restrict__ A, int64_t lda,
                                              const double *__restrict__ B, int64_t ldb, double beta,
                                              double *__restrict__ C, int64_t ldc, int mode, int64_t diag,
                                              const int *abort_flag) {
  if (abort_flag && *abort_flag) return;
  const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * BN;
  if (mode == TRI_LOWER && (m0 + BM - 1) - n0 + diag < 0) return;
  if (mode == TRI_UPPER && m0 - (n0 + BN - 1) + diag > 0) return;

  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; a++)
#pragma unroll
    for (int b = 0; b < 4; b++) acc[a][b] = 0.0;

  for (int64_t k0 = 0; k0 < K; k0 += BK) {
    // op(A) tile: BM x BK
#pragma unroll
    for (int q = 0; q < 4; q++) {
      int i, k;
      if (!transA) { i = t & 63; k = (t >> 6) + 4 * q; }
      else { k = t & 15; i = (t >> 4) + 16 * q; }
      int64_t gi = m0 + i, gk = k0 + k;
      double v = 0.0;
      if (gi < M && gk < K) v = transA ? A[GS_IDX(gk, gi, lda)] : A[GS_IDX(gi, gk, lda)];
      As[k][i] = v;
    }
    // op(B) tile: BK x BN
#pragma unroll
    for (int q = 0; q < 4; q++) {
      int j, k;
      if (!transB) { k = t & 15; j = (t >> 4) + 16 * q; }
      else { j = t & 63; k = (t >> 6) + 4 * q; }
      int64_t gj = n0 + j, gk = k0 + k;
      double v = 0.0;
      if (gj < N && gk < K) v = transB ? B[GS_IDX(gj, gk, ldb)] : B[GS_IDX(gk, gj, ldb)];
      Bs[k][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; k++) {
      double a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; r++) a[r] = As[k][tx + 16 * r];
#pragma unroll
      for (int r = 0; r < 4; r++) b[r] = Bs[k][ty + 16 * r];
#pragma unroll
      for (int r = 0; r < 4; r++)
#pragma unroll
        for (int c = 0; c < 4; c++) acc[r][c] = fma(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; r++) {
    int64_t gi = m0 + tx + 16 * r;
    if (gi >= M) continue;
#pragma unroll
    for (int c = 0; c < 4; c++) {
      int64_t gj = n0 + ty + 16 * c;
      if (gj >= N) continue;
      int64_t dd = gi - gj + diag;
      if (mode == TRI_LOWER && dd < 0) continue;
      if (mode == TRI_UPPER && dd > 0) continue;
      double *p = &C[GS_IDX(gi, gj, ldc)];
      double v = alpha * acc[r][c];
      if (beta != 0.0) v = fma(beta, *p, v);
      *p = v;
    }
  }
}

__global__ void k_copy_block(int64_t M, int64_t N, const double *__restrict__ src, int64_t lds,
                             double *__restrict__ dst, int64_t ldd, const int *abort_flag) {
  if (abort_flag && *abort_flag) return;
  for (int64_t j = blockIdx.y; j < N; j += gridDim.y)
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x)
      dst[GS_IDX(i, j, ldd)] = src[GS_IDX(i, j, lds)];
}

__global__ void k_axpy_block(int64_t M, int64_t N, double alpha, const double *__restrict__ X, int64_t ldx,
                             double *__restrict__ Y, int64_t ldy) {
  for (int64_t j = blockIdx.y; j < N; j += gridDim.y)
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x)
      Y[GS_IDX(i, j, ldy)] += alpha * X[GS_IDX(i, j, ldx)];
}

// 32 x 32 tiles: tile (bi, bj) with bi > bj is read coalesced and written
// transposed into tile (bj, bi); diagonal tiles mirror in place.
__global__ void k_symmetrize(int64_t n, double *A, int64_t lda, bool lower_to_upper) {
  __shared__ double tile[32][33];
  int64_t bi = blockIdx.x, bj = blockIdx.y;
  if (bi < bj) return;
  int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  // source tile is (bi, bj) for lower->upper, (bj, bi) for upper->lower
  int64_t sr0 = lower_to_upper ? bi * 32 : bj * 32, sc0 = lower_to_upper ? bj * 32 : bi * 32;
  for (int r = ty; r < 32; r += 8) {
    int64_t gi = sr0 + tx, gj = sc0 + r;
    tile[r][tx] = (gi < n && gj < n) ? A[GS_IDX(gi, gj, lda)] : 0.0;
  }
  __syncthreads();
  // destination: element (sc0 + c, sr0 + rr) = source (sr0 + rr, sc0 + c)
  for (int c = ty; c < 32; c += 8) {
    int64_t gi = sc0 + tx, gj = sr0 + c;  // dst row gi = sc0+tx, col gj = sr0+c  <- src (sr0+c, sc0+tx)
    if (gi >= n || gj >= n) continue;
    bool strict = lower_to_upper ? (gi < gj) : (gi > gj);
    if (bi == bj && !strict) continue;
    A[GS_IDX(gi, gj, lda)] = tile[tx][c];
  }
}

__global__ void k_identity(int64_t n, double *__restrict__ X, int64_t ldx) {
  for (int64_t j = blockIdx.y; j < n; j += gridDim.y)
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
      X[GS_IDX(i, j, ldx)] = (i == j) ? 1.0 : 0.0;
}

}  // namespace

// sum_{j=0}^{N-1} clamp(a + j, 0, M)
static double sum_clamp_inc(int64_t a, int64_t N, int64_t M) {
  const int64_t j0 = std::clamp<int64_t>(1 - a, 0, N);   // first j with a + j >= 1
  const int64_t j1 = std::clamp<int64_t>(M - a, j0, N);  // first j with a + j >= M
  const double lin = 0.5 * (double)(j1 - j0) * (double)((a + j0) + (a + j1 - 1));
  return lin + (double)M * (double)(N - j1);
}

// Number of (i, j), 0 <= i < M, 0 <= j < N, inside the written region:
// UPPER column j holds clamp(j - diag + 1, 0, M) rows, LOWER clamp(M - j + diag, 0, M).
double region_elems(int64_t M, int64_t N, TriMode mode, int64_t diag) {
  if (mode == TRI_ALL) return (double)M * (double)N;
  if (mode == TRI_UPPER) return sum_clamp_inc(1 - diag, N, M);
  return sum_clamp_inc(M + diag - N + 1, N, M);
}

int dgemm(cudaStream_t st, bool transA, bool transB, int64_t M, int64_t N, int64_t K, double alpha, const double *A,
          int64_t lda, const double *B, int64_t ldb, double beta, double *C, int64_t ldc, TriMode mode, int64_t diag,
          const int *abort_flag) {
  if (M <= 0 || N <= 0) return GSYEIG_SUCCESS;
  KernelProfiler *prof = current_profiler();
  size_t e0 = prof ? prof->start(st) : SIZE_MAX;
  GemmContext *gc = current_gemm();
  // the sliced engines take K in slabs (tcgen05: up to 512, exact chunks of
  // 128 inside; mma.sync: 128), C accumulating from the second slab on
  const int64_t kslab = (gc && gc->sliced) ? (gc->umma ? 512 : 128) : K;
  bool done = false;
  if (gc && gc->sliced && K >= 1) {
    const int64_t kc0 = std::min(K, kslab);
    const bool ws_ok = gc->umma ? gc->ws_bytes >= umma_workspace_bytes(M, N, kc0)
                                : gc->ws_bytes >= sliced_workspace_bytes(M, N, kc0);
    if (ws_ok) {
      for (int64_t k0 = 0; k0 < K; k0 += kslab) {
        const int64_t kc = std::min(kslab, K - k0);
        const double *Ak = transA ? A + k0 : A + k0 * lda;  // op(A) is M x K
        const double *Bk = transB ? B + k0 * ldb : B + k0;  // op(B) is K x N
        const double bk = (k0 == 0) ? beta : 1.0;
        if (gc->umma)
          GS_TRY(umma_gemm(st, transA, transB, M, N, kc, alpha, Ak, lda, Bk, ldb, bk, C, ldc, mode, diag, abort_flag,
                           gc->ws, gc->ws_bytes, gc->err, gc->spin, gc->max_ctas));
        else
          GS_TRY(sliced_gemm(st, transA, transB, M, N, kc, alpha, Ak, lda, Bk, ldb, bk, C, ldc, mode, diag, abort_flag,
                             gc->ws, gc->ws_bytes));
      }
      done = true;
    }
  }
  if (!done) {
    dim3 grid((unsigned)ceil_div(M, BM), (unsigned)ceil_div(N, BN));
    k_dgemm<<<grid, NT, 0, st>>>(transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, (int)mode, diag,
                                 abort_flag);
    count_launch();
    GS_CHECK_LAUNCH();
  }
  if (prof) {
    const double el = region_elems(M, N, mode, diag);
    // algorithmic: 2K flops per written element; bytes: op(A), op(B) once, C read (beta != 0) and written
    const double bytes = 8.0 * ((double)M * K + (double)K * N + el * (beta != 0.0 ? 2.0 : 1.0));
    prof->stop(st, e0, PROF_GEMM, 2.0 * (double)K * el, bytes);
  }
  return GSYEIG_SUCCESS;
}

int copy_block(cudaStream_t st, int64_t M, int64_t N, const double *src, int64_t lds, double *dst, int64_t ldd,
               const int *abort_flag) {
  if (M <= 0 || N <= 0) return GSYEIG_SUCCESS;
  dim3 grid((unsigned)std::min<int64_t>(ceil_div(M, 256), 64), (unsigned)std::min<int64_t>(N, 4096));
  k_copy_block<<<grid, 256, 0, st>>>(M, N, src, lds, dst, ldd, abort_flag);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

int axpy_block(cudaStream_t st, int64_t M, int64_t N, double alpha, const double *X, int64_t ldx, double *Y,
               int64_t ldy) {
  if (M <= 0 || N <= 0) return GSYEIG_SUCCESS;
  dim3 grid((unsigned)std::min<int64_t>(ceil_div(M, 256), 64), (unsigned)std::min<int64_t>(N, 4096));
  k_axpy_block<<<grid, 256, 0, st>>>(M, N, alpha, X, ldx, Y, ldy);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

int set_identity(cudaStream_t st, int64_t n, double *X, int64_t ldx) {
  if (n <= 0) return GSYEIG_SUCCESS;
  dim3 grid((unsigned)std::min<int64_t>(ceil_div(n, 256), 64), (unsigned)std::min<int64_t>(n, 4096));
  k_identity<<<grid, 256, 0, st>>>(n, X, ldx);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

int symmetrize(cudaStream_t st, int64_t n, double *A, int64_t lda, bool lower_to_upper) {
  if (n <= 1) return GSYEIG_SUCCESS;
  dim3 grid((unsigned)ceil_div(n, 32), (unsigned)ceil_div(n, 32));
  k_symmetrize<<<grid, dim3(32, 8), 0, st>>>(n, A, lda, lower_to_upper);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

}  // namespace gs
