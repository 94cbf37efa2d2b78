// Shared definitions for the GB300 (sm_103a) gsyeig library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <cstddef>
#include <vector>

#include "gsyeig.h"

#define GS_IDX(i, j, ld) ((size_t)(i) + (size_t)(j) * (size_t)(ld))

namespace gs {

// Process-wide count of kernels issued by this library (graph nodes counted
// when the graph is launched).
extern std::atomic<int64_t> g_launches;

inline void count_launch(int64_t k = 1) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// Status carried through the host-side drivers.
struct Status {
  int code = GSYEIG_SUCCESS;
  explicit operator bool() const { return code == GSYEIG_SUCCESS; }
};

#define GS_CUDA(call)                                      \
  do {                                                     \
    cudaError_t _e = (call);                               \
    if (_e != cudaSuccess) {                               \
      last_cuda_error() = _e;                              \
      return _e == cudaErrorMemoryAllocation ? GSYEIG_OOM  \
                                             : GSYEIG_CUDA_ERROR; \
    }                                                      \
  } while (0)

#define GS_CHECK_LAUNCH()                                  \
  do {                                                     \
    cudaError_t _e = cudaGetLastError();                   \
    if (_e != cudaSuccess) {                               \
      last_cuda_error() = _e;                              \
      return GSYEIG_CUDA_ERROR;                            \
    }                                                      \
  } while (0)

#define GS_TRY(expr)                  \
  do {                                \
    int _st = (expr);                 \
    if (_st != GSYEIG_SUCCESS) return _st; \
  } while (0)

cudaError_t &last_cuda_error();

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// cudaFuncAttributeMaxDynamicSharedMemorySize of kernel `fn` raised to
// `bytes` on the current device, once per (kernel, device): the attribute
// call costs host time that launch-bound sequences of small kernels feel.
int set_max_smem(const void *fn, int bytes);

// SMs of the current device (looked up once per device)
int num_sms_cached();

// ---------------------------------------------------------------------------
// Optional per-launch timing (opts.profile): CUDA events recorded on the
// launching stream around each GEMM-engine / symv launch, resolved after the
// call has synchronised.  One profiler per handle, installed for the
// duration of an API call on the calling thread.
// ---------------------------------------------------------------------------
// PROF_GEMM covers a whole GEMM-engine call (operand slicing included);
// PROF_GEMM_CORE only the tensor-core kernel k_sliced_umma inside it.
enum ProfClass {
  PROF_GEMM = 0,
  PROF_SYMV = 1,
  PROF_ORTH = 2,
  PROF_RESTART = 3,
  PROF_RITZ = 4,
  PROF_GEMM_CORE = 5,
  PROF_DIAG = 6,  // the diagonal-block factor and inverse kernels of gs1
  PROF_SLICE = 7,  // the kernels slicing GEMM operands into bf16 digit planes
  PROF_SYMV32 = 8, // the fp32 block operator of the mixed-precision stage
  PROF_NCLASS = 9
};

struct KernelProfiler {
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  struct Rec {
    int cls;
    double flops, bytes;
    size_t e0;
  };
  std::vector<Rec> recs;
  // start: returns the index of the start event (or SIZE_MAX on failure)
  size_t start(cudaStream_t st);
  void stop(cudaStream_t st, size_t e0, int cls, double flops, double bytes);
  // after synchronisation: per-class launches, ms, flops, bytes; then reset
  void resolve(int64_t launches[PROF_NCLASS], double ms[PROF_NCLASS], double flops[PROF_NCLASS],
               double bytes[PROF_NCLASS]);
  void release();
};

KernelProfiler *&current_profiler();

// ---------------------------------------------------------------------------
// GEMM engine (FP64):  C = alpha * op(A) * op(B) + beta * C on an M x N
// column-major block, op(X) = X or X^T.  `mode` restricts which elements
// of C are written: ALL, LOWER (i - j + diag >= 0) or UPPER (i - j + diag
// <= 0), with i, j the row/column inside the block; tiles wholly outside
// the region are skipped.  If abort_flag != nullptr and *abort_flag != 0
// the kernel returns without work (used to stop a factorisation after a
// failed pivot without a host round trip).
// ---------------------------------------------------------------------------
enum TriMode { TRI_ALL = 0, TRI_LOWER = 1, TRI_UPPER = 2 };

int dgemm(cudaStream_t st, bool transA, bool transB, int64_t M, int64_t N, int64_t K, double alpha,
          const double *A, int64_t lda, const double *B, int64_t ldb, double beta, double *C, int64_t ldc,
          TriMode mode = TRI_ALL, int64_t diag = 0, const int *abort_flag = nullptr);

// Elements of an M x N block inside the region `mode` writes.
double region_elems(int64_t M, int64_t N, TriMode mode, int64_t diag);

// How dgemm executes, installed per API call: sliced = true routes every
// call to the error-free bf16 tensor-core GEMM, in slabs of K (tcgen05
// engine gemm_umma.cu: up to 512, exact chunks of 128 inside; mma.sync
// engine gemm_sliced.cu: 128) using the workspace ws; otherwise the FP64
// FMA kernel.
struct GemmContext {
  bool sliced = false;
  bool umma = true;     // tcgen05 engine (else mma.sync engine)
  void *ws = nullptr;
  size_t ws_bytes = 0;
  int *err = nullptr;   // device flag: a bounded wait inside the tcgen05 engine expired
  uint32_t spin = 0;    // poll limit of the engine's main-loop waits (0 = the default bound)
  int max_ctas = 0;     // > 0: cap on the persistent grid (CTAs, one per SM)
};
GemmContext *&current_gemm();

size_t umma_workspace_bytes(int64_t M, int64_t N, int64_t K);
int umma_gemm(cudaStream_t st, bool transA, bool transB, int64_t M, int64_t N, int64_t K, double alpha,
              const double *A, int64_t lda, const double *B, int64_t ldb, double beta, double *C, int64_t ldc,
              TriMode mode, int64_t diag, const int *abort_flag, void *ws, size_t ws_bytes, int *err,
              uint32_t spin, int max_ctas);

size_t sliced_workspace_bytes(int64_t M, int64_t N, int64_t K);
int sliced_gemm(cudaStream_t st, bool transA, bool transB, int64_t M, int64_t N, int64_t K, double alpha,
                const double *A, int64_t lda, const double *B, int64_t ldb, double beta, double *C, int64_t ldc,
                TriMode mode, int64_t diag, const int *abort_flag, void *ws, size_t ws_bytes);

// Copy an M x N block (column-major, both with leading dimensions).
int copy_block(cudaStream_t st, int64_t M, int64_t N, const double *src, int64_t lds, double *dst, int64_t ldd,
               const int *abort_flag = nullptr);

// X = I (n x n, leading dimension ldx).
int set_identity(cudaStream_t st, int64_t n, double *X, int64_t ldx);
// Y += alpha X over an M x N block (column-major, leading dimensions ldx, ldy)
int axpy_block(cudaStream_t st, int64_t M, int64_t N, double alpha, const double *X, int64_t ldx, double *Y,
               int64_t ldy);

// Mirror one triangle of an n x n matrix into the other: lower_to_upper
// copies A[i][j] (i > j) to A[j][i]; otherwise the reverse.
int symmetrize(cudaStream_t st, int64_t n, double *A, int64_t lda, bool lower_to_upper);

// ---------------------------------------------------------------------------
// Dense factorisation drivers (factor.cu).
// ---------------------------------------------------------------------------
struct FactorWork {
  double *Uinv = nullptr;   // inverses of the nb x nb diagonal blocks of U, (nb x nb) each, ld nb
  double *panel = nullptr;  // staging buffer, max(nb, ...) x n
  size_t panel_elems = 0;
  int *flag = nullptr;      // device int: first failed pivot (1-based) or 0
  double *rdiag = nullptr;  // device, nb entries: 1 / U(i, i) of the diagonal block just factored
  // inverses of the NB x NB outer diagonal blocks of U (NB = outer_block(nb), ld NB, zeros below the
  // diagonal) and a staging buffer of NB x max(n, s) doubles for the outer panels
  double *UinvO = nullptr;
  double *panelO = nullptr;
  bool outer_ready = false;  // UinvO holds the current factor's outer inverses
  // look-ahead of potrf (NULL: none): a second stream for the diagonal-block
  // kernels and two events (the next diagonal block updated; it is factored)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_upd = nullptr, ev_diag = nullptr;
  // sygst's recursion: P = U12^T C11 of the top split (sygst_tmp_elems doubles; NULL: direct form)
  double *tmp = nullptr;
  size_t tmp_elems = 0;
};

// order NB of the outer blocks of the blocked factorisations for inner width nb
int64_t outer_block(int nb);

int potrf_blocked(cudaStream_t st, int64_t n, double *B, int64_t ldb, int nb, FactorWork &w);
int trtri_diag_blocks(cudaStream_t st, int64_t n, const double *U, int64_t ldu, int nb, double *Uinv);
int sygst_blocked(cudaStream_t st, int64_t n, double *A, int64_t lda, const double *U, int64_t ldu, int nb,
                  FactorWork &w, bool have_uinv);
// doubles of FactorWork::tmp that sygst_blocked's n^3 recursion needs at order n (0: none)
size_t sygst_tmp_elems(int64_t n, int nb);
int trsm_back_blocked(cudaStream_t st, int64_t n, const double *U, int64_t ldu, double *Y, int64_t ldy, int64_t s,
                      int nb, FactorWork &w, bool have_uinv);
// X = U^-1 for the upper-triangular U (X n x n, ld ldx; zeros below the diagonal).
int trtri_upper_blocked(cudaStream_t st, int64_t n, const double *U, int64_t ldu, double *X, int64_t ldx, int nb,
                        FactorWork &w, bool have_uinv);

// ---------------------------------------------------------------------------
// Operator application (symv.cu): z = C w, C full symmetric.
// ---------------------------------------------------------------------------
int symv_f64(cudaStream_t st, int64_t n, const double *C, int64_t ldc, const double *w, double *z);

// verify.cu: max normwise backward error and max |X^T B X - I| of a solve's
// pairs (w device, X device, ld ldx) against the full symmetric A0, B0, into
// out[0], out[1] (host); ws holds verify_workspace_doubles(n, s) doubles.
size_t verify_workspace_doubles(int64_t n, int64_t s);
int verify_solution(cudaStream_t st, int64_t n, int64_t s, const double *A0, int64_t lda, const double *B0,
                    int64_t ldb, const double *X, int64_t ldx, const double *w, double *ws, double out[2]);

}  // namespace gs
