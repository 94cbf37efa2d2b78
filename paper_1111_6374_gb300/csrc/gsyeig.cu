// C ABI of the library and the host-side driver of the KE route
// (Section 2.3 of the paper; Table 1 keys gs1, gs2, ke1-ke3, bt1).
// Device memory for inputs/outputs belongs to the caller; the handle owns a
// grow-on-demand workspace.  The driver only sequences kernels and reads
// back a few scalars per restart (converged count, breakdown flag).
#include <algorithm>
#include <array>
#include <chrono>
#include <map>
#include <mutex>
#include <thread>
#include <cmath>
#include <cstring>
#include <new>

#include "lanczos.cuh"
#include "mixed.cuh"
#include "symv_df.cuh"

namespace gs {

struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
  int ensure(size_t need) {
    if (need <= bytes) return GSYEIG_SUCCESS;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    cudaError_t e = cudaMalloc(&p, need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return GSYEIG_OOM;
    }
    bytes = need;
    return GSYEIG_SUCCESS;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  double *d() const { return static_cast<double *>(p); }
};

}  // namespace gs

using namespace gs;

struct gsyeig_ctx {
  int device = 0;
  cudaStream_t user = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t ev[10] = {};  // 0-6 stage marks, 7 first host matrix landed, 8 end mark, 9 user-stream ordering
  gsyeig_opts opts{};
  // workspace
  DevBuf uinv, panel, flag, diag;
  DevBuf uinvO;           // inverses of the outer diagonal blocks and the outer panel staging
  DevBuf gtmp;            // sygst's recursion buffer
  DevBuf V, Vq, z, h1, h2, sq, alpha, beta, alphaP, betaP, theta, S, Q, rot, invw, state, shifts, arrow;
  DevBuf hA, hB, hX, hw;  // device copies for host-pointer calls
  cudaStream_t side = nullptr;  // look-ahead of potrf: the diagonal-block kernels
  cudaEvent_t side_ev[2] = {};
  cudaStream_t cp = nullptr;  // host-pointer calls: the copy of the matrix needed second
  cudaEvent_t cp_ev = nullptr, cp_first = nullptr;
  DevBuf pA, pB;          // working copies when opts.preserve_inputs
  DevBuf vA, vB, vws;     // originals and workspace of opts.verify
  DevBuf gemm_ws;         // slices of the tensor-core GEMM
  DevBuf gemm_err;        // device error flag of the tcgen05 engine
  DevBuf dfop, dfpart;    // double-float operator tiles and symv partials
  DevBuf kinv, dfopL, kt; // variant KI: U^-1, the tiles of L = U^-T, two temporaries
  DevBuf tmin;            // smallest eigenvalue of the final projected matrix
  DevBuf wstart;          // start-block construction and Chebyshev filter vectors
  // mixed precision: fp32 operator and staging, block basis, projected matrices, refinement blocks
  DevBuf mx_op, mx_w, mx_z, mx_V, mx_Zd, mx_H, mx_part, mx_T, mx_small, mx_Sb, mx_CSb, mx_tmp, mx_fw, mx_ones;
  DfOperator op, opL;
  bool use_df = false;
  bool ki = false;        // the operator is U^-T G U^-1 applied implicitly (variant KI)
  KernelProfiler prof;
  GemmContext gemm;
  // opts.graph: instantiated graphs of Lanczos cycles, keyed by everything the captured launches use
  struct CycleGraph {
    std::array<uintptr_t, 12> key{};
    cudaGraphExec_t exec = nullptr;
    int64_t nodes = 0;
  };
  CycleGraph graphs[4];
  int graph_next = 0;
  // gsyeig_solve_batched: internal handles and the autotuned panel width per size class
  std::vector<gsyeig_ctx *> subs;
  std::map<int64_t, int> tuned;
  std::mutex tune_mu;
};

namespace {

constexpr int kDefaultBlock = 128;

// Installs the handle's profiler for the duration of one API call when
// opts.profile is set; fills the profile fields of info on request.
struct ProfScope {
  gsyeig_handle h;
  bool on;
  explicit ProfScope(gsyeig_handle hh) : h(hh), on(hh->opts.profile != 0) {
    if (on) current_profiler() = &h->prof;
  }
  void fill(gsyeig_info *info) {
    if (!on) return;
    int64_t l[PROF_NCLASS];
    double ms[PROF_NCLASS], fl[PROF_NCLASS], by[PROF_NCLASS];
    h->prof.resolve(l, ms, fl, by);
    if (!info) return;
    info->gemm_launches = l[PROF_GEMM];
    info->gemm_ms = ms[PROF_GEMM];
    info->gemm_flops = fl[PROF_GEMM];
    info->gemm_bytes = by[PROF_GEMM];
    info->symv_launches = l[PROF_SYMV];
    info->symv_ms = ms[PROF_SYMV];
    info->symv_flops = fl[PROF_SYMV];
    info->symv_bytes = by[PROF_SYMV];
    info->orth_ms = ms[PROF_ORTH];
    info->restart_ms = ms[PROF_RESTART];
    info->ritz_ms = ms[PROF_RITZ];
    info->gemm_core_launches = l[PROF_GEMM_CORE];
    info->gemm_core_ms = ms[PROF_GEMM_CORE];
    info->gemm_core_flops = fl[PROF_GEMM_CORE];
    info->diag_launches = l[PROF_DIAG];
    info->diag_ms = ms[PROF_DIAG];
    info->slice_ms = ms[PROF_SLICE];
    info->symm32_launches = l[PROF_SYMV32];
    info->symm32_ms = ms[PROF_SYMV32];
  }
  ~ProfScope() {
    if (on) {
      current_profiler() = nullptr;
      h->prof.recs.clear();
      h->prof.used = 0;
    }
  }
};

bool is_device_ptr(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Staging copy of a page-locked host buffer by the SMs: 16-byte loads
// through the buffer's device mapping, plus the last 8 bytes when the size
// is an odd number of doubles.
__global__ void k_stage_copy(const uint4 *__restrict__ src, uint4 *__restrict__ dst, size_t n16, bool tail8) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n16; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
  if (tail8 && blockIdx.x == 0 && threadIdx.x == 0)
    reinterpret_cast<double *>(dst + n16)[0] = reinterpret_cast<const double *>(src + n16)[0];
}

// n x n host matrix (leading dimension ld) into the contiguous device buffer
// d on stream s.  A contiguous page-locked source is read by k_stage_copy
// through its device mapping: on the GB300 hosts measured, the copy engines
// pulled a pinned 2 GB buffer at about 25 GB/s when they followed other GPU
// work (211 GB/s when repeated at once), while the SMs read it at 211 GB/s
// either way.  Pageable or strided sources go through cudaMemcpy(2D)Async.
int stage_h2d(double *d, const double *src, int64_t n, int64_t ld, cudaStream_t s) {
  const size_t bytes = (size_t)n * n * sizeof(double);
  if (ld == n && (uintptr_t)src % 16 == 0) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, src) == cudaSuccess) {
      if (a.type == cudaMemoryTypeHost && a.devicePointer && (uintptr_t)a.devicePointer % 16 == 0) {
        const size_t n16 = bytes / 16;
        const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(num_sms_cached(), ceil_div((int64_t)n16, 512)));
        k_stage_copy<<<grid, 512, 0, s>>>(static_cast<const uint4 *>(a.devicePointer), reinterpret_cast<uint4 *>(d), n16,
                                          bytes % 16 != 0);
        count_launch();
        GS_CHECK_LAUNCH();
        return GSYEIG_SUCCESS;
      }
    } else {
      cudaGetLastError();
    }
  }
  if (ld == n)
    GS_CUDA(cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, s));
  else
    GS_CUDA(cudaMemcpy2DAsync(d, n * sizeof(double), src, ld * sizeof(double), n * sizeof(double), n,
                              cudaMemcpyHostToDevice, s));
  return GSYEIG_SUCCESS;
}

int begin(gsyeig_handle h) {
  GS_CUDA(cudaSetDevice(h->device));
  GS_CUDA(cudaEventRecord(h->ev[9], h->user));
  GS_CUDA(cudaStreamWaitEvent(h->st, h->ev[9], 0));
  return GSYEIG_SUCCESS;
}

int finish(gsyeig_handle h) {
  GS_CUDA(cudaStreamSynchronize(h->st));
  GS_CUDA(cudaGetLastError());
  return GSYEIG_SUCCESS;
}

int nb_of(gsyeig_handle h, int64_t n) {
  int nb = h->opts.block > 0 ? h->opts.block : kDefaultBlock;
  if (nb > n) nb = (int)std::max<int64_t>(1, n);
  return nb;
}

// Install the GEMM mode for this call; the sliced GEMM needs slices of two
// operands of at most max(n, s) rows and K up to the outer block (the
// tcgen05 engine takes up to 512 per call).
int gemm_setup(gsyeig_handle h, int64_t n, int nb, int64_t s) {
  h->gemm.sliced = (h->opts.fp64_gemm != 1);
  h->gemm.umma = (h->opts.fp64_gemm == 0);
  if (h->gemm.sliced) {
    const int64_t r = std::max<int64_t>(n, s);
    GS_TRY(h->gemm_ws.ensure(
        std::max(sliced_workspace_bytes(r, r, nb), umma_workspace_bytes(r, r, 512))));
    h->gemm.ws = h->gemm_ws.p;
    h->gemm.ws_bytes = h->gemm_ws.bytes;
    GS_TRY(h->gemm_err.ensure(64));
    h->gemm.err = static_cast<int *>(h->gemm_err.p);
    GS_CUDA(cudaMemsetAsync(h->gemm.err, 0, sizeof(int), h->st));  // cudaMalloc does not zero
  }
  h->gemm.spin = (uint32_t)h->opts.wait_limit;
  h->gemm.max_ctas = h->opts.max_ctas;
  current_gemm() = &h->gemm;
  return GSYEIG_SUCCESS;
}

// After a call that used the tcgen05 engine: did any of its bounded waits expire?
int gemm_check(gsyeig_handle h) {
  if (!h->gemm.sliced || !h->gemm.umma || !h->gemm.err) return GSYEIG_SUCCESS;
  int e = 0;
  GS_CUDA(cudaMemcpyAsync(&e, h->gemm.err, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  GS_CUDA(cudaStreamSynchronize(h->st));
  if (e) {
    GS_CUDA(cudaMemsetAsync(h->gemm.err, 0, sizeof(int), h->st));
    return GSYEIG_TIMEOUT;
  }
  return GSYEIG_SUCCESS;
}

struct GemmScope {
  ~GemmScope() { current_gemm() = nullptr; }
};

int factor_ws(gsyeig_handle h, int64_t n, int nb, int64_t s, FactorWork &w) {
  GS_TRY(gemm_setup(h, n, nb, s));
  const int64_t nblk = ceil_div(n, nb);
  const int64_t NB = outer_block(nb), nout = ceil_div(n, NB);
  GS_TRY(h->uinvO.ensure(((size_t)nout * NB * NB + (size_t)NB * std::max<int64_t>(n, s)) * sizeof(double)));
  w.UinvO = h->uinvO.d();
  w.panelO = w.UinvO + (size_t)nout * NB * NB;
  GS_TRY(h->uinv.ensure((size_t)nblk * nb * nb * sizeof(double)));
  GS_TRY(h->panel.ensure((size_t)std::max<int64_t>(n, s) * nb * sizeof(double) + 64));
  GS_TRY(h->flag.ensure(256 + 160 * sizeof(double)));
  w.Uinv = h->uinv.d();
  w.panel = h->panel.d();
  w.flag = static_cast<int *>(h->flag.p);
  w.rdiag = reinterpret_cast<double *>(static_cast<char *>(h->flag.p) + 256);
  if (!h->side) {
    GS_CUDA(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
    for (cudaEvent_t &e : h->side_ev) GS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  w.side = h->side;
  w.ev_upd = h->side_ev[0];
  w.ev_diag = h->side_ev[1];
  return GSYEIG_SUCCESS;
}

// the recursion buffer of sygst (allocated only by the calls that run gs2)
int sygst_ws(gsyeig_handle h, int64_t n, int nb, FactorWork &w) {
  const size_t need = sygst_tmp_elems(n, nb);
  if (need == 0) return GSYEIG_SUCCESS;
  GS_TRY(h->gtmp.ensure(need * sizeof(double)));
  w.tmp = h->gtmp.d();
  w.tmp_elems = need;
  return GSYEIG_SUCCESS;
}

float elapsed(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
    cudaGetLastError();
    return 0.f;
  }
  return ms;
}

struct LanczosParams {
  int64_t m, k;
};

LanczosParams lanczos_params(const gsyeig_opts &o, int64_t n, int64_t s) {
  int64_t m = o.krylov_dim > 0 ? o.krylov_dim : std::min<int64_t>(n, std::max<int64_t>(3 * s, s + 16));
  m = std::min<int64_t>(m, n);
  int64_t k = o.keep > 0 ? o.keep : std::min<int64_t>(s + std::max<int64_t>(2, s / 4), m - 1);
  return {m, k};
}

// Coarse profiled region on the library stream (no-op without a profiler).
struct ProfRegion {
  cudaStream_t st;
  int cls;
  size_t e0 = SIZE_MAX;
  ProfRegion(cudaStream_t s, int c) : st(s), cls(c) {
    if (current_profiler()) e0 = current_profiler()->start(st);
  }
  ~ProfRegion() {
    if (current_profiler()) current_profiler()->stop(st, e0, cls, 0.0, 0.0);
  }
};

// The operator of ke1: z = C w with the explicit C (Eq. 3; double-float tiles
// or FP64), or, for variant KI, z = U^-T (G (U^-1 w)) as L (G (L^T w)) with
// L = U^-T held as lower-triangular double-float tiles.
int apply_operator(gsyeig_handle h, cudaStream_t st, int64_t n, const double *C, int64_t ldc, const double *w,
                   double *z) {
  if (h->ki) {
    double *t1 = h->kt.d(), *t2 = t1 + n;
    GS_TRY(df_symv(st, h->opL, w, t1, DF_COLS));
    GS_TRY(df_symv(st, h->op, t1, t2, DF_SYM));
    return df_symv(st, h->opL, t2, z, DF_ROWS);
  }
  if (h->use_df) return df_symv(st, h->op, w, z);
  return symv_f64(st, n, C, ldc, w, z);
}

// One Lanczos step j: z = C v_j, CGS2 against v_0..v_j, alpha_j, beta_j, v_{j+1}.
int lanczos_step(gsyeig_handle h, cudaStream_t st, int64_t n, int64_t m, int64_t j, const double *C, int64_t ldc) {
  double *V = h->V.d(), *z = h->z.d();
  GS_TRY(apply_operator(h, st, n, C, ldc, V + (size_t)j * n, z));
  ProfRegion pr(st, PROF_ORTH);
  GS_TRY(lz_cgs2(st, n, j + 1, V, n, z, h->h1.d(), h->h2.d(), h->sq.d()));
  GS_TRY(lz_finalize(st, j, m, h->h1.d(), h->h2.d(), h->sq.d(), lz_nparts(n), h->alpha.d(), h->beta.d(),
                     static_cast<LanczosState *>(h->state.p)));
  GS_TRY(lz_scale_into(st, n, z, V + (size_t)(j + 1) * n, static_cast<LanczosState *>(h->state.p)));
  return GSYEIG_SUCCESS;
}

// Steps j0..m-1 of a Lanczos cycle.  With opts.graph (and no profiler) the
// cycle's launches are captured once into a CUDA graph, kept while every
// buffer, size and operator it touches stays the same, and replayed: a
// cycle of m steps is one launch from the host instead of about 8 m.
int lanczos_cycle(gsyeig_handle h, cudaStream_t st, int64_t n, int64_t m, int64_t j0, const double *C, int64_t ldc) {
  if (h->opts.graph != 1 || current_profiler()) {
    for (int64_t j = j0; j < m; j++) GS_TRY(lanczos_step(h, st, n, m, j, C, ldc));
    return GSYEIG_SUCCESS;
  }
  const std::array<uintptr_t, 12> key = {
      (uintptr_t)h->V.p, (uintptr_t)h->z.p, (uintptr_t)h->h1.p, (uintptr_t)h->state.p, (uintptr_t)C,
      (uintptr_t)ldc, (uintptr_t)n, (uintptr_t)m, (uintptr_t)j0,
      (uintptr_t)(h->use_df ? h->op.hi : nullptr) ^ (uintptr_t)(h->ki ? h->opL.hi : nullptr) ^ (uintptr_t)h->ki,
      (uintptr_t)h->dfpart.p ^ (uintptr_t)h->kt.p, (uintptr_t)h->alpha.p ^ ((uintptr_t)h->beta.p << 1) ^ (uintptr_t)h->sq.p};
  gsyeig_ctx::CycleGraph *g = nullptr;
  for (auto &c : h->graphs)
    if (c.exec && c.key == key) g = &c;
  if (!g) {
    g = &h->graphs[h->graph_next];
    h->graph_next = (h->graph_next + 1) % 4;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    g->exec = nullptr;
    const int64_t l0 = g_launches.load();
    GS_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
    int rc = GSYEIG_SUCCESS;
    for (int64_t j = j0; j < m && rc == GSYEIG_SUCCESS; j++) rc = lanczos_step(h, st, n, m, j, C, ldc);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(st, &graph);
    g->nodes = g_launches.load() - l0;
    g_launches.fetch_sub(g->nodes);  // captured, not launched
    if (rc != GSYEIG_SUCCESS || ce != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return rc != GSYEIG_SUCCESS ? rc : GSYEIG_CUDA_ERROR;
    }
    const cudaError_t ie = cudaGraphInstantiate(&g->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
      g->exec = nullptr;
      cudaGetLastError();
      return GSYEIG_CUDA_ERROR;
    }
    g->key = key;
  }
  GS_CUDA(cudaGraphLaunch(g->exec, st));
  count_launch(g->nodes);
  return GSYEIG_SUCCESS;
}

// Put a fresh random unit vector, orthogonal to V[:, 0:ncols], in V[:, ncols].
int fresh_vector(gsyeig_handle h, cudaStream_t st, int64_t n, int64_t ncols, uint64_t stream_id, double *norm_out) {
  double *V = h->V.d(), *z = h->z.d();
  LanczosState *state = static_cast<LanczosState *>(h->state.p);
  GS_TRY(lz_random(st, n, h->opts.seed, stream_id, z));
  GS_TRY(lz_cgs2(st, n, ncols, V, n, z, h->h1.d(), h->h2.d(), h->sq.d()));
  GS_TRY(lz_norm_finish(st, h->sq.d(), lz_nparts(n), state, norm_out));
  GS_TRY(lz_scale_into(st, n, z, V + (size_t)ncols * n, state));
  return GSYEIG_SUCCESS;
}

// Copies the device fault flags of the kernels in use (bounded waits of the
// ke1 kernel and of the tensor-core GEMM) into f[0..1]; read them after the
// next stream synchronisation.
int fault_flags_async(gsyeig_handle h, cudaStream_t st, int f[2]) {
  f[0] = f[1] = 0;
  if (h->use_df || h->ki) GS_CUDA(cudaMemcpyAsync(&f[0], h->op.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  GemmContext *gc = current_gemm();
  if (gc && gc->sliced && gc->umma && gc->err)
    GS_CUDA(cudaMemcpyAsync(&f[1], gc->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  return GSYEIG_SUCCESS;
}

// Implicitly restarted Lanczos on the full symmetric C (ke1, ke2, ke3), or,
// with Uinv != NULL, on U^-T C U^-1 applied implicitly (variant KI: C is
// then the untransformed matrix G, Uinv the n x n inverse of the factor).
// Output: the s wanted Ritz values (ascending) in theta_out (device) and
// Ritz vectors in Y (n x s, ld ldy, device).  theta_min (host, optional):
// the smallest eigenvalue of the final projected matrix, an upper bound on
// the smallest eigenvalue of the operator.
// A caller's start block X0 (opts.start_block, eigenvector approximations
// of the pencil) is mapped to the operator's space by the upper-triangular
// factor F (F = U of gs1; NULL: X0 is already in the operator's space).
int lanczos_run(gsyeig_handle h, const double *C, int64_t ldc, int64_t n, int64_t s, int which, double *theta_out,
                double *Y, int64_t ldy, gsyeig_info *info, double *ms_ke3, const double *Uinv = nullptr,
                double *theta_min = nullptr, const double *F = nullptr, int64_t ldf = 0) {
  cudaStream_t st = h->st;
  const LanczosParams P = lanczos_params(h->opts, n, s);
  const int64_t m = P.m, k = P.k, p = m - k;
  if (!(s <= k && k < m && m <= n)) return GSYEIG_NOT_SUPPORTED;
  const int64_t np = lz_nparts(n);
  GS_TRY(h->V.ensure((size_t)n * (m + 1) * sizeof(double)));
  GS_TRY(h->Vq.ensure((size_t)n * (k + 1) * sizeof(double)));
  GS_TRY(h->z.ensure((size_t)n * sizeof(double)));
  GS_TRY(h->h1.ensure((size_t)(m + 1) * sizeof(double)));
  GS_TRY(h->h2.ensure((size_t)(m + 1) * sizeof(double)));
  GS_TRY(h->sq.ensure((size_t)(np + 1) * sizeof(double)));
  GS_TRY(h->alpha.ensure((size_t)m * sizeof(double)));
  GS_TRY(h->beta.ensure((size_t)m * sizeof(double)));
  GS_TRY(h->alphaP.ensure((size_t)m * sizeof(double)));
  GS_TRY(h->betaP.ensure((size_t)m * sizeof(double)));
  GS_TRY(h->theta.ensure((size_t)m * sizeof(double)));
  GS_TRY(h->S.ensure((size_t)m * k * sizeof(double)));
  GS_TRY(h->arrow.ensure((size_t)m * sizeof(double)));
  GS_TRY(h->Q.ensure((size_t)m * m * sizeof(double)));
  GS_TRY(h->rot.ensure((size_t)2 * std::max<int64_t>(p, 1) * (m - 1 + 1) * sizeof(double)));
  GS_TRY(h->invw.ensure((size_t)5 * m * k * sizeof(double)));
  GS_TRY(h->state.ensure(sizeof(LanczosState)));
  double *V = h->V.d();
  // ke1 operator: C's lower triangle as fp32 hi/lo tiles (default) or C
  // itself; variant KI: tiles of G and of L = U^-T
  h->ki = (Uinv != nullptr);
  h->use_df = (h->opts.fp64_symv == 0) || h->ki;
  if (h->use_df) {
    GS_TRY(h->dfop.ensure(df_operator_bytes(n)));
    GS_TRY(h->dfpart.ensure(df_partials_bytes(n)));
    h->op.hi = static_cast<float *>(h->dfop.p);
    h->op.W = static_cast<float2 *>(h->dfpart.p);
    const int64_t NTt = ceil_div(n, 64);
    h->op.wsplit = h->op.W + (size_t)NTt * NTt * 64;
    h->op.err = reinterpret_cast<int *>(h->op.wsplit + (size_t)NTt * 64);
    h->op.spin = (uint32_t)h->opts.wait_limit;
    GS_CUDA(cudaMemsetAsync(h->op.err, 0, sizeof(int), st));
    GS_TRY(df_operator_build(st, n, C, ldc, h->op));
    if (h->ki) {
      GS_TRY(h->dfopL.ensure(df_operator_bytes(n)));
      GS_TRY(h->kt.ensure((size_t)2 * n * sizeof(double)));
      h->opL = h->op;  // shares the partials, split vector and fault flag
      h->opL.hi = static_cast<float *>(h->dfopL.p);
      GS_TRY(df_operator_build(st, n, Uinv, n, h->opL, true, true));
    }
  }
  LanczosState *dstate = static_cast<LanczosState *>(h->state.p);
  LanczosState hs;
  std::memset(&hs, 0, sizeof(hs));
  hs.breakdown_at = -1;
  GS_CUDA(cudaMemcpyAsync(dstate, &hs, sizeof(hs), cudaMemcpyHostToDevice, st));
  GS_CUDA(cudaMemsetAsync(h->beta.p, 0, (size_t)m * sizeof(double), st));

  // v_0: built from the caller's start block, or the caller's start vector,
  // or a counter-based random one; optionally Chebyshev-filtered; normalised
  int64_t filter_mv = 0;
  const gsyeig_opts &o = h->opts;
  if (o.start_block && o.start_cols > 0) {
    if (o.ld_start < n) return GSYEIG_NOT_SUPPORTED;
    GS_TRY(h->wstart.ensure((size_t)3 * n * sizeof(double)));
    double *t = h->wstart.d();
    GS_TRY(lz_weighted_sum(st, n, o.start_cols, o.start_block, o.ld_start, o.start_weights, F ? t : h->z.d()));
    if (F) GS_TRY(lz_trmv_upper(st, n, F, ldf, t, h->z.d()));
  } else if (o.v0) {
    GS_CUDA(cudaMemcpyAsync(h->z.p, o.v0, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  } else {
    GS_TRY(lz_random(st, n, o.seed, 0, h->z.d()));
  }
  if (o.filter_degree > 0) {
    // Chebyshev filter p_d(C) z damping the unwanted end [cut, edge]
    // (Zhou and Saad's filtered subspace iteration, 2007): components below
    // the cut (above it, for the largest pairs) grow like T_d, the rest stay
    // bounded by 1
    GS_TRY(h->wstart.ensure((size_t)3 * n * sizeof(double)));
    double *y0 = h->wstart.d(), *y1 = y0 + n, *cy = y0 + 2 * n;
    const double a = std::min(o.filter_cut, o.filter_edge), b = std::max(o.filter_cut, o.filter_edge);
    const double e = 0.5 * (b - a), c = 0.5 * (b + a);
    GS_CUDA(cudaMemcpyAsync(y0, h->z.p, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    double *yp = y0, *yc = y1;
    for (int i = 1; i <= o.filter_degree; i++) {
      GS_TRY(apply_operator(h, st, n, C, ldc, i == 1 ? yp : yc, cy));
      // y_1 = (C - c) y_0 / e;  y_{i+1} = 2 (C - c) y_i / e - y_{i-1}
      GS_TRY(lz_cheb_step(st, n, cy, i == 1 ? yp : yc, yp, c, e, i == 1, i == 1 ? yc : yp));
      if (i > 1) std::swap(yp, yc);
      filter_mv++;
    }
    GS_CUDA(cudaMemcpyAsync(h->z.p, yc, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  }
  GS_TRY(lz_cgs2(st, n, 0, V, n, h->z.d(), h->h1.d(), h->h2.d(), h->sq.d()));
  GS_TRY(lz_norm_finish(st, h->sq.d(), (int)np, dstate, nullptr));
  GS_TRY(lz_scale_into(st, n, h->z.d(), V, dstate));

  const bool thick = (h->opts.qr_restart == 0);
  int64_t ka = 0;                                               // arrow rows of M (thick restart)
  const int64_t woff = (thick && which == GSYEIG_LARGEST) ? k - s : 0;  // wanted columns within S
  const double *shifts = (which == GSYEIG_LARGEST) ? h->theta.d() : h->theta.d() + k;
  const int dir = (which == GSYEIG_LARGEST) ? -1 : 1;  // nearest-to-wanted shift first
  int64_t j0 = 0, restarts = 0, matvecs = 0, breakdowns = 0;
  int status = GSYEIG_SUCCESS;
  auto t_start = std::chrono::steady_clock::now();
  int fault[2];
  // Ritz pairs of the leading mc x mc projected matrix (mc = m at the end of
  // a cycle; smaller at an early check) and the convergence test
  auto ritz = [&](int64_t mc) -> int {
    ProfRegion pr(st, PROF_RITZ);
    if (thick) {
      // the k kept Ritz pairs (the s wanted among them); M has an arrow after a restart
      const int64_t kf = (which == GSYEIG_LARGEST) ? mc - k : 0;
      GS_TRY(tri_bisect(st, mc, h->alpha.d(), h->beta.d(), ka, h->arrow.d(), kf, k, h->theta.d()));
      GS_TRY(tri_invit(st, mc, h->alpha.d(), h->beta.d(), ka, h->arrow.d(), k, h->theta.d(), h->S.d(), m,
                       h->invw.d()));
    } else {
      const int64_t wfc = (which == GSYEIG_LARGEST) ? mc - s : 0;
      GS_TRY(tri_bisect(st, mc, h->alpha.d(), h->beta.d(), 0, nullptr, 0, mc, h->theta.d()));
      GS_TRY(tri_invit(st, mc, h->alpha.d(), h->beta.d(), 0, nullptr, s, h->theta.d() + wfc, h->S.d(), m,
                       h->invw.d()));
    }
    GS_TRY(tri_converged(st, mc, s, h->theta.d(), h->beta.d(), h->S.d() + (size_t)woff * m, m, h->opts.tol, dstate));
    GS_CUDA(cudaMemcpyAsync(&hs, dstate, sizeof(hs), cudaMemcpyDeviceToHost, st));
    GS_TRY(fault_flags_async(h, st, fault));
    GS_CUDA(cudaStreamSynchronize(st));
    if (fault[0] || fault[1]) return GSYEIG_TIMEOUT;
    return GSYEIG_SUCCESS;
  };
  const int64_t ce = h->opts.check_every;        // 0: test only at the end of a cycle
  const int64_t first_check = thick ? k + 1 : s;  // smallest projected matrix holding the kept pairs
  int64_t mc = m;                                 // order of the projected matrix of the final Ritz pairs
  bool early = false;
  for (;;) {
    int64_t j = j0;
    bool stop_pass = false;
    while (j < m) {
      int64_t jend = m;
      if (ce > 0) {
        jend = std::max(j0 + ((j - j0) / ce + 1) * ce, first_check);
        jend = std::min(std::max(jend, j + 1), m);
      }
      const int64_t jb = j;
      if (ce == 0) {
        GS_TRY(lanczos_cycle(h, st, n, m, j, C, ldc));
        j = jend;
      } else {
        for (; j < jend; j++) GS_TRY(lanczos_step(h, st, n, m, j, C, ldc));
      }
      matvecs += jend - jb;
      if (jend == m) break;
      // an early convergence test on the leading jend x jend matrix
      GS_CUDA(cudaMemcpyAsync(&hs, dstate, sizeof(hs), cudaMemcpyDeviceToHost, st));
      GS_TRY(fault_flags_async(h, st, fault));
      GS_CUDA(cudaStreamSynchronize(st));
      if (fault[0] || fault[1]) return GSYEIG_TIMEOUT;
      if (hs.breakdown_at >= 0) {
        stop_pass = true;  // handled below, as at the end of a cycle
        break;
      }
      GS_TRY(ritz(jend));
      if (hs.nconv >= s) {
        mc = jend;
        early = true;
        break;
      }
    }
    if (early) break;
    if (stop_pass) {
      // finish the cycle's bookkeeping the same way as a full pass: the steps
      // after a breakdown were no-ops
      matvecs += m - j;
      for (; j < m; j++) GS_TRY(lanczos_step(h, st, n, m, j, C, ldc));
    }
    GS_CUDA(cudaMemcpyAsync(&hs, dstate, sizeof(hs), cudaMemcpyDeviceToHost, st));
    GS_TRY(fault_flags_async(h, st, fault));
    GS_CUDA(cudaStreamSynchronize(st));
    if (fault[0] || fault[1]) return GSYEIG_TIMEOUT;  // a bounded device wait ran out: results invalid
    if (hs.breakdown_at >= 0 && hs.breakdown_at < m - 1) {
      // invariant subspace met: continue from a fresh random direction
      const int64_t b = hs.breakdown_at;
      breakdowns++;
      hs.breakdown_at = -1;
      GS_CUDA(cudaMemcpyAsync(&dstate->breakdown_at, &hs.breakdown_at, sizeof(int64_t), cudaMemcpyHostToDevice, st));
      GS_TRY(fresh_vector(h, st, n, b + 1, 1000 + (uint64_t)breakdowns, nullptr));
      j0 = b + 1;
      if (breakdowns > m) return GSYEIG_NO_CONVERGENCE;
      continue;
    }
    // Ritz values of T_m, vectors of the wanted ones, convergence test
    GS_TRY(ritz(m));
    if (hs.nconv >= s) break;
    if (restarts >= h->opts.max_restarts) {
      status = GSYEIG_NO_CONVERGENCE;
      break;
    }
    if (h->opts.timeout_ms > 0) {
      double el = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
      if (el > h->opts.timeout_ms) {
        status = GSYEIG_TIMEOUT;
        break;
      }
    }
    ProfRegion pr(st, PROF_RESTART);
    if (thick) {
      // thick restart (same Krylov subspace and projection as the exact-shift
      // implicit restart): keep the k Ritz vectors, continue from v_m
      GS_TRY(dgemm(st, false, false, n, k, m, 1.0, V, n, h->S.d(), m, 0.0, h->Vq.d(), n));
      GS_TRY(copy_block(st, n, k, h->Vq.d(), n, V, n));
      GS_CUDA(cudaMemcpyAsync(V + (size_t)k * n, V + (size_t)m * n, (size_t)n * sizeof(double),
                              cudaMemcpyDeviceToDevice, st));
      GS_TRY(lz_thick_restart(st, m, k, h->theta.d(), h->S.d(), h->alpha.d(), h->beta.d(), h->arrow.d()));
      ka = k;
    } else {
      // implicit restart with the p unwanted Ritz values as exact shifts
      GS_TRY(tri_qr_shifts(st, m, p, h->alpha.d(), h->beta.d(), shifts, dir, h->alphaP.d(), h->betaP.d(), h->Q.d(),
                           m, h->rot.d()));
      GS_TRY(dgemm(st, false, false, n, k + 1, m, 1.0, V, n, h->Q.d(), m, 0.0, h->Vq.d(), n));
      GS_TRY(lz_restart_residual(st, n, k, m, h->Vq.d(), n, V + (size_t)m * n, h->betaP.d(), h->beta.d(), h->Q.d(),
                                 m, h->z.d()));
      GS_TRY(copy_block(st, n, k, h->Vq.d(), n, V, n));
      GS_CUDA(cudaMemcpyAsync(h->alpha.p, h->alphaP.p, (size_t)k * sizeof(double), cudaMemcpyDeviceToDevice, st));
      GS_CUDA(
          cudaMemcpyAsync(h->beta.p, h->betaP.p, (size_t)(k - 1) * sizeof(double), cudaMemcpyDeviceToDevice, st));
      GS_CUDA(cudaMemsetAsync(h->beta.d() + k, 0, (size_t)(m - k) * sizeof(double), st));
      // clean the new residual against V_k (CGS2), beta_{k-1} = ||f||, v_k = f / ||f||
      GS_TRY(lz_cgs2(st, n, k, V, n, h->z.d(), h->h1.d(), h->h2.d(), h->sq.d()));
      GS_TRY(lz_norm_finish(st, h->sq.d(), (int)np, dstate, h->beta.d() + (k - 1)));
      GS_TRY(lz_scale_into(st, n, h->z.d(), V + (size_t)k * n, dstate));
    }
    restarts++;
    j0 = k;
  }
  if (theta_min) {
    // the projected matrix of the last cycle is still in (alpha, beta, arrow)
    GS_TRY(h->tmin.ensure(sizeof(double)));
    const int64_t kam = thick ? ka : 0;
    GS_TRY(tri_bisect(st, mc, h->alpha.d(), h->beta.d(), kam, kam > 0 ? h->arrow.d() : nullptr, 0, 1, h->tmin.d()));
    GS_CUDA(cudaMemcpyAsync(theta_min, h->tmin.p, sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  // ke3: Ritz vectors Y = V_mc S
  cudaEvent_t e0 = h->ev[5], e1 = h->ev[6];
  GS_CUDA(cudaEventRecord(e0, st));
  GS_TRY(dgemm(st, false, false, n, s, mc, 1.0, V, n, h->S.d() + (size_t)woff * m, m, 0.0, Y, ldy));
  const int64_t wfin = thick ? woff : ((which == GSYEIG_LARGEST) ? mc - s : 0);
  GS_CUDA(cudaMemcpyAsync(theta_out, h->theta.d() + wfin, (size_t)s * sizeof(double), cudaMemcpyDeviceToDevice, st));
  GS_CUDA(cudaEventRecord(e1, st));
  GS_CUDA(cudaEventSynchronize(e1));
  if (ms_ke3) *ms_ke3 = elapsed(e0, e1);
  // a bounded wait that ran out inside the symv kernel or the GEMM engine invalidates the result
  GS_TRY(fault_flags_async(h, st, fault));
  GS_CUDA(cudaStreamSynchronize(st));
  if (fault[0] || fault[1]) return GSYEIG_TIMEOUT;
  if (info) {
    info->nconv = hs.nconv;
    info->restarts = restarts;
    info->matvecs = matvecs;
    info->krylov_dim = m;
    info->keep = k;
    info->breakdowns = breakdowns;
    info->max_ritz_estimate = hs.max_est;
    info->tnorm = hs.tnorm;
    info->filter_matvecs = filter_mv;
    info->matvecs = matvecs + filter_mv;
  }
  return status;
}


// ---- mixed precision (fp32 block Lanczos, FP64 block refinement) ----------

// cnt eigenpairs (the cnt smallest or largest, ascending) of a small dense
// symmetric H (m x m, ld m, device): Lanczos with full reorthogonalisation
// over the whole space (m steps, the tridiagonalisation Householder would
// give up to rounding) and the Ritz solve of T_m, on the handle's own
// kernels with the FP64 product.  th (cnt) and Z (m x cnt, ld ldz), device.
int small_syev(gsyeig_handle h, const double *H, int64_t m, int64_t cnt, int which, double *th, double *Z,
               int64_t ldz) {
  if (cnt < 1 || cnt >= m) return GSYEIG_NOT_SUPPORTED;
  const gsyeig_opts saved = h->opts;
  KernelProfiler *prof = current_profiler();
  GemmContext *gc = current_gemm();
  current_profiler() = nullptr;
  current_gemm() = nullptr;
  gsyeig_opts &o = h->opts;
  o.krylov_dim = m;
  o.keep = 0;
  o.fp64_symv = 1;
  o.qr_restart = 0;
  o.check_every = 0;
  o.start_block = nullptr;
  o.v0 = nullptr;
  o.filter_degree = 0;
  o.max_restarts = 4;
  o.timeout_ms = 0;
  const int st = lanczos_run(h, H, m, m, cnt, which, th, Z, ldz, nullptr, nullptr);
  h->opts = saved;
  current_profiler() = prof;
  current_gemm() = gc;
  return st;
}

// A small factorisation workspace (the solve's own diagonal-block inverses
// stay intact for bt1).
struct SmallFactor {
  FactorWork w;
  double *G, *Rinv, *R1, *R2, *norms;
};

int small_factor(gsyeig_handle h, int64_t bmax, SmallFactor &f) {
  const int nb = 128;
  const int64_t nblk = ceil_div(bmax, nb);
  const int64_t NB = outer_block(nb), nout = ceil_div(bmax, NB);
  const size_t need = (size_t)nblk * nb * nb + (size_t)bmax * nb + 4 * (size_t)bmax * bmax + (size_t)bmax + 512 +
                      (size_t)nout * NB * NB + (size_t)NB * bmax;
  GS_TRY(h->mx_fw.ensure(need * sizeof(double)));
  double *p = h->mx_fw.d();
  f.w.UinvO = p;
  p += (size_t)nout * NB * NB;
  f.w.panelO = p;
  p += (size_t)NB * bmax;
  f.w.Uinv = p;
  p += (size_t)nblk * nb * nb;
  f.w.panel = p;
  p += (size_t)bmax * nb;
  f.G = p;
  p += (size_t)bmax * bmax;
  f.Rinv = p;
  p += (size_t)bmax * bmax;
  f.R1 = p;
  p += (size_t)bmax * bmax;
  f.R2 = p;
  p += (size_t)bmax * bmax;
  f.norms = p;
  p += bmax;
  f.w.flag = reinterpret_cast<int *>(p);
  f.w.rdiag = p + 32;
  return GSYEIG_SUCCESS;
}

// Orthonormalise the n x b block Z (ld ldz) by Cholesky QR twice: G = Z^T Z
// = R^T R, Z <- Z R^-1, twice (the products on the GEMM engine in use, or
// the FP64 tall-skinny kernels for b <= 16).  The same right factors are
// applied to CZ (if not NULL), so that CZ stays C Z.  With Rout != NULL,
// Rout (b x b, ld b) = R2 R1 (Z_in = Z_out Rout).  Returns GSYEIG_NOT_SPD if
// a Gram matrix is not numerically positive definite (Z rank deficient).
int cholqr2(gsyeig_handle h, cudaStream_t st, int64_t n, int64_t b, double *Z, int64_t ldz, double *CZ, int64_t ldcz,
            double *Rout, SmallFactor &f, double *tmp, double *part) {
  const int nb = (int)std::min<int64_t>(128, b);
  for (int pass = 0; pass < 2; pass++) {
    if (b <= 16)
      GS_TRY(ts_dots(st, n, b, (int)b, Z, ldz, Z, ldz, part, f.G, b));
    else
      GS_TRY(dgemm(st, true, false, b, b, n, 1.0, Z, ldz, Z, ldz, 0.0, f.G, b));
    GS_TRY(potrf_blocked(st, b, f.G, b, nb, f.w));
    int flag = 0;
    GS_CUDA(cudaMemcpyAsync(&flag, f.w.flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    GS_CUDA(cudaStreamSynchronize(st));
    if (flag) return GSYEIG_NOT_SPD;
    GS_TRY(trtri_upper_blocked(st, b, f.G, b, f.Rinv, b, nb, f.w, true));
    GS_TRY(dgemm(st, false, false, n, b, b, 1.0, Z, ldz, f.Rinv, b, 0.0, tmp, n));
    GS_TRY(copy_block(st, n, b, tmp, n, Z, ldz));
    if (CZ) {
      GS_TRY(dgemm(st, false, false, n, b, b, 1.0, CZ, ldcz, f.Rinv, b, 0.0, tmp, n));
      GS_TRY(copy_block(st, n, b, tmp, n, CZ, ldcz));
    }
    // the factor is the upper triangle of G (its strict lower triangle still holds Gram entries)
    if (Rout) GS_TRY(copy_upper(st, b, f.G, b, pass == 0 ? f.R1 : f.R2, b));
  }
  if (Rout) GS_TRY(dgemm(st, false, false, b, b, b, 1.0, f.R2, b, f.R1, b, 0.0, Rout, b));
  return GSYEIG_SUCCESS;
}

// Lanczos stage of the mixed-precision route (C full symmetric, FP64):
// block Lanczos (b = 16) with C streamed as fp32 tiles and fp32
// accumulation, the reorthogonalisation (CGS2) and the projected band
// matrix in FP64; the k = s + guard Ritz vectors of that stage then go
// through an FP64 block refinement (LOBPCG: Rayleigh-Ritz on [X, R, P],
// C products on the FP64-accurate GEMM engine) until the s wanted residuals
// meet tol ||C||.  Ritz values ascending into theta_out, vectors into Y.
//
// With warm = true (opts.block_start and a start block of at least s
// columns) the fp32 stage is skipped: the refinement starts from the start
// block mapped into the operator's space by the factor F (F X0), with
// max(8, s/4) random guard columns, and ||C|| is bounded by its 1-norm.
//
// With stage_out != NULL (opts.mixed = 1) the function stops after the fp32
// stage: *stage_out = the k = s + guard Ritz vectors of the band matrix at
// the wanted end (n x k, ld n, in the handle's workspace), the start of the
// FP64 Lanczos stage, and *stage_cols = k.
int lanczos_mixed(gsyeig_handle h, const double *C, int64_t ldc, int64_t n, int64_t s, int which, double *theta_out,
                  double *Y, int64_t ldy, gsyeig_info *info, double *ms_ke3, const double *F = nullptr,
                  int64_t ldf = 0, const double **stage_out = nullptr, int64_t *stage_cols = nullptr) {
  cudaStream_t st = h->st;
  constexpr int BK = 16;
  const gsyeig_opts &o = h->opts;
  const bool warm = o.block_start == 1 && o.start_block && o.start_cols >= s;
  // the fp32 stage feeding the FP64 Lanczos (stage_out) needs approximations,
  // not converged pairs: a smaller block Krylov space by default
  int64_t mb = o.krylov_dim > 0 ? o.krylov_dim : std::max<int64_t>((stage_out ? 3 : 5) * s, s + 64);
  mb = std::min<int64_t>(ceil_div(mb, BK) * BK, (n / BK) * BK - BK);
  const int64_t g = warm ? std::max<int64_t>(8, s / 4) : std::max<int64_t>(16, s / 8);
  const int64_t k = warm ? std::min<int64_t>(o.start_cols + g, n / 4) : std::min<int64_t>(s + g, mb - BK);
  if (warm && (o.ld_start < n || k <= s || 3 * k >= n)) return GSYEIG_NOT_SUPPORTED;
  if (!warm && (n < 8 * BK || mb < 2 * BK || s >= k || 3 * k >= n)) return GSYEIG_NOT_SUPPORTED;
  if (warm && stage_out) return GSYEIG_NOT_SUPPORTED;
  if (warm) mb = BK;  // no fp32 stage
  const int64_t nblk = mb / BK;
  // ---- workspace
  if (!warm) {
    GS_TRY(h->mx_op.ensure(f32_operator_bytes(n)));
    GS_TRY(h->mx_w.ensure(f32_block_bytes(n)));
    GS_TRY(h->mx_z.ensure(f32_block_bytes(n)));
  }
  GS_TRY(h->mx_V.ensure((size_t)n * (mb + BK) * sizeof(double)));
  GS_TRY(h->mx_Zd.ensure((size_t)n * BK * sizeof(double)));
  GS_TRY(h->mx_H.ensure((size_t)2 * (mb + BK) * BK * sizeof(double)));
  GS_TRY(h->mx_part.ensure(ts_part_doubles(n, mb + BK) * sizeof(double)));
  GS_TRY(h->mx_T.ensure((size_t)mb * mb * sizeof(double) + 64));
  const int64_t zrows = std::max<int64_t>(mb, 3 * k);
  GS_TRY(h->mx_small.ensure(((size_t)12 * k * k + (size_t)zrows * k + 5 * k + 64) * sizeof(double)));
  GS_TRY(h->mx_Sb.ensure((size_t)n * 3 * k * sizeof(double)));
  GS_TRY(h->mx_CSb.ensure((size_t)n * 3 * k * sizeof(double)));
  GS_TRY(h->mx_tmp.ensure((size_t)n * 4 * k * sizeof(double)));
  SmallFactor sf;
  GS_TRY(small_factor(h, 2 * k, sf));
  F32Operator op;
  op.tiles = static_cast<float *>(h->mx_op.p);
  op.W = static_cast<float *>(h->mx_w.p);
  op.Z = static_cast<float *>(h->mx_z.p);
  double *V = h->mx_V.d(), *Zd = h->mx_Zd.d(), *H1 = h->mx_H.d(), *H2 = H1 + (mb + BK) * BK;
  double *part = h->mx_part.d(), *T = h->mx_T.d(), *cn = T + (size_t)mb * mb;
  double *Hs = h->mx_small.d(), *Zs = Hs + 9 * k * k, *thv = Zs + zrows * k, *res = thv + 3 * k;
  double *Sb = h->mx_Sb.d(), *CSb = h->mx_CSb.d(), *tmp = h->mx_tmp.d();
  GemmContext *gc = current_gemm();  // the FP64-accurate engine of the solve
  cudaEvent_t ev0, ev1, ev2;
  GS_CUDA(cudaEventCreate(&ev0));
  GS_CUDA(cudaEventCreate(&ev1));
  GS_CUDA(cudaEventCreate(&ev2));
  struct EvGuard {
    cudaEvent_t a, b, c;
    ~EvGuard() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
      cudaEventDestroy(c);
    }
  } evg{ev0, ev1, ev2};
  GS_CUDA(cudaEventRecord(ev0, st));
  GemmContext *gc0 = current_gemm();
  int64_t blocks = 0;
  double cnorm = 0.0;
  int rc = GSYEIG_SUCCESS;
  if (warm) {
    // ---- the caller's block, mapped by F, plus random guard columns, orthonormal
    for (int64_t c = 0; c < o.start_cols; c++) {
      const double *xc = o.start_block + (size_t)c * o.ld_start;
      if (F) GS_TRY(lz_trmv_upper(st, n, F, ldf, xc, Sb + (size_t)c * n));
      else GS_CUDA(cudaMemcpyAsync(Sb + (size_t)c * n, xc, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    }
    for (int64_t c = o.start_cols; c < k; c++) GS_TRY(lz_random(st, n, o.seed, 3000 + (uint64_t)c, Sb + (size_t)c * n));
    GS_TRY(col_norms(st, n, k, Sb, n, sf.norms));
    GS_TRY(scale_cols(st, n, k, Sb, n, sf.norms));
    rc = cholqr2(h, st, n, k, Sb, n, nullptr, 0, nullptr, sf, tmp, part);
    if (rc != GSYEIG_SUCCESS) return rc == GSYEIG_NOT_SPD ? GSYEIG_NOT_SUPPORTED : rc;
    GS_TRY(mat_norm1(st, n, C, ldc, cn));
    GS_CUDA(cudaMemcpyAsync(&cnorm, cn, sizeof(double), cudaMemcpyDeviceToHost, st));
    GS_CUDA(cudaStreamSynchronize(st));
  } else {
  // ---- fp32 operator and a random orthonormal start block
  GS_TRY(f32_operator_build(st, n, C, ldc, op));
  for (int c = 0; c < BK; c++) GS_TRY(lz_random(st, n, h->opts.seed, 2000 + (uint64_t)c, V + (size_t)c * n));
  GS_CUDA(cudaMemsetAsync(T, 0, (size_t)mb * mb * sizeof(double), st));
  current_gemm() = nullptr;  // small products in FP64
  rc = cholqr2(h, st, n, BK, V, n, nullptr, 0, nullptr, sf, tmp, part);
  if (rc != GSYEIG_SUCCESS) {
    current_gemm() = gc;
    return rc;
  }
  // ---- block Lanczos: Z = C V_j (fp32), CGS2 in FP64, Z = V_{j+1} B_j
  for (int64_t j = 0; j < nblk; j++) {
    double *Vj = V + (size_t)j * BK * n;
    GS_TRY(f32_symm(st, op, Vj, n, Zd, n));
    blocks++;
    const int64_t w = (j + 1) * BK;
    {
      ProfRegion pr(st, PROF_ORTH);
      GS_TRY(ts_dots(st, n, w, BK, V, n, Zd, n, part, H1, w));
      GS_TRY(ts_update(st, n, w, BK, V, n, H1, w, Zd, n));
      GS_TRY(ts_dots(st, n, w, BK, V, n, Zd, n, part, H2, w));
      GS_TRY(ts_update(st, n, w, BK, V, n, H2, w, Zd, n));
      GS_TRY(put_sum(st, BK, H1 + j * BK, H2 + j * BK, w, T, mb, j * BK));
      if (j + 1 < nblk) {
        double *R = Hs;  // 16 x 16
        rc = cholqr2(h, st, n, BK, Zd, n, nullptr, 0, R, sf, tmp, part);
        if (rc != GSYEIG_SUCCESS) {
          current_gemm() = gc;
          return rc == GSYEIG_NOT_SPD ? GSYEIG_NO_CONVERGENCE : rc;
        }
        GS_TRY(copy_block(st, n, BK, Zd, n, V + (size_t)(j + 1) * BK * n, n));
        GS_TRY(put_block(st, BK, R, BK, T, mb, (j + 1) * BK, j * BK, true));
      }
    }
  }
  GS_TRY(sym_avg(st, mb, T, mb));
  GS_TRY(inf_norm(st, mb, T, mb, cn));
  GS_CUDA(cudaMemcpyAsync(&cnorm, cn, sizeof(double), cudaMemcpyDeviceToHost, st));
  // ---- the k wanted Ritz pairs of the band matrix, X = V S
  {
    ProfRegion pr(st, PROF_RITZ);
    GS_TRY(small_syev(h, T, mb, k, which, thv, Zs, mb));
  }
  current_gemm() = gc;
  GS_TRY(dgemm(st, false, false, n, k, mb, 1.0, V, n, Zs, mb, 0.0, Sb, n));
  }
  (void)gc0;
  GS_CUDA(cudaEventRecord(ev1, st));
  if (stage_out) {
    *stage_out = Sb;
    if (stage_cols) *stage_cols = k;
    GS_CUDA(cudaStreamSynchronize(st));
    if (info) {
      info->block_steps = blocks;
      info->ms_block_lanczos = elapsed(ev0, ev1);
      info->matvecs = blocks * BK;
    }
    return GSYEIG_SUCCESS;
  }
  // ---- FP64 block refinement on C: LOBPCG (Knyazev 2001) with soft locking
  // (columns whose residual meets the tolerance leave the search space) on an
  // orthonormal basis S = [X, P, W] chosen as Hetmaniuk and Lehoucq (2006)
  // do: the new directions W are made orthonormal against [X, P] before
  // their product with C is taken, and P is chosen in the coordinates of S
  // (P = S Q, C P = (C S) Q with Q orthonormal), so that no carried product
  // passes through the inverse of an ill-conditioned factor.
  double *X = Sb, *CX = CSb;
  int *idx = reinterpret_cast<int *>(res + k);
  double *Qs = res + 2 * k;  // ms x na coordinates of the next P
  GS_TRY(dgemm(st, false, false, n, k, n, 1.0, C, ldc, X, n, 0.0, CX, n));
  GS_TRY(column_dots(st, n, k, X, n, CX, n, thv));  // Rayleigh quotients of the columns
  const int64_t w0 = (which == GSYEIG_LARGEST) ? k - s : 0;  // wanted columns w0..w0+s-1
  const double tol = h->opts.tol;
  std::vector<double> hres(k), hist;
  std::vector<int> act;
  int64_t iters = 0, products = k, qr_fail = 0, stop = 0;
  int64_t np = 0;  // columns of P, stored after X in S
  bool done = false;
  for (; iters < 60; iters++) {
    double *Rf = tmp;  // the k residuals
    GS_TRY(block_resid(st, n, k, CX, X, n, thv, Rf));
    GS_TRY(col_norms(st, n, k, Rf, n, res));
    GS_CUDA(cudaMemcpyAsync(hres.data(), res, (size_t)k * sizeof(double), cudaMemcpyDeviceToHost, st));
    GS_CUDA(cudaStreamSynchronize(st));
    double mx = 0.0;
    for (int64_t i = w0; i < w0 + s; i++) mx = std::max(mx, hres[i]);
    if (mx <= tol * cnorm) {
      done = true;
      break;
    }
    // the rate over the last 4 steps predicts the steps still needed; when
    // they do not fit in the limit (small relative gaps at the wanted end),
    // stop now and leave the pairs to the FP64 Lanczos stage
    hist.push_back(mx);
    if (iters >= 6) {
      const double r = std::pow(mx / hist[iters - 4], 0.25);
      if (!(r < 1.0) || (double)iters + std::log(tol * cnorm / mx) / std::log(r) > 60.0) {
        stop = 2;
        break;
      }
    }
    act.clear();
    for (int64_t i = 0; i < k; i++)
      if (hres[i] > tol * cnorm) act.push_back((int)i);
    const int64_t na = (int64_t)act.size();
    ProfRegion pr(st, PROF_RESTART);
    GS_CUDA(cudaMemcpyAsync(idx, act.data(), (size_t)na * sizeof(int), cudaMemcpyHostToDevice, st));
    const int64_t kp = k + np;  // [X, P], orthonormal
    double *W = Sb + (size_t)kp * n, *CW = CSb + (size_t)kp * n;
    GS_TRY(gather_cols(st, n, na, idx, Rf, n, W, n));
    // W against [X, P], then orthonormal (Cholesky QR twice); the factor
    // R^-1 of nearly dependent residuals magnifies what is left of [X, P]
    // in W, so the projection and the Cholesky QR are repeated on the
    // well-conditioned result
    rc = GSYEIG_SUCCESS;
    for (int round = 0; round < 2 && rc == GSYEIG_SUCCESS; round++) {
      for (int pass = 0; pass < 2 - round; pass++) {
        GS_TRY(dgemm(st, true, false, kp, na, n, 1.0, Sb, n, W, n, 0.0, Hs, kp));
        GS_TRY(dgemm(st, false, false, n, na, kp, -1.0, Sb, n, Hs, kp, 1.0, W, n));
      }
      if (round == 0) {
        GS_TRY(col_norms(st, n, na, W, n, sf.norms));
        GS_TRY(scale_cols(st, n, na, W, n, sf.norms));
      }
      rc = cholqr2(h, st, n, na, W, n, nullptr, 0, nullptr, sf, tmp + (size_t)k * n, part);
      if (rc != GSYEIG_SUCCESS && rc != GSYEIG_NOT_SPD) return rc;
    }
    if (rc != GSYEIG_SUCCESS) {  // the residuals are numerically dependent: keep the current pairs
      qr_fail++;
      stop = 1;
      break;
    }
    GS_TRY(dgemm(st, false, false, n, na, n, 1.0, C, ldc, W, n, 0.0, CW, n));
    products += na;
    // Rayleigh-Ritz on S = [X, P, W]
    const int64_t ms = kp + na;
    GS_TRY(dgemm(st, true, false, ms, ms, n, 1.0, Sb, n, CSb, n, 0.0, Hs, ms));
    GS_TRY(sym_avg(st, ms, Hs, ms));
    GS_TRY(small_syev(h, Hs, ms, k, which, thv, Zs, ms));
    // the next P: the active Ritz vectors' components outside the old X
    // (the rows of Z below the first k), made orthonormal against Z in the
    // coordinates of S; if they are numerically dependent, the next step
    // goes without P
    int64_t np_new = na;
    GS_TRY(gather_cols(st, ms, na, idx, Zs, ms, Qs, ms));
    GS_CUDA(cudaMemset2DAsync(Qs, (size_t)ms * sizeof(double), 0, (size_t)k * sizeof(double), (size_t)na, st));
    rc = GSYEIG_SUCCESS;
    for (int round = 0; round < 2 && rc == GSYEIG_SUCCESS; round++) {
      for (int pass = 0; pass < 2 - round; pass++) {
        GS_TRY(dgemm(st, true, false, k, na, ms, 1.0, Zs, ms, Qs, ms, 0.0, Hs, k));
        GS_TRY(dgemm(st, false, false, ms, na, k, -1.0, Zs, ms, Hs, k, 1.0, Qs, ms));
      }
      if (round == 0) {
        GS_TRY(col_norms(st, ms, na, Qs, ms, sf.norms));
        GS_TRY(scale_cols(st, ms, na, Qs, ms, sf.norms));
      }
      rc = cholqr2(h, st, ms, na, Qs, ms, nullptr, 0, nullptr, sf, tmp, part);
      if (rc != GSYEIG_SUCCESS && rc != GSYEIG_NOT_SPD) return rc;
    }
    if (rc != GSYEIG_SUCCESS) {
      qr_fail++;
      np_new = 0;
    }
    // X <- S Z, C X <- (C S) Z, P <- S Q, C P <- (C S) Q
    double *Xn = tmp, *CXn = tmp + (size_t)k * n, *Pn = tmp + (size_t)2 * k * n, *CPn = tmp + (size_t)3 * k * n;
    GS_TRY(dgemm(st, false, false, n, k, ms, 1.0, Sb, n, Zs, ms, 0.0, Xn, n));
    GS_TRY(dgemm(st, false, false, n, k, ms, 1.0, CSb, n, Zs, ms, 0.0, CXn, n));
    if (np_new > 0) {
      GS_TRY(dgemm(st, false, false, n, np_new, ms, 1.0, Sb, n, Qs, ms, 0.0, Pn, n));
      GS_TRY(dgemm(st, false, false, n, np_new, ms, 1.0, CSb, n, Qs, ms, 0.0, CPn, n));
      GS_TRY(copy_block(st, n, np_new, Pn, n, Sb + (size_t)k * n, n));
      GS_TRY(copy_block(st, n, np_new, CPn, n, CSb + (size_t)k * n, n));
    }
    GS_TRY(copy_block(st, n, k, Xn, n, X, n));
    GS_TRY(copy_block(st, n, k, CXn, n, CX, n));
    np = np_new;
  }
  // ke3: the s wanted pairs
  GS_CUDA(cudaEventRecord(ev2, st));
  GS_TRY(copy_block(st, n, s, X + (size_t)w0 * n, n, Y, ldy));
  GS_CUDA(cudaMemcpyAsync(theta_out, thv + w0, (size_t)s * sizeof(double), cudaMemcpyDeviceToDevice, st));
  GS_CUDA(cudaStreamSynchronize(st));
  if (ms_ke3) *ms_ke3 = 0.0;
  if (info) {
    info->nconv = done ? s : 0;
    info->restarts = 0;
    info->matvecs = blocks * BK + products;
    info->krylov_dim = mb;
    info->keep = k;
    info->block_steps = blocks;
    info->refine_iters = iters;
    info->breakdowns = qr_fail;      // Gram matrices of the search directions that were not definite
    info->refine_stop = stop;        // 1: residuals numerically dependent, 2: too slow to converge
    info->ms_block_lanczos = elapsed(ev0, ev1);
    info->ms_refine = elapsed(ev1, ev2);
    info->tnorm = cnorm;
    double mx = 0.0;
    for (int64_t i = w0; i < w0 + s; i++) mx = std::max(mx, hres[i]);
    info->max_ritz_estimate = cnorm > 0 ? mx / cnorm : mx;
  }
  return done ? GSYEIG_SUCCESS : GSYEIG_NO_CONVERGENCE;
}

// Inverse route (Section 3.1): the pairs of the pencil are x = L^-1 y /
// sqrt(mu), so X^T B X = D^-1/2 Y^T C' Y D^-1/2 (D = diag(mu)), and any
// defect of Y^T C' Y is divided by sqrt(mu_i mu_j): for a wide range of the
// wanted mu (a lambda near zero) the Ritz vectors' B-orthonormality suffers.
// This makes it exact to rounding before the back-transform: M = D^-1/2
// (Y^T C' Y) D^-1/2 (C' stored full; products on the FP64-accurate engine),
// M = R^T R, Y <- Y D^-1/2 R^-1 D^1/2, so that X^T B X = R^-T M R^-1 = I.
// theta (device, s, positive) = the mu of the columns of Y.  A Gram matrix
// that is not positive definite leaves Y as it was.
int b_orthonormalise_inverse(gsyeig_handle h, cudaStream_t st, int64_t n, int64_t s, const double *Cp, int64_t ldc,
                             double *Y, int64_t ldy, const double *theta) {
  GS_TRY(h->mx_tmp.ensure((size_t)n * s * sizeof(double)));
  GS_TRY(h->mx_small.ensure((size_t)2 * s * s * sizeof(double)));
  SmallFactor sf;
  GS_TRY(small_factor(h, s, sf));
  double *W = h->mx_tmp.d(), *M = h->mx_small.d(), *K = M + (size_t)s * s;
  GS_TRY(dgemm(st, false, false, n, s, n, 1.0, Cp, ldc, Y, ldy, 0.0, W, n));
  GS_TRY(dgemm(st, true, false, s, s, n, 1.0, Y, ldy, W, n, 0.0, M, s));
  GS_TRY(sym_avg(st, s, M, s));
  GS_TRY(scale_by_powers(st, s, M, s, theta, -0.5, -0.5));
  GS_TRY(potrf_blocked(st, s, M, s, (int)std::min<int64_t>(128, s), sf.w));
  int flag = 0;
  GS_CUDA(cudaMemcpyAsync(&flag, sf.w.flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  GS_CUDA(cudaStreamSynchronize(st));
  if (flag) return GSYEIG_SUCCESS;
  GS_TRY(trtri_upper_blocked(st, s, M, s, K, s, (int)std::min<int64_t>(128, s), sf.w, true));
  GS_TRY(scale_by_powers(st, s, K, s, theta, -0.5, 0.5));
  GS_TRY(dgemm(st, false, false, n, s, s, 1.0, Y, ldy, K, s, 0.0, W, n));
  GS_TRY(copy_block(st, n, s, W, n, Y, ldy));
  return GSYEIG_SUCCESS;
}

int check_solve_args(int64_t lda, int64_t ldb, int64_t n, int64_t s, int which, const void *A, const void *B,
                     const void *w, const void *X, int64_t ldx) {
  if (!A) return -2;
  if (lda < std::max<int64_t>(1, n)) return -3;
  if (!B) return -4;
  if (ldb < std::max<int64_t>(1, n)) return -5;
  if (n < 2) return -6;
  if (s < 1 || s >= n) return -7;
  if (which != GSYEIG_SMALLEST && which != GSYEIG_LARGEST) return -8;
  if (!w) return -9;
  if (!X) return -10;
  if (ldx < n) return -11;
  return 0;
}

}  // namespace

extern "C" {

int gsyeig_default_options(gsyeig_opts *o) {
  if (!o) return -1;
  std::memset(o, 0, sizeof(*o));
  o->tol = 1e-12;
  o->max_restarts = 2000;
  return GSYEIG_SUCCESS;
}

int gsyeig_create(gsyeig_handle *hp, int device, void *cuda_stream) {
  if (!hp) return -1;
  *hp = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    cudaGetLastError();
    return GSYEIG_CUDA_ERROR;
  }
  if (device < 0 || device >= ndev) return -2;
  gsyeig_ctx *h = new (std::nothrow) gsyeig_ctx();
  if (!h) return GSYEIG_OOM;
  h->device = device;
  h->user = static_cast<cudaStream_t>(cuda_stream);
  gsyeig_default_options(&h->opts);
  if (cudaSetDevice(device) != cudaSuccess || cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return GSYEIG_CUDA_ERROR;
  }
  for (auto &e : h->ev)
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      gsyeig_destroy(h);
      return GSYEIG_CUDA_ERROR;
    }
  *hp = h;
  return GSYEIG_SUCCESS;
}

int gsyeig_destroy(gsyeig_handle h) {
  if (!h) return -1;
  cudaSetDevice(h->device);
  if (h->st) cudaStreamSynchronize(h->st);
  DevBuf *bufs[] = {&h->uinvO, &h->gtmp, &h->mx_ones, &h->mx_op, &h->mx_w, &h->mx_z, &h->mx_V, &h->mx_Zd, &h->mx_H, &h->mx_part, &h->mx_T,
                    &h->mx_small, &h->mx_Sb, &h->mx_CSb, &h->mx_tmp, &h->mx_fw, &h->wstart, &h->kinv, &h->dfopL, &h->kt, &h->tmin, &h->pA, &h->pB, &h->vA, &h->vB, &h->vws, &h->diag, &h->arrow, &h->gemm_err, &h->dfop, &h->dfpart, &h->gemm_ws, &h->uinv, &h->panel, &h->flag, &h->V, &h->Vq, &h->z, &h->h1, &h->h2, &h->sq, &h->alpha,
                    &h->beta, &h->alphaP, &h->betaP, &h->theta, &h->S, &h->Q, &h->rot, &h->invw, &h->state,
                    &h->shifts, &h->hA, &h->hB, &h->hX, &h->hw};
  for (DevBuf *b : bufs) b->release();
  h->prof.release();
  for (auto &g : h->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  for (gsyeig_ctx *sub : h->subs) gsyeig_destroy(sub);
  for (auto &e : h->ev)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : h->side_ev)
    if (e) cudaEventDestroy(e);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->cp_ev) cudaEventDestroy(h->cp_ev);
  if (h->cp_first) cudaEventDestroy(h->cp_first);
  if (h->cp) cudaStreamDestroy(h->cp);
  if (h->st) cudaStreamDestroy(h->st);
  delete h;
  return GSYEIG_SUCCESS;
}

int gsyeig_set_options(gsyeig_handle h, const gsyeig_opts *o) {
  if (!h) return -1;
  if (!o) return -2;
  if (!(o->tol > 0.0) || o->krylov_dim < 0 || o->keep < 0 || o->max_restarts < 0 || o->timeout_ms < 0 ||
      o->block < 0 || o->block > 160 || (o->block > 0 && o->block < 16) || o->profile < 0 || o->profile > 1 ||
      o->fp64_gemm < 0 || o->fp64_gemm > 2 || o->fp64_symv < 0 || o->fp64_symv > 1 || o->qr_restart < 0 ||
      o->qr_restart > 1 || o->inverse < 0 || o->inverse > 1 || o->preserve_inputs < 0 ||
      o->preserve_inputs > 1 || o->verify < 0 || o->verify > 1 || o->implicit < 0 || o->implicit > 1 ||
      o->wait_limit < 0 || o->filter_degree < 0 || o->filter_degree > 64 || o->check_every < 0 ||
      o->start_cols < 0 || (o->start_block && o->start_cols > 0 && o->ld_start < 1) ||
      (o->filter_degree > 0 && !(o->filter_cut != o->filter_edge)) || o->mixed < 0 || o->mixed > 2 || !std::isfinite(o->shift) ||
      o->graph < 0 || o->graph > 1 || o->max_ctas < 0 || o->block_start < 0 || o->block_start > 1)
    return -2;
  if (o->krylov_dim > 0 && o->keep > 0 && o->keep >= o->krylov_dim) return -2;
  h->opts = *o;
  return GSYEIG_SUCCESS;
}

const char *gsyeig_strerror(int status) {
  switch (status) {
    case GSYEIG_SUCCESS: return "success";
    case GSYEIG_NOT_SPD: return "B is not positive definite (Cholesky pivot <= 0)";
    case GSYEIG_NO_CONVERGENCE: return "Lanczos did not converge within max_restarts";
    case GSYEIG_TIMEOUT: return "time budget exhausted";
    case GSYEIG_CUDA_ERROR: return "CUDA runtime error";
    case GSYEIG_OOM: return "out of device memory";
    case GSYEIG_NOT_SUPPORTED: return "unsupported parameter combination";
    case GSYEIG_SCRATCH_TOO_SMALL:
      return "problem too large for the fixed scratch of the allocation-free entry point (needs 5*m*cnt <= 1048576 doubles)";
    default: return status < 0 ? "invalid argument" : "unknown status";
  }
}

int64_t gsyeig_kernel_launches(void) { return g_launches.load(); }

int gsyeig_potrf(gsyeig_handle h, double *dB, int64_t ldb, int64_t n, int64_t *potrf_index) {
  if (!h) return -1;
  if (!dB) return -2;
  if (ldb < std::max<int64_t>(1, n)) return -3;
  if (n < 1) return -4;
  GS_TRY(begin(h));
  GemmScope gscope;
  const int nb = nb_of(h, n);
  FactorWork w;
  GS_TRY(factor_ws(h, n, nb, 1, w));
  GS_TRY(potrf_blocked(h->st, n, dB, ldb, nb, w));
  int flag = 0;
  GS_CUDA(cudaMemcpyAsync(&flag, w.flag, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  GS_TRY(finish(h));
  GS_TRY(gemm_check(h));
  if (potrf_index) *potrf_index = flag;
  return flag ? GSYEIG_NOT_SPD : GSYEIG_SUCCESS;
}

int gsyeig_sygst(gsyeig_handle h, double *dA, int64_t lda, const double *dU, int64_t ldu, int64_t n) {
  if (!h) return -1;
  if (!dA) return -2;
  if (lda < std::max<int64_t>(1, n)) return -3;
  if (!dU) return -4;
  if (ldu < std::max<int64_t>(1, n)) return -5;
  if (n < 1) return -6;
  GS_TRY(begin(h));
  GemmScope gscope;
  const int nb = nb_of(h, n);
  FactorWork w;
  GS_TRY(factor_ws(h, n, nb, 1, w));
  GS_TRY(sygst_ws(h, n, nb, w));
  GS_TRY(sygst_blocked(h->st, n, dA, lda, dU, ldu, nb, w, false));
  GS_TRY(finish(h));
  return gemm_check(h);
}

int gsyeig_symv(gsyeig_handle h, const double *dC, int64_t ldc, int64_t n, const double *dw, double *dz) {
  if (!h) return -1;
  if (!dC) return -2;
  if (ldc < std::max<int64_t>(1, n)) return -3;
  if (n < 1) return -4;
  if (!dw) return -5;
  if (!dz) return -6;
  GS_TRY(begin(h));
  ProfScope prof(h);
  if (h->opts.fp64_symv == 1) {
    GS_TRY(symv_f64(h->st, n, dC, ldc, dw, dz));
    return finish(h);
  }
  // the solver's default ke1 operator: C's lower triangle as fp32 hi/lo tiles
  GS_TRY(h->dfop.ensure(df_operator_bytes(n)));
  GS_TRY(h->dfpart.ensure(df_partials_bytes(n)));
  DfOperator op;
  op.hi = static_cast<float *>(h->dfop.p);
  op.W = static_cast<float2 *>(h->dfpart.p);
  const int64_t NTt = ceil_div(n, 64);
  op.wsplit = op.W + (size_t)NTt * NTt * 64;
  op.err = reinterpret_cast<int *>(op.wsplit + (size_t)NTt * 64);
  op.spin = (uint32_t)h->opts.wait_limit;
  GS_CUDA(cudaMemsetAsync(op.err, 0, sizeof(int), h->st));
  GS_TRY(df_operator_build(h->st, n, dC, ldc, op));
  GS_TRY(df_symv(h->st, op, dw, dz));
  int e = 0;
  GS_CUDA(cudaMemcpyAsync(&e, op.err, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  GS_TRY(finish(h));
  return e ? GSYEIG_TIMEOUT : GSYEIG_SUCCESS;
}

int gsyeig_trsm_back(gsyeig_handle h, const double *dU, int64_t ldu, int64_t n, double *dY, int64_t ldy, int64_t s) {
  if (!h) return -1;
  if (!dU) return -2;
  if (ldu < std::max<int64_t>(1, n)) return -3;
  if (n < 1) return -4;
  if (!dY) return -5;
  if (ldy < n) return -6;
  if (s < 1) return -7;
  GS_TRY(begin(h));
  GemmScope gscope;
  const int nb = nb_of(h, n);
  FactorWork w;
  GS_TRY(factor_ws(h, n, nb, s, w));
  GS_TRY(trsm_back_blocked(h->st, n, dU, ldu, dY, ldy, s, nb, w, false));
  GS_TRY(finish(h));
  return gemm_check(h);
}

int gsyeig_gemm(gsyeig_handle h, int transA, int transB, int64_t M, int64_t N, int64_t K, double alpha, const double *A,
                int64_t lda, const double *B, int64_t ldb, double beta, double *C, int64_t ldc) {
  if (!h) return -1;
  if (M < 0) return -4;
  if (N < 0) return -5;
  if (K < 0) return -6;
  if (!A && M > 0 && K > 0) return -8;
  if (lda < std::max<int64_t>(1, transA ? K : M)) return -9;
  if (!B && N > 0 && K > 0) return -10;
  if (ldb < std::max<int64_t>(1, transB ? N : K)) return -11;
  if (!C && M > 0 && N > 0) return -13;
  if (ldc < std::max<int64_t>(1, M)) return -14;
  if (M == 0 || N == 0) return GSYEIG_SUCCESS;
  GS_TRY(begin(h));
  GemmScope gscope;
  GS_TRY(gemm_setup(h, std::max(M, N), 128, 1));  // K = 0 scales C by beta in the FP64 kernel
  GS_TRY(dgemm(h->st, transA != 0, transB != 0, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc));
  GS_TRY(finish(h));
  return gemm_check(h);
}

int gsyeig_tridiag_eig(gsyeig_handle h, const double *d, const double *e, int64_t m, int64_t first, int64_t cnt,
                       double *lam, double *dZ, int64_t ldz) {
  if (!h) return -1;
  if (!d) return -2;
  if (!e && m > 1) return -3;
  if (m < 1) return -4;
  if (first < 0 || first >= m) return -5;
  if (cnt < 1 || first + cnt > m) return -6;
  if (!lam) return -7;
  if (dZ && ldz < m) return -9;
  GS_TRY(begin(h));
  GS_TRY(tri_bisect(h->st, m, d, e, 0, nullptr, first, cnt, lam));
  if (dZ) {
    GS_TRY(h->invw.ensure((size_t)5 * m * cnt * sizeof(double)));
    GS_TRY(tri_invit(h->st, m, d, e, 0, nullptr, cnt, lam, dZ, ldz, h->invw.d()));
  }
  return finish(h);
}

int gsyeig_syev_lanczos(gsyeig_handle h, const double *dC, int64_t ldc, int64_t n, int64_t s, int which, double *w,
                        double *dY, int64_t ldy, gsyeig_info *info) {
  if (!h) return -1;
  if (!dC) return -2;
  if (ldc < std::max<int64_t>(1, n)) return -3;
  if (n < 2) return -4;
  if (s < 1 || s >= n) return -5;
  if (which != GSYEIG_SMALLEST && which != GSYEIG_LARGEST) return -6;
  if (!w) return -7;
  if (!dY) return -8;
  if (ldy < n) return -9;
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->n = n;
    info->s = s;
  }
  const int64_t l0 = g_launches.load();
  GS_TRY(begin(h));
  ProfScope prof(h);
  GemmScope gscope;
  current_gemm() = nullptr;  // no slicing workspace here: the basis products use the FP64 engine
  GS_TRY(h->hw.ensure((size_t)s * sizeof(double)));
  double ms_ke3 = 0;
  cudaEventRecord(h->ev[0], h->st);
  int st = lanczos_run(h, dC, ldc, n, s, which, h->hw.d(), dY, ldy, info, &ms_ke3);
  if (st != GSYEIG_SUCCESS && st != GSYEIG_NO_CONVERGENCE && st != GSYEIG_TIMEOUT) return st;
  GS_CUDA(cudaMemcpyAsync(w, h->hw.p, (size_t)s * sizeof(double), cudaMemcpyDefault, h->st));
  cudaEventRecord(h->ev[1], h->st);
  GS_TRY(finish(h));
  prof.fill(info);
  if (info) {
    info->ms_ke = elapsed(h->ev[0], h->ev[1]) - ms_ke3;
    info->ms_ke3 = ms_ke3;
    info->ms_total = elapsed(h->ev[0], h->ev[1]);
    info->kernel_launches = g_launches.load() - l0;
  }
  return st;
}

int gsyeig_solve(gsyeig_handle h, double *A, int64_t lda, double *B, int64_t ldb, int64_t n, int64_t s, int which,
                 double *w, double *X, int64_t ldx, gsyeig_info *info) {
  if (!h) return -1;
  int bad = check_solve_args(lda, ldb, n, s, which, A, B, w, X, ldx);
  if (bad) return bad;
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->n = n;
    info->s = s;
  }
  const int64_t l0 = g_launches.load();
  GS_TRY(begin(h));
  ProfScope prof(h);
  GemmScope gscope;
  cudaStream_t st = h->st;
  // host inputs: stage them in the handle's device buffers
  const bool hostA = !is_device_ptr(A), hostB = !is_device_ptr(B), hostX = !is_device_ptr(X);
  if (hostA != hostB || hostA != hostX) return -10;
  double *dA = A, *dB = B, *dX = X;
  int64_t dlda = lda, dldb = ldb, dldx = ldx;
  // every return waits for a copy still in flight on the second stream (the
  // caller may free its host buffer once the call returns)
  struct CopyGuard {
    cudaStream_t st = nullptr;
    ~CopyGuard() {
      if (st) cudaStreamSynchronize(st);
    }
  } copy_pending;
  GS_CUDA(cudaEventRecord(h->ev[0], st));
  if (hostA) {
    GS_TRY(h->hA.ensure((size_t)n * n * sizeof(double)));
    GS_TRY(h->hB.ensure((size_t)n * n * sizeof(double)));
    GS_TRY(h->hX.ensure((size_t)n * s * sizeof(double)));
    dA = h->hA.d();
    dB = h->hB.d();
    dX = h->hX.d();
    dlda = dldb = dldx = n;
    // the matrix factored first (A on the inverse route, else B) on the
    // solve's stream; the other on a second stream once the first has landed
    // (the two would otherwise share the link and delay the factorisation),
    // so that its transfer overlaps the Cholesky factorisation; the solve
    // waits for it just before its first read
    if (!h->cp) {
      GS_CUDA(cudaStreamCreateWithFlags(&h->cp, cudaStreamNonBlocking));
      GS_CUDA(cudaEventCreateWithFlags(&h->cp_ev, cudaEventDisableTiming));
      GS_CUDA(cudaEventCreateWithFlags(&h->cp_first, cudaEventDisableTiming));
    }
    const bool a_first = h->opts.inverse == 1 && which == GSYEIG_SMALLEST;
    double *d1 = a_first ? dA : dB, *d2 = a_first ? dB : dA;
    const double *s1 = a_first ? A : B, *s2 = a_first ? B : A;
    const int64_t l1 = a_first ? lda : ldb, l2 = a_first ? ldb : lda;
    auto h2d = [&](double *d, const double *src, int64_t ld, cudaStream_t s) { return stage_h2d(d, src, n, ld, s); };
    const auto tq0 = std::chrono::steady_clock::now();
    GS_TRY(h2d(d1, s1, l1, st));
    GS_CUDA(cudaEventRecord(h->cp_first, st));
    GS_CUDA(cudaEventRecord(h->ev[7], st));
    GS_CUDA(cudaStreamWaitEvent(h->cp, h->cp_first, 0));
    GS_TRY(h2d(d2, s2, l2, h->cp));
    GS_CUDA(cudaEventRecord(h->cp_ev, h->cp));
    copy_pending.st = h->cp;
    if (info)
      info->host_ms_h2d_enqueue = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tq0).count();
  }
  // the second matrix has landed (no-op for device inputs)
  auto second_ready = [&]() -> int {
    if (hostA) GS_CUDA(cudaStreamWaitEvent(st, h->cp_ev, 0));
    return GSYEIG_SUCCESS;
  };
  if (!hostA && h->opts.preserve_inputs == 1) {  // solve on copies; the caller's A, B stay as they were
    GS_TRY(h->pA.ensure((size_t)n * n * sizeof(double)));
    GS_TRY(h->pB.ensure((size_t)n * n * sizeof(double)));
    GS_CUDA(cudaMemcpy2DAsync(h->pA.p, n * sizeof(double), A, lda * sizeof(double), n * sizeof(double), n,
                              cudaMemcpyDeviceToDevice, st));
    GS_CUDA(cudaMemcpy2DAsync(h->pB.p, n * sizeof(double), B, ldb * sizeof(double), n * sizeof(double), n,
                              cudaMemcpyDeviceToDevice, st));
    dA = h->pA.d();
    dB = h->pB.d();
    dlda = dldb = n;
  }
  const bool verify = h->opts.verify == 1;
  if (verify) {  // the originals, completed from the triangles the route reads (A lower, B upper)
    GS_TRY(second_ready());
    GS_TRY(h->vA.ensure((size_t)n * n * sizeof(double)));
    GS_TRY(h->vB.ensure((size_t)n * n * sizeof(double)));
    GS_CUDA(cudaMemcpy2DAsync(h->vA.p, n * sizeof(double), dA, dlda * sizeof(double), n * sizeof(double), n,
                              cudaMemcpyDeviceToDevice, st));
    GS_CUDA(cudaMemcpy2DAsync(h->vB.p, n * sizeof(double), dB, dldb * sizeof(double), n * sizeof(double), n,
                              cudaMemcpyDeviceToDevice, st));
    GS_TRY(symmetrize(st, n, h->vA.d(), n, true));
    GS_TRY(symmetrize(st, n, h->vB.d(), n, false));
  }
  const int nb = nb_of(h, n);
  FactorWork fw;
  GS_TRY(factor_ws(h, n, nb, s, fw));
  GS_TRY(h->hw.ensure((size_t)s * sizeof(double)));
  // Inverse problem (Section 3.1): with A positive definite as well, the
  // smallest lambda of (A, B) are the largest mu = 1/lambda of (B, A), the
  // end of C' = L^-T B L^-1 that Lanczos resolves fastest when the wanted
  // lambda sit at the bottom of a wide spectrum.  The factored matrix F and
  // the transformed matrix G swap roles.
  bool inv = h->opts.inverse == 1 && which == GSYEIG_SMALLEST;
  double *dF = dB, *dG = dA;
  int64_t dldf = dldb, dldg = dlda;
  int flag = 0;
  GS_CUDA(cudaEventRecord(h->ev[1], st));
  if (inv) {
    // A's lower triangle is the one read: mirror it, keep its diagonal (the
    // only part of the lower triangle a failed Cholesky overwrites)
    GS_TRY(symmetrize(st, n, dA, dlda, true));
    GS_TRY(h->diag.ensure((size_t)n * sizeof(double)));
    GS_CUDA(cudaMemcpy2DAsync(h->diag.p, sizeof(double), dA, (size_t)(dlda + 1) * sizeof(double), sizeof(double), n,
                              cudaMemcpyDeviceToDevice, st));
    if (h->opts.shift != 0.0) {  // the upper triangle of A - shift B (B's upper triangle is the one read)
      GS_TRY(second_ready());
      GS_TRY(lz_shift_upper(st, n, dA, dlda, dB, dldb, h->opts.shift));
    }
    GS_TRY(potrf_blocked(st, n, dA, dlda, nb, fw));
    GS_CUDA(cudaMemcpyAsync(&flag, fw.flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    GS_CUDA(cudaStreamSynchronize(st));
    GS_TRY(gemm_check(h));  // an expired GEMM wait, not a pivot, may have set the flag
    GS_TRY(second_ready());
    if (flag) {  // A indefinite: put its diagonal back, take the direct route
      GS_CUDA(cudaMemcpy2DAsync(dA, (size_t)(dlda + 1) * sizeof(double), h->diag.p, sizeof(double), sizeof(double), n,
                                cudaMemcpyDeviceToDevice, st));
      inv = false;
      flag = 0;
    } else {
      dF = dA;
      dldf = dlda;
      dG = dB;
      dldg = dldb;
      // B's upper triangle is the one read: mirror it into the lower
      GS_TRY(symmetrize(st, n, dB, dldb, false));
    }
  }
  // gs1: F = U^T U
  if (!inv) {
    GS_TRY(potrf_blocked(st, n, dB, dldb, nb, fw));
    GS_CUDA(cudaMemcpyAsync(&flag, fw.flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  }
  GS_CUDA(cudaEventRecord(h->ev[2], st));
  GS_CUDA(cudaStreamSynchronize(st));
  GS_TRY(gemm_check(h));
  if (flag) {
    if (info) info->potrf_index = flag;
    return GSYEIG_NOT_SPD;
  }
  GS_TRY(second_ready());
  const bool ki = h->opts.implicit == 1;
  if (ki && h->opts.fp64_symv == 1) return GSYEIG_NOT_SUPPORTED;  // KI runs on the double-float tiles
  if (ki && (h->opts.mixed != 0 || h->opts.block_start == 1)) return GSYEIG_NOT_SUPPORTED;
  if (!ki) {
    // gs2: C = U^-T G U^-1 over G (diagonal-block inverses reused from gs1)
    GS_TRY(sygst_ws(h, n, nb, fw));
    GS_TRY(sygst_blocked(st, n, dG, dldg, dF, dldf, nb, fw, true));
  } else {
    // variant KI: G stays; U^-1 is formed once (n^3/3 flops on the GEMM
    // engine) so that both triangular solves of every step become
    // triangular products over stored tiles
    if (!inv) GS_TRY(symmetrize(st, n, dG, dldg, true));  // A's lower triangle is the one read
    GS_TRY(h->kinv.ensure((size_t)n * n * sizeof(double)));
    GS_TRY(trtri_upper_blocked(st, n, dF, dldf, h->kinv.d(), n, nb, fw, true));
  }
  GS_CUDA(cudaEventRecord(h->ev[3], st));
  // ke: Lanczos on C; Ritz vectors land in X.  On the inverse route the
  // smallest Ritz value of the final projected matrix bounds the smallest
  // eigenvalue of L^-T B L^-1 from above: if it is not positive, B is not
  // positive definite (the direct route's Cholesky of B would fail).
  double ms_ke3 = 0, theta_min = 1.0;
  int status;
  if (h->opts.mixed == 1) {
    // fp32 block Lanczos, then the FP64-accurate Lanczos started from the sum
    // of the fp32 Ritz vectors, with Ritz tests every check_every (default
    // 32) steps: the start vector lies in the wanted invariant subspace up to
    // the fp32 stage's error, so the FP64 stage stops early
    const double *blk = nullptr;
    int64_t bcols = 0;
    status = lanczos_mixed(h, dG, dldg, n, s, inv ? GSYEIG_LARGEST : which, h->hw.d(), dX, dldx, info, &ms_ke3,
                           nullptr, 0, &blk, &bcols);
    if (status != GSYEIG_SUCCESS && status != GSYEIG_NOT_SUPPORTED) return status;
    gsyeig_info keep{};
    if (info) keep = *info;
    const gsyeig_opts saved = h->opts;
    if (status == GSYEIG_SUCCESS) {
      // every Ritz vector of the fp32 stage, guard columns included: the
      // Lanczos stage then resolves s + guard pairs, and the wanted s see
      // the wider gap to the first pair outside that set
      GS_TRY(h->mx_ones.ensure((size_t)bcols * sizeof(double)));
      const std::vector<double> ones((size_t)bcols, 1.0);
      GS_CUDA(cudaMemcpyAsync(h->mx_ones.p, ones.data(), (size_t)bcols * sizeof(double), cudaMemcpyHostToDevice, st));
      h->opts.start_block = blk;
      h->opts.start_cols = bcols;
      h->opts.ld_start = n;
      h->opts.start_weights = h->mx_ones.d();
      h->opts.filter_degree = 0;
      if (h->opts.check_every == 0) h->opts.check_every = 32;
    }
    status = lanczos_run(h, dG, dldg, n, s, inv ? GSYEIG_LARGEST : which, h->hw.d(), dX, dldx, info, &ms_ke3,
                         nullptr, inv ? &theta_min : nullptr, nullptr, 0);
    h->opts = saved;
    if (info) {  // ms_refine (the FP64 stage) is set with the stage times below
      info->block_steps = keep.block_steps;
      info->ms_block_lanczos = keep.ms_block_lanczos;
      info->matvecs += keep.matvecs;
    }
  } else if (h->opts.mixed == 2 || (h->opts.block_start == 1 && h->opts.start_block)) {
    // fp32 block Lanczos (or the caller's block) + FP64 block refinement;
    // B's definiteness is not checked here on the inverse route
    status = lanczos_mixed(h, dG, dldg, n, s, inv ? GSYEIG_LARGEST : which, h->hw.d(), dX, dldx, info, &ms_ke3,
                           dF, dldf);
    if (status == GSYEIG_NO_CONVERGENCE || status == GSYEIG_NOT_SUPPORTED) {
      // the block refinement did not reach the tolerance (small relative
      // gaps at the wanted end, e.g. the smallest eigenvalues on the direct
      // route): the FP64-accurate Lanczos stage takes over
      gsyeig_info keep{};
      if (info) keep = *info;
      status = lanczos_run(h, dG, dldg, n, s, inv ? GSYEIG_LARGEST : which, h->hw.d(), dX, dldx, info, &ms_ke3,
                           nullptr, inv ? &theta_min : nullptr, dF, dldf);
      if (info) {
        info->refine_fallback = 1;
        info->block_steps = keep.block_steps;
        info->refine_iters = keep.refine_iters;
        info->ms_block_lanczos = keep.ms_block_lanczos;
        info->ms_refine = keep.ms_refine;
        info->matvecs += keep.matvecs;
      }
    }
  } else {
    status = lanczos_run(h, dG, dldg, n, s, inv ? GSYEIG_LARGEST : which, h->hw.d(), dX, dldx, info, &ms_ke3,
                         ki ? h->kinv.d() : nullptr, inv ? &theta_min : nullptr, dF, dldf);
  }
  if (status != GSYEIG_SUCCESS && status != GSYEIG_NO_CONVERGENCE && status != GSYEIG_TIMEOUT) return status;
  if (inv && !(theta_min > 0.0)) {
    if (info) info->inverse = 1;
    return GSYEIG_NOT_SPD;
  }
  if (inv && !ki) {  // (variant KI holds the untransformed matrix, not C')
    // needed when the wanted mu span a wide range (a lambda near zero): the
    // defect of X^T B X grows like mu_max / mu_min times the rounding level
    double mu_lo = 0.0, mu_hi = 0.0;  // the wanted mu, ascending: all must be positive
    GS_CUDA(cudaMemcpyAsync(&mu_lo, h->hw.d(), sizeof(double), cudaMemcpyDeviceToHost, st));
    GS_CUDA(cudaMemcpyAsync(&mu_hi, h->hw.d() + (s - 1), sizeof(double), cudaMemcpyDeviceToHost, st));
    GS_CUDA(cudaStreamSynchronize(st));
    if (mu_lo > 0.0 && theta_min > 0.0 && mu_hi > 1e5 * mu_lo)
      GS_TRY(b_orthonormalise_inverse(h, st, n, s, dG, dldg, dX, dldx, h->hw.d()));
  }
  GS_CUDA(cudaEventRecord(h->ev[4], st));
  // bt1: X = U^-1 Y
  GS_TRY(trsm_back_blocked(st, n, dF, dldf, dX, dldx, s, nb, fw, true));
  if (inv) {
    // B is assumed positive definite on this route (it is never factored);
    // a wanted mu <= 0 shows it is not
    double mu_min = 0.0;
    GS_CUDA(cudaMemcpyAsync(&mu_min, h->hw.d(), sizeof(double), cudaMemcpyDeviceToHost, st));
    GS_CUDA(cudaStreamSynchronize(st));
    if (!(mu_min > 0.0)) return GSYEIG_NOT_SPD;
    GS_TRY(lz_invert_pairs(st, n, s, h->hw.d(), dX, dldx, h->opts.shift));
  }
  GS_CUDA(cudaMemcpyAsync(w, h->hw.p, (size_t)s * sizeof(double), cudaMemcpyDefault, st));
  if (hostA)
    GS_CUDA(cudaMemcpy2DAsync(X, ldx * sizeof(double), dX, n * sizeof(double), n * sizeof(double), s,
                              cudaMemcpyDeviceToHost, st));
  GS_CUDA(cudaEventRecord(h->ev[8], st));
  GS_TRY(finish(h));
  GS_TRY(gemm_check(h));
  prof.fill(info);
  if (verify) {  // after the end mark: not part of the stage times
    double vout[2] = {0.0, 0.0};
    GS_TRY(h->vws.ensure(verify_workspace_doubles(n, s) * sizeof(double)));
    GS_TRY(verify_solution(st, n, s, h->vA.d(), n, h->vB.d(), n, dX, dldx, h->hw.d(), h->vws.d(), vout));
    GS_TRY(gemm_check(h));
    if (info) {
      info->max_eta = vout[0];
      info->orth_err = vout[1];
    }
  }
  if (info) {
    info->ms_gs1 = elapsed(h->ev[1], h->ev[2]);
    info->ms_gs2 = elapsed(h->ev[2], h->ev[3]);
    const double ke = elapsed(h->ev[3], h->ev[4]);
    info->ms_ke3 = ms_ke3;
    info->ms_ke = ke - ms_ke3;
    if (h->opts.mixed == 1) info->ms_refine = ke - info->ms_block_lanczos;  // the FP64 Lanczos stage
    info->ms_bt1 = elapsed(h->ev[4], h->ev[8]);
    info->ms_total = elapsed(h->ev[0], h->ev[8]);
    if (hostA) info->ms_h2d_first = elapsed(h->ev[0], h->ev[7]);
    info->kernel_launches = g_launches.load() - l0;
    info->inverse = inv ? 1 : 0;
  }
  return status;
}

}  // extern "C"

// ---- batches ---------------------------------------------------------------

namespace {

__global__ void k_tune_matrix(int64_t n, double *M) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n * n; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % n, j = idx / n;
    const uint64_t a = (uint64_t)std::min(i, j) * 0x9E3779B97F4A7C15ull ^ (uint64_t)std::max(i, j) * 0xBF58476D1CE4E5B9ull;
    M[idx] = (i == j) ? (double)n : (double)((a >> 11) & 0xFFFFF) * 0x1p-20 - 0.5;
  }
}

// Time gs1 + gs2 of a synthetic diagonally dominant SPD pencil of order n
// with each candidate panel width; the fastest wins.
int autotune(gsyeig_handle h, int64_t n) {
  const int cand[] = {64, 128};
  GS_TRY(h->pA.ensure((size_t)n * n * sizeof(double)));
  GS_TRY(h->pB.ensure((size_t)n * n * sizeof(double)));
  cudaStream_t st = h->st;
  float best_ms = 1e30f;
  int best = 128;
  const gsyeig_opts saved = h->opts;
  for (int rep = 0; rep < 2; rep++)  // the first pass warms the workspace up
    for (int nb : cand) {
      if (nb > n) continue;
      h->opts.block = nb;
      FactorWork fw;
      GS_TRY(factor_ws(h, n, nb, 1, fw));
      GS_TRY(sygst_ws(h, n, nb, fw));
      const unsigned g = (unsigned)std::min<int64_t>(ceil_div(n * n, 256), 4096);
      k_tune_matrix<<<g, 256, 0, st>>>(n, h->pA.d());
      k_tune_matrix<<<g, 256, 0, st>>>(n, h->pB.d());
      count_launch(2);
      GS_CHECK_LAUNCH();
      GS_CUDA(cudaEventRecord(h->ev[1], st));
      GS_TRY(potrf_blocked(st, n, h->pB.d(), n, nb, fw));
      GS_TRY(sygst_blocked(st, n, h->pA.d(), n, h->pB.d(), n, nb, fw, true));
      GS_CUDA(cudaEventRecord(h->ev[2], st));
      GS_CUDA(cudaEventSynchronize(h->ev[2]));
      const float ms = elapsed(h->ev[1], h->ev[2]);
      if (rep == 1 && ms < best_ms) {
        best_ms = ms;
        best = nb;
      }
    }
  current_gemm() = nullptr;
  h->opts = saved;
  return best;
}

int tuned_block(gsyeig_handle h, gsyeig_handle worker, int64_t n) {
  const int64_t cls = ceil_div(n, 512) * 512;
  {
    std::lock_guard<std::mutex> lock(h->tune_mu);
    auto it = h->tuned.find(cls);
    if (it != h->tuned.end()) return it->second;
  }
  const int nb = autotune(worker, cls);
  std::lock_guard<std::mutex> lock(h->tune_mu);
  h->tuned[cls] = nb;
  return nb;
}

}  // namespace

extern "C" int gsyeig_solve_batched(gsyeig_handle h, int64_t count, const gsyeig_problem *probs, int32_t nstreams,
                                    int32_t *statuses, gsyeig_info *infos) {
  if (!h) return -1;
  if (count < 0) return -2;
  if (!probs && count > 0) return -3;
  if (nstreams < 1 || nstreams > 16) return -4;
  for (int64_t i = 0; i < count; i++) {
    const gsyeig_problem &p = probs[i];
    if (check_solve_args(p.lda, p.ldb, p.n, p.s, p.which, p.A, p.B, p.w, p.X, p.ldx) != 0) return -3;
  }
  if (count == 0) return GSYEIG_SUCCESS;
  GS_TRY(begin(h));
  while ((int)h->subs.size() < nstreams) {
    gsyeig_handle sub = nullptr;
    GS_TRY(gsyeig_create(&sub, h->device, h->st));  // ordered after the caller's stream through h->st
    h->subs.push_back(sub);
  }
  gsyeig_opts o = h->opts;
  o.graph = 1;
  o.profile = 0;
  if (o.max_ctas == 0) o.max_ctas = (int32_t)ceil_div(num_sms_cached(), nstreams);
  // largest problems first
  std::vector<int64_t> order((size_t)count);
  for (int64_t i = 0; i < count; i++) order[(size_t)i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return probs[a].n > probs[b].n; });
  std::atomic<int64_t> next{0};
  std::vector<int> st((size_t)count, GSYEIG_SUCCESS);
  auto work = [&](int t) {
    gsyeig_handle sub = h->subs[(size_t)t];
    cudaSetDevice(h->device);
    for (;;) {
      const int64_t q = next.fetch_add(1);
      if (q >= count) break;
      const int64_t i = order[(size_t)q];
      const gsyeig_problem &p = probs[i];
      gsyeig_opts oi = o;
      if (h->opts.block == 0) oi.block = tuned_block(h, sub, p.n);
      sub->opts = oi;
      gsyeig_info inf;
      st[(size_t)i] = gsyeig_solve(sub, p.A, p.lda, p.B, p.ldb, p.n, p.s, p.which, p.w, p.X, p.ldx, &inf);
      if (infos) infos[i] = inf;
    }
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < nstreams; t++) pool.emplace_back(work, t);
  work(0);
  for (auto &th : pool) th.join();
  int rc = GSYEIG_SUCCESS;
  for (int64_t i = 0; i < count; i++) {
    if (statuses) statuses[i] = st[(size_t)i];
    if (rc == GSYEIG_SUCCESS && st[(size_t)i] != GSYEIG_SUCCESS) rc = st[(size_t)i];
  }
  // the caller's stream orders after every internal stream
  for (gsyeig_handle sub : h->subs) {
    GS_CUDA(cudaEventRecord(sub->ev[8], sub->st));
    GS_CUDA(cudaStreamWaitEvent(h->user, sub->ev[8], 0));
  }
  return rc;
}

extern "C" int32_t gsyeig_autotuned_block(gsyeig_handle h, int64_t n) {
  if (!h || n < 1) return 0;
  if (begin(h) != GSYEIG_SUCCESS) return 0;
  if (h->subs.empty()) {
    gsyeig_handle sub = nullptr;
    if (gsyeig_create(&sub, h->device, h->st) != GSYEIG_SUCCESS) return 0;
    h->subs.push_back(sub);
  }
  return tuned_block(h, h->subs[0], n);
}
