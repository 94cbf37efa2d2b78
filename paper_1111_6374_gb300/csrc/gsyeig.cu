// C ABI of the library and the host-side driver of the KE route
// (Section 2.3 of the paper; Table 1 keys gs1, gs2, ke1-ke3, bt1).
// Device memory for inputs/outputs belongs to the caller; the handle owns a
// grow-on-demand workspace.  The driver only sequences kernels and reads
// back a few scalars per restart (converged count, breakdown flag).
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>

#include "lanczos.cuh"
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
  cudaEvent_t ev[10] = {};  // 0-6 stage marks, 8 end mark, 9 user-stream ordering
  gsyeig_opts opts{};
  // workspace
  DevBuf uinv, panel, flag, diag;
  DevBuf V, Vq, z, h1, h2, sq, alpha, beta, alphaP, betaP, theta, S, Q, rot, invw, state, shifts, arrow;
  DevBuf hA, hB, hX, hw;  // device copies for host-pointer calls
  DevBuf pA, pB;          // working copies when opts.preserve_inputs
  DevBuf vA, vB, vws;     // originals and workspace of opts.verify
  DevBuf gemm_ws;         // slices of the tensor-core GEMM
  DevBuf gemm_err;        // device error flag of the tcgen05 engine
  DevBuf dfop, dfpart;    // double-float operator tiles and symv partials
  DevBuf kinv, dfopL, kt; // variant KI: U^-1, the tiles of L = U^-T, two temporaries
  DevBuf tmin;            // smallest eigenvalue of the final projected matrix
  DevBuf wstart;          // start-block construction and Chebyshev filter vectors
  DfOperator op, opL;
  bool use_df = false;
  bool ki = false;        // the operator is U^-T G U^-1 applied implicitly (variant KI)
  KernelProfiler prof;
  GemmContext gemm;
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
// operands of at most max(n, s) rows and K up to the outer block 4 nb (the
// tcgen05 engine takes up to 512 per call).
int gemm_setup(gsyeig_handle h, int64_t n, int nb, int64_t s) {
  h->gemm.sliced = (h->opts.fp64_gemm != 1);
  h->gemm.umma = (h->opts.fp64_gemm == 0);
  if (h->gemm.sliced) {
    const int64_t r = std::max<int64_t>(n, s);
    GS_TRY(h->gemm_ws.ensure(
        std::max(sliced_workspace_bytes(r, r, nb), umma_workspace_bytes(r, r, std::min<int64_t>(512, 4 * (int64_t)nb)))));
    h->gemm.ws = h->gemm_ws.p;
    h->gemm.ws_bytes = h->gemm_ws.bytes;
    GS_TRY(h->gemm_err.ensure(64));
    h->gemm.err = static_cast<int *>(h->gemm_err.p);
    GS_CUDA(cudaMemsetAsync(h->gemm.err, 0, sizeof(int), h->st));  // cudaMalloc does not zero
  }
  h->gemm.spin = (uint32_t)h->opts.wait_limit;
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
  GS_TRY(h->uinv.ensure((size_t)nblk * nb * nb * sizeof(double)));
  GS_TRY(h->panel.ensure((size_t)std::max<int64_t>(n, s) * nb * sizeof(double) + 64));
  GS_TRY(h->flag.ensure(256 + 160 * sizeof(double)));
  w.Uinv = h->uinv.d();
  w.panel = h->panel.d();
  w.flag = static_cast<int *>(h->flag.p);
  w.rdiag = reinterpret_cast<double *>(static_cast<char *>(h->flag.p) + 256);
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
  const int64_t wf = (which == GSYEIG_LARGEST) ? m - s : 0;  // first wanted index among the m Ritz values
  const int64_t kfirst = (which == GSYEIG_LARGEST) ? m - k : 0;  // first kept index (thick restart)
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
      for (; j < jend; j++) GS_TRY(lanczos_step(h, st, n, m, j, C, ldc));
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
  DevBuf *bufs[] = {&h->wstart, &h->kinv, &h->dfopL, &h->kt, &h->tmin, &h->pA, &h->pB, &h->vA, &h->vB, &h->vws, &h->diag, &h->arrow, &h->gemm_err, &h->dfop, &h->dfpart, &h->gemm_ws, &h->uinv, &h->panel, &h->flag, &h->V, &h->Vq, &h->z, &h->h1, &h->h2, &h->sq, &h->alpha,
                    &h->beta, &h->alphaP, &h->betaP, &h->theta, &h->S, &h->Q, &h->rot, &h->invw, &h->state,
                    &h->shifts, &h->hA, &h->hB, &h->hX, &h->hw};
  for (DevBuf *b : bufs) b->release();
  h->prof.release();
  for (auto &e : h->ev)
    if (e) cudaEventDestroy(e);
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
      (o->filter_degree > 0 && !(o->filter_cut != o->filter_edge)))
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
  GS_CUDA(cudaEventRecord(h->ev[0], st));
  if (hostA) {
    GS_TRY(h->hA.ensure((size_t)n * n * sizeof(double)));
    GS_TRY(h->hB.ensure((size_t)n * n * sizeof(double)));
    GS_TRY(h->hX.ensure((size_t)n * s * sizeof(double)));
    dA = h->hA.d();
    dB = h->hB.d();
    dX = h->hX.d();
    dlda = dldb = dldx = n;
    GS_CUDA(cudaMemcpy2DAsync(dA, n * sizeof(double), A, lda * sizeof(double), n * sizeof(double), n,
                              cudaMemcpyHostToDevice, st));
    GS_CUDA(cudaMemcpy2DAsync(dB, n * sizeof(double), B, ldb * sizeof(double), n * sizeof(double), n,
                              cudaMemcpyHostToDevice, st));
  }
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
    GS_TRY(potrf_blocked(st, n, dA, dlda, nb, fw));
    GS_CUDA(cudaMemcpyAsync(&flag, fw.flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    GS_CUDA(cudaStreamSynchronize(st));
    GS_TRY(gemm_check(h));  // an expired GEMM wait, not a pivot, may have set the flag
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
  const bool ki = h->opts.implicit == 1;
  if (ki && h->opts.fp64_symv == 1) return GSYEIG_NOT_SUPPORTED;  // KI runs on the double-float tiles
  if (!ki) {
    // gs2: C = U^-T G U^-1 over G (diagonal-block inverses reused from gs1)
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
  int status = lanczos_run(h, dG, dldg, n, s, inv ? GSYEIG_LARGEST : which, h->hw.d(), dX, dldx, info, &ms_ke3,
                           ki ? h->kinv.d() : nullptr, inv ? &theta_min : nullptr);
  if (status != GSYEIG_SUCCESS && status != GSYEIG_NO_CONVERGENCE && status != GSYEIG_TIMEOUT) return status;
  if (inv && !(theta_min > 0.0)) {
    if (info) info->inverse = 1;
    return GSYEIG_NOT_SPD;
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
    GS_TRY(lz_invert_pairs(st, n, s, h->hw.d(), dX, dldx));
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
    info->ms_bt1 = elapsed(h->ev[4], h->ev[8]);
    info->ms_total = elapsed(h->ev[0], h->ev[8]);
    info->kernel_launches = g_launches.load() - l0;
    info->inverse = inv ? 1 : 0;
  }
  return status;
}

}  // extern "C"
