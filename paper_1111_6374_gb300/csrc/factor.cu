// Blocked dense steps of the route (gs1, gs2, bt1 in Table 1 of the paper):
//   potrf  B = U^T U                    (Eq. 2)   n^3/3 flops
//   sygst  C = U^-T A U^-1              (Eq. 3)   n^3 flops (+ lower order)
//   trsm   X = U^-1 Y                   (Eq. 4)   n^2 s flops
// All bulk work goes through the GEMM engine; the only other kernels are the
// nb x nb diagonal-block factor/inverse (one CTA each), copies and axpys.
//
// sygst: the paper computes C with two triangular solves (2n^3, Section 4.1)
// or, exploiting symmetry, with n^3.  The n^3 form here is a recursion on a
// 2 x 2 split of A and U (sygst_rec): C11 recursively; the off-diagonal block
// through Y = A21 U11^-1, Z = Y - P/2, W = Z - P/2 with P = U12^T C11; the
// symmetric rank-2n1 update A22 -= Z U12 + U12^T Z^T; C22 recursively; and
// C21 = U22^-T W.  Every step is a large GEMM.  Blocks of at most 4 outer
// blocks use the direct form (sygst_leaf): step 1 forms W = U^-T A in full
// (n^3) and step 2 only the lower triangle of C = W U^-1 (n^3/3).
#include "common.cuh"

namespace gs {
namespace {

// Shared-memory nb x nb block, column-major with leading dimension nb + 1.
struct SmemBlock {
  double *p;
  int ld;
  __device__ double &operator()(int i, int j) { return p[i + j * ld]; }
};

// The diagonal block B[k0:k0+kb, k0:k0+kb] (upper triangle) is factored in
// place, B_kk = U_kk^T U_kk, by a right-looking Cholesky over sub-panels of
// PW rows, three launches each: the PW x PW diagonal sub-block (one CTA),
// the sub-panel's rows right of it (U_pp^-T times the block row, one warp
// per column, many CTAs) and the rank-PW update of the rest of the block
// (16 x 16 tiles of its upper triangle, many CTAs).  GB300's FP64 pipe is
// narrow, so the flops of the block (kb^3/3) are spread over several SMs;
// only the sub-blocks' pivots stay serial.  1 / U(i, i) is left in
// rdiag[0..kb).  A non-positive or NaN pivot records its global 1-based
// index in *flag and stops; every later launch of the block (and every GEMM
// given the flag) then returns at once.  Only the upper triangle of the
// block is written.
constexpr int PW = 32;

// 1/d to within about an ulp for any positive finite d: d = f 2^k with f in
// [1/2, 1) (frexp, exact), an fp32 seed of 1/f refined by two Newton steps
// in FP64, scaled back by 2^-k (ldexp, exact unless the result leaves the
// FP64 range).  GB300's FP64 divide is a long sequence on a narrow pipe; this
// takes four FP64 FMAs.
__device__ __forceinline__ double recip(double d) {
  int k;
  const double f = frexp(d, &k);
  double r = (double)(1.0f / (float)f);
  double e = fma(-f, r, 1.0);
  r = fma(r, e, r);
  e = fma(-f, r, 1.0);
  r = fma(r, e, r);
  return ldexp(r, -k);
}

// Cholesky of the pw x pw diagonal sub-block at (q0, q0), padded to PW x PW
// with the identity, on one CTA of four warps (one per SMSP) in shared
// memory.  Right-looking on the unscaled rows: step j updates
// A(r, c) -= A(j, r) A(j, c) / A(j, j) for j < r <= c, with the active
// trailing triangle packed over all 128 threads (the elements are listed by
// row, last row first, so that step j's are the first (31-j)(32-j)/2), and
// only the pivot's reciprocal is serial.  At the end U(r, c) = A(r, c) /
// sqrt(A(r, r)).
constexpr int SUB_T = 128;
constexpr int SUB_ELEMS = PW * (PW - 1) / 2;  // (r, c), 1 <= r <= c < PW
__global__ void __launch_bounds__(SUB_T) k_chol_sub(double *B, int64_t ldb, int64_t q0, int pw, double *rd, int *flag) {
  if (*flag) return;
  __shared__ double S[PW][PW + 1];  // S[c][r] = A(r, c)
  __shared__ double u[PW], v[PW];
  __shared__ unsigned char er[SUB_ELEMS], ec[SUB_ELEMS];
  const int t = threadIdx.x;
  for (int idx = t; idx < PW * PW; idx += SUB_T) {
    const int r = idx % PW, c = idx / PW;
    S[c][r] = (c < pw && r <= c) ? B[GS_IDX(q0 + r, q0 + c, ldb)] : (r == c ? 1.0 : 0.0);
  }
  for (int e = t; e < SUB_ELEMS; e += SUB_T) {
    int r = PW - 1, base = 0;  // row r holds PW - r elements, rows PW-1, PW-2, ... first
    while (e >= base + (PW - r)) {
      base += PW - r;
      r--;
    }
    er[e] = (unsigned char)r;
    ec[e] = (unsigned char)(r + (e - base));
  }
  __syncthreads();
  int bad = 0;
  for (int j = 0; j < PW; j++) {
    const double d = S[j][j];  // the same in every thread: a uniform exit
    if (!(d > 0.0)) {
      bad = j + 1;
      break;
    }
    if (t < PW) {
      const double a = (t > j) ? S[t][j] : 0.0;  // A(j, t)
      u[t] = a;
      v[t] = a * recip(d);
    }
    __syncthreads();
    const int nact = (PW - 1 - j) * (PW - j) / 2;
    for (int e = t; e < nact; e += SUB_T) {
      const int r = er[e], c = ec[e];
      S[c][r] = fma(-u[r], v[c], S[c][r]);
    }
    __syncthreads();
  }
  if (bad) {
    if (t == 0) atomicCAS(flag, 0, (int)(q0 + bad));
    return;
  }
  if (t < PW) {
    const double sq = sqrt(S[t][t]);
    u[t] = sq;
    v[t] = 1.0 / sq;
    if (t < pw) rd[t] = v[t];
  }
  __syncthreads();
  for (int idx = t; idx < PW * PW; idx += SUB_T) {
    const int r = idx % PW, c = idx / PW;
    if (c < pw && r <= c) B[GS_IDX(q0 + r, q0 + c, ldb)] = (r == c) ? u[r] : S[c][r] * v[r];
  }
}

// Rows q0..q0+pw-1 of the ncols columns from c0 on: x = U_pp^-T b by
// forward substitution, x_j = b_j / U(j, j), then b_i -= U(j, i) x_j for
// i > j; one warp per column (lane i holds row i), 8 columns per CTA.
__global__ void __launch_bounds__(256) k_chol_panel(double *B, int64_t ldb, int64_t q0, int pw, int64_t c0, int ncols,
                                                    const double *rd, const int *flag) {
  if (*flag) return;
  __shared__ double U[PW][PW + 1];  // U[j][i] = U(j, i)
  __shared__ double ri[PW];
  for (int idx = threadIdx.x; idx < PW * PW; idx += blockDim.x) {
    const int j = idx % PW, i = idx / PW;
    U[j][i] = (i < pw && j <= i) ? B[GS_IDX(q0 + j, q0 + i, ldb)] : 0.0;
  }
  if (threadIdx.x < PW) ri[threadIdx.x] = (threadIdx.x < pw) ? rd[threadIdx.x] : 0.0;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cl = blockIdx.x * 8 + warp;
  if (cl >= ncols) return;
  const int64_t col = c0 + cl;
  double b = (lane < pw) ? B[GS_IDX(q0 + lane, col, ldb)] : 0.0;
  double x = 0.0;
  for (int j = 0; j < pw; j++) {
    const double xj = __shfl_sync(0xffffffffu, b, j) * ri[j];
    if (lane == j) x = xj;
    if (lane > j) b = fma(-U[j][lane], xj, b);
  }
  if (lane < pw) B[GS_IDX(q0 + lane, col, ldb)] = x;
}

// The rank-pw update of the upper triangle of the m x m block at (r0, r0):
// A(r, c) -= sum_i U(q0 + i, r) U(q0 + i, c), r <= c, one 16 x 16 tile of
// the upper triangle per CTA (tiles numbered row by row), one element per
// thread.
__global__ void __launch_bounds__(256) k_chol_update(double *B, int64_t ldb, int64_t q0, int pw, int64_t r0, int m,
                                                     const int *flag) {
  if (*flag) return;
  const int nt = (m + 15) / 16;
  int t = blockIdx.x, tr = 0;
  while (tr < nt && t >= nt - tr) {
    t -= nt - tr;
    tr++;
  }
  const int tc = tr + t;
  __shared__ double Ur[PW][17], Uc[PW][17];
  for (int idx = threadIdx.x; idx < PW * 16; idx += blockDim.x) {
    const int i = idx % PW, k = idx / PW;
    const int rr = tr * 16 + k, cc = tc * 16 + k;
    Ur[i][k] = (i < pw && rr < m) ? B[GS_IDX(q0 + i, r0 + rr, ldb)] : 0.0;
    Uc[i][k] = (i < pw && cc < m) ? B[GS_IDX(q0 + i, r0 + cc, ldb)] : 0.0;
  }
  __syncthreads();
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  const int r = tr * 16 + ty, c = tc * 16 + tx;
  if (tr < nt && r < m && c < m && r <= c) {
    double acc = B[GS_IDX(r0 + r, r0 + c, ldb)];
    for (int i = 0; i < pw; i++) acc = fma(-Ur[i][ty], Uc[i][tx], acc);
    B[GS_IDX(r0 + r, r0 + c, ldb)] = acc;
  }
}

// Inverses of upper-triangular kb x kb diagonal blocks into nb x nb blocks
// of Uinv (ld nb, zeros below the diagonal), spread over many SMs: block
// q = blockIdx.y starts at row/column q nb; each CTA stages that block of U in
// shared memory and each of its warps back-substitutes one column c,
// x_k = b_k / U(k, k), b_i -= U(i, k) x_k for i < k, with lane l holding
// rows l, l + 32, ...: no reductions and no FP64 divides in the loop.
// rdiag (or NULL: computed here) holds 1 / U(k, k) of block 0.
constexpr int INV_WARPS = 16;
__global__ void __launch_bounds__(INV_WARPS * 32) k_trtri_cols(int64_t n, const double *U, int64_t ldu, int64_t k0,
                                                                int nb, const double *rdiag, double *Uinv,
                                                                const int *flag) {
  extern __shared__ double smem[];
  if (flag && *flag) return;
  SmemBlock S{smem, nb + 1};
  double *ri = smem + (size_t)(nb + 1) * nb;
  const int64_t b0 = k0 + (int64_t)blockIdx.y * nb;
  const int kb = (int)((n - b0 < nb) ? n - b0 : nb);
  double *X = Uinv + (size_t)blockIdx.y * nb * nb;
  for (int idx = threadIdx.x; idx < kb * kb; idx += blockDim.x) {
    const int i = idx % kb, j = idx / kb;
    if (i <= j) S(i, j) = U[GS_IDX(b0 + i, b0 + j, ldu)];
  }
  for (int k = threadIdx.x; k < kb; k += blockDim.x)
    ri[k] = (rdiag && blockIdx.y == 0) ? rdiag[k] : 1.0 / U[GS_IDX(b0 + k, b0 + k, ldu)];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * INV_WARPS + (threadIdx.x >> 5);
  if (c >= nb) return;
  double *x = X + (size_t)c * nb;
  if (c >= kb) {
    for (int i = lane; i < nb; i += 32) x[i] = 0.0;
    return;
  }
  constexpr int MR = 5;  // rows per lane: nb <= 160
  double b[MR];
#pragma unroll
  for (int m = 0; m < MR; m++) b[m] = (lane + 32 * m == c) ? 1.0 : 0.0;
  for (int k = c; k >= 0; k--) {
    const int mk = k >> 5;
    double bk = 0.0;
#pragma unroll
    for (int m = 0; m < MR; m++)
      if (m == mk) bk = b[m];
    const double xk = __shfl_sync(0xffffffffu, bk, k & 31) * ri[k];
    // rows 32 m + lane with m > k / 32 all lie below row k: nothing to do
    // (k is the same in every lane, so the skip costs no divergence and the
    // narrow FP64 pipe only sees the rows that change)
#pragma unroll
    for (int m = 0; m < MR; m++) {
      if (m > mk) break;
      const int i = lane + 32 * m;
      if (i < k) b[m] = fma(-S(i, k), xk, b[m]);
      else if (i == k) b[m] = xk;
    }
  }
#pragma unroll
  for (int m = 0; m < MR; m++) {
    const int i = lane + 32 * m;
    if (i < nb) x[i] = (i <= c) ? b[m] : 0.0;
  }
}

// shared memory of k_trtri_cols: the block plus two rows
size_t diag_smem_bytes(int nb) { return (size_t)(nb + 3) * nb * sizeof(double); }

int set_smem(const void *fn, size_t bytes) {
  if (bytes > 48 * 1024) GS_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return GSYEIG_SUCCESS;
}

}  // namespace

int trtri_diag_blocks(cudaStream_t st, int64_t n, const double *U, int64_t ldu, int nb, double *Uinv) {
  size_t sm = diag_smem_bytes(nb);
  GS_TRY(set_smem((const void *)k_trtri_cols, sm));
  k_trtri_cols<<<dim3((unsigned)ceil_div(nb, INV_WARPS), (unsigned)ceil_div(n, nb)), INV_WARPS * 32, sm, st>>>(
      n, U, ldu, 0, nb, nullptr, Uinv, nullptr);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

// Two-level blocking: inner steps of nb (the diagonal-block kernels, one
// CTA each) and outer blocks of NB = outer_block(nb) (512 when nb divides
// it, else kOuter nb).  The inner steps stay inside an outer diagonal block;
// everything beyond it goes through the inverse U_JJ^-1 of the whole outer
// block, so that each outer block costs one GEMM with K = NB per pass
// instead of several narrow ones (each GEMM call slices its operands into
// digit planes, a cost proportional to the operand, not to K).
constexpr int kOuter = 4;

int64_t outer_block(int nb) { return (512 % nb == 0) ? 512 : (int64_t)kOuter * nb; }

namespace {

// U_JJ^-1 of the outer diagonal block J (order jb, starting at J0) into
// w.UinvO, from the inverses of its nb x nb blocks (already in w.Uinv).
int outer_inverse(cudaStream_t st, int64_t J0, int64_t jb, const double *U, int64_t ldu, int nb, FactorWork &w) {
  const int64_t NB = outer_block(nb);
  FactorWork wj = w;
  wj.Uinv = w.Uinv + (size_t)(J0 / nb) * nb * nb;
  return trtri_upper_blocked(st, jb, &U[GS_IDX(J0, J0, ldu)], ldu, w.UinvO + (size_t)(J0 / NB) * NB * NB, NB, nb, wj,
                             true);
}

}  // namespace

// Right-looking blocked Cholesky in two levels: inner steps of nb (the
// diagonal kernels, the panel U_k,rest = U_kk^-T B_k,rest over the whole
// rest of the row, and the update of the rows of the outer block below the
// step), and one rank-NB update of the trailing matrix per outer block.
// The panels use the nb x nb inverses only (explicit inverses of whole
// outer blocks would cost backward stability on badly scaled matrices).
int potrf_blocked(cudaStream_t st, int64_t n, double *B, int64_t ldb, int nb, FactorWork &w) {
  size_t sm = diag_smem_bytes(nb);
  GS_TRY(set_smem((const void *)k_trtri_cols, sm));
  GS_CUDA(cudaMemsetAsync(w.flag, 0, sizeof(int), st));
  w.outer_ready = false;
  const int64_t NB = outer_block(nb);
  // Look-ahead (w.side set): the diagonal-block kernels are FP64-bound on a
  // few SMs and lie on the serial chain.  Each time the next diagonal block
  // is about to be reached, it is updated first (a small GEMM), factored and
  // inverted on the side stream, while the main stream applies the rest of
  // the same update with the persistent GEMM kept off kDiagSMs SMs.
  const bool la = w.side != nullptr && w.ev_upd != nullptr && w.ev_diag != nullptr;
  constexpr int kDiagSMs = 9;  // the k_chol_* launches (up to 36 small CTAs) and k_trtri_cols (8 CTAs)
  GemmContext *gc = current_gemm();
  const int ctas0 = gc ? gc->max_ctas : 0;
  auto reserve = [&](bool on) {
    if (!gc) return;
    const int cap = std::max(1, num_sms_cached() - kDiagSMs);
    gc->max_ctas = on ? (ctas0 > 0 ? std::min(ctas0, cap) : cap) : ctas0;
  };
  // U_kk and U_kk^-1 of the diagonal block at k0 (order kb) on stream s
  auto diag = [&](cudaStream_t s, int64_t k0, int kb) -> int {
    double *Uinv_k = w.Uinv + (size_t)(k0 / nb) * nb * nb;
    KernelProfiler *prof = current_profiler();
    const size_t e0 = prof ? prof->start(s) : SIZE_MAX;
    int launches = 1;
    for (int p0 = 0; p0 < kb; p0 += PW) {
      const int pw = std::min(PW, kb - p0), rest = kb - p0 - pw;
      const int64_t q0 = k0 + p0;
      k_chol_sub<<<1, SUB_T, 0, s>>>(B, ldb, q0, pw, w.rdiag + p0, w.flag);
      launches++;
      if (rest <= 0) continue;
      const int nt = (int)ceil_div(rest, 16);
      k_chol_panel<<<(unsigned)ceil_div(rest, 8), 256, 0, s>>>(B, ldb, q0, pw, q0 + pw, rest, w.rdiag + p0, w.flag);
      k_chol_update<<<(unsigned)(nt * (nt + 1) / 2), 256, 0, s>>>(B, ldb, q0, pw, q0 + pw, rest, w.flag);
      launches += 2;
    }
    k_trtri_cols<<<dim3((unsigned)ceil_div(nb, INV_WARPS), 1), INV_WARPS * 32, sm, s>>>(n, B, ldb, k0, nb, w.rdiag,
                                                                                        Uinv_k, w.flag);
    count_launch(launches);
    GS_CHECK_LAUNCH();
    if (prof) prof->stop(s, e0, PROF_DIAG, 0.0, 0.0);
    return GSYEIG_SUCCESS;
  };
  // the diagonal block at k1 (order kb1) once the main stream has updated it
  auto diag_ahead = [&](int64_t k1, int kb1) -> int {
    GS_CUDA(cudaEventRecord(w.ev_upd, st));
    GS_CUDA(cudaStreamWaitEvent(w.side, w.ev_upd, 0));
    GS_TRY(diag(w.side, k1, kb1));
    GS_CUDA(cudaEventRecord(w.ev_diag, w.side));
    return GSYEIG_SUCCESS;
  };
  bool ahead = false;  // the current diagonal block was factored on the side stream
  int rc = GSYEIG_SUCCESS;
  for (int64_t J0 = 0; J0 < n && rc == GSYEIG_SUCCESS; J0 += NB) {
    const int64_t J1 = std::min(n, J0 + NB);
    for (int64_t k0 = J0; k0 < J1; k0 += nb) {
      const int kb = (int)std::min<int64_t>(nb, J1 - k0);
      double *Uinv_k = w.Uinv + (size_t)(k0 / nb) * nb * nb;
      // U_kk (one CTA), then U_kk^-1 (one warp per column, many SMs)
      if (ahead) {
        GS_CUDA(cudaStreamWaitEvent(st, w.ev_diag, 0));
        ahead = false;
      } else {
        GS_TRY(diag(st, k0, kb));
      }
      const int64_t rest = n - k0 - kb;
      if (rest <= 0) break;
      double *Bk = &B[GS_IDX(k0, k0 + kb, ldb)];
      // U_k,rest = U_kk^-T B_k,rest  (panel, kb x rest, staged)
      GS_TRY(dgemm(st, true, false, kb, rest, kb, 1.0, Uinv_k, nb, Bk, ldb, 0.0, w.panel, kb, TRI_ALL, 0, w.flag));
      GS_TRY(copy_block(st, kb, rest, w.panel, kb, Bk, ldb, w.flag));
      // rows of the outer block below this step: B (upper) -= U_k,.^T U_k,.
      const int64_t rin = J1 - k0 - kb;
      if (rin <= 0) continue;
      const int64_t k1 = k0 + kb;
      double *Bn = &B[GS_IDX(k1, k1, ldb)];
      if (!la) {
        GS_TRY(dgemm(st, true, false, rin, rest, kb, -1.0, w.panel, kb, w.panel, kb, 1.0, Bn, ldb, TRI_UPPER, 0,
                     w.flag));
        continue;
      }
      // the next diagonal block first, then the rest of the update beside its factorisation
      const int64_t kb1 = std::min<int64_t>(nb, rin);
      GS_TRY(dgemm(st, true, false, kb1, kb1, kb, -1.0, w.panel, kb, w.panel, kb, 1.0, Bn, ldb, TRI_UPPER, 0, w.flag));
      GS_TRY(diag_ahead(k1, (int)kb1));
      ahead = true;
      reserve(true);
      if (rest > kb1)
        rc = dgemm(st, true, false, kb1, rest - kb1, kb, -1.0, w.panel, kb, w.panel + (size_t)kb1 * kb, kb, 1.0,
                   &B[GS_IDX(k1, k1 + kb1, ldb)], ldb, TRI_ALL, 0, w.flag);
      if (rc == GSYEIG_SUCCESS && rin > kb1)
        rc = dgemm(st, true, false, rin - kb1, rest - kb1, kb, -1.0, w.panel + (size_t)kb1 * kb, kb,
                   w.panel + (size_t)kb1 * kb, kb, 1.0, &B[GS_IDX(k1 + kb1, k1 + kb1, ldb)], ldb, TRI_UPPER, 0,
                   w.flag);
      reserve(false);
      if (rc != GSYEIG_SUCCESS) break;
    }
    if (rc != GSYEIG_SUCCESS) break;
    // trailing matrix beyond the outer block (upper) -= U_J,rest^T U_J,rest
    const int64_t r2 = n - J1;
    if (r2 <= 0) break;
    const double *UJ = &B[GS_IDX(J0, J1, ldb)];
    if (!la) {
      GS_TRY(dgemm(st, true, false, r2, r2, J1 - J0, -1.0, UJ, ldb, UJ, ldb, 1.0, &B[GS_IDX(J1, J1, ldb)], ldb,
                   TRI_UPPER, 0, w.flag));
      continue;
    }
    // the first diagonal block of the next outer block first, as above
    const int64_t kbn = std::min<int64_t>(nb, r2);
    GS_TRY(dgemm(st, true, false, kbn, kbn, J1 - J0, -1.0, UJ, ldb, UJ, ldb, 1.0, &B[GS_IDX(J1, J1, ldb)], ldb,
                 TRI_UPPER, 0, w.flag));
    GS_TRY(diag_ahead(J1, (int)kbn));
    ahead = true;
    reserve(true);
    if (r2 > kbn) {
      const double *UJn = &B[GS_IDX(J0, J1 + kbn, ldb)];
      rc = dgemm(st, true, false, kbn, r2 - kbn, J1 - J0, -1.0, UJ, ldb, UJn, ldb, 1.0, &B[GS_IDX(J1, J1 + kbn, ldb)],
                 ldb, TRI_ALL, 0, w.flag);
      if (rc == GSYEIG_SUCCESS)
        rc = dgemm(st, true, false, r2 - kbn, r2 - kbn, J1 - J0, -1.0, UJn, ldb, UJn, ldb, 1.0,
                   &B[GS_IDX(J1 + kbn, J1 + kbn, ldb)], ldb, TRI_UPPER, 0, w.flag);
    }
    reserve(false);
  }
  // every diagonal block factored on the side stream is ordered before the caller's next step
  if (ahead) GS_CUDA(cudaStreamWaitEvent(st, w.ev_diag, 0));
  return rc;
}

// The outer-block inverses U_JJ^-1 of every outer block (have_uinv: the
// nb x nb inverses are in w.Uinv already).
int outer_inverses(cudaStream_t st, int64_t n, const double *U, int64_t ldu, int nb, FactorWork &w, bool have_uinv) {
  if (!have_uinv) GS_TRY(trtri_diag_blocks(st, n, U, ldu, nb, w.Uinv));
  const int64_t NB = outer_block(nb);
  for (int64_t J0 = 0; J0 < n; J0 += NB) GS_TRY(outer_inverse(st, J0, std::min(n, J0 + NB) - J0, U, ldu, nb, w));
  w.outer_ready = true;
  return GSYEIG_SUCCESS;
}

namespace {

// Direct sygst of one diagonal sub-block (its first row/column is a
// multiple of NB, UiO its first outer inverse): C = U^-T A U^-1 from A's
// lower triangle, stored full.  Step 1: W = U^-T A, block row by block row:
// W_J = U_JJ^-T A_J, then the rows below, A_rest -= U_J,rest^T W_J.  Step 2:
// the lower triangle of C = W U^-1, block column by block column:
// C_{J0:, J} = W_{J0:, J} U_JJ^-1 (rows above the block's diagonal are not
// needed), then C_rest,rest (lower) -= C_rest,J U_J,rest.  4n^3/3 flops.
int sygst_leaf(cudaStream_t st, int64_t n, double *A, int64_t lda, const double *U, int64_t ldu,
               const double *UiO, int64_t NB, FactorWork &w) {
  GS_TRY(symmetrize(st, n, A, lda, true));
  for (int64_t J0 = 0; J0 < n; J0 += NB) {
    const int64_t J1 = std::min(n, J0 + NB), jb = J1 - J0;
    const double *UiJ = UiO + (size_t)(J0 / NB) * NB * NB;
    double *AJ = &A[GS_IDX(J0, 0, lda)];
    GS_TRY(dgemm(st, true, false, jb, n, jb, 1.0, UiJ, NB, AJ, lda, 0.0, w.panelO, jb));
    GS_TRY(copy_block(st, jb, n, w.panelO, jb, AJ, lda));
    const int64_t r2 = n - J1;
    if (r2 > 0)
      GS_TRY(dgemm(st, true, false, r2, n, jb, -1.0, &U[GS_IDX(J0, J1, ldu)], ldu, AJ, lda, 1.0,
                   &A[GS_IDX(J1, 0, lda)], lda));
  }
  for (int64_t J0 = 0; J0 < n; J0 += NB) {
    const int64_t J1 = std::min(n, J0 + NB), jb = J1 - J0, rows = n - J0;
    const double *UiJ = UiO + (size_t)(J0 / NB) * NB * NB;
    double *CJ = &A[GS_IDX(J0, J0, lda)];
    GS_TRY(dgemm(st, false, false, rows, jb, jb, 1.0, CJ, lda, UiJ, NB, 0.0, w.panelO, rows));
    GS_TRY(copy_block(st, rows, jb, w.panelO, rows, CJ, lda));
    const int64_t r2 = n - J1;
    if (r2 > 0)
      GS_TRY(dgemm(st, false, false, r2, r2, jb, -1.0, &A[GS_IDX(J1, J0, lda)], lda, &U[GS_IDX(J0, J1, ldu)], ldu,
                   1.0, &A[GS_IDX(J1, J1, lda)], lda, TRI_LOWER, 0));
  }
  return symmetrize(st, n, A, lda, true);
}

// X <- X U^-1 for the k x k upper-triangular diagonal sub-block U whose
// outer inverses start at UiO (X m x k): forward over the outer column
// blocks, X_J = X_J U_JJ^-1, then X_rest -= X_J U_J,rest.
int trsm_right_upper(cudaStream_t st, int64_t m, int64_t k, double *X, int64_t ldx, const double *U, int64_t ldu,
                     const double *UiO, int64_t NB, FactorWork &w) {
  for (int64_t J0 = 0; J0 < k; J0 += NB) {
    const int64_t J1 = std::min(k, J0 + NB), jb = J1 - J0;
    const double *UiJ = UiO + (size_t)(J0 / NB) * NB * NB;
    double *XJ = X + J0 * ldx;
    GS_TRY(dgemm(st, false, false, m, jb, jb, 1.0, XJ, ldx, UiJ, NB, 0.0, w.panelO, m));
    GS_TRY(copy_block(st, m, jb, w.panelO, m, XJ, ldx));
    if (J1 < k)
      GS_TRY(dgemm(st, false, false, m, k - J1, jb, -1.0, XJ, ldx, &U[GS_IDX(J0, J1, ldu)], ldu, 1.0, X + J1 * ldx,
                   ldx));
  }
  return GSYEIG_SUCCESS;
}

// X <- U^-T X for the same kind of sub-block (X k x m): forward over the
// outer row blocks, X_J = U_JJ^-T X_J, then X_rest -= U_J,rest^T X_J.
int trsm_left_upper_t(cudaStream_t st, int64_t k, int64_t m, double *X, int64_t ldx, const double *U, int64_t ldu,
                      const double *UiO, int64_t NB, FactorWork &w) {
  for (int64_t J0 = 0; J0 < k; J0 += NB) {
    const int64_t J1 = std::min(k, J0 + NB), jb = J1 - J0;
    const double *UiJ = UiO + (size_t)(J0 / NB) * NB * NB;
    double *XJ = X + J0;
    GS_TRY(dgemm(st, true, false, jb, m, jb, 1.0, UiJ, NB, XJ, ldx, 0.0, w.panelO, jb));
    GS_TRY(copy_block(st, jb, m, w.panelO, jb, XJ, ldx));
    if (J1 < k)
      GS_TRY(dgemm(st, true, false, k - J1, m, jb, -1.0, &U[GS_IDX(J0, J1, ldu)], ldu, XJ, ldx, 1.0, X + J1, ldx));
  }
  return GSYEIG_SUCCESS;
}

// split point of an n-row block for the recursion: the first half of its
// outer blocks (rounded up)
int64_t sygst_split(int64_t n, int64_t NB) { return ((ceil_div(n, NB) + 1) / 2) * NB; }
bool sygst_recurses(int64_t n, int64_t NB) { return n > 4 * NB; }

// C = U^-T A U^-1 of a diagonal sub-block by the 2 x 2 recursion: with
// U = [U11 U12; 0 U22] and A's lower triangle [A11; A21 A22],
//   C11 = sygst(A11, U11)
//   Y = A21 U11^-1,  P = U12^T C11,  Z = Y - P/2
//   A22 <- A22 - Z U12 - U12^T Z^T        (lower triangle)
//   C22 = sygst(A22, U22)
//   C21 = U22^-T (Z - P/2)
// (expanding C = V^T A V with V = U^-1 blockwise gives C21 = U22^-T (Y - P) and
// C22 = U22^-T (A22 - Y U12 - U12^T Y^T + U12^T C11 U12) U22^-1, which the
// half-steps through Z reproduce).  Only A's lower triangle is read; the
// result is stored full.  P lives in w.tmp (the calls below a node reuse it
// once its P is consumed).
int sygst_rec(cudaStream_t st, int64_t n, double *A, int64_t lda, const double *U, int64_t ldu, const double *UiO,
              int64_t NB, FactorWork &w) {
  if (!sygst_recurses(n, NB)) return sygst_leaf(st, n, A, lda, U, ldu, UiO, NB, w);
  const int64_t n1 = sygst_split(n, NB), n2 = n - n1;
  double *A21 = A + n1, *A22 = A + n1 + n1 * lda;
  const double *U12 = U + n1 * ldu, *U22 = U + n1 + n1 * ldu;
  const double *UiO2 = UiO + (size_t)(n1 / NB) * NB * NB;
  double *P = w.tmp;
  GS_TRY(sygst_rec(st, n1, A, lda, U, ldu, UiO, NB, w));
  GS_TRY(trsm_right_upper(st, n2, n1, A21, lda, U, ldu, UiO, NB, w));
  GS_TRY(dgemm(st, true, false, n2, n1, n1, 1.0, U12, ldu, A, lda, 0.0, P, n2));
  GS_TRY(axpy_block(st, n2, n1, -0.5, P, n2, A21, lda));
  GS_TRY(dgemm(st, false, false, n2, n2, n1, -1.0, A21, lda, U12, ldu, 1.0, A22, lda, TRI_LOWER, 0));
  GS_TRY(dgemm(st, true, true, n2, n2, n1, -1.0, U12, ldu, A21, lda, 1.0, A22, lda, TRI_LOWER, 0));
  GS_TRY(axpy_block(st, n2, n1, -0.5, P, n2, A21, lda));
  GS_TRY(sygst_rec(st, n2, A22, lda, U22, ldu, UiO2, NB, w));
  GS_TRY(trsm_left_upper_t(st, n2, n1, A21, lda, U22, ldu, UiO2, NB, w));
  return symmetrize(st, n, A, lda, true);
}

}  // namespace

size_t sygst_tmp_elems(int64_t n, int nb) {
  const int64_t NB = outer_block(nb);
  if (!sygst_recurses(n, NB)) return 0;
  const int64_t n1 = sygst_split(n, NB);
  return (size_t)n1 * (size_t)(n - n1);  // the largest P is the top split's
}

// sygst: C = U^-T A U^-1 from A's lower triangle, stored full; n^3 flops by
// the recursion when w.tmp holds sygst_tmp_elems(n, nb) doubles, else the
// direct 4n^3/3 form on the whole matrix.
int sygst_blocked(cudaStream_t st, int64_t n, double *A, int64_t lda, const double *U, int64_t ldu, int nb,
                  FactorWork &w, bool have_uinv) {
  if (!have_uinv || !w.outer_ready) GS_TRY(outer_inverses(st, n, U, ldu, nb, w, have_uinv));
  const int64_t NB = outer_block(nb);
  const size_t need = sygst_tmp_elems(n, nb);
  if (need > 0 && w.tmp && w.tmp_elems >= need) return sygst_rec(st, n, A, lda, U, ldu, w.UinvO, NB, w);
  return sygst_leaf(st, n, A, lda, U, ldu, w.UinvO, NB, w);
}

// X = U^-1 (upper triangular, zeros below the diagonal) by the backward
// block substitution U X = I restricted to the columns that can be nonzero:
// block row k of X has nonzeros only in columns >= k0, so its update of the
// rows above touches columns k0..n-1 only (n^3/3 flops in all).
int trtri_upper_blocked(cudaStream_t st, int64_t n, const double *U, int64_t ldu, double *X, int64_t ldx, int nb,
                        FactorWork &w, bool have_uinv) {
  if (!have_uinv) GS_TRY(trtri_diag_blocks(st, n, U, ldu, nb, w.Uinv));
  GS_TRY(set_identity(st, n, X, ldx));
  const int64_t last = ((n - 1) / nb) * nb;
  for (int64_t k0 = last; k0 >= 0; k0 -= nb) {
    const int kb = (int)std::min<int64_t>(nb, n - k0);
    const int64_t nc = n - k0;  // columns k0..n-1
    const double *Uinv_k = w.Uinv + (size_t)(k0 / nb) * nb * nb;
    double *Xk = &X[GS_IDX(k0, k0, ldx)];
    GS_TRY(dgemm(st, false, false, kb, nc, kb, 1.0, Uinv_k, nb, Xk, ldx, 0.0, w.panel, kb));
    GS_TRY(copy_block(st, kb, nc, w.panel, kb, Xk, ldx));
    if (k0 > 0)
      GS_TRY(dgemm(st, false, false, k0, nc, kb, -1.0, &U[GS_IDX(0, k0, ldu)], ldu, w.panel, kb, 1.0,
                   &X[GS_IDX(0, k0, ldx)], ldx));
  }
  return GSYEIG_SUCCESS;
}

// bt1: Y <- U^-1 Y by backward block substitution over the outer blocks,
// Y_J = U_JJ^-1 Y_J, then the rows above, Y_top -= U_top,J Y_J.
int trsm_back_blocked(cudaStream_t st, int64_t n, const double *U, int64_t ldu, double *Y, int64_t ldy, int64_t s,
                      int nb, FactorWork &w, bool have_uinv) {
  if (!have_uinv || !w.outer_ready) GS_TRY(outer_inverses(st, n, U, ldu, nb, w, have_uinv));
  const int64_t NB = outer_block(nb);
  const int64_t last = ((n - 1) / NB) * NB;
  for (int64_t J0 = last; J0 >= 0; J0 -= NB) {
    const int64_t jb = std::min(NB, n - J0);
    const double *UiJ = w.UinvO + (size_t)(J0 / NB) * NB * NB;
    double *YJ = &Y[GS_IDX(J0, 0, ldy)];
    GS_TRY(dgemm(st, false, false, jb, s, jb, 1.0, UiJ, NB, YJ, ldy, 0.0, w.panelO, jb));
    GS_TRY(copy_block(st, jb, s, w.panelO, jb, YJ, ldy));
    if (J0 > 0)
      GS_TRY(dgemm(st, false, false, J0, s, jb, -1.0, &U[GS_IDX(0, J0, ldu)], ldu, w.panelO, jb, 1.0, Y, ldy));
  }
  return GSYEIG_SUCCESS;
}

}  // namespace gs
