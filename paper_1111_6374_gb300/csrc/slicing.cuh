// Error-free slicing of FP64 GEMM operands into bf16 digit planes, shared
// by the tcgen05 engine (gemm_umma.cu) and the mma.sync engine
// (gemm_sliced.cu).  See gemm_sliced.cu for the digit scheme.
//
// Scaling.  Before digits are taken, column k of op(A) is multiplied by
// 2^{s_k} and row k of op(B) by 2^{-s_k} (exact; the product is unchanged),
// with s_k = floor((b_k - a_k) / 2) from the largest exponents a_k of
// column k of op(A) and b_k of row k of op(B).  This equalises scalings
// that cancel inside each product a_ik b_kj (e.g. D^-1 and D from a
// diagonally scaled pencil), which a per-row/per-column scale alone would
// turn into lost digits.  Then every row r of op(A) gets its own exponent
// e_r (entries below 2^{e_r - 1}) and every column c of op(B) its f_c.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace gs {
namespace slicing {
namespace {  // each including translation unit gets its own kernels

constexpr int S = 7;
constexpr int EXP_NONE = -100000;
constexpr int SHIFT_MAX = 400;

// smallest e with |v| < 2^e (EXP_NONE for 0)
__device__ __forceinline__ int exp_bound(double v) {
  const uint64_t u = (uint64_t)__double_as_longlong(v);
  const int E = (int)((u >> 52) & 0x7FF);
  const uint64_t man = u & ((1ull << 52) - 1);
  if (E != 0) return E - 1022;
  if (man == 0) return EXP_NONE;
  return (64 - __clzll((long long)man)) - 1074;
}

// element (r, k) of op(X): X[k + r ld] (kcontig) or X[r + k ld]
__device__ __forceinline__ double opx(const double *X, int64_t ld, bool kcontig, int64_t r, int64_t k) {
  return kcontig ? X[k + r * ld] : X[r + k * ld];
}

// Digit layouts: plain rows (mma.sync engine: (p * Rpad + r) * Kpad + k
// bf16 elements) or UMMA core-matrix tiles (tcgen05 engine, row blocks of rb).
struct DigitLayout {
  bool umma;
  int rb;  // UMMA row block (128 for A, 32 for B)
};

__device__ __forceinline__ size_t digit_off(const DigitLayout &L, int p, int64_t r, int64_t k, int64_t Rpad,
                                            int64_t Kpad) {
  if (!L.umma) return (((size_t)p * Rpad + r) * Kpad + k) * 2;
  const int rb = L.rb;
  const int64_t nks = Kpad / 16;  // one stage = one k16 block of all S slices
  const int64_t blk = r / rb, ii = r % rb;
  const int64_t ks = k / 16;
  const int k16 = (int)(k % 16);
  const int ki = k16 / 8, kc = k16 % 8, mi = (int)(ii / 8), rr = (int)(ii % 8);
  const size_t k16bytes = (size_t)rb * 32;
  return ((size_t)(blk * nks + ks) * S + p) * k16bytes + (size_t)mi * 256 + ki * 128 + rr * 16 + kc * 2;
}

// Per-k maxima kA[k] (over the rows of op(A)) and kB[k] (over the columns of
// op(B)) in one launch: blockIdx.z selects the operand.  kA, kB start at the
// memset sentinel KNONE (below every exponent bound).
constexpr int KNONE = (int)0x80808080;

__global__ void k_inner_exp2(int64_t M, int64_t N, int64_t K, const double *__restrict__ A, int64_t lda, bool a_kc,
                             const double *__restrict__ B, int64_t ldb, bool b_kc, int *__restrict__ kA,
                             int *__restrict__ kB) {
  const bool isB = blockIdx.z != 0;
  const int64_t R = isB ? N : M;
  const int64_t r0 = (int64_t)blockIdx.x * 32, k0 = (int64_t)blockIdx.y * 32;
  if (r0 >= R) return;
  const double *X = isB ? B : A;
  const int64_t ld = isB ? ldb : lda;
  const bool kcontig = isB ? b_kc : a_kc;
  int *ek = isB ? kB : kA;
  __shared__ int sm[32][33];
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int j = ty; j < 32; j += 8) {
    int64_t r = kcontig ? r0 + j : r0 + tx, k = kcontig ? k0 + tx : k0 + j;
    int e = EXP_NONE;
    if (r < R && k < K) e = exp_bound(opx(X, ld, kcontig, r, k));
    if (kcontig) sm[j][tx] = e; else sm[tx][j] = e;  // sm[row][k]
  }
  __syncthreads();
  if (ty == 0 && k0 + tx < K) {
    int best = EXP_NONE;
    for (int j = 0; j < 32; j++) best = max(best, sm[j][tx]);
    if (best != EXP_NONE) atomicMax(&ek[k0 + tx], best);
  }
}

// the equalising shift s_k of column k (0 when either side is all zeros)
__device__ __forceinline__ int kshift_of(const int *kA, const int *kB, int64_t k) {
  const int a = kA[k], b = kB[k];
  if (a == KNONE || b == KNONE) return 0;
  const int d = b - a;
  const int sft = (d >= 0) ? d / 2 : -((-d + 1) / 2);
  return max(-SHIFT_MAX, min(SHIFT_MAX, sft));
}

// Raw row maxima rX[r] = max over k of (exp_bound(v_rk) + sgn s_k), by
// atomicMax over K chunks of 128: grid (rows / 32, K / 128, operand).
// kA == nullptr: no equalising shift (a symmetric rank-K update).
__global__ void k_rowmax2(int64_t M, int64_t N, int64_t K, const double *__restrict__ A, int64_t lda, bool a_kc,
                          const double *__restrict__ B, int64_t ldb, bool b_kc, const int *__restrict__ kA,
                          const int *__restrict__ kB, int *__restrict__ rA, int *__restrict__ rB) {
  const bool isB = blockIdx.z != 0;
  const int64_t R = isB ? N : M;
  const int64_t r0 = (int64_t)blockIdx.x * 32, kc0 = (int64_t)blockIdx.y * 128;
  if (r0 >= R) return;
  const double *X = isB ? B : A;
  const int64_t ld = isB ? ldb : lda;
  const bool kcontig = isB ? b_kc : a_kc;
  const int sgn = isB ? -1 : 1;
  int *rx = isB ? rB : rA;
  __shared__ int red[8][33];
  const int tx = threadIdx.x, ty = threadIdx.y;
  if (kcontig) {
    // a warp per row (rows r0 + ty + 8 i), lanes along k: coalesced
    for (int i = 0; i < 4; i++) {
      const int64_t r = r0 + ty + 8 * i;
      int best = EXP_NONE;
      if (r < R)
        for (int64_t k = kc0 + tx; k < kc0 + 128 && k < K; k += 32) {
          int e = exp_bound(X[k + r * ld]);
          if (e != EXP_NONE && kA) e += sgn * kshift_of(kA, kB, k);
          best = max(best, e);
        }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
      if (tx == 0 && r < R && best != EXP_NONE) atomicMax(&rx[r], best);
    }
  } else {
    // lanes along rows (coalesced), the 8 warps split the k chunk
    const int64_t r = r0 + tx;
    int best = EXP_NONE;
    if (r < R)
      for (int64_t k = kc0 + ty; k < kc0 + 128 && k < K; k += 8) {
        int e = exp_bound(X[r + k * ld]);
        if (e != EXP_NONE && kA) e += sgn * kshift_of(kA, kB, k);
        best = max(best, e);
      }
    red[ty][tx] = best;
    __syncthreads();
    if (ty == 0) {
      for (int j = 1; j < 8; j++) best = max(best, red[j][tx]);
      if (r < R && best != EXP_NONE) atomicMax(&rx[r], best);
    }
  }
}

// Digits of a 32 x 32 tile of one operand (grid (rows / 32, Kpad / 32,
// operand)): entry v of row r becomes X = round(|v| 2^{56 - e_r + sgn s_k})
// with e_r = 1 + rX[r], written as balanced base-256 digits (d_0 in
// [0, 128], the others in [-128, 127]) times sign(v); rows R..Rpad-1 and
// columns K..Kpad-1 are zeros.  The CTAs of the first K tile also store
// the final row exponents e_r (EXP_NONE for a zero row).
__global__ void k_split2(int64_t M, int64_t N, int64_t K, int64_t Mpad, int64_t Npad, int64_t Kpad,
                         const double *__restrict__ A, int64_t lda, bool a_kc, const double *__restrict__ B,
                         int64_t ldb, bool b_kc, const int *__restrict__ kA, const int *__restrict__ kB,
                         const int *__restrict__ rA, const int *__restrict__ rB, int *__restrict__ ea,
                         int *__restrict__ eb, DigitLayout LA, DigitLayout LB, unsigned char *__restrict__ SA,
                         unsigned char *__restrict__ SB) {
  const bool isB = blockIdx.z != 0;
  const int64_t R = isB ? N : M, Rpad = isB ? Npad : Mpad;
  const int64_t r0 = (int64_t)blockIdx.x * 32, k0 = (int64_t)blockIdx.y * 32;
  if (r0 >= Rpad) return;
  const double *X = isB ? B : A;
  const int64_t ld = isB ? ldb : lda;
  const bool kcontig = isB ? b_kc : a_kc;
  const int sgn = isB ? -1 : 1;
  const int *rx = isB ? rB : rA;
  int *ex = isB ? eb : ea;
  const DigitLayout L = isB ? LB : LA;
  unsigned char *dst = isB ? SB : SA;
  __shared__ double tile[32][33];
  __shared__ int rowe[32];
  const int tx = threadIdx.x, ty = threadIdx.y;
  if (ty == 0) {
    const int64_t r = r0 + tx;
    const int raw = (r < R) ? rx[r] : KNONE;
    const int e = (raw == KNONE) ? EXP_NONE : raw + 1;
    rowe[tx] = e;
    if (blockIdx.y == 0 && r < R) ex[r] = e;
  }
  for (int j = ty; j < 32; j += 8) {
    int64_t r = kcontig ? r0 + j : r0 + tx, k = kcontig ? k0 + tx : k0 + j;
    double v = 0.0;
    if (r < R && k < K) v = opx(X, ld, kcontig, r, k);
    if (kcontig) tile[j][tx] = v; else tile[tx][j] = v;
  }
  __syncthreads();
  // digits: thread u < 128 takes row j = u / 4 and the 8 consecutive k of
  // group u % 4, so that the 8 digits of one slice (contiguous in both
  // layouts, 16-byte aligned since Kpad is a multiple of 32) leave as one
  // 16-byte store; all tests on the values are integer ones
  const int u = ty * 32 + tx;
  if (u >= 128) return;
  const int j = u >> 2, q = u & 3;
  const int64_t r = r0 + j, kb = k0 + 8 * q;
  if (r >= Rpad || kb >= Kpad) return;
  const int e = rowe[j];
  uint32_t packed[S][4];
#pragma unroll
  for (int p = 0; p < S; p++)
#pragma unroll
    for (int w = 0; w < 4; w++) packed[p][w] = 0u;
#pragma unroll
  for (int kk = 0; kk < 8; kk++) {
    const int64_t k = kb + kk;
    const uint64_t ub = (uint64_t)__double_as_longlong(tile[j][8 * q + kk]);
    uint64_t Xm = 0;
    const bool neg = (ub >> 63) != 0;
    if ((ub << 1) != 0 && e != EXP_NONE) {  // v != 0
      const int E = (int)((ub >> 52) & 0x7FF);
      uint64_t m = ub & ((1ull << 52) - 1);
      int Eeff = E;
      if (E != 0) m |= (1ull << 52); else Eeff = 1;
      const int ks = (kA && k < K) ? sgn * kshift_of(kA, kB, k) : 0;
      const int sh = Eeff - 1019 - e + ks;  // |v 2^ks| 2^{56 - e} = m 2^sh <= 2^55
      if (sh >= 0) Xm = m << sh;
      else if (sh > -60) Xm = (m + (1ull << (-sh - 1))) >> (-sh);
    }
    int dg[S];
    uint64_t t = Xm;
#pragma unroll
    for (int p = S - 1; p > 0; p--) {
      int rr = (int)(t & 255u);
      t >>= 8;
      if (rr >= 128) {
        rr -= 256;
        t += 1;
      }
      dg[p] = rr;
    }
    dg[0] = (int)t;
#pragma unroll
    for (int p = 0; p < S; p++) {
      const int d = neg ? -dg[p] : dg[p];
      const uint32_t bits = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn((float)d));
      packed[p][kk >> 1] |= bits << (16 * (kk & 1));
    }
  }
#pragma unroll
  for (int p = 0; p < S; p++)
    *reinterpret_cast<uint4 *>(dst + digit_off(L, p, r, kb, Rpad, Kpad)) =
        make_uint4(packed[p][0], packed[p][1], packed[p][2], packed[p][3]);
}

// Host side: digits and exponents of op(A) (M x K) and op(B) (rows = its N
// columns).  Workspace (ints, slice_ints): the final row exponents ea[Mpad],
// eb[Npad], then the raw row maxima rA[Mpad], rB[Npad] and the per-k
// maxima kA[Kpad], kB[Kpad] (one memset clears those four).  When the two
// operands are the same set of vectors (op(A) = op(B)^T, a symmetric
// rank-K update), the inner equalisation is skipped (s_k = 0).
struct SlicePlan {
  int64_t Mpad, Npad, Kpad;
  unsigned char *SA, *SB;
  int *ea, *eb, *rA, *rB, *kA, *kB;
};

inline size_t slice_ints(int64_t Mpad, int64_t Npad, int64_t Kpad) { return (size_t)(2 * (Mpad + Npad) + 2 * Kpad); }

// the ints of the plan laid out from `base`
inline void slice_layout(SlicePlan &P, int *base) {
  P.ea = base;
  P.eb = P.ea + P.Mpad;
  P.rA = P.eb + P.Npad;
  P.rB = P.rA + P.Mpad;
  P.kA = P.rB + P.Npad;
  P.kB = P.kA + P.Kpad;
}

inline int slice_operands(cudaStream_t st, bool transA, bool transB, int64_t M, int64_t N, int64_t K,
                          const double *A, int64_t lda, const double *B, int64_t ldb, const SlicePlan &P,
                          DigitLayout LA, DigitLayout LB) {
  const bool a_kc = transA, b_kc = !transB;
  const bool same = (A == B) && (lda == ldb) && (transA != transB) && (M == N);
  dim3 tb(32, 8);
  KernelProfiler *prof = current_profiler();
  const size_t e0 = prof ? prof->start(st) : SIZE_MAX;
  // per-k maxima (unless same), per-row maxima, digits: three launches
  GS_CUDA(cudaMemsetAsync(P.rA, 0x80, (size_t)(P.Mpad + P.Npad + 2 * P.Kpad) * sizeof(int), st));
  const int64_t Rmax = std::max(M, N);
  if (!same)
    k_inner_exp2<<<dim3((unsigned)ceil_div(Rmax, 32), (unsigned)ceil_div(K, 32), 2), tb, 0, st>>>(
        M, N, K, A, lda, a_kc, B, ldb, b_kc, P.kA, P.kB);
  const int *kA = same ? nullptr : P.kA, *kB = same ? nullptr : P.kB;
  k_rowmax2<<<dim3((unsigned)ceil_div(Rmax, 32), (unsigned)ceil_div(K, 128), 2), tb, 0, st>>>(
      M, N, K, A, lda, a_kc, B, ldb, b_kc, kA, kB, P.rA, P.rB);
  k_split2<<<dim3((unsigned)(std::max(P.Mpad, P.Npad) / 32), (unsigned)(P.Kpad / 32), 2), tb, 0, st>>>(
      M, N, K, P.Mpad, P.Npad, P.Kpad, A, lda, a_kc, B, ldb, b_kc, kA, kB, P.rA, P.rB, P.ea, P.eb, LA, LB, P.SA,
      P.SB);
  count_launch(same ? 2 : 3);
  GS_CHECK_LAUNCH();
  if (prof) prof->stop(st, e0, PROF_SLICE, 0.0, 0.0);
  return GSYEIG_SUCCESS;
}

}  // namespace
}  // namespace slicing
}  // namespace gs
