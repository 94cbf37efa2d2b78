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
  int rb;  // UMMA row block (128 for A, 64 for B)
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

__global__ void k_fill(int n, int *p, int v) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = v;
}

// per-k maximum exponent of op(X) (R x K) over its rows, by atomicMax
__global__ void k_inner_exp(int64_t R, int64_t K, const double *__restrict__ X, int64_t ld, bool kcontig,
                            int *__restrict__ ek) {
  const int64_t r0 = (int64_t)blockIdx.x * 32, k0 = (int64_t)blockIdx.y * 32;
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

__global__ void k_kshift(int64_t K, const int *__restrict__ ea, const int *__restrict__ eb, int *__restrict__ sh) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < K; k += (int64_t)gridDim.x * blockDim.x) {
    int s = 0;
    if (ea[k] != EXP_NONE && eb[k] != EXP_NONE) {
      const int d = eb[k] - ea[k];
      s = (d >= 0) ? d / 2 : -((-d + 1) / 2);
      s = max(-SHIFT_MAX, min(SHIFT_MAX, s));
    }
    sh[k] = s;
  }
}

// row exponents of op(X) * 2^{sgn s_k}: e_r = 1 + max_k (exp_bound + sgn s_k)
__global__ void k_row_exp(int64_t R, int64_t K, const double *__restrict__ X, int64_t ld, bool kcontig,
                          const int *__restrict__ kshift, int sgn, int *__restrict__ ex) {
  const int64_t r0 = (int64_t)blockIdx.x * 32;
  __shared__ int sm[32][33];
  int best = EXP_NONE;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int64_t k0 = 0; k0 < K; k0 += 32) {
    for (int j = ty; j < 32; j += 8) {
      int64_t r = kcontig ? r0 + j : r0 + tx, k = kcontig ? k0 + tx : k0 + j;
      int e = EXP_NONE;
      if (r < R && k < K) {
        e = exp_bound(opx(X, ld, kcontig, r, k));
        if (e != EXP_NONE && kshift) e += sgn * kshift[k];
      }
      if (kcontig) sm[j][tx] = e; else sm[tx][j] = e;
    }
    __syncthreads();
    if (ty == 0)
      for (int j = 0; j < 32; j++) best = max(best, sm[tx][j]);
    __syncthreads();
  }
  if (ty == 0 && r0 + tx < R) ex[r0 + tx] = (best == EXP_NONE) ? EXP_NONE : best + 1;
}

// Digits of row r of op(X) * 2^{sgn s_k}, scaled by 2^{-e_r}: X = round(|v| 2^{56 - e_r + sgn s_k})
// written as balanced base-256 digits (d_0 in [0, 128], others in [-128, 127]) times sign(v).
__global__ void k_split(int64_t R, int64_t K, int64_t Rpad, int64_t Kpad, const double *__restrict__ X, int64_t ld,
                        bool kcontig, const int *__restrict__ kshift, int sgn, const int *__restrict__ ex,
                        DigitLayout L, unsigned char *__restrict__ dst) {
  __shared__ double tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32, k0 = (int64_t)blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int j = ty; j < 32; j += 8) {
    int64_t r = kcontig ? r0 + j : r0 + tx, k = kcontig ? k0 + tx : k0 + j;
    double v = 0.0;
    if (r < R && k < K) v = opx(X, ld, kcontig, r, k);
    if (kcontig) tile[j][tx] = v; else tile[tx][j] = v;
  }
  __syncthreads();
  for (int j = ty; j < 32; j += 8) {
    const int64_t r = r0 + j, k = k0 + tx;
    if (r >= Rpad || k >= Kpad) continue;
    const double v = tile[j][tx];
    const int e = (r < R) ? ex[r] : EXP_NONE;
    uint64_t Xm = 0;
    bool neg = false;
    if (v != 0.0 && e != EXP_NONE) {
      const uint64_t u = (uint64_t)__double_as_longlong(v);
      neg = (u >> 63) != 0;
      const int E = (int)((u >> 52) & 0x7FF);
      uint64_t m = u & ((1ull << 52) - 1);
      int Eeff = E;
      if (E != 0) m |= (1ull << 52); else Eeff = 1;
      const int ks = (kshift && k < K) ? sgn * kshift[k] : 0;
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
      *reinterpret_cast<__nv_bfloat16 *>(dst + digit_off(L, p, r, k, Rpad, Kpad)) = __float2bfloat16_rn((float)d);
    }
  }
}

// Host side: digits and exponents of op(A) (M x K) and op(B) (rows = its N
// columns).  Workspace (ints) holds ea[Mpad], eb[Npad], then 3 K-arrays.
// When the two operands are the same set of vectors (op(A) = op(B)^T, a
// symmetric rank-K update), the inner equalisation is skipped (s_k = 0).
struct SlicePlan {
  int64_t Mpad, Npad, Kpad;
  unsigned char *SA, *SB;
  int *ea, *eb, *kA, *kB, *ksh;
};

inline size_t slice_ints(int64_t Mpad, int64_t Npad, int64_t Kpad) { return (size_t)(Mpad + Npad + 3 * Kpad); }

inline int slice_operands(cudaStream_t st, bool transA, bool transB, int64_t M, int64_t N, int64_t K,
                          const double *A, int64_t lda, const double *B, int64_t ldb, const SlicePlan &P,
                          DigitLayout LA, DigitLayout LB) {
  const bool a_kc = transA, b_kc = !transB;
  const bool same = (A == B) && (lda == ldb) && (transA != transB) && (M == N);
  dim3 tb(32, 8);
  int nl = 0;
  const int *ksh = nullptr;
  if (!same) {
    k_fill<<<(unsigned)ceil_div(2 * P.Kpad, 256), 256, 0, st>>>((int)(2 * P.Kpad), P.kA, EXP_NONE);
    k_inner_exp<<<dim3((unsigned)ceil_div(M, 32), (unsigned)ceil_div(K, 32)), tb, 0, st>>>(M, K, A, lda, a_kc, P.kA);
    k_inner_exp<<<dim3((unsigned)ceil_div(N, 32), (unsigned)ceil_div(K, 32)), tb, 0, st>>>(N, K, B, ldb, b_kc, P.kB);
    k_kshift<<<(unsigned)ceil_div(K, 256), 256, 0, st>>>(K, P.kA, P.kB, P.ksh);
    ksh = P.ksh;
    nl += 4;
  }
  k_row_exp<<<(unsigned)ceil_div(M, 32), tb, 0, st>>>(M, K, A, lda, a_kc, ksh, +1, P.ea);
  k_split<<<dim3((unsigned)(P.Mpad / 32), (unsigned)(P.Kpad / 32)), tb, 0, st>>>(M, K, P.Mpad, P.Kpad, A, lda, a_kc, ksh,
                                                                                  +1, P.ea, LA, P.SA);
  k_row_exp<<<(unsigned)ceil_div(N, 32), tb, 0, st>>>(N, K, B, ldb, b_kc, ksh, -1, P.eb);
  k_split<<<dim3((unsigned)(P.Npad / 32), (unsigned)(P.Kpad / 32)), tb, 0, st>>>(N, K, P.Npad, P.Kpad, B, ldb, b_kc, ksh,
                                                                                  -1, P.eb, LB, P.SB);
  count_launch(nl + 4);
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

}  // namespace
}  // namespace slicing
}  // namespace gs
