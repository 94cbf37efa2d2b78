// FP64-accurate GEMM on the bf16 tensor cores by error-free slicing.
//
// GB300 retires ~2 FP64 FMAs per SM-clock but ~1,600 bf16 MACs: so every
// O(n^3) flop of gs1/gs2/bt1 (Eqs. 2-4) is cheaper on the tensor pipe if it
// can be made exact.  Each row r of op(A) is scaled by a power of two 2^-e_r
// so that its entries are below 1/2, rounded to 56 fractional bits, and the
// resulting integer X (< 2^55) is written in S = 7 balanced base-256 digits
// d_0..d_6 with d_0 in [0, 128] and the others in [-128, 127]; slice p
// holds digit p of every entry (times the entry's sign), an integer that
// bf16 represents exactly.  Columns of op(B) likewise.  Then
//
//   op(A) op(B) = 2^{e_r + f_c} sum_{p,q} 2^{-8(p+q+2)} A_p B_q
//
// and every product A_p B_q is an integer matrix.  Pairs are summed per
// level d = p + q <= 6 (28 pairs); the dropped levels weigh about 2^-58 of
// the row/column maxima and, like the rounding of the inputs, carry random
// signs, so the result is as accurate as an FP64 dot product (checked
// against the oracle).  A level holds at most 7 pairs and each digit
// product is at most 2^14, so with K <= 128 a level sum stays below 2^24
// and the fp32 tensor-core accumulator is exact.  The seven exact level
// sums are recombined in int64 (levels 0-3 and 4-6 in two integers) and
// converted to FP64 once per output, where the caller's alpha/beta update
// happens.
//
// Error model: |error| <~ 2^-55 K max_k|a_rk| max_k|b_kc| (normwise), where
// a DGEMM guarantees gamma_K sum_k |a_rk||b_kc| (componentwise): rows or
// columns whose entries span many orders of magnitude lose relative
// accuracy in small products.  The solver exposes opts.fp64_gemm = 1 for
// such inputs.
//
// Kernels: k_inner_exp2 / k_rowsplit2 (exponents and digits, written K-major
// as bf16 slices padded to 64 rows x 32 k), k_sliced_gemm (mma.sync bf16 ->
// fp32 on 64 x 64 output tiles, 8 warps, 7 level accumulators per warp).
#include <cuda_bf16.h>

#include "slicing.cuh"

namespace gs {
namespace {

using slicing::S;
using slicing::EXP_NONE;
constexpr int TM = 64, TN = 64, TK = 32;  // CTA tile; K stage
constexpr int ROWB = TK * 2 + 16;          // smem bytes per tile row (64 B of data + 16 B pad)
constexpr int SLICE_TILE_BYTES = TM * ROWB;
constexpr int STAGE_BYTES = 2 * S * SLICE_TILE_BYTES;  // A and B, all slices
constexpr int NSTAGE = 2;
constexpr int GEMM_THREADS = 256;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src));
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// One K stage (TK = 32) of all slices of the A tile and the B tile into smem.
__device__ __forceinline__ void load_stage(unsigned char *st, const __nv_bfloat16 *SA, const __nv_bfloat16 *SB,
                                           int64_t Mpad, int64_t Npad, int64_t Kpad, int64_t m0, int64_t n0,
                                           int64_t k0) {
  // 2 operands x S slices x 64 rows x 4 chunks of 16 B
  for (int c = threadIdx.x; c < 2 * S * TM * 4; c += GEMM_THREADS) {
    const int op = c / (S * TM * 4), rem = c % (S * TM * 4);
    const int p = rem / (TM * 4), row = (rem / 4) % TM, ch = rem % 4;
    const __nv_bfloat16 *src = (op == 0) ? SA + ((int64_t)p * Mpad + m0 + row) * Kpad + k0 + ch * 8
                                         : SB + ((int64_t)p * Npad + n0 + row) * Kpad + k0 + ch * 8;
    const uint32_t dst = smem_u32(st + (size_t)op * S * SLICE_TILE_BYTES + (size_t)p * SLICE_TILE_BYTES +
                                  (size_t)row * ROWB + ch * 16);
    cp_async16(dst, src);
  }
  asm volatile("cp.async.commit_group;\n" ::);
}

__global__ void __launch_bounds__(GEMM_THREADS, 1)
    k_sliced_gemm(int64_t M, int64_t N, int64_t Mpad, int64_t Npad, int64_t Kpad, const __nv_bfloat16 *__restrict__ SA,
                  const __nv_bfloat16 *__restrict__ SB, const int *__restrict__ ea, const int *__restrict__ eb,
                  double alpha, double beta, double *__restrict__ C, int64_t ldc, int mode, int64_t diag,
                  const int *abort_flag) {
  if (abort_flag && *abort_flag) return;
  const int64_t m0 = (int64_t)blockIdx.x * TM, n0 = (int64_t)blockIdx.y * TN;
  if (mode == TRI_LOWER && (m0 + TM - 1) - n0 + diag < 0) return;
  if (mode == TRI_UPPER && m0 - (n0 + TN - 1) + diag > 0) return;
  extern __shared__ __align__(128) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wm = (warp & 3) * 16, wn = (warp >> 2) * 32;  // warp tile: 16 rows x 32 cols
  float acc[S][4][4];
#pragma unroll
  for (int d = 0; d < S; d++)
#pragma unroll
    for (int t = 0; t < 4; t++)
#pragma unroll
      for (int q = 0; q < 4; q++) acc[d][t][q] = 0.f;

  const int nk = (int)(Kpad / TK);
  load_stage(smem, SA, SB, Mpad, Npad, Kpad, m0, n0, 0);
  for (int ks = 0; ks < nk; ks++) {
    if (ks + 1 < nk) {
      load_stage(smem + (size_t)((ks + 1) % NSTAGE) * STAGE_BYTES, SA, SB, Mpad, Npad, Kpad, m0, n0,
                 (int64_t)(ks + 1) * TK);
      asm volatile("cp.async.wait_group 1;\n" ::);
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::);
    }
    __syncthreads();
    const unsigned char *st = smem + (size_t)(ks % NSTAGE) * STAGE_BYTES;
    const unsigned char *sA = st, *sB = st + (size_t)S * SLICE_TILE_BYTES;
#pragma unroll
    for (int kk = 0; kk < TK; kk += 16) {
      // A fragments of all slices: rows wm..wm+15, k kk..kk+15
      uint32_t a[S][4];
      {
        const int r = wm + (lane & 7) + ((lane >> 3) & 1) * 8, kc = kk + (lane >> 4) * 8;
#pragma unroll
        for (int p = 0; p < S; p++)
          ldsm_x4(smem_u32(sA + (size_t)p * SLICE_TILE_BYTES + (size_t)r * ROWB + kc * 2), a[p][0], a[p][1], a[p][2],
                  a[p][3]);
      }
#pragma unroll
      for (int q = 0; q < S; q++) {
        // B fragments of slice q for the warp's four n8 tiles
        uint32_t b[4][2];
#pragma unroll
        for (int h = 0; h < 2; h++) {
          const int nr = wn + h * 16 + (lane & 7) + (lane >> 4) * 8, kc = kk + ((lane >> 3) & 1) * 8;
          ldsm_x4(smem_u32(sB + (size_t)q * SLICE_TILE_BYTES + (size_t)nr * ROWB + kc * 2), b[2 * h][0], b[2 * h][1],
                  b[2 * h + 1][0], b[2 * h + 1][1]);
        }
#pragma unroll
        for (int p = 0; p < S - q; p++)
#pragma unroll
          for (int t = 0; t < 4; t++) mma_bf16(acc[p + q][t], a[p], b[t][0], b[t][1]);
      }
    }
    __syncthreads();
  }
  // epilogue: exact level sums -> int64 (levels 0-3, 4-7) -> FP64 update
  const int g = lane >> 2, c2 = (lane & 3) * 2;
#pragma unroll
  for (int t = 0; t < 4; t++)
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int64_t gi = m0 + wm + g + (q >> 1) * 8;
      const int64_t gj = n0 + wn + t * 8 + c2 + (q & 1);
      if (gi >= M || gj >= N) continue;
      const int64_t dd = gi - gj + diag;
      if (mode == TRI_LOWER && dd < 0) continue;
      if (mode == TRI_UPPER && dd > 0) continue;
      long long hi = 0, lo = 0;
#pragma unroll
      for (int d = 0; d < 4; d++) hi = hi * 256 + (long long)__float2int_rn(acc[d][t][q]);
#pragma unroll
      for (int d = 4; d < S; d++) lo = lo * 256 + (long long)__float2int_rn(acc[d][t][q]);
      const int er = ea[gi], ec = eb[gj];
      double v = 0.0;
      if (er != EXP_NONE && ec != EXP_NONE) {
        // value = (hi + lo 2^-24) 2^-40 2^{er + ec}; hi, lo < 2^50 convert exactly
        const double r = fma((double)lo, 0x1p-24, (double)hi);
        v = r * ldexp(alpha, er + ec - 40);
      }
      double *pc = &C[gi + gj * ldc];
      *pc = (beta != 0.0) ? fma(beta, *pc, v) : v;
    }
}

}  // namespace

size_t sliced_workspace_bytes(int64_t M, int64_t N, int64_t K) {
  const int64_t Mpad = ceil_div(M, TM) * TM, Npad = ceil_div(N, TN) * TN, Kpad = ceil_div(K, TK) * TK;
  return (size_t)S * (size_t)(Mpad + Npad) * (size_t)Kpad * 2 + slicing::slice_ints(Mpad, Npad, Kpad) * sizeof(int) +
         1024;
}

int sliced_gemm(cudaStream_t st, bool transA, bool transB, int64_t M, int64_t N, int64_t K, double alpha,
                const double *A, int64_t lda, const double *B, int64_t ldb, double beta, double *C, int64_t ldc,
                TriMode mode, int64_t diag, const int *abort_flag, void *ws, size_t ws_bytes) {
  if (M <= 0 || N <= 0) return GSYEIG_SUCCESS;
  if (K > 128 || K <= 0) return GSYEIG_NOT_SUPPORTED;
  const int64_t Mpad = ceil_div(M, TM) * TM, Npad = ceil_div(N, TN) * TN, Kpad = ceil_div(K, TK) * TK;
  if (ws_bytes < sliced_workspace_bytes(M, N, K)) return GSYEIG_NOT_SUPPORTED;
  slicing::SlicePlan P;
  P.Mpad = Mpad;
  P.Npad = Npad;
  P.Kpad = Kpad;
  P.SA = static_cast<unsigned char *>(ws);
  P.SB = P.SA + (size_t)S * Mpad * Kpad * 2;
  slicing::slice_layout(P, reinterpret_cast<int *>(P.SB + (size_t)S * Npad * Kpad * 2));
  GS_TRY(slicing::slice_operands(st, transA, transB, M, N, K, A, lda, B, ldb, P, {false, 0}, {false, 0}));
  const size_t smem = (size_t)NSTAGE * STAGE_BYTES;
  GS_TRY(set_max_smem((const void *)k_sliced_gemm, (int)smem));
  dim3 grid((unsigned)(Mpad / TM), (unsigned)(Npad / TN));
  k_sliced_gemm<<<grid, GEMM_THREADS, smem, st>>>(M, N, Mpad, Npad, Kpad, reinterpret_cast<__nv_bfloat16 *>(P.SA),
                                                  reinterpret_cast<__nv_bfloat16 *>(P.SB), P.ea, P.eb, alpha, beta, C,
                                                  ldc, (int)mode, diag, abort_flag);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

}  // namespace gs
