// tcgen05 (5th-generation tensor core) engine of the error-free sliced GEMM
// (the digit scheme is described in gemm_sliced.cu; this file only changes
// how the 28 digit-pair products are issued and how the exact level sums are
// turned into FP64).
//
//  * Operands are pre-split by k_split_umma straight into the UMMA
//    "no-swizzle K-major" core-matrix layout (8 rows x 16 bytes per core
//    matrix, K-adjacent cores 128 B apart, row-adjacent cores 256 B apart),
//    grouped so that one K stage (32 k) of all 7 slices of a 128-row A block
//    (56 KB) or a 64-row B block (28 KB) is one contiguous run: each stage is
//    brought in by a single cp.async.bulk per operand, completing on an
//    mbarrier (no tensor map needed).
//  * One thread issues tcgen05.mma.kind::f16 (bf16 x bf16 -> fp32, M = 128,
//    N = 64, K = 16); the accumulator of level d lives in TMEM columns
//    [64 d, 64 d + 64) (7 levels, 448 columns, 512 allocated).  Each K stage
//    is 2 x 28 MMAs; tcgen05.commit releases the stage buffer.
//  * Epilogue (16 warps; warp w reads TMEM lane quarter w % 4, a quarter of
//    the columns each): tcgen05.ld of the 7 level sums of a row, exact
//    recombination in 128-bit integers and a
//    correctly rounded integer-only conversion to FP64 with the row/column
//    exponents folded in; the FP64 pipe only does the final C update.
//  * Every mbarrier wait is bounded; on expiry the kernel records the fault
//    in *err, still waits (bounded) for its own copies, frees its TMEM and
//    returns.
#include <cuda_bf16.h>

#include "slicing.cuh"

namespace gs {
namespace {

using slicing::S;
using slicing::EXP_NONE;
constexpr int UM = 128, UN = 64, UKS = 32;  // tile rows, tile cols, K per stage
constexpr int A_K16_BYTES = UM * 16 * 2;     // one slice, one k16 block: 4096
constexpr int B_K16_BYTES = UN * 16 * 2;     // 2048
constexpr int A_STAGE = S * 2 * A_K16_BYTES; // 57344
constexpr int B_STAGE = S * 2 * B_K16_BYTES; // 28672
constexpr int NBUF = 2;
constexpr int UMMA_THREADS = 512;  // 16 warps: the epilogue splits each TMEM lane quarter over 4 warps
constexpr int TMEM_COLS = 512;
constexpr uint32_t SPIN_LIMIT = 1u << 24;

// ---------------------------------------------------------------- PTX -----
__device__ __forceinline__ uint32_t sptr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(sptr(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(sptr(bar)), "r"(bytes) : "memory");
}

// bounded wait for the phase with the given parity; false on expiry
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  const uint32_t a = sptr(bar);
  for (uint32_t it = 0; it < SPIN_LIMIT; it++) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (it > 64) __nanosleep(64);
  }
  return false;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   sptr(dst)),
               "l"(src), "r"(bytes), "r"(sptr(bar))
               : "memory");
}

// SM100 shared-memory matrix descriptor, no swizzle, K-major
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
  // base offset 0, lbo mode 0, layout type 0 (no swizzle)
  return d;
}

// instruction descriptor: kind::f16, bf16 A/B, fp32 D, K-major A/B, M = 128, N = 64
__host__ __device__ constexpr uint32_t instr_desc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(UN >> 3) << 17) | ((uint32_t)(UM >> 4) << 24);
}

__device__ __forceinline__ void umma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void umma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(sptr(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&v)[4]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
               : "r"(taddr));
}

// Out-of-range tail of i128_ldexp (result subnormal or infinite): kept out of
// line so that the compiler cannot if-convert its FP64 instructions into the
// common path (GB300's FP64 pipe is narrow).
__device__ __noinline__ double i128_ldexp_slow(uint64_t w, int e, bool neg) {
  const double v = ldexp((double)w, e);
  return neg ? -v : v;
}

// alpha * v for an alpha that is not a power of two (not used by the solver)
__device__ __noinline__ double scale_slow(double alpha, double v) { return alpha * v; }

// Signed 128-bit integer (h:l) times 2^e2 as a correctly rounded double
// (round to nearest even), integer operations only.  |value| must lie in the
// normal range (checked by the caller's exponent bounds).
__device__ __forceinline__ double i128_ldexp(int64_t h, uint64_t l, int e2, bool flip) {
  const bool neg = (h < 0) != flip;
  const bool vneg = h < 0;
  uint64_t ah = (uint64_t)h, al = l;
  if (vneg) {  // two's complement negate
    al = ~al + 1;
    ah = ~ah + (al == 0 ? 1 : 0);
  }
  if (ah == 0 && al == 0) return 0.0;
  int lz = ah ? __clzll((long long)ah) : 64 + __clzll((long long)al);
  const int top = 127 - lz;  // index of the leading bit
  // bring the leading bit to position 63 of a 64-bit word, keep a sticky bit
  uint64_t w, rest;
  const int s = 63 - top;  // left shift of the 128-bit value so that bit `top` lands at 127
  const int shl = lz;      // same thing for the 128-bit word
  if (shl == 0) {
    w = ah;
    rest = al;
  } else if (shl < 64) {
    w = (ah << shl) | (al >> (64 - shl));
    rest = al << shl;
  } else {
    w = al << (shl - 64);
    rest = 0;
  }
  (void)s;
  // w holds bits [top, top-63]; mantissa = top 53 bits of w
  uint64_t mant = w >> 11;
  const uint64_t rbits = w & 0x7FF;  // 11 dropped bits of w
  const bool half = (rbits & 0x400) != 0;
  const bool sticky = ((rbits & 0x3FF) != 0) || (rest != 0);
  if (half && (sticky || (mant & 1))) mant++;
  int expo = top + e2;  // value = 1.f * 2^(top + e2)
  if (mant >> 53) {      // rounding carried into a new leading bit
    mant >>= 1;
    expo++;
  }
  const int64_t be = (int64_t)expo + 1023;
  if (be <= 0 || be >= 2047) return i128_ldexp_slow(w, top - 63 + e2, neg);
  const uint64_t bits = ((uint64_t)neg << 63) | ((uint64_t)be << 52) | (mant & ((1ull << 52) - 1));
  return __longlong_as_double((long long)bits);
}

__global__ void __launch_bounds__(UMMA_THREADS, 1)
    k_sliced_umma(int64_t M, int64_t N, int64_t nks, const unsigned char *__restrict__ SA,
                  const unsigned char *__restrict__ SB, const int *__restrict__ ea, const int *__restrict__ eb,
                  double alpha, double beta, double *__restrict__ C, int64_t ldc, int mode, int64_t diag,
                  const int *abort_flag, int *err) {
  if (abort_flag && *abort_flag) return;
  const int64_t m0 = (int64_t)blockIdx.x * UM, n0 = (int64_t)blockIdx.y * UN;
  if (mode == TRI_LOWER && (m0 + UM - 1) - n0 + diag < 0) return;
  if (mode == TRI_UPPER && m0 - (n0 + UN - 1) + diag > 0) return;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char *bufA = smem;                             // NBUF x A_STAGE
  unsigned char *bufB = smem + NBUF * A_STAGE;            // NBUF x B_STAGE
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + NBUF * (A_STAGE + B_STAGE));
  uint64_t *full = bars, *empty = bars + NBUF, *accb = bars + 2 * NBUF;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * NBUF + 1);
  __shared__ int s_fail;
  __shared__ int s_issued;  // stages whose bulk copies were issued
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int i = 0; i < NBUF; i++) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(accb, 1);
    s_fail = 0;
    s_issued = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(sptr(tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const unsigned char *gA = SA + (size_t)blockIdx.x * nks * A_STAGE;
  const unsigned char *gB = SB + (size_t)blockIdx.y * nks * B_STAGE;

  if (warp == 0 && lane == 0) {
    // producer: one bulk copy per operand per stage
    for (int64_t ks = 0; ks < nks; ks++) {
      const int b = (int)(ks % NBUF);
      if (ks >= NBUF && !mbar_wait(&empty[b], (uint32_t)(((ks / NBUF) - 1) & 1))) {
        atomicExch(&s_fail, 1);
        break;
      }
      mbar_expect_tx(&full[b], A_STAGE + B_STAGE);
      bulk_g2s(bufA + (size_t)b * A_STAGE, gA + (size_t)ks * A_STAGE, A_STAGE, &full[b]);
      bulk_g2s(bufB + (size_t)b * B_STAGE, gB + (size_t)ks * B_STAGE, B_STAGE, &full[b]);
      s_issued = (int)ks + 1;
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    const uint32_t idesc = instr_desc();
    bool ok = true;
    for (int64_t ks = 0; ks < nks && ok; ks++) {
      const int b = (int)(ks % NBUF);
      if (!mbar_wait(&full[b], (uint32_t)((ks / NBUF) & 1))) {
        atomicExch(&s_fail, 1);
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t a0 = sptr(bufA + (size_t)b * A_STAGE), b0 = sptr(bufB + (size_t)b * B_STAGE);
#pragma unroll
      for (int kb2 = 0; kb2 < 2; kb2++)
#pragma unroll
        for (int q = 0; q < S; q++) {
          const uint64_t bd = smem_desc(b0 + (uint32_t)((q * 2 + kb2) * B_K16_BYTES), 128, 256);
#pragma unroll
          for (int p = 0; p < S - q; p++) {
            const uint64_t ad = smem_desc(a0 + (uint32_t)((p * 2 + kb2) * A_K16_BYTES), 128, 256);
            // level d = p + q is first written at (ks, kb2, q) = (0, 0, 0), p = d: start it fresh there
            const uint32_t acc = (ks == 0 && kb2 == 0 && q == 0) ? 0u : 1u;
            umma(tmem + (uint32_t)((p + q) * UN), ad, bd, idesc, acc);
          }
        }
      umma_commit(&empty[b]);
    }
    umma_commit(accb);
  }
  __syncwarp();
  // epilogue: 16 warps; warp w reads TMEM lane quarter (w % 4) (rows 32 (w % 4) + lane)
  // and columns [16 (w / 4), 16 (w / 4) + 16) of every level
  const bool got = mbar_wait(accb, 0);
  if (!got) atomicExch(&s_fail, 1);
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const int quarter = warp & 3, cgroup = warp >> 2;
  const int64_t gi = m0 + quarter * 32 + lane;
  const int er = (got && gi < M) ? ea[gi] : EXP_NONE;
  const bool neg_alpha = alpha < 0.0;
  const int ea2 = (alpha == 0.0) ? 0 : (int)((__double_as_longlong(fabs(alpha)) >> 52) & 0x7FF) - 1023;
  const bool alpha_pow2 = (alpha != 0.0) && ((__double_as_longlong(alpha) & ((1ll << 52) - 1)) == 0);
  const int beta_mode = (beta == 0.0) ? 0 : (beta == 1.0 ? 1 : 2);
  for (int c0 = cgroup * (UN / 4); c0 < (cgroup + 1) * (UN / 4); c0 += 4) {
    uint32_t v[S][4];
#pragma unroll
    for (int d = 0; d < S; d++) tmem_ld4(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(d * UN + c0), v[d]);
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
    if (!got || gi >= M) continue;
    // gather first (independent loads in flight together), then convert, then store
    bool ok[4];
    int ecv[4];
    double cold[4];
#pragma unroll
    for (int c = 0; c < 4; c++) {
      const int64_t gj = n0 + c0 + c;
      const int64_t dd = gi - gj + diag;
      ok[c] = (gj < N) && !(mode == TRI_LOWER && dd < 0) && !(mode == TRI_UPPER && dd > 0);
      ecv[c] = ok[c] ? eb[gj] : EXP_NONE;
      cold[c] = (ok[c] && beta_mode != 0) ? C[gi + gj * ldc] : 0.0;
    }
#pragma unroll
    for (int c = 0; c < 4; c++) {
      if (!ok[c]) continue;
      const int ec = ecv[c];
      double val = 0.0;
      if (er != EXP_NONE && ec != EXP_NONE) {
        int64_t hi = 0, lo = 0;
#pragma unroll
        for (int d = 0; d < 4; d++) hi = hi * 256 + (int64_t)__float2int_rn(__uint_as_float(v[d][c]));
#pragma unroll
        for (int d = 4; d < S; d++) lo = lo * 256 + (int64_t)__float2int_rn(__uint_as_float(v[d][c]));
        // V = hi 2^24 + lo as a signed 128-bit integer; value = V 2^(er + ec - 64)
        const uint64_t hl = (uint64_t)hi << 24;
        int64_t vh = hi >> 40;  // arithmetic shift keeps the sign
        uint64_t vl = hl + (uint64_t)lo;
        // carry / borrow of the low-word addition
        if (lo >= 0) vh += (vl < hl) ? 1 : 0;
        else vh -= (vl > hl) ? 1 : 0;
        if (alpha_pow2) val = i128_ldexp(vh, vl, er + ec - 64 + ea2, neg_alpha);
        else val = scale_slow(alpha, i128_ldexp(vh, vl, er + ec - 64, false));
      }
      const int64_t gj = n0 + c0 + c;
      C[gi + gj * ldc] = (beta_mode == 0) ? val : (beta_mode == 1 ? cold[c] + val : fma(beta, cold[c], val));
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0) {
    // no bulk copy of ours may still be landing in shared memory when the CTA exits
    for (int ks = max(0, s_issued - NBUF); ks < s_issued; ks++)
      if (!mbar_wait(&full[ks % NBUF], (uint32_t)((ks / NBUF) & 1))) s_fail = 1;
    if (s_fail) atomicExch(err, 1);
  }
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS));
}

}  // namespace

size_t umma_workspace_bytes(int64_t M, int64_t N, int64_t K) {
  const int64_t Mpad = ceil_div(M, UM) * UM, Npad = ceil_div(N, UN) * UN, Kpad = ceil_div(K, UKS) * UKS;
  return (size_t)S * (size_t)(Mpad + Npad) * (size_t)Kpad * 2 + slicing::slice_ints(Mpad, Npad, Kpad) * sizeof(int) +
         4096;
}

int umma_gemm(cudaStream_t st, bool transA, bool transB, int64_t M, int64_t N, int64_t K, double alpha,
              const double *A, int64_t lda, const double *B, int64_t ldb, double beta, double *C, int64_t ldc,
              TriMode mode, int64_t diag, const int *abort_flag, void *ws, size_t ws_bytes, int *err) {
  if (M <= 0 || N <= 0) return GSYEIG_SUCCESS;
  if (K > 128 || K <= 0) return GSYEIG_NOT_SUPPORTED;
  const int64_t Mpad = ceil_div(M, UM) * UM, Npad = ceil_div(N, UN) * UN, Kpad = ceil_div(K, UKS) * UKS;
  if (ws_bytes < umma_workspace_bytes(M, N, K)) return GSYEIG_NOT_SUPPORTED;
  slicing::SlicePlan P;
  P.Mpad = Mpad;
  P.Npad = Npad;
  P.Kpad = Kpad;
  P.SA = static_cast<unsigned char *>(ws);
  P.SB = P.SA + (size_t)S * Mpad * Kpad * 2;
  P.ea = reinterpret_cast<int *>(P.SB + (size_t)S * Npad * Kpad * 2);
  P.eb = P.ea + Mpad;
  P.kA = P.eb + Npad;
  P.kB = P.kA + Kpad;
  P.ksh = P.kB + Kpad;
  GS_TRY(slicing::slice_operands(st, transA, transB, M, N, K, A, lda, B, ldb, P, {true, UM}, {true, UN}));
  const size_t smem = (size_t)NBUF * (A_STAGE + B_STAGE) + 128;
  GS_CUDA(cudaFuncSetAttribute((const void *)k_sliced_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid((unsigned)(Mpad / UM), (unsigned)(Npad / UN));
  k_sliced_umma<<<grid, UMMA_THREADS, smem, st>>>(M, N, Kpad / UKS, P.SA, P.SB, P.ea, P.eb, alpha, beta, C, ldc,
                                                  (int)mode, diag, abort_flag, err);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

}  // namespace gs
