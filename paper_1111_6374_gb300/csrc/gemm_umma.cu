// tcgen05 (5th-generation tensor core) engine of the error-free sliced GEMM
// (the digit scheme is described in gemm_sliced.cu; this file only changes
// how the 28 digit-pair products are issued and how the exact level sums are
// turned into FP64).
//
//  * Operands are pre-split by k_rowsplit2 straight into the UMMA
//    "no-swizzle K-major" core-matrix layout (8 rows x 16 bytes per core
//    matrix, K-adjacent cores 128 B apart, row-adjacent cores 256 B apart),
//    grouped so that one K stage (32 k: two k16 blocks of all 7 slices) of a
//    128-row A block (56 KB) or a 32-row B block (14 KB) is one contiguous
//    run: each stage is brought in by a single cp.async.bulk per operand into
//    a 3-deep ring, completing on an mbarrier (no tensor map needed).
//  * Persistent CTAs (one per SM) walk the 128 x 32 tiles of C with
//    warp-specialised roles: a producer lane, an MMA lane and 16 epilogue
//    warps.  One thread issues tcgen05.mma.kind::f16 (bf16 x bf16 -> fp32,
//    M = 128, K = 16); the accumulator of level d lives in TMEM columns
//    [32 d, 32 d + 32) of one of two sets (columns 0 and 256; 7 levels, 224
//    columns each, 512 allocated).  The 28 digit products of a k16 block go
//    out as 7 MMAs of N = 32..224 (the B slices 0..6-p against A slice p
//    fill levels p..6); tcgen05.commit releases the stage buffer.
//  * Consecutive K chunks alternate between the two sets, so the epilogue
//    folds one chunk out of TMEM while the MMAs of the next one run.
//  * K up to 512 per call, in exact chunks of K = 128: after each chunk the
//    epilogue (warp w reads TMEM lane quarter w % 4, a quarter of the
//    columns each) reads the 7 level sums with tcgen05.ld, recombines them
//    exactly into a 128-bit integer per element added to a register
//    accumulator, and hands TMEM back to the next chunk's MMAs; after the
//    last chunk the exact sum V, scaled by the row and column exponents, is
//    faithfully rounded to FP64 in integer arithmetic and added to C with
//    one FP64 add.
//  * Every mbarrier wait is bounded; on expiry the kernel records the fault
//    in *err, still waits (bounded) for its own copies, frees its TMEM and
//    returns.
#include <cuda_bf16.h>

#include "slicing.cuh"

namespace gs {
namespace {

using slicing::S;
using slicing::EXP_NONE;
#ifndef UMMA_UKS
#define UMMA_UKS 32
#endif
#ifndef UMMA_NBUF
#define UMMA_NBUF 3
#endif
constexpr int UM = 128, UN = 32, UKS = UMMA_UKS;  // tile rows, tile cols, K per stage (16 or 32)
constexpr int KB2 = UKS / 16;                // k16 blocks per stage
constexpr int KPAD = 32;                     // K padding of the digit planes
constexpr int A_K16_BYTES = UM * 16 * 2;     // one slice, one k16 block: 4096
constexpr int B_K16_BYTES = UN * 16 * 2;     // 1024
constexpr int A_STAGE = KB2 * S * A_K16_BYTES;  // 57344
constexpr int B_STAGE = KB2 * S * B_K16_BYTES;  // 14336
constexpr int NBUF = UMMA_NBUF;  // stages in the ring
static_assert(UKS == 16 || UKS == 32, "a stage is one or two k16 blocks");
// after the ring: full[NBUF], empty[NBUF], acc_full[2], acc_empty[2], fin (8 bytes each), the TMEM
// slot (4 bytes), rounded up to 16
constexpr int BAR_BYTES = (((2 * NBUF + 5) * 8 + 4) + 15) / 16 * 16;
constexpr size_t UMMA_SMEM = (size_t)NBUF * (KB2 * S * (UM + UN) * 32) + BAR_BYTES;
static_assert(UMMA_SMEM <= 227 * 1024 - 1024, "the stage ring and its barriers exceed shared memory");
constexpr int CH_STAGES = 128 / UKS;  // K stages per exact chunk (level sums exact for K <= 128)
constexpr int UMMA_MAX_K = 512;
constexpr int TMEM_COLS = 512;
constexpr int SET_COLS = 256;  // two accumulator sets of 7 levels x UN columns, at columns 0 and 256
constexpr int NGROUP = S;      // MMAs per k16 block
constexpr uint32_t SPIN_LIMIT = 1u << 24;

int num_sms() { return num_sms_cached(); }

// ---------------------------------------------------------------- PTX -----
__device__ __forceinline__ uint32_t sptr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(sptr(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(sptr(bar)), "r"(bytes) : "memory");
}

// bounded wait for the phase with the given parity (at most `limit` polls);
// false on expiry
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t limit = SPIN_LIMIT) {
  const uint32_t a = sptr(bar);
  for (uint32_t it = 0; it < limit; it++) {
    uint32_t done;
    if (limit < SPIN_LIMIT) {
      // a test limit: poll without the hardware's suspended wait, so that
      // the limit counts polls and the wait can run out
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(done)
          : "r"(a), "r"(parity)
          : "memory");
      if (done) return true;
      continue;
    }
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

// instruction descriptor: kind::f16, bf16 A/B, fp32 D, K-major A/B, M = 128, N = n
__host__ __device__ constexpr uint32_t instr_desc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(UM >> 4) << 24);
}

// The 28 digit products (p, q), p + q <= 6, as 7 MMAs: the B slices
// 0..6 - p lie back to back in shared memory (one UN-row block each) and
// level d's accumulator is TMEM columns [UN d, UN d + UN) of a set, so A_p
// times the (UN (7 - p))-row block of those slices (N = UN (7 - p) <= 224)
// writes levels p .. 6 in one instruction.  The MMA of p = 0 covers every
// level once: it starts a chunk's accumulators.
struct MmaGroup {
  int p, q0, nq;
};
__host__ __device__ constexpr MmaGroup mma_group(int i) { return MmaGroup{i, 0, S - i}; }

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

// The registers written by tcgen05.ld are valid only after tcgen05.wait::ld;
// this empty asm makes every later use depend on a point after the wait.
__device__ __forceinline__ void reg_fence(uint32_t &x) { asm volatile("" : "+r"(x)); }

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
  const int lz = ah ? __clzll((long long)ah) : 64 + __clzll((long long)al);
  const int top = 127 - lz;  // index of the leading bit
  // shift the 128-bit magnitude left by lz: bit `top` lands at bit 127;
  // w = bits [top, top - 63], rest = everything below (sticky)
  uint64_t w, rest;
  if (lz == 0) {
    w = ah;
    rest = al;
  } else if (lz < 64) {
    w = (ah << lz) | (al >> (64 - lz));
    rest = al << lz;
  } else {
    w = al << (lz - 64);
    rest = 0;
  }
  uint64_t mant = w >> 11;  // top 53 bits
  const uint64_t rbits = w & 0x7FF;
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

// (-1)^flip V 2^e2 for V = h:l, |V| < 2^73, faithfully rounded to a double
// (error < 1 ulp) in 64-bit integer arithmetic, branch-free so that the
// elements of a thread interleave: T = V >> 10 fits in an int64 and carries
// every bit a double keeps (the 10 bits shifted out can only move a rounding
// tie).  *slow is set when the result leaves the normal range (the caller
// then takes i128_ldexp).  GB300 runs FP64 adds at about 1.6 per clock per
// SM and integer-to-float conversions at 16, so the C update is this, plus
// one FP64 add.
__device__ __forceinline__ double i128_to_double(int32_t h, uint64_t l, int e2, bool flip, bool &slow) {
  const int64_t T = (int64_t)(((uint64_t)(int64_t)h << 54) | (l >> 10));
  const bool neg = (T < 0) != flip;
  const uint64_t a = (uint64_t)(T < 0 ? -T : T);
  const bool zero = a == 0;
  const int lz = __clzll((long long)a);
  const uint64_t w = a << (lz & 63);
  uint64_t mant = w >> 11;
  const uint64_t rbits = w & 0x7FF;
  const bool up = (rbits & 0x400) && ((rbits & 0x3FF) || (mant & 1));
  mant += up ? 1ull : 0ull;
  const int carry = (int)(mant >> 53);
  mant >>= carry;
  const int be = (63 - lz) + e2 + 10 + carry + 1023;
  slow = !zero && (be <= 0 || be >= 2047);
  const double r = __longlong_as_double(
      (long long)(((uint64_t)neg << 63) | ((uint64_t)(be & 0x7FF) << 52) | (mant & ((1ull << 52) - 1))));
  return zero ? 0.0 : r;
}

// Persistent CTAs, one per SM; tile t = blockIdx.x + i gridDim.x over the
// (M / 128) x (N / 64) grid of C (column-major in m), tiles outside the
// triangle of a TRI mode skipped by every role alike.
//   warp 16 (one lane): producer -- bulk copies of each K stage into a
//       3-deep ring, released by the MMA commits;
//   warp 17 (one lane): MMA issuer -- before each K chunk waits for the
//       epilogue to have folded the chunk two before (the same accumulator
//       set), then 7 x 2 MMAs per stage;
//   warps 0-15: epilogue -- read the 7 level sums of 8 elements each from
//       TMEM, fold them into 128-bit integers in registers, hand the set back
//       (the MMAs of the chunk after next may start), and after a tile's
//       last chunk update C from the registers.
// Every wait is bounded; a wait that runs out sets s_fail, every role leaves
// its loop, the MMA issuer waits (bounded) for its own MMAs and thread 0 for
// the producer's copies before TMEM is freed.
constexpr int EPI_WARPS = 16;
constexpr int PRODUCER_WARP = EPI_WARPS, MMA_WARP = EPI_WARPS + 1;
constexpr int UMMA_THREADS = (EPI_WARPS + 2) * 32;
constexpr int EPI_COLS = UN / (EPI_WARPS / 4);  // columns of a tile per epilogue warp (8)

// Exact integer value of a level sum (an integer-valued fp32, |x| < 2^24).
__device__ __forceinline__ int32_t lvl(uint32_t bits) { return __float2int_rn(__uint_as_float(bits)); }

// The same for |x| <= 2^22 without the conversion unit (16 per clock per SM
// on GB300): x + 1.5 2^23 lies in [2^23, 2^24], where every integer is an
// fp32, so the addition is exact and the bit pattern minus that of 1.5 2^23
// is x.  Levels 0 and 1 of a K <= 128 chunk qualify (|L_d| <= (d + 1) 2^21).
__device__ __forceinline__ int32_t lvl22(uint32_t bits) {
  return __float_as_int(__uint_as_float(bits) + 12582912.0f) - 0x4B400000;
}

// (vh:vl) += V for the 7 level sums v[0..6] of one element,
// V = sum_d L_d 256^(6-d), |L_d| <= (d + 1) 128 2^14 (K <= 128 per chunk):
// a = L0 256 + L1 and b = L2 256 + L3 fit in int32, P = a 2^16 + b < 2^47,
// Q = (L4 256 + L5) 256 + L6 < 2^41, V = P 2^24 + Q.
__device__ __forceinline__ void fold_add(const uint32_t (&v)[S], int32_t &vh, uint64_t &vl) {
  const int32_t a = lvl22(v[0]) * 256 + lvl22(v[1]);
  const int32_t b = lvl(v[2]) * 256 + lvl(v[3]);
  const int64_t P = (int64_t)a * 65536 + (int64_t)b;
  const int64_t Q = ((int64_t)lvl(v[4]) * 256 + (int64_t)lvl(v[5])) * 256 + (int64_t)lvl(v[6]);
  const uint64_t pl = (uint64_t)P << 24;
  const uint64_t l1 = pl + (uint64_t)Q;
  int32_t h = (int32_t)(P >> 40) + (int32_t)(Q >> 63) + (l1 < pl ? 1 : 0);
  const uint64_t l2 = vl + l1;
  vh += h + (l2 < vl ? 1 : 0);
  vl = l2;
}

struct TileGrid {
  int64_t M, N, diag;
  int mt, nt, mode;
  __device__ bool get(int t, int64_t &m0, int64_t &n0) const {
    m0 = (int64_t)(t % mt) * UM;
    n0 = (int64_t)(t / mt) * UN;
    if (mode == TRI_LOWER && (m0 + UM - 1) - n0 + diag < 0) return false;
    if (mode == TRI_UPPER && m0 - (n0 + UN - 1) + diag > 0) return false;
    return true;
  }
};

__device__ __forceinline__ bool failed(const int *f) { return *(volatile const int *)f != 0; }

__global__ void __launch_bounds__(UMMA_THREADS, 1)
    k_sliced_umma(TileGrid g, int64_t nks, const unsigned char *__restrict__ SA, const unsigned char *__restrict__ SB,
                  const int *__restrict__ ea, const int *__restrict__ eb, double alpha, double beta,
                  double *__restrict__ C, int64_t ldc, const int *abort_flag, int *err, uint32_t spin) {
  if (abort_flag && *abort_flag) return;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char *bufA = smem;                   // NBUF x A_STAGE
  unsigned char *bufB = smem + NBUF * A_STAGE;  // NBUF x B_STAGE
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + NBUF * (A_STAGE + B_STAGE));
  // per accumulator set: acc_full (the chunk's MMAs are done), acc_empty (the epilogue has folded it)
  uint64_t *full = bars, *empty = bars + NBUF, *acc_full = bars + 2 * NBUF, *acc_empty = acc_full + 2,
           *fin = acc_full + 4;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * NBUF + 5);
  __shared__ int s_fail;
  __shared__ int64_t s_issued;  // stages whose bulk copies were issued
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntile = g.mt * g.nt;

  if (threadIdx.x == 0) {
    for (int i = 0; i < NBUF; i++) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; i++) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], EPI_WARPS);
    }
    mbar_init(fin, 1);
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

  if (warp == PRODUCER_WARP) {
    if (lane == 0) {
      int64_t it = 0;
      for (int t = blockIdx.x; t < ntile && !failed(&s_fail); t += gridDim.x) {
        int64_t m0, n0;
        if (!g.get(t, m0, n0)) continue;
        const unsigned char *gA = SA + (size_t)(m0 / UM) * nks * A_STAGE;
        const unsigned char *gB = SB + (size_t)(n0 / UN) * nks * B_STAGE;
        for (int64_t ks = 0; ks < nks; ks++, it++) {
          const int b = (int)(it % NBUF);
          if (it >= NBUF && !mbar_wait(&empty[b], (uint32_t)(((it / NBUF) - 1) & 1), spin)) {
            atomicExch(&s_fail, 1);
            break;
          }
          if (failed(&s_fail)) break;
          mbar_expect_tx(&full[b], A_STAGE + B_STAGE);
          bulk_g2s(bufA + (size_t)b * A_STAGE, gA + (size_t)ks * A_STAGE, A_STAGE, &full[b]);
          bulk_g2s(bufB + (size_t)b * B_STAGE, gB + (size_t)ks * B_STAGE, B_STAGE, &full[b]);
          s_issued = it + 1;
        }
      }
    }
  } else if (warp == MMA_WARP) {
    if (lane == 0) {
      uint32_t idesc[S + 1];
#pragma unroll
      for (int q = 0; q <= S; q++) idesc[q] = instr_desc(q > 0 ? q * UN : UN);
      int64_t it = 0;
      int64_t fc = 0;  // chunks issued
      uint32_t set_base = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntile && ok; t += gridDim.x) {
        int64_t m0, n0;
        if (!g.get(t, m0, n0)) continue;
        for (int64_t ks = 0; ks < nks; ks++, it++) {
          const int b = (int)(it % NBUF);
          const bool first = (ks % CH_STAGES) == 0;  // first stage of an exact K chunk
          if (first) {
            // this chunk's set (fc & 1) was folded out of TMEM by the epilogue (chunk fc - 2)
            const int set = (int)(fc & 1);
            if (fc >= 2 && !mbar_wait(&acc_empty[set], (uint32_t)(((fc >> 1) - 1) & 1), spin)) {
              ok = false;
              break;
            }
            set_base = (uint32_t)(set * SET_COLS);
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
          }
          if (failed(&s_fail) || !mbar_wait(&full[b], (uint32_t)((it / NBUF) & 1), spin)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
          const uint32_t a0 = sptr(bufA + (size_t)b * A_STAGE), b0 = sptr(bufB + (size_t)b * B_STAGE);
#pragma unroll
          for (int kb2 = 0; kb2 < KB2; kb2++)
#pragma unroll
            for (int gq = 0; gq < NGROUP; gq++) {
              const MmaGroup gr = mma_group(gq);
              const uint64_t ad = smem_desc(a0 + (uint32_t)((kb2 * S + gr.p) * A_K16_BYTES), 128, 256);
              const uint64_t bd = smem_desc(b0 + (uint32_t)((kb2 * S + gr.q0) * B_K16_BYTES), 128, 256);
              const uint32_t acc = (first && kb2 == 0 && gr.p == 0) ? 0u : 1u;
              umma(tmem + set_base + (uint32_t)((gr.p + gr.q0) * UN), ad, bd, idesc[gr.nq], acc);
            }
          umma_commit(&empty[b]);
          if ((ks % CH_STAGES) == CH_STAGES - 1 || ks == nks - 1) {
            umma_commit(&acc_full[fc & 1]);
            fc++;
          }
        }
        if (!ok) break;
      }
      if (!ok) atomicExch(&s_fail, 1);
      // every MMA of ours has finished before TMEM can be freed
      umma_commit(fin);
      if (!mbar_wait(fin, 0)) atomicExch(&s_fail, 1);
    }
  } else {
    // epilogue: warp w reads TMEM lane quarter w % 4 (rows 32 (w % 4) + lane)
    // and columns [8 (w / 4), 8 (w / 4) + 8) of every level
    const int quarter = warp & 3, cgroup = warp >> 2;
    const bool neg_alpha = alpha < 0.0;
    const int ea2 = (alpha == 0.0) ? 0 : (int)((__double_as_longlong(fabs(alpha)) >> 52) & 0x7FF) - 1023;
    const bool alpha_pow2 = (alpha != 0.0) && ((__double_as_longlong(alpha) & ((1ll << 52) - 1)) == 0);
    const int beta_mode = (beta == 0.0) ? 0 : (beta == 1.0 ? 1 : 2);
    const int64_t nch = (nks + CH_STAGES - 1) / CH_STAGES;
    int64_t fc = 0;  // chunks folded
    bool ok = true;
    for (int t = blockIdx.x; t < ntile && ok; t += gridDim.x) {
      int64_t m0, n0;
      if (!g.get(t, m0, n0)) continue;
      const int64_t gi = m0 + quarter * 32 + lane;
      const int64_t gjb = n0 + cgroup * EPI_COLS;
      // the exponents this thread needs: its row's, and lane j < 16 holds column gjb + j's
      const int er_pre = (gi < g.M) ? ea[gi] : EXP_NONE;
      const int ec_pre = (lane < EPI_COLS && gjb + lane < g.N) ? eb[gjb + lane] : EXP_NONE;
      const bool row_ok = gi < g.M;  // (no early exit: the warp shuffles below need every lane)
      const int er = er_pre;
      // which of this thread's elements it writes (bit c), and their column exponents
      uint32_t okm = 0;
      int ecv[EPI_COLS];
#pragma unroll
      for (int c = 0; c < EPI_COLS; c++) {
        const int64_t gj = gjb + c, dd = gi - gj + g.diag;
        const bool ok = row_ok && (gj < g.N) && !(g.mode == TRI_LOWER && dd < 0) && !(g.mode == TRI_UPPER && dd > 0);
        const int ecs = __shfl_sync(0xffffffffu, ec_pre, c);
        ecv[c] = ok ? ecs : EXP_NONE;
        okm |= ok ? (1u << c) : 0u;
      }
      // the solver's updates (C += +-2^k A B) read C: its lines are brought
      // into L2 while the tile's last K chunk is still in the tensor cores
      // (a prefetch holds no registers: 18 warps leave at most 96 per thread)
      const bool prefetch = alpha_pow2 && beta_mode == 1;
      // V = sum over chunks of the recombined level sums, a signed 128-bit
      // integer (vh:vl) per element, held in registers
      int32_t vh[EPI_COLS];
      uint64_t vl[EPI_COLS];
#pragma unroll
      for (int c = 0; c < EPI_COLS; c++) {
        vh[c] = 0;
        vl[c] = 0;
      }
      for (int64_t ch = 0; ch < nch; ch++, fc++) {
        if (prefetch && ch == nch - 1) {
#pragma unroll
          for (int c = 0; c < EPI_COLS; c++)
            if ((okm >> c) & 1) asm volatile("prefetch.global.L2 [%0];\n" ::"l"(C + gi + (gjb + c) * ldc));
        }
        // the warp decides together (the TMEM loads and shuffles below are
        // .sync.aligned: no lane may leave on its own)
        const int set = (int)(fc & 1);
        const bool got = mbar_wait(&acc_full[set], (uint32_t)((fc >> 1) & 1), spin);
        if (!__all_sync(0xffffffffu, got)) {
          if (lane == 0) atomicExch(&s_fail, 1);
          ok = false;
          break;
        }
        if (__any_sync(0xffffffffu, failed(&s_fail))) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
        for (int c0 = 0; c0 < EPI_COLS; c0 += 4) {
          uint32_t v[S][4];
#pragma unroll
          for (int d = 0; d < S; d++)
            tmem_ld4(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(set * SET_COLS + d * UN + cgroup * EPI_COLS + c0),
                     v[d]);
          asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
          for (int d = 0; d < S; d++)
#pragma unroll
            for (int c = 0; c < 4; c++) reg_fence(v[d][c]);
#pragma unroll
          for (int c = 0; c < 4; c++) {
            const uint32_t lv[S] = {v[0][c], v[1][c], v[2][c], v[3][c], v[4][c], v[5][c], v[6][c]};
            fold_add(lv, vh[c0 + c], vl[c0 + c]);
          }
        }
        // TMEM is free for the next chunk's MMAs
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(sptr(&acc_empty[set])) : "memory");
      }
      if (!ok) break;
      if (alpha_pow2 && beta_mode != 2) {
        // the solver's updates, C = +-2^k A B (+ C): V rounded to FP64 first
        // (branch-free; the 128-bit accumulators die here), then every load
        // of C in one burst (a store may alias a later load, so the compiler
        // would not hoist them), then one FP64 add per element
        double val[EPI_COLS];
#pragma unroll
        for (int c = 0; c < EPI_COLS; c++) {
          const bool live = (er != EXP_NONE && ecv[c] != EXP_NONE);
          bool slow;
          val[c] = i128_to_double(live ? vh[c] : 0, live ? vl[c] : 0ull, er + ecv[c] - 64 + ea2, neg_alpha, slow);
          if (slow) val[c] = i128_ldexp(vh[c], vl[c], er + ecv[c] - 64 + ea2, neg_alpha);
        }
        if (beta_mode == 1) {
          double cold[EPI_COLS];
#pragma unroll
          for (int c = 0; c < EPI_COLS; c++) cold[c] = ((okm >> c) & 1) ? C[gi + (gjb + c) * ldc] : 0.0;
#pragma unroll
          for (int c = 0; c < EPI_COLS; c++)
            if ((okm >> c) & 1) C[gi + (gjb + c) * ldc] = cold[c] + val[c];
        } else {
#pragma unroll
          for (int c = 0; c < EPI_COLS; c++)
            if ((okm >> c) & 1) C[gi + (gjb + c) * ldc] = val[c];
        }
      } else {
#pragma unroll
        for (int c = 0; c < EPI_COLS; c++) {
          if (!((okm >> c) & 1)) continue;
          const int ec = ecv[c];
          double ab = 0.0;
          if (er != EXP_NONE && ec != EXP_NONE)
            ab = alpha_pow2 ? i128_ldexp(vh[c], vl[c], er + ec - 64 + ea2, neg_alpha)
                            : scale_slow(alpha, i128_ldexp(vh[c], vl[c], er + ec - 64, false));
          const double cold = (beta_mode != 0) ? C[gi + (gjb + c) * ldc] : 0.0;
          C[gi + (gjb + c) * ldc] = (beta_mode == 0) ? ab : (beta_mode == 1 ? cold + ab : fma(beta, cold, ab));
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0) {
    // none of the producer's bulk copies may still be landing when the CTA exits
    const int64_t iss = s_issued;
    for (int64_t i = (iss > NBUF ? iss - NBUF : 0); i < iss; i++)
      if (!mbar_wait(&full[i % NBUF], (uint32_t)((i / NBUF) & 1))) s_fail = 1;
    if (s_fail) atomicExch(err, 1);
  }
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS));
}

}  // namespace

size_t umma_workspace_bytes(int64_t M, int64_t N, int64_t K) {
  const int64_t Mpad = ceil_div(M, UM) * UM, Npad = ceil_div(N, UN) * UN, Kpad = ceil_div(K, KPAD) * KPAD;
  return (size_t)S * (size_t)(Mpad + Npad) * (size_t)Kpad * 2 + slicing::slice_ints(Mpad, Npad, Kpad) * sizeof(int) +
         4096;
}

int umma_gemm(cudaStream_t st, bool transA, bool transB, int64_t M, int64_t N, int64_t K, double alpha,
              const double *A, int64_t lda, const double *B, int64_t ldb, double beta, double *C, int64_t ldc,
              TriMode mode, int64_t diag, const int *abort_flag, void *ws, size_t ws_bytes, int *err,
              uint32_t spin, int max_ctas) {
  if (M <= 0 || N <= 0) return GSYEIG_SUCCESS;
  if (K > UMMA_MAX_K || K <= 0) return GSYEIG_NOT_SUPPORTED;
  const int64_t Mpad = ceil_div(M, UM) * UM, Npad = ceil_div(N, UN) * UN, Kpad = ceil_div(K, KPAD) * KPAD;
  if (ws_bytes < umma_workspace_bytes(M, N, K)) return GSYEIG_NOT_SUPPORTED;
  slicing::SlicePlan P;
  P.Mpad = Mpad;
  P.Npad = Npad;
  P.Kpad = Kpad;
  P.SA = static_cast<unsigned char *>(ws);
  P.SB = P.SA + (size_t)S * Mpad * Kpad * 2;
  slicing::slice_layout(P, reinterpret_cast<int *>(P.SB + (size_t)S * Npad * Kpad * 2));
  GS_TRY(slicing::slice_operands(st, transA, transB, M, N, K, A, lda, B, ldb, P, {true, UM}, {true, UN}));
  const size_t smem = UMMA_SMEM;
  GS_TRY(set_max_smem((const void *)k_sliced_umma, (int)smem));
  TileGrid g{M, N, diag, (int)(Mpad / UM), (int)(Npad / UN), (int)mode};
  // CTAs without an active tile (TRI modes) only set up and leave
  const int64_t tiles = (int64_t)g.mt * g.nt;
  const int64_t ctas = max_ctas > 0 ? std::min(max_ctas, num_sms()) : num_sms();
  const unsigned grid = (unsigned)std::min<int64_t>(tiles, ctas);
  KernelProfiler *prof = current_profiler();
  const size_t e0 = prof ? prof->start(st) : SIZE_MAX;
  k_sliced_umma<<<grid, UMMA_THREADS, smem, st>>>(g, Kpad / UKS, P.SA, P.SB, P.ea, P.eb, alpha, beta, C, ldc,
                                                  abort_flag, err, spin > 0 ? spin : SPIN_LIMIT);
  count_launch();
  GS_CHECK_LAUNCH();
  if (prof) {
    // the tensor-core kernel alone: 2K FP64-equivalent flops per written element
    prof->stop(st, e0, PROF_GEMM_CORE, 2.0 * (double)K * region_elems(M, N, mode, diag), 0.0);
  }
  return GSYEIG_SUCCESS;
}

}  // namespace gs
