// ke1 on the FP32 pipes: z = C w with C held as a pair of fp32 matrices
// (C = C_hi + C_lo to about 2^-48 relative per entry) and only its lower
// triangle stored, in 64 x 64 tiles.
//
// In FP64 the product is bound by GB300's FP64 pipe (2n^2 flops at ~1.26
// TFLOP/s, 0.43 ms at n = 16384), not by HBM.  Here every product of
// (c_hi + c_lo)(w_hi + w_lo) is formed with an error-free product on the
// fp32 pipe and summed with compensated (twice-working-precision) dot
// products (Ogita, Rump, Oishi, "Accurate sum and dot product", 2005), so
// the operator applied is C_hi + C_lo to ~2^-48 and each 64-term partial is
// accurate to ~2^-48; partials are combined in double-float and rounded to
// FP64 once per row.  The stored bytes are
// 4 n(n+1)/2 * 2 = half of the full FP64 square, and each stored tile is
// used twice (C_ij w_j and C_ij^T w_i): the kernel is HBM-bound.
//
// Layout: tile t = bi (bi + 1) / 2 + bj for bi >= bj; within a tile,
// element (r, c) at (r ^ 2 (c & 15)) + 64 c (column-major, the row index
// XOR-swizzled by an even amount that depends on the column: rows 2m and
// 2m + 1 stay adjacent, so a thread reads a pair of rows with one 64-bit
// load, and both a warp reading 64 rows of one column and a warp reading
// one row pair of 32 columns are free of bank conflicts); hi and lo in two
// arrays.
// The arithmetic runs on packed pairs (fma/mul/add.rn.f32x2): a thread
// carries two compensated accumulators, one per row of its pair.
// C is stored scaled by the power of two 2^-e that brings max|C| into
// [1/2, 1), so that neither fp32 half overflows or underflows for pencils
// of any scale; the row sums are scaled back by 2^e.
// Diagonal tiles hold the full symmetric 64 x 64 block.  Partials go to
// W[slot][row]: tile (bi, bj) writes its row sums to slot bj of rows in
// block bi and (off-diagonal) its column sums to slot bi of rows in block
// bj, so each (slot, row) is written exactly once; a second kernel sums the
// NT slots of every row in double-float.  Deterministic.
#include "symv_df.cuh"

namespace gs {
namespace {

constexpr int TS = 64;           // tile size
constexpr int DF_THREADS = 256;  // 8 warps: row pairs x column groups of 8 (row sums); columns x row groups of 16

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// packed pairs of fp32 (low half: first element) and their arithmetic
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 pmul(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f32x2 padd(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f32x2 psub(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f32x2 pfma(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ float2 unpack(f32x2 v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}

// One compensated step on both lanes: (s, c) += (c_hi + c_lo)(x_hi + x_lo)
// with p = c_hi x_hi, its exact error from an FMA, the cross terms
// c_hi x_lo + c_lo x_hi in plain fp32, and the two-sum error of s + p
// (Ogita, Rump, Oishi 2005).  The negated x halves come precomputed, so
// en = p - c_hi x_hi - c_hi x_lo - c_lo x_hi is the negated low-order part.
__device__ __forceinline__ void dot2_step(f32x2 &s, f32x2 &c, f32x2 ch, f32x2 cl, f32x2 xh, f32x2 nxh, f32x2 nxl) {
  const f32x2 p = pmul(ch, xh);
  f32x2 en = pfma(ch, nxh, p);
  en = pfma(ch, nxl, en);
  en = pfma(cl, nxh, en);
  const f32x2 t = padd(s, p);
  const f32x2 bb = psub(t, s);
  const f32x2 q = padd(psub(s, psub(t, bb)), psub(p, bb));
  c = psub(padd(c, q), en);
  s = t;
}

// Largest |entry| of the stored part of M (as its bit pattern: for
// non-negative doubles the integer order is the numeric order) into *amax.
__global__ void k_op_absmax(int64_t n, const double *__restrict__ C, int64_t ldc, int tri, int trans,
                            unsigned long long *amax) {
  const int64_t bi = blockIdx.y, bj = blockIdx.x;
  if (bj > bi) return;
  unsigned long long mx = 0;
  for (int idx = threadIdx.x; idx < TS * TS; idx += blockDim.x) {
    const int r = idx % TS, c = idx / TS;
    const int64_t i = bi * TS + r, j = bj * TS + c;
    if (i < n && j < n && !(tri && j > i)) {
      const double v = trans ? C[j + i * ldc] : C[i + j * ldc];
      const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(v));
      if (b < 0x7FF0000000000000ull && b > mx) mx = b;  // finite entries only
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = y > mx ? y : mx;
  }
  if ((threadIdx.x & 31) == 0 && mx) atomicMax(amax, mx);
}

// the power of two 2^e with max|M| 2^-e in [1/2, 1) (e = 0 for M = 0)
__device__ __forceinline__ int op_exponent(const unsigned long long *amax) {
  const unsigned long long b = *amax;
  if (b == 0) return 0;
  int e;
  frexp(__longlong_as_double((long long)b), &e);
  return e;
}

// Tiles of the lower triangle of M 2^-e: M = C (trans = 0) or M = C^T (trans
// = 1, read from C's upper triangle); with tri = 1 the entries above the
// diagonal of the diagonal tiles are stored as zeros (M lower triangular),
// else the diagonal tiles hold the full symmetric block.  The exact scaling
// by 2^-e (e from op_exponent) keeps the fp32 hi/lo pair inside fp32's range
// whatever the magnitude of M; the products are scaled back by 2^e.
__global__ void k_op_build(int64_t n, int64_t NT, const double *__restrict__ C, int64_t ldc, int tri, int trans,
                           const unsigned long long *amax, float *__restrict__ hi, float *__restrict__ lo) {
  const int64_t bi = blockIdx.y, bj = blockIdx.x;
  if (bj > bi) return;
  const int64_t t = bi * (bi + 1) / 2 + bj;
  float *h = hi + t * TS * TS, *l = lo + t * TS * TS;
  const int e = op_exponent(amax);
  for (int idx = threadIdx.x; idx < TS * TS; idx += blockDim.x) {
    const int r = idx % TS, c = idx / TS;
    const int64_t i = bi * TS + r, j = bj * TS + c;
    double v = 0.0;
    if (i < n && j < n && !(tri && j > i)) v = ldexp(trans ? C[j + i * ldc] : C[i + j * ldc], -e);
    const float vh = (float)v;
    const int pos = (r ^ (2 * (c & 15))) + TS * c;
    h[pos] = vh;
    l[pos] = (float)(v - (double)vh);
  }
}

__global__ void k_vec_split(int64_t n, int64_t npad, const double *__restrict__ w, float2 *__restrict__ ws) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npad; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = (i < n) ? w[i] : 0.0;
    const float vh = (float)v;
    ws[i] = make_float2(vh, (float)(v - (double)vh));
  }
}

// (bi, bj) of packed tile t (32-bit: the tile count stays below 2^31);
// fp32 estimate corrected by integer steps (no FP64 instruction).
__device__ __forceinline__ void tile_of(int t, int &bi, int &bj) {
  int b = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
  while (b * (b + 1) / 2 > t) b--;
  while ((b + 1) * (b + 2) / 2 <= t) b++;
  bi = b;
  bj = t - b * (b + 1) / 2;
}

__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
  float s, q;
  two_sum(a.x, b.x, s, q);
  return make_float2(s, a.y + b.y + q);
}

__device__ __forceinline__ uint32_t sptr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

constexpr uint32_t SPIN_LIMIT = 1u << 24;

// bounded mbarrier wait, at most `limit` polls (false on expiry)
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t limit) {
  for (uint32_t it = 0; it < limit; it++) {
    uint32_t done;
    if (limit < SPIN_LIMIT) {
      // a test limit: poll without the hardware's suspended wait, so that
      // the limit counts polls and the wait can run out
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(done)
          : "r"(sptr(bar)), "r"(parity)
          : "memory");
      if (done) return true;
      continue;
    }
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(sptr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if (it > 64) __nanosleep(64);
  }
  return false;
}

#ifndef SYMV_DF_NSTAGE
#define SYMV_DF_NSTAGE 1
#endif
#ifndef SYMV_DF_CTAS_PER_SM
#define SYMV_DF_CTAS_PER_SM 4
#endif
constexpr int NSTAGE = SYMV_DF_NSTAGE;        // tiles in flight per CTA
constexpr int CTAS_PER_SM = SYMV_DF_CTAS_PER_SM;
constexpr int TILE_BYTES = TS * TS * 4;  // one of hi / lo

// Persistent CTAs; tiles t = blockIdx.x + i gridDim.x.  Thread 0 keeps
// NSTAGE tiles in flight with cp.async.bulk (hi and lo, 16 KB each) into
// shared memory; all 8 warps compute on the oldest one.  A wait that runs
// out (after `spin` polls) sets *err and ends the CTA after draining its own
// copies (those waits keep the full bound).
// mode DF_SYM: z = M w for the symmetric M whose lower triangle is stored
// (row sums of every tile, column sums of the off-diagonal ones);
// DF_ROWS: z = L w and DF_COLS: z = L^T w for the lower-triangular L stored.
__global__ void __launch_bounds__(DF_THREADS, CTAS_PER_SM) k_symv_df(int NT, int64_t npad, const float *__restrict__ hi,
                                                        const float *__restrict__ lo, const float2 *__restrict__ ws,
                                                        float2 *__restrict__ W, int *err, int mode, uint32_t spin) {
  extern __shared__ __align__(128) unsigned char smem[];
  float *sh = reinterpret_cast<float *>(smem);                       // NSTAGE x (hi tile, lo tile)
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + (size_t)NSTAGE * 2 * TILE_BYTES);
  // w of the tile's column block for the row sums, as duplicated pairs (x_hi, x_hi), (-x_hi, -x_hi),
  // (-x_lo, -x_lo); w of its row block for the column sums, as arrays read in row pairs
  __shared__ f32x2 xrh[TS], xrnh[TS], xrnl[TS];
  __shared__ __align__(8) float xch[TS], xcnh[TS], xcnl[TS];
  __shared__ float2 rowp[8][TS];  // row-sum partials of the 8 column groups
  __shared__ float2 colp[4][TS];  // column-sum partials of the 4 row groups
  __shared__ int s_fail;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = NT * (NT + 1) / 2;
  const int mine = (blockIdx.x < (unsigned)ntiles) ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < NSTAGE; i++) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(sptr(&full[i])));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    s_fail = 0;
  }
  __syncthreads();
  auto issue = [&](int i) {  // thread 0: copies of this CTA's i-th tile into stage i % NSTAGE
    const int t = (int)blockIdx.x + i * (int)gridDim.x;
    const int b = i % NSTAGE;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(sptr(&full[b])),
                 "r"(2 * TILE_BYTES)
                 : "memory");
    const float *srcs[2] = {hi + (size_t)t * TS * TS, lo + (size_t)t * TS * TS};
    for (int q = 0; q < 2; q++)
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                       sptr(sh + (size_t)(b * 2 + q) * TS * TS)),
                   "l"(srcs[q]), "r"(TILE_BYTES), "r"(sptr(&full[b]))
                   : "memory");
  };
  if (threadIdx.x == 0)
    for (int i = 0; i < NSTAGE && i < mine; i++) issue(i);
  int issued = (mine < NSTAGE) ? mine : NSTAGE;
  for (int i = 0; i < mine; i++) {
    const int t = (int)blockIdx.x + i * (int)gridDim.x;
    int bi, bj;
    tile_of(t, bi, bj);
    const bool diag = (bi == bj);
    const bool do_rows = mode != DF_COLS;                          // block-uniform
    const bool do_cols = (mode == DF_SYM && !diag) || mode == DF_COLS;
    if (threadIdx.x < TS) {
      const float2 v = ws[(int64_t)bj * TS + threadIdx.x];
      const int q = threadIdx.x;
      asm("mov.b64 %0, {%1, %1};" : "=l"(xrh[q]) : "f"(v.x));
      asm("mov.b64 %0, {%1, %1};" : "=l"(xrnh[q]) : "f"(-v.x));
      asm("mov.b64 %0, {%1, %1};" : "=l"(xrnl[q]) : "f"(-v.y));
    } else if (threadIdx.x < 2 * TS) {
      const int q = threadIdx.x - TS;
      const float2 v = ws[(int64_t)bi * TS + q];
      xch[q] = v.x;
      xcnh[q] = -v.x;
      xcnl[q] = -v.y;
    }
    const int b = i % NSTAGE;
    const bool ok = mbar_wait(&full[b], (uint32_t)((i / NSTAGE) & 1), spin);
    if (!ok) s_fail = 1;
    __syncthreads();
    if (s_fail) break;
    const f32x2 *h2 = reinterpret_cast<const f32x2 *>(sh + (size_t)(b * 2) * TS * TS);
    const f32x2 *l2 = h2 + TS * TS / 2;
    if (do_rows) {
      // row sums: thread (rows 2 lane, 2 lane + 1) over the 8 columns of its
      // warp; (c & 15) = 8 (warp & 1) + k, so the swizzle is rb ^ 2k
      const int rb = (2 * lane) ^ (16 * (warp & 1));
      f32x2 sr = 0ull, cr = 0ull;
#pragma unroll
      for (int k = 0; k < 8; k++) {
        const int col = 8 * warp + k;
        const int pos = (rb ^ (2 * k)) + TS * col;
        dot2_step(sr, cr, h2[pos >> 1], l2[pos >> 1], xrh[col], xrnh[col], xrnl[col]);
      }
      const float2 a = unpack(sr), c = unpack(cr);
      *reinterpret_cast<float4 *>(&rowp[warp][2 * lane]) = make_float4(a.x, c.x, a.y, c.y);
    }
    if (do_cols) {
      // column sums (C_ij^T w_i): thread (column cc, row group g) over the
      // 8 row pairs 16 g + 2k, 16 g + 2k + 1, one accumulator per row parity
      const int cc = lane + 32 * (warp & 1), g = warp >> 1;
      const int cb = (16 * g) ^ (2 * (cc & 15));
      f32x2 sc = 0ull, ccp = 0ull;
#pragma unroll
      for (int k = 0; k < 8; k++) {
        const int row = 16 * g + 2 * k;
        const int pos = (cb ^ (2 * k)) + TS * cc;
        dot2_step(sc, ccp, h2[pos >> 1], l2[pos >> 1], *reinterpret_cast<const f32x2 *>(&xch[row]),
                  *reinterpret_cast<const f32x2 *>(&xcnh[row]), *reinterpret_cast<const f32x2 *>(&xcnl[row]));
      }
      const float2 a = unpack(sc), c = unpack(ccp);
      colp[g][cc] = df_add(make_float2(a.x, c.x), make_float2(a.y, c.y));
    }
    __syncthreads();  // stage b fully read; partials complete
    if (threadIdx.x == 0 && issued < mine) {
      issue(issued);
      issued++;
    }
    if (do_rows && threadIdx.x < TS) {
      // rows of block bi: combine the 4 column groups
      const int rr = threadIdx.x;
      const float2 a = df_add(df_add(df_add(rowp[0][rr], rowp[1][rr]), df_add(rowp[2][rr], rowp[3][rr])),
                              df_add(df_add(rowp[4][rr], rowp[5][rr]), df_add(rowp[6][rr], rowp[7][rr])));
      W[(int64_t)bj * npad + (int64_t)bi * TS + rr] = a;
    } else if (do_cols && threadIdx.x >= TS && threadIdx.x < 2 * TS) {
      const int cc = threadIdx.x - TS;
      W[(int64_t)bi * npad + (int64_t)bj * TS + cc] = df_add(df_add(colp[0][cc], colp[1][cc]), df_add(colp[2][cc], colp[3][cc]));
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    // none of our bulk copies may still be landing when the CTA exits
    for (int i = (issued > NSTAGE ? issued - NSTAGE : 0); i < issued; i++)
      if (!mbar_wait(&full[i % NSTAGE], (uint32_t)((i / NSTAGE) & 1), SPIN_LIMIT)) s_fail = 1;
    if (s_fail) atomicExch(err, 1);
  }
}

// z_i = sum over the slots of W[slot][i] written for row i (all NT for
// DF_SYM; the tiles' column blocks 0..b for DF_ROWS and b..NT-1 for DF_COLS,
// b = i / 64), accumulated in double-float and rounded to FP64 once.
__global__ void k_reduce_slots(int64_t n, int64_t npad, int64_t NT, const float2 *__restrict__ W, double *__restrict__ z,
                               int mode, const unsigned long long *amax) {
  const int e = op_exponent(amax);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
    const int64_t blk = i / TS;
    int64_t q = (mode == DF_COLS) ? blk : 0;
    const int64_t q1 = (mode == DF_ROWS) ? blk + 1 : NT;
    for (; q + 1 < q1; q += 2) {
      a = df_add(a, W[q * npad + i]);
      b = df_add(b, W[(q + 1) * npad + i]);
    }
    if (q < q1) a = df_add(a, W[q * npad + i]);
    a = df_add(a, b);
    z[i] = ldexp((double)a.x + (double)a.y, e);
  }
}

}  // namespace

size_t df_tile_bytes(int64_t n) {
  const int64_t NT = ceil_div(n, TS);
  return (size_t)NT * (NT + 1) / 2 * TS * TS * sizeof(float) * 2;
}

size_t df_operator_bytes(int64_t n) { return df_tile_bytes(n) + 256; }

size_t df_partials_bytes(int64_t n) {
  const int64_t NT = ceil_div(n, TS);
  return (size_t)NT * NT * TS * sizeof(float2) + (size_t)NT * TS * sizeof(float2) + 256;
}

int df_operator_build(cudaStream_t st, int64_t n, const double *C, int64_t ldc, DfOperator &op, bool tri, bool trans) {
  const int64_t NT = ceil_div(n, TS);
  op.n = n;
  op.NT = NT;
  op.npad = NT * TS;
  const size_t tiles = (size_t)NT * (NT + 1) / 2 * TS * TS;
  op.lo = op.hi + tiles;
  op.amax = reinterpret_cast<unsigned long long *>(reinterpret_cast<char *>(op.hi) + df_tile_bytes(n));
  GS_CUDA(cudaMemsetAsync(op.amax, 0, sizeof(unsigned long long), st));
  k_op_absmax<<<dim3((unsigned)NT, (unsigned)NT), 256, 0, st>>>(n, C, ldc, tri ? 1 : 0, trans ? 1 : 0, op.amax);
  k_op_build<<<dim3((unsigned)NT, (unsigned)NT), 256, 0, st>>>(n, NT, C, ldc, tri ? 1 : 0, trans ? 1 : 0, op.amax,
                                                               op.hi, op.lo);
  count_launch(2);
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

int num_sms_cached() {
  static int sms[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (sms[dev] <= 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      v = 1;
    }
    sms[dev] = v > 0 ? v : 1;
  }
  return sms[dev];
}

int df_symv(cudaStream_t st, const DfOperator &op, const double *w, double *z, int mode) {
  KernelProfiler *prof = current_profiler();
  size_t e0 = prof ? prof->start(st) : SIZE_MAX;
  const int64_t ntiles = op.NT * (op.NT + 1) / 2;
  k_vec_split<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(op.npad, 256), 1024)), 256, 0, st>>>(
      op.n, op.npad, w, op.wsplit);
  const size_t smem = (size_t)NSTAGE * 2 * TILE_BYTES + NSTAGE * sizeof(uint64_t);
  GS_TRY(set_max_smem((const void *)k_symv_df, (int)smem));
  k_symv_df<<<(unsigned)std::min<int64_t>(ntiles, (int64_t)num_sms_cached() * CTAS_PER_SM), DF_THREADS, smem, st>>>(
      (int)op.NT, op.npad, op.hi, op.lo, op.wsplit, op.W, op.err, mode, op.spin > 0 ? op.spin : SPIN_LIMIT);
  k_reduce_slots<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(op.n, 256), 1024)), 256, 0, st>>>(
      op.n, op.npad, op.NT, op.W, z, mode, op.amax);
  count_launch(3);
  GS_CHECK_LAUNCH();
  if (prof) {
    const double n = (double)op.n;
    // algorithmic: 2n^2 flops (n^2 for a triangular product); the stored
    // triangle (hi + lo, 8 bytes per entry of n(n+1)/2) plus w and z
    prof->stop(st, e0, PROF_SYMV, (mode == DF_SYM ? 2.0 : 1.0) * n * n, 8.0 * (n * (n + 1) / 2) + 16.0 * n);
  }
  return GSYEIG_SUCCESS;
}

}  // namespace gs
