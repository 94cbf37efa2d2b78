// The learned warm start for sequences of related problems (the paper's
// Section 3 motivates them with the dozens of related eigenproblems of each
// DFT self-consistency cycle).  A small MLP (n_in -> 256 -> 256 -> n_out,
// ReLU) reads the previous two problems' eigenvalues and the overlaps of
// their eigenvectors and predicts, per wanted pair, how far to extrapolate
// the eigenvector along the sequence; the extrapolated block builds the next
// solve's start vector, and the solver's residual test alone decides
// acceptance.
//
// Every GEMM of the network's forward and backward pass runs on the bf16
// tensor cores (tcgen05.mma kind::f16, fp32 accumulation in TMEM).  The
// matrices are small (at most 256 x 256 x 256), so one CTA of 128 threads
// computes a 128 x N (N <= 256) tile: the threads round the fp32 operands
// to bf16 into the no-swizzle K-major core-matrix layout in shared memory
// (any strides, so transposed products need no copies), one thread issues
// the K/16 MMAs, and the four warps read their 32 TMEM lanes back for the
// epilogue (bias, ReLU, or a ReLU mask for back-propagation).  Parameters,
// Adam moments and gradients stay fp32.
//
// Layout of the packed parameters: W1 (H x n_in, row-major), b1 (H), W2
// (H x H), b2 (H), W3 (n_out x H), b3 (n_out).
#include <cuda_bf16.h>

#include "common.cuh"

namespace gs {
namespace {

constexpr int MT = 128;        // rows of a tile (the MMA's M)
constexpr int MAXN = 256;      // columns of a tile (the MMA's N, TMEM columns)
constexpr int MAXK = 256;      // reduction length held in shared memory
constexpr int MLP_THREADS = 128;
constexpr uint32_t SPIN = 1u << 24;

__device__ __forceinline__ uint32_t sptr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool bar_wait(uint64_t *bar, uint32_t parity) {
  for (uint32_t it = 0; it < SPIN; it++) {
    uint32_t done;
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

// shared-memory matrix descriptor: no swizzle, K-major core matrices of 8
// rows x 16 bytes, K-adjacent cores `lbo` bytes apart, row-adjacent `sbo`
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((256u >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// kind::f16 instruction descriptor: bf16 A and B, fp32 D, both K-major, M = 128
__device__ __forceinline__ uint32_t idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(MT >> 4) << 24);
}

// byte offset of element (r, k) in a tile of `rows` rows: k16 blocks of
// rows x 16, each an array of 8 x 8 core matrices (row groups 256 B apart,
// the two K halves 128 B apart)
__device__ __forceinline__ uint32_t tile_off(int r, int k, int rows) {
  return (uint32_t)((k >> 4) * (rows * 32) + (r >> 3) * 256 + ((k >> 3) & 1) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

enum Epi { EPI_NONE = 0, EPI_RELU = 1, EPI_MASK = 2 };

// D(m, n) = epi( sum_k A(m, k) B(n, k) + bias(n) ), with A(m, k) =
// A[m sam + k sak] and B(n, k) = B[n sbn + k sbk] rounded to bf16 (round to
// nearest even); EPI_MASK multiplies by (mask(m, n) > 0), mask laid out as
// D.  Tile: rows blockIdx.x * 128 .., all N <= 256 columns; K <= 256.
__global__ void __launch_bounds__(MLP_THREADS) k_mlp_gemm(int M, int N, int K, const float *__restrict__ A, int64_t sam,
                                                          int64_t sak, const float *__restrict__ B, int64_t sbn,
                                                          int64_t sbk, const float *__restrict__ bias, int epi,
                                                          const float *__restrict__ mask, float *__restrict__ D,
                                                          int64_t ldd, int *err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tslot;
  const int Kp = (K + 15) & ~15, Np = (N + 15) & ~15;
  unsigned char *sa = smem, *sb = smem + MT * Kp * 2;
  const int m0 = blockIdx.x * MT;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(sptr(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(sptr(&tslot)), "r"(MAXN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  // operands to bf16 in the core-matrix layout (zero padding)
  for (int idx = t; idx < MT * Kp; idx += MLP_THREADS) {
    const int r = idx / Kp, k = idx % Kp;
    const float v = (m0 + r < M && k < K) ? A[(int64_t)(m0 + r) * sam + (int64_t)k * sak] : 0.f;
    *reinterpret_cast<__nv_bfloat16 *>(sa + tile_off(r, k, MT)) = __float2bfloat16_rn(v);
  }
  for (int idx = t; idx < Np * Kp; idx += MLP_THREADS) {
    const int r = idx / Kp, k = idx % Kp;
    const float v = (r < N && k < K) ? B[(int64_t)r * sbn + (int64_t)k * sbk] : 0.f;
    *reinterpret_cast<__nv_bfloat16 *>(sb + tile_off(r, k, Np)) = __float2bfloat16_rn(v);
  }
  // the tensor core reads shared memory through the async proxy
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tslot;
  if (t == 0) {
    const uint32_t id = idesc(Np);
    for (int kb = 0; kb < Kp / 16; kb++) {
      const uint64_t ad = sdesc(sptr(sa + kb * MT * 32)), bd = sdesc(sptr(sb + kb * Np * 32));
      asm volatile(
          "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
          " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
          "l"(ad), "l"(bd), "r"(id), "r"(kb > 0 ? 1u : 0u));
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(sptr(&bar))
                 : "memory");
  }
  bool ok = bar_wait(&bar, 0);
  ok = __all_sync(0xffffffffu, ok);
  if (!ok) {
    // the MMAs may still run: record the fault, wait once more (bounded),
    // and never read the accumulator
    if (lane == 0) atomicExch(err, 1);
    bar_wait(&bar, 0);
  }
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (ok) {
    const int row = m0 + warp * 32 + lane;
    for (int c0 = 0; c0 < Np; c0 += 8) {
      uint32_t v[8];
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                   : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                   : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
      for (int c = 0; c < 8; c++) {
        asm volatile("" : "+r"(v[c]));
        const int col = c0 + c;
        if (row < M && col < N) {
          float x = __uint_as_float(v[c]) + (bias ? bias[col] : 0.f);
          if (epi == EPI_RELU) x = fmaxf(x, 0.f);
          else if (epi == EPI_MASK) x = (mask[(int64_t)row * ldd + col] > 0.f) ? x : 0.f;
          D[(int64_t)row * ldd + col] = x;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(MAXN));
}

// db(n) = sum over rows b of G(b, n) (G rows x cols, row-major)
__global__ void k_colsum(int rows, int cols, const float *__restrict__ G, float *__restrict__ db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= cols) return;
  float a = 0.f;
  for (int b = 0; b < rows; b++) a += G[(int64_t)b * cols + n];
  db[n] = a;
}

// MSE with per-output weights wo: loss = sum_{b,o} wo (Y - T)^2 / (2 batch);
// dY = wo (Y - T) / batch.  One CTA; loss into *loss.
__global__ void k_mse(int batch, int nout, const float *__restrict__ Y, const float *__restrict__ T,
                      const float *__restrict__ wo, float *__restrict__ dY, float *__restrict__ loss) {
  __shared__ float red[32];
  float acc = 0.f;
  for (int i = threadIdx.x; i < batch * nout; i += blockDim.x) {
    const int o = i % nout;
    const float w = wo ? wo[o] : 1.f;
    const float d = Y[i] - T[i];
    dY[i] = w * d / (float)batch;
    acc += w * d * d;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); i++) s += red[i];
    *loss = s / (2.f * (float)batch);
  }
}

// Adam (Kingma and Ba, 2015) with bias correction.
__global__ void k_adam(int64_t P, float *__restrict__ p, float *__restrict__ m, float *__restrict__ v,
                       const float *__restrict__ g, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// SplitMix64 (Steele, Lea, Flood 2014) on (seed, i) -> uniform [-1, 1)
__device__ __forceinline__ float u11(uint64_t seed, uint64_t i) {
  uint64_t x = seed * 0x9E3779B97F4A7C15ull + i + 0x632BE59BD9B4E019ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  x ^= x >> 31;
  return (float)((double)(x >> 11) * 0x1p-52 - 1.0);
}

// weights uniform in +-sqrt(6 / fan_in) (He et al. 2015 for ReLU layers), biases 0
__global__ void k_mlp_init(int nin, int H, int nout, uint64_t seed, float *__restrict__ p) {
  const int64_t w1 = (int64_t)H * nin, w2 = (int64_t)H * H, w3 = (int64_t)nout * H;
  const int64_t P = w1 + H + w2 + H + w3 + nout;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t j = i;
    float v = 0.f;
    if (j < w1) v = u11(seed, i) * sqrtf(6.f / nin);
    else if ((j -= w1) < H) v = 0.f;
    else if ((j -= H) < w2) v = u11(seed, i) * sqrtf(6.f / H);
    else if ((j -= w2) < H) v = 0.f;
    else if ((j -= H) < w3) v = u11(seed, i) * sqrtf(6.f / H);
    else v = 0.f;
    p[i] = v;
  }
}

// Alignment of two sets of eigenvectors through their overlaps P (s x s,
// P[j, i] = x_j^T B y_i): out_j = sgn_j y_{pi_j} - x_j with pi_j the best
// match of x_j among the y and sgn_j the sign of that overlap; columns whose
// best |overlap| is below 1/2 (a crossing) get out_j = 0.  match[j] (may be
// NULL) = the best |overlap|.
__global__ void k_ws_align(int64_t n, int s, const double *__restrict__ X, int64_t ldx, const double *__restrict__ Y,
                           int64_t ldy, const double *__restrict__ P, int64_t ldp, double *__restrict__ out,
                           int64_t ldo, float *__restrict__ match) {
  const int j = blockIdx.y;
  __shared__ int pi;
  __shared__ double sg;
  if (threadIdx.x == 0) {
    int bi = 0;
    double bv = -1.0;
    for (int i = 0; i < s; i++) {
      const double v = fabs(P[j + (int64_t)i * ldp]);
      if (v > bv) {
        bv = v;
        bi = i;
      }
    }
    pi = bi;
    sg = (bv >= 0.5) ? (P[j + (int64_t)bi * ldp] >= 0.0 ? 1.0 : -1.0) : 0.0;
    if (match && blockIdx.x == 0) match[j] = (float)bv;
  }
  __syncthreads();
  const double *y = Y + (int64_t)pi * ldy, *x = X + (int64_t)j * ldx;
  double *o = out + (int64_t)j * ldo;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    o[i] = (sg != 0.0) ? sg * y[i] - x[i] : 0.0;
}

// targets t_j = clamp(-(D_j . BE_j) / (D_j . BD_j), lo, hi) (0 where D_j = 0)
__global__ void k_ws_coef(int64_t n, int s, const double *__restrict__ D, int64_t ldd, const double *__restrict__ BD,
                          int64_t ldbd, const double *__restrict__ BE, int64_t ldbe, double lo, double hi,
                          float *__restrict__ t) {
  __shared__ double r1[32], r2[32];
  const int j = blockIdx.x;
  double a = 0.0, b = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double d = D[i + (int64_t)j * ldd];
    a = fma(d, BE[i + (int64_t)j * ldbe], a);
    b = fma(d, BD[i + (int64_t)j * ldbd], b);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    r1[threadIdx.x >> 5] = a;
    r2[threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double num = 0.0, den = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) {
      num += r1[k];
      den += r2[k];
    }
    t[j] = (den > 0.0) ? (float)fmin(hi, fmax(lo, -num / den)) : 0.f;
  }
}

// out_j = X_j - clamp(c_j, lo, hi) D_j (the extrapolated start block)
__global__ void k_ws_extrapolate(int64_t n, int s, const double *__restrict__ X, int64_t ldx,
                                 const double *__restrict__ D, int64_t ldd, const float *__restrict__ c, double lo,
                                 double hi, double *__restrict__ out, int64_t ldo) {
  const int j = blockIdx.y;
  const double cj = fmin(hi, fmax(lo, (double)c[j]));
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i + (int64_t)j * ldo] = X[i + (int64_t)j * ldx] - cj * D[i + (int64_t)j * ldd];
}

// the extrapolation coefficient of the smallest eigenvalue along the
// sequence: t = clamp((l(t) - l(t-1)) / (l(t-1) - l(t-2)), lo, hi), 0 when
// the previous step did not move it
__global__ void k_ws_shift_target(const double *w2, const double *w1, const double *w, double lo, double hi,
                                  float *t) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double d = w1[0] - w2[0];
  const double c = (fabs(d) > 0.0) ? (w[0] - w1[0]) / d : 0.0;
  t[0] = (float)fmin(fmax(c, lo), hi);
}

// shift = l(t-1) + clamp(c, lo, hi) (l(t-1) - l(t-2)) - frac (l_s(t-1) - l(t-1)) / s
// (c = 0 without a coefficient): below the predicted smallest eigenvalue by a
// fraction of the mean spacing of the wanted ones
__global__ void k_ws_shift(int s, const double *w2, const double *w1, const float *coef, double lo, double hi,
                           double frac, double *shift) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double c = coef ? fmin(fmax((double)coef[0], lo), hi) : 0.0;
  const double step = w2 ? w1[0] - w2[0] : 0.0;
  shift[0] = w1[0] + c * step - frac * (w1[s - 1] - w1[0]) / (double)s;
}

// Features of the problem at step t for the next one: with g the mean
// spacing of theta(t) (s ascending Ritz values), f_j = (theta_j(t) -
// theta_s(t)) / g, f_{s+j} = (theta_j(t) - theta_j(t-1)) / g, f_{2s} =
// dt / dt_ref.  Also writes scal[0] = theta_s(t), scal[1] = g.
__global__ void k_ws_features(int s, const double *__restrict__ th, const double *__restrict__ thp, double dt_rel,
                              float *__restrict__ f, double *__restrict__ scal) {
  const double top = th[s - 1];
  const double g = (s > 1) ? fmax((th[s - 1] - th[0]) / (double)(s - 1), 1e-300) : fmax(fabs(top), 1e-300);
  for (int j = threadIdx.x; j < s; j += blockDim.x) {
    f[j] = (float)((th[j] - top) / g);
    f[s + j] = (float)((th[j] - thp[j]) / g);
  }
  if (threadIdx.x == 0) {
    f[2 * s] = (float)dt_rel;
    scal[0] = top;
    scal[1] = g;
  }
}



int mlp_gemm(cudaStream_t st, int M, int N, int K, const float *A, int64_t sam, int64_t sak, const float *B,
             int64_t sbn, int64_t sbk, const float *bias, int epi, const float *mask, float *D, int64_t ldd, int *err) {
  if (M <= 0 || N <= 0 || N > MAXN || K <= 0 || K > MAXK) return GSYEIG_NOT_SUPPORTED;
  GS_TRY(set_max_smem((const void *)k_mlp_gemm, (MT + MAXN) * MAXK * 2));
  const int Kp = (K + 15) & ~15, Np = (N + 15) & ~15;
  const size_t smem = (size_t)(MT + Np) * Kp * 2;
  k_mlp_gemm<<<(unsigned)ceil_div(M, MT), MLP_THREADS, smem, st>>>(M, N, K, A, sam, sak, B, sbn, sbk, bias, epi, mask,
                                                                   D, ldd, err);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

struct Net {
  int nin, H, nout;
  const float *W1, *b1, *W2, *b2, *W3, *b3;
};

Net net_of(const float *p, int nin, int H, int nout) {
  Net n{nin, H, nout};
  n.W1 = p;
  n.b1 = n.W1 + (int64_t)H * nin;
  n.W2 = n.b1 + H;
  n.b2 = n.W2 + (int64_t)H * H;
  n.W3 = n.b2 + H;
  n.b3 = n.W3 + (int64_t)nout * H;
  return n;
}

bool dims_ok(int nin, int H, int nout) {
  return nin >= 1 && nin <= MAXK && H >= 16 && H <= MAXN && H % 16 == 0 && nout >= 1 && nout <= MAXN;
}

// workspace: H1, H2 (batch x H), Y (batch x nout), then for back-propagation
// dY (batch x nout), dZ2, dZ1 (batch x H), the loss and the fault flag
struct Ws {
  float *H1, *H2, *Y, *dY, *dZ2, *dZ1, *loss;
  int *err;
};
Ws ws_of(float *w, int H, int nout, int64_t batch) {
  Ws s;
  s.H1 = w;
  s.H2 = s.H1 + batch * H;
  s.Y = s.H2 + batch * H;
  s.dY = s.Y + batch * nout;
  s.dZ2 = s.dY + batch * nout;
  s.dZ1 = s.dZ2 + batch * H;
  s.loss = s.dZ1 + batch * H;
  s.err = reinterpret_cast<int *>(s.loss + 4);
  return s;
}

int forward(cudaStream_t st, const Net &n, const float *X, int batch, const Ws &w, float *Y) {
  // H1 = relu(X W1^T + b1), H2 = relu(H1 W2^T + b2), Y = H2 W3^T + b3
  GS_TRY(mlp_gemm(st, batch, n.H, n.nin, X, n.nin, 1, n.W1, n.nin, 1, n.b1, EPI_RELU, nullptr, w.H1, n.H, w.err));
  GS_TRY(mlp_gemm(st, batch, n.H, n.H, w.H1, n.H, 1, n.W2, n.H, 1, n.b2, EPI_RELU, nullptr, w.H2, n.H, w.err));
  GS_TRY(mlp_gemm(st, batch, n.nout, n.H, w.H2, n.H, 1, n.W3, n.H, 1, n.b3, EPI_NONE, nullptr, Y, n.nout, w.err));
  return GSYEIG_SUCCESS;
}

int fault_status(cudaStream_t st, const int *err) {
  int e = 0;
  GS_CUDA(cudaMemcpyAsync(&e, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  GS_CUDA(cudaStreamSynchronize(st));
  GS_CUDA(cudaGetLastError());
  return e ? GSYEIG_TIMEOUT : GSYEIG_SUCCESS;
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" {

int64_t gsyeig_mlp_param_count(int32_t n_in, int32_t n_hidden, int32_t n_out) {
  if (!dims_ok(n_in, n_hidden, n_out)) return -1;
  const int64_t H = n_hidden;
  return H * n_in + H + H * H + H + (int64_t)n_out * H + n_out;
}

int64_t gsyeig_mlp_workspace_floats(int32_t n_in, int32_t n_hidden, int32_t n_out, int64_t batch) {
  if (!dims_ok(n_in, n_hidden, n_out) || batch < 1) return -1;
  return batch * (4 * (int64_t)n_hidden + 2 * n_out) + 8;
}

int gsyeig_mlp_init(float *params, int32_t n_in, int32_t n_hidden, int32_t n_out, uint64_t seed, void *stream) {
  if (!params) return -1;
  if (!dims_ok(n_in, n_hidden, n_out)) return -2;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_mlp_init<<<256, 256, 0, st>>>(n_in, n_hidden, n_out, seed, params);
  count_launch();
  GS_CHECK_LAUNCH();
  GS_CUDA(cudaStreamSynchronize(st));
  return GSYEIG_SUCCESS;
}

int gsyeig_mlp_forward(const float *params, int32_t n_in, int32_t n_hidden, int32_t n_out, const float *X,
                       int64_t batch, float *Y, float *ws, void *stream) {
  if (!params) return -1;
  if (!dims_ok(n_in, n_hidden, n_out)) return -2;
  if (!X) return -5;
  if (batch < 1 || batch > (1 << 20)) return -6;
  if (!Y) return -7;
  if (!ws) return -8;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const Net n = net_of(params, n_in, n_hidden, n_out);
  const Ws w = ws_of(ws, n_hidden, n_out, batch);
  GS_CUDA(cudaMemsetAsync(w.err, 0, sizeof(int), st));
  GS_TRY(forward(st, n, X, (int)batch, w, Y));
  return fault_status(st, w.err);
}

int gsyeig_mlp_grad(const float *params, int32_t n_in, int32_t n_hidden, int32_t n_out, const float *X,
                    const float *T, const float *out_weights, int64_t batch, float *grad, float *loss, float *ws,
                    void *stream) {
  if (!params) return -1;
  if (!dims_ok(n_in, n_hidden, n_out)) return -2;
  if (!X) return -5;
  if (!T) return -6;
  if (batch < 1 || batch > MAXK) return -8;
  if (!grad) return -9;
  if (!ws) return -11;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int H = n_hidden, B = (int)batch;
  const Net n = net_of(params, n_in, H, n_out);
  const Ws w = ws_of(ws, H, n_out, batch);
  float *gW1 = grad, *gb1 = gW1 + (int64_t)H * n_in, *gW2 = gb1 + H, *gb2 = gW2 + (int64_t)H * H, *gW3 = gb2 + H,
        *gb3 = gW3 + (int64_t)n_out * H;
  GS_CUDA(cudaMemsetAsync(w.err, 0, sizeof(int), st));
  GS_TRY(forward(st, n, X, B, w, w.Y));
  k_mse<<<1, 256, 0, st>>>(B, n_out, w.Y, T, out_weights, w.dY, w.loss);
  count_launch();
  GS_CHECK_LAUNCH();
  // layer 3: dW3 = dY^T H2, db3 = sum_b dY, dZ2 = (dY W3) * (H2 > 0)
  GS_TRY(mlp_gemm(st, n_out, H, B, w.dY, 1, n_out, w.H2, 1, H, nullptr, EPI_NONE, nullptr, gW3, H, w.err));
  k_colsum<<<(unsigned)ceil_div(n_out, 128), 128, 0, st>>>(B, n_out, w.dY, gb3);
  GS_TRY(mlp_gemm(st, B, H, n_out, w.dY, n_out, 1, n.W3, 1, H, nullptr, EPI_MASK, w.H2, w.dZ2, H, w.err));
  // layer 2: dW2 = dZ2^T H1, db2, dZ1 = (dZ2 W2) * (H1 > 0)
  GS_TRY(mlp_gemm(st, H, H, B, w.dZ2, 1, H, w.H1, 1, H, nullptr, EPI_NONE, nullptr, gW2, H, w.err));
  k_colsum<<<(unsigned)ceil_div(H, 128), 128, 0, st>>>(B, H, w.dZ2, gb2);
  GS_TRY(mlp_gemm(st, B, H, H, w.dZ2, H, 1, n.W2, 1, H, nullptr, EPI_MASK, w.H1, w.dZ1, H, w.err));
  // layer 1: dW1 = dZ1^T X, db1
  GS_TRY(mlp_gemm(st, H, n_in, B, w.dZ1, 1, H, X, 1, n_in, nullptr, EPI_NONE, nullptr, gW1, n_in, w.err));
  k_colsum<<<(unsigned)ceil_div(H, 128), 128, 0, st>>>(B, H, w.dZ1, gb1);
  count_launch(3);
  GS_CHECK_LAUNCH();
  if (loss) GS_CUDA(cudaMemcpyAsync(loss, w.loss, sizeof(float), cudaMemcpyDeviceToDevice, st));
  return fault_status(st, w.err);
}

int gsyeig_mlp_adam(float *params, float *m, float *v, const float *grad, int64_t count, int64_t step, float lr,
                    float beta1, float beta2, float eps, void *stream) {
  if (!params) return -1;
  if (!m) return -2;
  if (!v) return -3;
  if (!grad) return -4;
  if (count < 1) return -5;
  if (step < 1) return -6;
  if (!(lr > 0.f)) return -7;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  k_adam<<<(unsigned)std::min<int64_t>(ceil_div(count, 256), 1024), 256, 0, st>>>(count, params, m, v, grad, lr, beta1,
                                                                                  beta2, eps, c1, c2);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

int gsyeig_ws_features(int64_t s, const double *theta, const double *theta_prev, double dt_rel, float *features,
                       double *scal, void *stream) {
  if (s < 1 || s > 4096) return -1;
  if (!theta) return -2;
  if (!theta_prev) return -3;
  if (!features) return -5;
  if (!scal) return -6;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_ws_features<<<1, 256, 0, st>>>((int)s, theta, theta_prev, dt_rel, features, scal);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

int gsyeig_ws_align(int64_t n, int64_t s, const double *X, int64_t ldx, const double *Y, int64_t ldy, const double *P,
                    int64_t ldp, double *out, int64_t ldo, float *match, void *stream) {
  if (n < 1) return -1;
  if (s < 1 || s > 4096) return -2;
  if (!X || ldx < n) return -3;
  if (!Y || ldy < n) return -5;
  if (!P || ldp < s) return -7;
  if (!out || ldo < n) return -9;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_ws_align<<<dim3((unsigned)std::min<int64_t>(ceil_div(n, 256), 64), (unsigned)s), 256, 0, st>>>(
      n, (int)s, X, ldx, Y, ldy, P, ldp, out, ldo, match);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

int gsyeig_ws_coef_targets(int64_t n, int64_t s, const double *D, int64_t ldd, const double *BD, int64_t ldbd,
                           const double *BE, int64_t ldbe, double lo, double hi, float *targets, void *stream) {
  if (n < 1) return -1;
  if (s < 1 || s > 4096) return -2;
  if (!D || !BD || !BE) return -3;
  if (!targets) return -11;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_ws_coef<<<(unsigned)s, 256, 0, st>>>(n, (int)s, D, ldd, BD, ldbd, BE, ldbe, lo, hi, targets);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

int gsyeig_ws_extrapolate(int64_t n, int64_t s, const double *X, int64_t ldx, const double *D, int64_t ldd,
                          const float *coef, double lo, double hi, double *out, int64_t ldo, void *stream) {
  if (n < 1) return -1;
  if (s < 1 || s > 4096) return -2;
  if (!X || ldx < n) return -3;
  if (!D || ldd < n) return -5;
  if (!coef) return -7;
  if (!out || ldo < n) return -10;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_ws_extrapolate<<<dim3((unsigned)std::min<int64_t>(ceil_div(n, 256), 64), (unsigned)s), 256, 0, st>>>(
      n, (int)s, X, ldx, D, ldd, coef, lo, hi, out, ldo);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

int gsyeig_ws_shift_target(const double *w_prev2, const double *w_prev, const double *w, double lo, double hi,
                           float *target, void *stream) {
  if (!w_prev2 || !w_prev || !w) return -1;
  if (!target) return -6;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_ws_shift_target<<<1, 32, 0, st>>>(w_prev2, w_prev, w, lo, hi, target);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

int gsyeig_ws_shift(int64_t s, const double *w_prev2, const double *w_prev, const float *coef, double lo, double hi,
                    double frac, double *shift, void *stream) {
  if (s < 2 || s > 4096) return -1;
  if (!w_prev) return -3;
  if (!shift) return -8;
  if (coef && !w_prev2) return -2;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_ws_shift<<<1, 32, 0, st>>>((int)s, w_prev2, w_prev, coef, lo, hi, frac, shift);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

}  // extern "C"
