// ke2 (Table 1): the Lanczos recurrence with full reorthogonalisation
// (Section 2.3).  Each step j turns z = C v_j into v_{j+1}:
//
//   h1 = V_j^T z,  z -= V_j h1          classical Gram-Schmidt against all of
//   h2 = V_j^T z,  z -= V_j h2          V_j = [v_0..v_j], done twice ("twice
//                                        is enough", Kahan / Giraud et al.)
//   alpha_j = h1[j] + h2[j],  beta_j = ||z||,  v_{j+1} = z / beta_j
//
// The coefficients h1[i], h2[i] for i < j are roundoff and are dropped, so
// T_m stays tridiagonal.  Everything stays on the device: the reductions
// are deterministic two-level sums (no atomics), scalars live in device
// memory, and a breakdown (beta_j ~ 0) is flagged for the host.
#include "common.cuh"
#include "lanczos.cuh"

namespace gs {
namespace {

constexpr int DOT_THREADS = 256;
constexpr int SUB_ROWS = 64, SUB_GROUPS = 4;  // 256 threads: 64 rows x 4 column groups

__device__ __forceinline__ double block_sum(double v, double *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); i++) s += red[i];
  return s;  // valid in thread 0 only
}

// h[c] = V[:, c] . z for c < ncols; one CTA per column.
__global__ void __launch_bounds__(DOT_THREADS) k_dots(int64_t n, int64_t ncols, const double *__restrict__ V,
                                                     int64_t ldv, const double *__restrict__ z, double *__restrict__ h) {
  __shared__ double red[DOT_THREADS / 32];
  const int64_t c = blockIdx.x;
  if (c >= ncols) return;
  const double *v = V + (size_t)c * ldv;
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += DOT_THREADS) acc = fma(v[i], z[i], acc);
  double s = block_sum(acc, red);
  if (threadIdx.x == 0) h[c] = s;
}

// z -= V[:, 0:ncols] h for a 64-row slice per CTA; the four column groups
// of a CTA combine in shared memory.  If sq != nullptr the CTA also writes
// the sum of squares of its updated slice to sq[blockIdx.x].
__global__ void __launch_bounds__(SUB_ROWS *SUB_GROUPS) k_sub(int64_t n, int64_t ncols, const double *__restrict__ V,
                                                             int64_t ldv, const double *__restrict__ h,
                                                             double *__restrict__ z, double *__restrict__ sq) {
  extern __shared__ double hs[];  // ncols coefficients
  __shared__ double part[SUB_GROUPS][SUB_ROWS];
  __shared__ double red[SUB_ROWS * SUB_GROUPS / 32];
  for (int64_t c = threadIdx.x; c < ncols; c += blockDim.x) hs[c] = h[c];
  __syncthreads();
  const int r = threadIdx.x % SUB_ROWS, g = threadIdx.x / SUB_ROWS;
  const int64_t i = (int64_t)blockIdx.x * SUB_ROWS + r;
  double acc = 0.0;
  if (i < n)
    for (int64_t c = g; c < ncols; c += SUB_GROUPS) acc = fma(V[(size_t)c * ldv + i], hs[c], acc);
  part[g][r] = acc;
  __syncthreads();
  double zi = 0.0;
  if (g == 0 && i < n) {
    double t = (part[0][r] + part[1][r]) + (part[2][r] + part[3][r]);
    zi = z[i] - t;
    z[i] = zi;
  }
  if (sq) {
    double s = block_sum(zi * zi, red);
    if (threadIdx.x == 0) sq[blockIdx.x] = s;
  }
}

// sum of squares of z, per 64-row slice (same slicing as k_sub)
__global__ void __launch_bounds__(SUB_ROWS *SUB_GROUPS) k_sumsq(int64_t n, const double *__restrict__ z,
                                                               double *__restrict__ sq) {
  __shared__ double red[SUB_ROWS * SUB_GROUPS / 32];
  const int64_t i = (int64_t)blockIdx.x * SUB_ROWS + threadIdx.x;
  double zi = (threadIdx.x < SUB_ROWS && i < n) ? z[i] : 0.0;
  double s = block_sum(zi * zi, red);
  if (threadIdx.x == 0) sq[blockIdx.x] = s;
}

// Finish step j: alpha_j, beta_j, breakdown test, 1/beta_j for the scaling.
__global__ void k_finalize(int64_t j, int64_t m, const double *h1, const double *h2, const double *sq, int nparts,
                           double *alpha, double *beta, LanczosState *state) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += sq[i];
  double ss = block_sum(acc, red);
  if (threadIdx.x != 0) return;
  double a = h1[j] + h2[j];
  double b = sqrt(ss);
  double prev = (j > 0) ? fabs(beta[j - 1]) : 0.0;
  double tn = fmax(state->tnorm, fabs(a) + b + prev);
  state->tnorm = tn;
  alpha[j] = a;
  bool bad = (j < m - 1) && !(b > 1e-13 * tn);
  if (state->breakdown_at >= 0 && state->breakdown_at <= j) bad = true;  // earlier breakdown in this pass
  if (bad) {
    if (state->breakdown_at < 0) state->breakdown_at = j;
    beta[j] = 0.0;
    state->inv_beta = 0.0;
  } else {
    beta[j] = b;
    state->inv_beta = (b > 0.0) ? 1.0 / b : 0.0;
  }
}

__global__ void k_scale_into(int64_t n, const double *__restrict__ z, double *__restrict__ out,
                             const LanczosState *state) {
  const double s = state->inv_beta;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = z[i] * s;
}

// Norm from slice partials into state->inv_beta and *norm_out (optional).
__global__ void k_norm_finish(const double *sq, int nparts, LanczosState *state, double *norm_out) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += sq[i];
  double ss = block_sum(acc, red);
  if (threadIdx.x != 0) return;
  double b = sqrt(ss);
  state->inv_beta = (b > 0.0) ? 1.0 / b : 0.0;
  if (norm_out) *norm_out = b;
}

// Counter-based uniform(-1/2, 1/2) vector: SplitMix64 (Steele, Lea, Flood,
// OOPSLA 2014) applied to (seed, stream, i).
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

__global__ void k_random(int64_t n, uint64_t seed, uint64_t stream, double *v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t r = splitmix64(splitmix64(seed ^ (stream * 0xD1B54A32D192ED03ull)) + (uint64_t)i);
    v[i] = (double)(r >> 11) * 0x1p-53 - 0.5;
  }
}

// Restart residual: f = Vq[:, k] * betaP[k-1] + vm * beta_m * Q[m-1, k-1]
__global__ void k_restart_residual(int64_t n, int64_t k, int64_t m, const double *__restrict__ Vq, int64_t ldvq,
                                   const double *__restrict__ vm, const double *betaP, const double *beta,
                                   const double *Q, int64_t ldq, double *__restrict__ f) {
  const double c1 = betaP[k - 1];
  const double c2 = beta[m - 1] * Q[(m - 1) + (size_t)(k - 1) * ldq];
  const double *vk = Vq + (size_t)k * ldvq;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    f[i] = vk[i] * c1 + vm[i] * c2;
}

__global__ void k_thick_restart(int64_t m, int64_t k, const double *theta, const double *S, double *d, double *e,
                                double *b) {
  const double bm = e[m - 1];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x) {
    b[i] = bm * S[(m - 1) + (size_t)i * m];
    d[i] = theta[i];
  }
}

__global__ void k_zero(int64_t n, double *p) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = 0.0;
}

unsigned grid1d(int64_t n, int threads) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, threads), 152 * 8)); }

// Column pairs (i, s-1-i) of X swapped and scaled by 1/sqrt(mu); theta read only.
__global__ void k_invert_cols(int64_t n, int64_t s, const double *__restrict__ theta, double *X, int64_t ldx) {
  const int64_t half = (s + 1) / 2;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n * half;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx % n, i = idx / n, k = s - 1 - i;
    const double a = X[GS_IDX(r, i, ldx)], b = X[GS_IDX(r, k, ldx)];
    X[GS_IDX(r, i, ldx)] = b / sqrt(theta[k]);
    if (k != i) X[GS_IDX(r, k, ldx)] = a / sqrt(theta[i]);
  }
}

// theta[i] <- 1 / theta[s-1-i] (one thread per pair)
// theta (mu ascending) <- shift + 1/mu, ascending
__global__ void k_invert_vals(int64_t s, double *theta, double shift) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (s + 1) / 2; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = s - 1 - i;
    const double a = theta[i], b = theta[k];
    theta[i] = shift + 1.0 / b;
    theta[k] = shift + 1.0 / a;
  }
}

// A(i, j) -= shift B(i, j) for i <= j (the upper triangles)
__global__ void k_shift_upper(int64_t n, double *__restrict__ A, int64_t lda, const double *__restrict__ B,
                              int64_t ldb, double shift) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n * n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % n, j = idx / n;
    if (i <= j) A[i + j * lda] = fma(-shift, B[i + j * ldb], A[i + j * lda]);
  }
}

__global__ void k_weighted_sum(int64_t n, int64_t k, const double *__restrict__ X, int64_t ldx,
                               const double *__restrict__ w, double *__restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int64_t c = 0; c < k; c++) acc = fma(X[(size_t)c * ldx + i], w ? w[c] : 1.0, acc);
    out[i] = acc;
  }
}

// row i of U v over columns j >= i; lanes of a warp take consecutive rows,
// so every column's reads are coalesced
__global__ void k_trmv_upper(int64_t n, const double *__restrict__ U, int64_t ldu, const double *__restrict__ v,
                             double *__restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int64_t j = i; j < n; j++) acc = fma(U[i + (size_t)j * ldu], v[j], acc);
    out[i] = acc;
  }
}

__global__ void k_cheb_step(int64_t n, const double *__restrict__ Cy, const double *__restrict__ y,
                            const double *yprev, double c, double inv_e, int first, double *out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double t = (Cy[i] - c * y[i]) * inv_e;
    out[i] = first ? t : 2.0 * t - yprev[i];
  }
}

}  // namespace

int lz_weighted_sum(cudaStream_t st, int64_t n, int64_t k, const double *X, int64_t ldx, const double *w,
                    double *out) {
  k_weighted_sum<<<grid1d(n, 256), 256, 0, st>>>(n, k, X, ldx, w, out);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

int lz_trmv_upper(cudaStream_t st, int64_t n, const double *U, int64_t ldu, const double *v, double *out) {
  k_trmv_upper<<<(unsigned)ceil_div(n, 128), 128, 0, st>>>(n, U, ldu, v, out);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

int lz_cheb_step(cudaStream_t st, int64_t n, const double *Cy, const double *y, const double *yprev, double c,
                 double e, bool first, double *out) {
  k_cheb_step<<<grid1d(n, 256), 256, 0, st>>>(n, Cy, y, yprev, c, 1.0 / e, first ? 1 : 0, out);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

int lz_nparts(int64_t n) { return (int)ceil_div(n, SUB_ROWS); }

int lz_dots(cudaStream_t st, int64_t n, int64_t ncols, const double *V, int64_t ldv, const double *z, double *h) {
  if (ncols <= 0) return GSYEIG_SUCCESS;
  k_dots<<<(unsigned)ncols, DOT_THREADS, 0, st>>>(n, ncols, V, ldv, z, h);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

int lz_sub(cudaStream_t st, int64_t n, int64_t ncols, const double *V, int64_t ldv, const double *h, double *z,
           double *sq) {
  size_t smem = (size_t)std::max<int64_t>(ncols, 1) * sizeof(double);
  if (smem > 48 * 1024) GS_CUDA(cudaFuncSetAttribute((const void *)k_sub, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_sub<<<(unsigned)lz_nparts(n), SUB_ROWS * SUB_GROUPS, smem, st>>>(n, ncols, V, ldv, h, z, sq);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

int lz_cgs2(cudaStream_t st, int64_t n, int64_t ncols, const double *V, int64_t ldv, double *z, double *h1,
            double *h2, double *sq) {
  if (ncols > 0) {
    GS_TRY(lz_dots(st, n, ncols, V, ldv, z, h1));
    GS_TRY(lz_sub(st, n, ncols, V, ldv, h1, z, nullptr));
    GS_TRY(lz_dots(st, n, ncols, V, ldv, z, h2));
    GS_TRY(lz_sub(st, n, ncols, V, ldv, h2, z, sq));
  } else {
    k_sumsq<<<(unsigned)lz_nparts(n), SUB_ROWS * SUB_GROUPS, 0, st>>>(n, z, sq);
    count_launch();
    GS_CHECK_LAUNCH();
  }
  return GSYEIG_SUCCESS;
}

int lz_finalize(cudaStream_t st, int64_t j, int64_t m, const double *h1, const double *h2, const double *sq,
                int nparts, double *alpha, double *beta, LanczosState *state) {
  k_finalize<<<1, 256, 0, st>>>(j, m, h1, h2, sq, nparts, alpha, beta, state);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

int lz_invert_pairs(cudaStream_t st, int64_t n, int64_t s, double *theta, double *X, int64_t ldx, double shift) {
  k_invert_cols<<<grid1d(n * ((s + 1) / 2), 256), 256, 0, st>>>(n, s, theta, X, ldx);
  k_invert_vals<<<1, 128, 0, st>>>(s, theta, shift);
  count_launch(2);
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

int lz_shift_upper(cudaStream_t st, int64_t n, double *A, int64_t lda, const double *B, int64_t ldb, double shift) {
  k_shift_upper<<<grid1d(n * n, 256), 256, 0, st>>>(n, A, lda, B, ldb, shift);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

int lz_scale_into(cudaStream_t st, int64_t n, const double *z, double *out, const LanczosState *state) {
  k_scale_into<<<grid1d(n, 256), 256, 0, st>>>(n, z, out, state);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

int lz_norm_finish(cudaStream_t st, const double *sq, int nparts, LanczosState *state, double *norm_out) {
  k_norm_finish<<<1, 256, 0, st>>>(sq, nparts, state, norm_out);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

int lz_random(cudaStream_t st, int64_t n, uint64_t seed, uint64_t stream, double *v) {
  k_random<<<grid1d(n, 256), 256, 0, st>>>(n, seed, stream, v);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

int lz_thick_restart(cudaStream_t st, int64_t m, int64_t k, const double *theta, const double *S, double *d, double *e,
                     double *b) {
  // b and d first (they read e[m - 1]); the couplings e[0..k-1] are then cleared
  k_thick_restart<<<grid1d(k, 256), 256, 0, st>>>(m, k, theta, S, d, e, b);
  k_zero<<<grid1d(k, 256), 256, 0, st>>>(k, e);
  count_launch(2);
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

int lz_restart_residual(cudaStream_t st, int64_t n, int64_t k, int64_t m, const double *Vq, int64_t ldvq,
                        const double *vm, const double *betaP, const double *beta, const double *Q, int64_t ldq,
                        double *f) {
  k_restart_residual<<<grid1d(n, 256), 256, 0, st>>>(n, k, m, Vq, ldvq, vm, betaP, beta, Q, ldq, f);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

}  // namespace gs
