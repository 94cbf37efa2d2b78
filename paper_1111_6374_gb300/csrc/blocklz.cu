// FP64 kernels of the block Lanczos / block refinement stage (the
// mixed-precision route): tall-skinny products against the basis, residuals
// and column norms.  The basis products keep the reorthogonalisation in
// FP64 as the route prescribes; GB300's FP64 pipe bounds them, so they are
// spread over every SM: H = V^T Z splits the n rows into slices whose
// partial products are summed by a second kernel (deterministic, no
// atomics), and Z -= V H gives each thread one row.
#include "mixed.cuh"

namespace gs {
namespace {

constexpr int TSC = 32;       // basis columns per CTA of k_ts_dots
constexpr int TS_ROWS = 512;  // rows of a slice

// part[slice][c][q] = sum over the slice's rows i of V(i, c) Z(i, q), for
// the TSC columns c of this CTA and the b <= 16 columns q of Z.  32-row
// chunks of V and Z are staged in shared memory with coalesced loads (lanes
// along rows); thread (column lane, warp g) then sums rows g, g + 8, ...
__global__ void __launch_bounds__(256) k_ts_dots(int64_t n, int64_t w, int b, const double *__restrict__ V, int64_t ldv,
                                                 const double *__restrict__ Z, int64_t ldz, double *__restrict__ part) {
  __shared__ double vs[32][TSC + 1];
  __shared__ double zs[32][16];
  __shared__ double red[8][TSC][16];
  const int64_t c0 = (int64_t)blockIdx.x * TSC;
  const int64_t r0 = (int64_t)blockIdx.y * TS_ROWS;
  const int t = threadIdx.x, lane = t & 31, wp = t >> 5;
  double acc[16];
#pragma unroll
  for (int q = 0; q < 16; q++) acc[q] = 0.0;
  for (int64_t rb = r0; rb < r0 + TS_ROWS && rb < n; rb += 32) {
    __syncthreads();
    for (int cc = wp; cc < TSC; cc += 8) {  // lane = row: coalesced down each column
      const int64_t col = c0 + cc, row = rb + lane;
      vs[lane][cc] = (col < w && row < n) ? V[row + col * ldv] : 0.0;
    }
    for (int idx = t; idx < 32 * 16; idx += 256) {
      const int rr = idx % 32, q = idx / 32;
      zs[rr][q] = (rb + rr < n && q < b) ? Z[(rb + rr) + (int64_t)q * ldz] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int rr = wp; rr < 32; rr += 8) {
      const double v = vs[rr][lane];
#pragma unroll
      for (int q = 0; q < 16; q++) acc[q] = fma(v, zs[rr][q], acc[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < 16; q++) red[wp][lane][q] = acc[q];
  __syncthreads();
  for (int idx = t; idx < TSC * 16; idx += 256) {
    const int cc = idx / 16, q = idx % 16;
    double s = 0.0;
    for (int k = 0; k < 8; k++) s += red[k][cc][q];
    if (c0 + cc < w && q < b) part[((int64_t)blockIdx.y * w + c0 + cc) * 16 + q] = s;
  }
}

// H(c, q) (column-major, ld ldh) = sum over slices of part[slice][c][q]
__global__ void k_ts_reduce(int64_t w, int b, int nslice, const double *__restrict__ part, double *__restrict__ H,
                            int64_t ldh) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < w * b; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = idx / b;
    const int q = (int)(idx % b);
    double s = 0.0;
    for (int sl = 0; sl < nslice; sl++) s += part[((int64_t)sl * w + c) * 16 + q];
    H[c + q * ldh] = s;
  }
}

// Z(i, q) -= sum_c V(i, c) H(c, q): one thread per row, H staged in shared memory
__global__ void __launch_bounds__(128) k_ts_update(int64_t n, int64_t w, int b, const double *__restrict__ V,
                                                   int64_t ldv, const double *__restrict__ H, int64_t ldh,
                                                   double *__restrict__ Z, int64_t ldz) {
  extern __shared__ double hs[];  // w x 16
  for (int64_t idx = threadIdx.x; idx < w * 16; idx += blockDim.x) {
    const int64_t c = idx / 16;
    const int q = (int)(idx % 16);
    hs[idx] = (q < b) ? H[c + q * ldh] : 0.0;
  }
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc[16];
#pragma unroll
  for (int q = 0; q < 16; q++) acc[q] = 0.0;
  for (int64_t c = 0; c < w; c++) {
    const double v = V[i + c * ldv];
#pragma unroll
    for (int q = 0; q < 16; q++) acc[q] = fma(v, hs[c * 16 + q], acc[q]);
  }
  for (int q = 0; q < b; q++) Z[i + q * ldz] -= acc[q];
}

// norms[c] = ||X(:, c)||_2 (one CTA per column)
__global__ void k_colnorms(int64_t n, const double *__restrict__ X, int64_t ldx, double *__restrict__ norms) {
  __shared__ double red[32];
  const double *x = X + (int64_t)blockIdx.x * ldx;
  double a = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) a = fma(x[i], x[i], a);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) s += red[k];
    norms[blockIdx.x] = sqrt(s);
  }
}

// X(:, c) *= 1 / norms[c] (columns of zero norm left as they are)
__global__ void k_scale_cols(int64_t n, int64_t cols, double *__restrict__ X, int64_t ldx,
                             const double *__restrict__ norms) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n * cols;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % n, c = idx / n;
    const double nr = norms[c];
    if (nr > 0.0) X[i + c * ldx] /= nr;
  }
}

// R = CX - X diag(theta)
__global__ void k_block_resid(int64_t n, int64_t k, const double *__restrict__ CX, const double *__restrict__ X,
                              int64_t ld, const double *__restrict__ theta, double *__restrict__ R) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n * k;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % n, c = idx / n;
    R[i + c * ld] = CX[i + c * ld] - theta[c] * X[i + c * ld];
  }
}

// T(r0 + i, c0 + j) = M(i, j) for an m x m block (ld ldm); with mirror also
// T(c0 + j, r0 + i) = M(i, j)
__global__ void k_put_block(int m, const double *__restrict__ M, int64_t ldm, double *__restrict__ T, int64_t ldt,
                            int64_t r0, int64_t c0, int mirror) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < m * m; idx += gridDim.x * blockDim.x) {
    const int i = idx % m, j = idx / m;
    const double v = M[i + (int64_t)j * ldm];
    T[(r0 + i) + (c0 + j) * ldt] = v;
    if (mirror) T[(c0 + j) + (r0 + i) * ldt] = v;
  }
}

// T <- (T + T^T) / 2 (a square m x m, ld ldt)
__global__ void k_sym_avg(int64_t m, double *__restrict__ T, int64_t ldt) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < m * m;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % m, j = idx / m;
    if (i < j) {
      const double a = 0.5 * (T[i + j * ldt] + T[j + i * ldt]);
      T[i + j * ldt] = a;
      T[j + i * ldt] = a;
    }
  }
}

// out[0] = max_i sum_j |T(i, j)| (the infinity norm, an upper bound on |lambda| of T)
__global__ void k_inf_norm(int64_t m, const double *__restrict__ T, int64_t ldt, double *out) {
  __shared__ double red[32];
  double mx = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
    double a = 0.0;
    for (int64_t j = 0; j < m; j++) a += fabs(T[i + j * ldt]);
    mx = fmax(mx, a);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) v = fmax(v, red[k]);
    out[0] = v;
  }
}

// M1 + M2 (b x b, ld ldm) into T at (r0, r0)
__global__ void k_put_sum(int b, const double *__restrict__ M1, const double *__restrict__ M2, int64_t ldm,
                          double *__restrict__ T, int64_t ldt, int64_t r0) {
  for (int idx = threadIdx.x; idx < b * b; idx += blockDim.x) {
    const int i = idx % b, j = idx / b;
    T[(r0 + i) + (r0 + j) * ldt] = M1[i + (int64_t)j * ldm] + M2[i + (int64_t)j * ldm];
  }
}

// out[c] = X(:, c) . Y(:, c) (one CTA per column)
__global__ void k_coldots(int64_t n, const double *__restrict__ X, int64_t ldx, const double *__restrict__ Y,
                          int64_t ldy, double *__restrict__ out) {
  __shared__ double red[32];
  const double *x = X + (int64_t)blockIdx.x * ldx, *y = Y + (int64_t)blockIdx.x * ldy;
  double a = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) a = fma(x[i], y[i], a);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) s += red[k];
    out[blockIdx.x] = s;
  }
}

// dst = the upper triangle of src (zeros below the diagonal), b x b
__global__ void k_copy_upper(int64_t b, const double *__restrict__ src, int64_t lds, double *__restrict__ dst,
                             int64_t ldd) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < b * b;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % b, j = idx / b;
    dst[i + j * ldd] = (i <= j) ? src[i + j * lds] : 0.0;
  }
}

// dst(:, c) = src(:, idx[c]) for c < cnt
__global__ void k_gather_cols(int64_t n, int64_t cnt, const int *__restrict__ idx, const double *__restrict__ src,
                              int64_t lds, double *__restrict__ dst, int64_t ldd) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n * cnt; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = q % n, c = q / n;
    dst[i + c * ldd] = src[i + (int64_t)idx[c] * lds];
  }
}

// out[0] = max_c sum_i |M(i, c)| (the 1-norm; the infinity norm of a
// symmetric M), one CTA per column, combined by atomicMax on the bits of
// the non-negative sums; out[0] must start at 0
__global__ void k_norm1(int64_t n, const double *__restrict__ M, int64_t ldm, unsigned long long *out) {
  __shared__ double red[32];
  const double *col = M + (int64_t)blockIdx.x * ldm;
  double a = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) a += fabs(col[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) v += red[k];
    atomicMax(out, (unsigned long long)__double_as_longlong(v));
  }
}

// M(i, j) *= theta_i^pa theta_j^pb (m x m, theta > 0)
__global__ void k_scale_by_powers(int64_t m, double *__restrict__ M, int64_t ldm, const double *__restrict__ theta,
                                  double pa, double pb) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < m * m;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % m, j = idx / m;
    M[i + j * ldm] *= pow(theta[i], pa) * pow(theta[j], pb);
  }
}

unsigned g1(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), 4096)); }

}  // namespace

size_t ts_part_doubles(int64_t n, int64_t w) { return (size_t)ceil_div(n, TS_ROWS) * (size_t)w * 16; }

int ts_dots(cudaStream_t st, int64_t n, int64_t w, int b, const double *V, int64_t ldv, const double *Z, int64_t ldz,
            double *part, double *H, int64_t ldh) {
  if (w <= 0) return GSYEIG_SUCCESS;
  if (b < 1 || b > 16) return GSYEIG_NOT_SUPPORTED;
  const int nslice = (int)ceil_div(n, TS_ROWS);
  k_ts_dots<<<dim3((unsigned)ceil_div(w, TSC), (unsigned)nslice), 256, 0, st>>>(n, w, b, V, ldv, Z, ldz, part);
  k_ts_reduce<<<g1(w * b), 256, 0, st>>>(w, b, nslice, part, H, ldh);
  count_launch(2);
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

int ts_update(cudaStream_t st, int64_t n, int64_t w, int b, const double *V, int64_t ldv, const double *H, int64_t ldh,
              double *Z, int64_t ldz) {
  if (w <= 0) return GSYEIG_SUCCESS;
  if (b < 1 || b > 16) return GSYEIG_NOT_SUPPORTED;
  const size_t smem = (size_t)w * 16 * sizeof(double);
  if (smem > 200 * 1024) return GSYEIG_NOT_SUPPORTED;
  GS_TRY(set_max_smem((const void *)k_ts_update, 200 * 1024));
  k_ts_update<<<(unsigned)ceil_div(n, 128), 128, smem, st>>>(n, w, b, V, ldv, H, ldh, Z, ldz);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

int col_norms(cudaStream_t st, int64_t n, int64_t cols, const double *X, int64_t ldx, double *norms) {
  if (cols <= 0) return GSYEIG_SUCCESS;
  k_colnorms<<<(unsigned)cols, 256, 0, st>>>(n, X, ldx, norms);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

int scale_cols(cudaStream_t st, int64_t n, int64_t cols, double *X, int64_t ldx, const double *norms) {
  k_scale_cols<<<g1(n * cols), 256, 0, st>>>(n, cols, X, ldx, norms);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

int block_resid(cudaStream_t st, int64_t n, int64_t k, const double *CX, const double *X, int64_t ld,
                const double *theta, double *R) {
  k_block_resid<<<g1(n * k), 256, 0, st>>>(n, k, CX, X, ld, theta, R);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

int put_block(cudaStream_t st, int m, const double *M, int64_t ldm, double *T, int64_t ldt, int64_t r0, int64_t c0,
              bool mirror) {
  k_put_block<<<g1((int64_t)m * m), 256, 0, st>>>(m, M, ldm, T, ldt, r0, c0, mirror ? 1 : 0);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

int sym_avg(cudaStream_t st, int64_t m, double *T, int64_t ldt) {
  k_sym_avg<<<g1(m * m), 256, 0, st>>>(m, T, ldt);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

int inf_norm(cudaStream_t st, int64_t m, const double *T, int64_t ldt, double *out) {
  k_inf_norm<<<1, 256, 0, st>>>(m, T, ldt, out);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

int put_sum(cudaStream_t st, int b, const double *M1, const double *M2, int64_t ldm, double *T, int64_t ldt,
            int64_t r0) {
  k_put_sum<<<1, 256, 0, st>>>(b, M1, M2, ldm, T, ldt, r0);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

int column_dots(cudaStream_t st, int64_t n, int64_t cols, const double *X, int64_t ldx, const double *Y, int64_t ldy,
                double *out) {
  if (cols <= 0) return GSYEIG_SUCCESS;
  k_coldots<<<(unsigned)cols, 256, 0, st>>>(n, X, ldx, Y, ldy, out);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

int copy_upper(cudaStream_t st, int64_t b, const double *src, int64_t lds, double *dst, int64_t ldd) {
  k_copy_upper<<<g1(b * b), 256, 0, st>>>(b, src, lds, dst, ldd);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

int gather_cols(cudaStream_t st, int64_t n, int64_t cnt, const int *idx, const double *src, int64_t lds, double *dst,
                int64_t ldd) {
  if (cnt <= 0) return GSYEIG_SUCCESS;
  k_gather_cols<<<g1(n * cnt), 256, 0, st>>>(n, cnt, idx, src, lds, dst, ldd);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

int scale_by_powers(cudaStream_t st, int64_t m, double *M, int64_t ldm, const double *theta, double pa, double pb) {
  if (m <= 0) return GSYEIG_SUCCESS;
  k_scale_by_powers<<<g1(m * m), 256, 0, st>>>(m, M, ldm, theta, pa, pb);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

int mat_norm1(cudaStream_t st, int64_t n, const double *M, int64_t ldm, double *out) {
  GS_CUDA(cudaMemsetAsync(out, 0, sizeof(double), st));
  k_norm1<<<(unsigned)n, 256, 0, st>>>(n, M, ldm, reinterpret_cast<unsigned long long *>(out));
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

}  // namespace gs
