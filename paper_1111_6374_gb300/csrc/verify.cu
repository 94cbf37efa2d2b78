// Optional check of a solve's result against the original pencil, in FP64
// on the device (gsyeig_opts.verify): the per-column normwise backward error
//   eta_i = ||A x_i - lambda_i B x_i||_2 / ((||A||_2 + |lambda_i| ||B||_2) ||x_i||_2)
// and the B-orthonormality error max |X^T B X - I|.  ||A||_2 and ||B||_2 are
// estimated by power iteration (from below, so eta is not understated by
// the estimate).  A X and B X go through the solve's GEMM engine; the
// symmetric products of the power iteration through the FP64 symv.
#include "lanczos.cuh"

namespace gs {
namespace {

constexpr int VT = 512;  // threads of the reduction kernels

__device__ double block_sum(double v, double *red) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = (threadIdx.x < (int)(blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;  // valid in thread 0
}

// column i: rn[i] = ||AX_i - w_i BX_i||, xn[i] = ||X_i|| (one CTA per column)
__global__ void __launch_bounds__(VT) k_resid_cols(int64_t n, const double *AX, const double *BX, const double *w,
                                                   const double *X, int64_t ldx, double *rn, double *xn) {
  __shared__ double red[VT / 32];
  const int64_t i = blockIdx.x;
  const double wi = w[i];
  double r2 = 0.0, x2 = 0.0;
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
    const double r = AX[k + i * n] - wi * BX[k + i * n];
    const double x = X[k + i * ldx];
    r2 = fma(r, r, r2);
    x2 = fma(x, x, x2);
  }
  const double R = block_sum(r2, red);
  const double Xs = block_sum(x2, red);
  if (threadIdx.x == 0) {
    rn[i] = sqrt(R);
    xn[i] = sqrt(Xs);
  }
}

// v = z / ||z||, *nrm = ||z|| (one CTA)
__global__ void __launch_bounds__(VT) k_power_normalize(int64_t n, const double *z, double *v, double *nrm) {
  __shared__ double red[VT / 32];
  __shared__ double s_inv;
  double z2 = 0.0;
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) z2 = fma(z[k], z[k], z2);
  const double t = block_sum(z2, red);
  if (threadIdx.x == 0) {
    const double nz = sqrt(t);
    *nrm = nz;
    s_inv = nz > 0.0 ? 1.0 / nz : 0.0;
  }
  __syncthreads();
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) v[k] = z[k] * s_inv;
}

// out[0] = max_i eta_i, out[1] = max |G - I| (one CTA; G s x s, ld s)
__global__ void __launch_bounds__(VT) k_verify_finish(int64_t s, const double *rn, const double *xn, const double *w,
                                                      const double *nA, const double *nB, const double *G,
                                                      double *out) {
  __shared__ double red[VT / 32];
  double e = 0.0, o = 0.0;
  for (int64_t i = threadIdx.x; i < s; i += blockDim.x) {
    const double den = (*nA + fabs(w[i]) * *nB) * xn[i];
    e = fmax(e, den > 0.0 ? rn[i] / den : INFINITY);
  }
  for (int64_t idx = threadIdx.x; idx < s * s; idx += blockDim.x) {
    const int64_t r = idx % s, c = idx / s;
    o = fmax(o, fabs(G[idx] - (r == c ? 1.0 : 0.0)));
  }
  for (int off = 16; off; off >>= 1) {
    e = fmax(e, __shfl_xor_sync(0xffffffffu, e, off));
    o = fmax(o, __shfl_xor_sync(0xffffffffu, o, off));
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[warp] = e;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) m = fmax(m, red[k]);
    out[0] = m;
  }
  __syncthreads();
  if (lane == 0) red[warp] = o;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) m = fmax(m, red[k]);
    out[1] = m;
  }
}

constexpr int POWER_ITERS = 40;

// ||M||_2 estimate of a full symmetric M into *nrm (device)
int power_norm(cudaStream_t st, int64_t n, const double *M, int64_t ldm, double *v, double *z, double *nrm) {
  GS_TRY(lz_random(st, n, 0x5eed, 7, z));
  k_power_normalize<<<1, VT, 0, st>>>(n, z, v, nrm);
  count_launch();
  for (int it = 0; it < POWER_ITERS; it++) {
    GS_TRY(symv_f64(st, n, M, ldm, v, z));
    k_power_normalize<<<1, VT, 0, st>>>(n, z, v, nrm);
    count_launch();
  }
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

}  // namespace

size_t verify_workspace_doubles(int64_t n, int64_t s) { return (size_t)(2 * n * s + s * s + 2 * n + 2 * s + 8); }

int verify_solution(cudaStream_t st, int64_t n, int64_t s, const double *A0, int64_t lda, const double *B0,
                    int64_t ldb, const double *X, int64_t ldx, const double *w, double *ws, double out[2]) {
  double *AX = ws, *BX = AX + n * s, *G = BX + n * s, *v = G + s * s, *z = v + n, *rn = z + n, *xn = rn + s,
         *sc = xn + s;  // sc: ||A||, ||B||, max eta, orth error
  GS_TRY(dgemm(st, false, false, n, s, n, 1.0, A0, lda, X, ldx, 0.0, AX, n));
  GS_TRY(dgemm(st, false, false, n, s, n, 1.0, B0, ldb, X, ldx, 0.0, BX, n));
  GS_TRY(dgemm(st, true, false, s, s, n, 1.0, X, ldx, BX, n, 0.0, G, s));
  k_resid_cols<<<(unsigned)s, VT, 0, st>>>(n, AX, BX, w, X, ldx, rn, xn);
  count_launch();
  GS_TRY(power_norm(st, n, A0, lda, v, z, sc));
  GS_TRY(power_norm(st, n, B0, ldb, v, z, sc + 1));
  k_verify_finish<<<1, VT, 0, st>>>(s, rn, xn, w, sc, sc + 1, G, sc + 2);
  count_launch();
  GS_CHECK_LAUNCH();
  GS_CUDA(cudaMemcpyAsync(out, sc + 2, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  GS_CUDA(cudaStreamSynchronize(st));
  return GSYEIG_SUCCESS;
}

}  // namespace gs
