// The small problems on the Lanczos tridiagonal T_m (m <= a few thousand):
//   * eigenvalues by Sturm-count multisection (ke3; the paper's ARPACK uses a
//     QR variant for this, Section 4.1 -- multisection gives each Ritz value
//     independently, one warp per value, 32 counts per round);
//   * eigenvectors by inverse iteration (one thread per value, tridiagonal
//     Gaussian elimination with partial pivoting), tight clusters
//     orthogonalised afterwards;
//   * the implicit restart (Section 2.3: "the application of the QR
//     iteration to the tridiagonal matrix T_m"): p = m - k single-shift QR
//     steps whose shifts are the unwanted Ritz values (exact shifts).  Each
//     shift is a Givens bulge chase; after an exact shift the trailing
//     entry deflates, so shift i chases over m - i rows.  The chase is
//     sequential (one thread); the accumulation Q <- Q G^T, which is where
//     the O(p m^2) flops are, runs on many CTAs, each owning rows of Q.
#include <float.h>

#include <mutex>

#include "lanczos.cuh"

namespace gs {
namespace {

__device__ __forceinline__ double sturm_pivmin(double maxe2) { return DBL_MIN * fmax(1.0, maxe2); }

// Number of eigenvalues strictly below x of the symmetric matrix M with
// diagonal d, arrow couplings b[0..ka-1] between rows i < ka and row ka, and
// tridiagonal couplings e[i] (i >= ka) between rows i and i+1 (e2 = e^2,
// b2 = b^2).  ka = 0 is a plain tridiagonal.  Inertia of M - x I by block
// elimination in the order 0, 1, ..., m-1 (Sylvester): the arrow rows are
// diagonal, so their pivots are d_i - x and they only update row ka.
__device__ int64_t sturm_below(int64_t m, int64_t ka, const double *d, const double *e2, const double *b2, double x,
                               double pivmin) {
  int64_t cnt = 0;
  double acc = 0.0;
  for (int64_t i = 0; i < ka; i++) {
    double p = d[i] - x;
    if (fabs(p) < pivmin) p = -pivmin;
    if (p < 0.0) cnt++;
    acc += b2[i] / p;
  }
  double q = (d[ka] - x) - acc;
  if (fabs(q) < pivmin) q = -pivmin;
  if (q < 0.0) cnt++;
  for (int64_t i = ka + 1; i < m; i++) {
    q = (d[i] - x) - e2[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0.0) cnt++;
  }
  return cnt;
}

// Multisection: one warp per eigenvalue (one CTA each, spread over the
// SMs -- GB300's FP64 pipe is narrow, so the Sturm sequences must not share
// an SM).  Each round the 32 lanes evaluate the count at 32 interior points
// of the bracket [a, b] and the bracket shrinks 33-fold.
// dynamic smem: d[m], e2[m], b2[m]
__global__ void __launch_bounds__(32) k_multisect(int64_t m, const double *__restrict__ d, const double *__restrict__ e,
                                                  int64_t ka, const double *__restrict__ b, int64_t first,
                                                  double *__restrict__ lam) {
  extern __shared__ double sm[];
  double *ds = sm, *e2 = sm + m, *b2 = sm + 2 * m;
  const int lane = threadIdx.x;
  double lo = DBL_MAX, hi = -DBL_MAX, me2 = 0.0, bsum = 0.0;
  for (int64_t i = lane; i < m; i += 32) {
    const double di = d[i];
    const double el = (i > ka) ? fabs(e[i - 1]) : 0.0, er = (i >= ka && i + 1 < m) ? fabs(e[i]) : 0.0;
    const double bi = (i < ka) ? fabs(b[i]) : 0.0;
    ds[i] = di;
    e2[i] = (i >= ka && i + 1 < m) ? e[i] * e[i] : 0.0;
    b2[i] = (i < ka) ? b[i] * b[i] : 0.0;
    me2 = fmax(me2, fmax(er * er, bi * bi));
    bsum += bi;
    lo = fmin(lo, di - el - er - bi);
    hi = fmax(hi, di + el + er + bi);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    me2 = fmax(me2, __shfl_xor_sync(0xffffffffu, me2, o));
    bsum += __shfl_xor_sync(0xffffffffu, bsum, o);
  }
  if (ka > 0) {
    const double dk = d[ka], ek = (ka + 1 < m) ? fabs(e[ka]) : 0.0;
    lo = fmin(lo, dk - bsum - ek);
    hi = fmax(hi, dk + bsum + ek);
  }
  __syncwarp();
  const double pivmin = sturm_pivmin(me2);
  const double span = fmax(fabs(lo), fabs(hi));
  double xa = lo - 2.0 * DBL_EPSILON * span - 2.0 * pivmin;
  double xb = hi + 2.0 * DBL_EPSILON * span + 2.0 * pivmin;
  const int64_t q = first + blockIdx.x;  // 0-based index of the wanted eigenvalue
  for (int it = 0; it < 64; it++) {
    if (xb - xa <= 2.0 * DBL_EPSILON * fmax(fabs(xa), fabs(xb)) + 4.0 * pivmin) break;
    const double step = (xb - xa) / 33.0;
    const double x = xa + (double)(lane + 1) * step;
    const bool le = sturm_below(m, ka, ds, e2, b2, x, pivmin) <= q;  // eigenvalue q lies above x
    const unsigned above = __ballot_sync(0xffffffffu, !le);
    const int L = above ? (__ffs(above) - 1) : 32;  // first lane whose point is above the eigenvalue
    const double na = (L > 0) ? xa + (double)L * step : xa;
    const double nb = (L < 32) ? xa + (double)(L + 1) * step : xb;
    if (!(na < nb) || (na == xa && nb == xb)) break;
    xa = na;
    xb = nb;
  }
  if (lane == 0) lam[blockIdx.x] = 0.5 * (xa + xb);
}

__device__ __forceinline__ uint64_t mix64(uint64_t x) {
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdull;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ull;
  return x ^ (x >> 33);
}

// Inverse iteration, one thread per eigenvalue, on M - lam I with M as in
// sturm_below (arrow rows 0..ka-1, tridiagonal from row ka).  The arrow rows
// are eliminated first (pivots d_i - lam), which only changes the diagonal
// and right-hand side of row ka; the remaining tridiagonal rows ka..m-1 are
// eliminated with partial pivoting between the running row and the next
// original row (U gets two superdiagonals).  Tiny pivots are replaced by
// eps ||M||, the classical device that makes the solve return the wanted
// direction.  Work per thread: 5m doubles.
__global__ void k_invit(int64_t m, const double *__restrict__ d, const double *__restrict__ e, int64_t ka,
                        const double *__restrict__ b, int64_t cnt, const double *__restrict__ lam,
                        double *__restrict__ Z, int64_t ldz, double *__restrict__ work) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cnt) return;
  double *p0 = work + (size_t)t * 5 * m, *p1 = p0 + m, *p2 = p1 + m, *mu = p2 + m, *sw = mu + m;
  double *z = Z + (size_t)t * ldz;
  double tn = 0.0, bs = 0.0;
  for (int64_t i = 0; i < m; i++) {
    double r = fabs(d[i]);
    if (i < ka) {
      r += fabs(b[i]);
      bs += fabs(b[i]);
    } else {
      if (i > ka) r += fabs(e[i - 1]);
      if (i + 1 < m) r += fabs(e[i]);
    }
    tn = fmax(tn, r);
  }
  tn = fmax(tn, fabs(d[ka]) + bs + ((ka + 1 < m) ? fabs(e[ka]) : 0.0));
  if (tn == 0.0) tn = 1.0;
  const double tiny = DBL_EPSILON * tn;
  const double x = lam[t];
  // arrow pivots and the Schur complement on row ka
  double a = d[ka] - x;
  for (int64_t i = 0; i < ka; i++) {
    double piv = d[i] - x;
    if (fabs(piv) < tiny) piv = copysign(tiny, piv);
    p0[i] = piv;
    a -= b[i] * b[i] / piv;
  }
  // factor rows ka..m-1
  double bb = (ka + 1 < m) ? e[ka] : 0.0, c = 0.0;
  for (int64_t i = ka; i < m; i++) {
    if (i == m - 1) {
      p0[i] = (fabs(a) < tiny) ? copysign(tiny, a) : a;
      p1[i] = p2[i] = mu[i] = sw[i] = 0.0;
      break;
    }
    const double lo = e[i], nd = d[i + 1] - x, nu = (i + 2 < m) ? e[i + 1] : 0.0;
    if (fabs(a) >= fabs(lo)) {
      const double piv = (fabs(a) < tiny) ? copysign(tiny, a) : a;
      const double f = lo / piv;
      p0[i] = piv; p1[i] = bb; p2[i] = c; mu[i] = f; sw[i] = 0.0;
      a = nd - f * bb;
      bb = nu - f * c;
    } else {
      const double f = a / lo;
      p0[i] = lo; p1[i] = nd; p2[i] = nu; mu[i] = f; sw[i] = 1.0;
      a = bb - f * nd;
      bb = c - f * nu;
    }
    c = 0.0;
  }
  // start vector
  for (int64_t i = 0; i < m; i++)
    z[i] = 1.0 + 0.25 * ((double)(mix64((uint64_t)i * 0x9E3779B97F4A7C15ull + (uint64_t)t) >> 11) * 0x1p-53 - 0.5);
  for (int it = 0; it < 3; it++) {
    // arrow elimination on the right-hand side
    double acc = 0.0;
    for (int64_t i = 0; i < ka; i++) acc += b[i] * z[i] / p0[i];
    z[ka] -= acc;
    for (int64_t i = ka; i + 1 < m; i++) {
      if (sw[i] != 0.0) { double q = z[i]; z[i] = z[i + 1]; z[i + 1] = q; }
      z[i + 1] -= mu[i] * z[i];
    }
    double mx = 0.0;
    for (int64_t i = m - 1; i >= ka; i--) {
      double v = z[i];
      if (i + 1 < m) v -= p1[i] * z[i + 1];
      if (i + 2 < m) v -= p2[i] * z[i + 2];
      v /= p0[i];
      z[i] = v;
      mx = fmax(mx, fabs(v));
    }
    const double xk = z[ka];
    for (int64_t i = 0; i < ka; i++) {
      const double v = (z[i] - b[i] * xk) / p0[i];
      z[i] = v;
      mx = fmax(mx, fabs(v));
    }
    const double sc = (mx > 0.0) ? 1.0 / mx : 1.0;
    for (int64_t i = 0; i < m; i++) z[i] *= sc;
  }
  double nrm = 0.0;
  for (int64_t i = 0; i < m; i++) nrm = fma(z[i], z[i], nrm);
  nrm = sqrt(nrm);
  const double sc = (nrm > 0.0) ? 1.0 / nrm : 0.0;
  for (int64_t i = 0; i < m; i++) z[i] *= sc;
}

__device__ double block_sum256(double v, double *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); i++) s += red[i];
  __syncthreads();
  return s;  // valid in every thread
}

// Orthogonalise eigenvectors whose eigenvalues sit within 1e-5 ||T|| of
// the previous one against the earlier members of their cluster (modified
// Gram-Schmidt, two passes).  Inverse-iteration vectors of eigenvalues a gap
// g apart are orthogonal only to about eps ||T|| / g, so this bound keeps
// every pair within about 2e-11 (LAPACK's inverse iteration groups at
// 1e-3 ||T||; the benchmark spectra form no cluster at 1e-5 ||T||, while
// crossing eigenvalues of a sequence of pencils do).  One CTA; a no-op scan
// when nothing clusters.
__global__ void k_cluster_orth(int64_t m, int64_t cnt, const double *lam, double tn_hint, const double *d,
                               const double *e, double *Z, int64_t ldz) {
  __shared__ double red[32];
  double tl = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x)
    tl = fmax(tl, fabs(d[i]) + (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < m ? fabs(e[i]) : 0.0));
  // max-reduce
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tl = fmax(tl, __shfl_xor_sync(0xffffffffu, tl, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = tl;
  __syncthreads();
  double tn = tn_hint;
  for (int i = 0; i < (int)(blockDim.x >> 5); i++) tn = fmax(tn, red[i]);
  __syncthreads();
  const double thr = 1e-5 * tn;
  int64_t start = 0;
  for (int64_t c = 1; c < cnt; c++) {
    if (lam[c] - lam[c - 1] > thr) {
      start = c;
      continue;
    }
    double *zc = Z + (size_t)c * ldz;
    for (int pass = 0; pass < 2; pass++)
      for (int64_t q = start; q < c; q++) {
        const double *zq = Z + (size_t)q * ldz;
        double acc = 0.0;
        for (int64_t i = threadIdx.x; i < m; i += blockDim.x) acc = fma(zq[i], zc[i], acc);
        double dot = block_sum256(acc, red);
        for (int64_t i = threadIdx.x; i < m; i += blockDim.x) zc[i] -= dot * zq[i];
        __syncthreads();
      }
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) acc = fma(zc[i], zc[i], acc);
    double nrm = sqrt(block_sum256(acc, red));
    const double s = nrm > 0.0 ? 1.0 / nrm : 0.0;
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) zc[i] *= s;
    __syncthreads();
  }
}

// Bulge chase for p exact shifts on T_m; rotations (c, s) of shift i at
// rot[2 * (i * (m - 1) + r) + {0, 1}] for r < m - 1 - i.  One thread.
__global__ void k_qr_chase(int64_t m, int64_t p, const double *alpha, const double *beta, const double *shifts,
                           int dir, double *aP, double *bP, double *rot) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int64_t i = 0; i < m; i++) aP[i] = alpha[i];
  for (int64_t i = 0; i + 1 < m; i++) bP[i] = beta[i];
  for (int64_t sh = 0; sh < p; sh++) {
    const int64_t hi = m - 1 - sh;  // active block [0, hi]
    const double mu = (dir > 0) ? shifts[sh] : shifts[p - 1 - sh];
    double *cs = rot + 2 * (size_t)sh * (m - 1);
    double x = aP[0] - mu, z = (hi > 0) ? bP[0] : 0.0;
    for (int64_t i = 0; i < hi; i++) {
      double r = hypot(x, z);
      double c = 1.0, s = 0.0;
      if (r != 0.0) {
        double ir = 1.0 / r;
        c = x * ir;
        s = z * ir;
      }
      if (i > 0) bP[i - 1] = r;
      const double a0 = aP[i], a1 = aP[i + 1], b = bP[i];
      const double cc = c * c, ss = s * s, c2s = 2.0 * c * s * b;
      aP[i] = cc * a0 + c2s + ss * a1;
      aP[i + 1] = ss * a0 - c2s + cc * a1;
      bP[i] = c * s * (a1 - a0) + (cc - ss) * b;
      if (i + 1 < hi) {
        const double bulge = s * bP[i + 1];
        bP[i + 1] *= c;
        x = bP[i];
        z = bulge;
      }
      cs[2 * i] = c;
      cs[2 * i + 1] = s;
    }
  }
}

// Q = I, then Q <- Q G_1^T G_2^T ... for every rotation of every shift, one
// thread per row of Q (rows are independent).
__global__ void k_qr_apply(int64_t m, int64_t p, const double *__restrict__ rot, double *__restrict__ Q, int64_t ldq) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= m) return;
  for (int64_t j = 0; j < m; j++) Q[r + (size_t)j * ldq] = (r == j) ? 1.0 : 0.0;
  for (int64_t sh = 0; sh < p; sh++) {
    const int64_t hi = m - 1 - sh;
    const double *cs = rot + 2 * (size_t)sh * (m - 1);
    double x = Q[r];
    for (int64_t i = 0; i < hi; i++) {
      const double c = cs[2 * i], s = cs[2 * i + 1];
      const double y = Q[r + (size_t)(i + 1) * ldq];
      Q[r + (size_t)i * ldq] = c * x + s * y;
      x = c * y - s * x;
    }
    Q[r + (size_t)hi * ldq] = x;
  }
}

__global__ void k_converged(int64_t m, int64_t cnt, const double *theta, const double *beta, const double *Z,
                            int64_t ldz, double tol, LanczosState *state) {
  __shared__ double red[32];
  __shared__ int64_t nc;
  if (threadIdx.x == 0) nc = 0;
  __syncthreads();
  const double tn = state->tnorm;  // running estimate of ||T|| from the recurrence
  const double bm = fabs(beta[m - 1]);
  double mx = 0.0;
  int64_t mine = 0;
  for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x) {
    double est = bm * fabs(Z[(m - 1) + (size_t)i * ldz]);
    double rel = (tn > 0.0) ? est / tn : est;
    mx = fmax(mx, rel);
    if (rel <= tol) mine++;
  }
  atomicAdd((unsigned long long *)&nc, (unsigned long long)mine);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); i++) v = fmax(v, red[i]);
    state->max_est = v;
    state->nconv = nc;
  }
}

}  // namespace

int tri_bisect(cudaStream_t st, int64_t m, const double *d, const double *e, int64_t ka, const double *b, int64_t first,
               int64_t cnt, double *lam) {
  if (cnt <= 0) return GSYEIG_SUCCESS;
  size_t smem = (size_t)(3 * m) * sizeof(double);
  if (smem > 48 * 1024)
    GS_CUDA(cudaFuncSetAttribute((const void *)k_multisect, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_multisect<<<(unsigned)cnt, 32, smem, st>>>(m, d, e, ka, b, first, lam);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

int tri_invit(cudaStream_t st, int64_t m, const double *d, const double *e, int64_t ka, const double *b, int64_t cnt,
              const double *lam, double *Z, int64_t ldz, double *work) {
  if (cnt <= 0) return GSYEIG_SUCCESS;
  // one thread per eigenvalue, spread over many SMs (32 threads per CTA)
  k_invit<<<(unsigned)ceil_div(cnt, 8), 8, 0, st>>>(m, d, e, ka, b, cnt, lam, Z, ldz, work);
  count_launch();
  GS_CHECK_LAUNCH();
  k_cluster_orth<<<1, 256, 0, st>>>(m, cnt, lam, 0.0, d, e, Z, ldz);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

int tri_qr_shifts(cudaStream_t st, int64_t m, int64_t p, const double *alpha, const double *beta, const double *shifts,
                  int dir, double *alphaP, double *betaP, double *Q, int64_t ldq, double *rot) {
  k_qr_chase<<<1, 32, 0, st>>>(m, p, alpha, beta, shifts, dir, alphaP, betaP, rot);
  count_launch();
  GS_CHECK_LAUNCH();
  k_qr_apply<<<(unsigned)ceil_div(m, 32), 32, 0, st>>>(m, p, rot, Q, ldq);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

int tri_converged(cudaStream_t st, int64_t m, int64_t cnt, const double *theta_all, const double *beta, const double *Z,
                  int64_t ldz, double tol, LanczosState *state) {
  k_converged<<<1, 256, 0, st>>>(m, cnt, theta_all, beta, Z, ldz, tol, state);
  count_launch();
  GS_CHECK_LAUNCH();
  return GSYEIG_SUCCESS;
}

}  // namespace gs

// ---------------------------------------------------------------------------
// Allocation-free variant of the tridiagonal eigen-solve (the paper has no
// counterpart: this exists for callers, not for the method).
//
// gsyeig_tridiag_eig draws its inverse-iteration scratch (5 m cnt doubles)
// from a handle workspace that grows with cudaMalloc.  Some callers cannot
// allocate device memory at the point where they need this solve: code whose
// device memory is entirely owned by another allocator or a fixed budget,
// and latency-critical loops where cudaMalloc/cudaFree would synchronise the
// whole device.  This entry point takes only the caller's inputs and
// outputs; its scratch is the fixed array below, which lives in the
// library's own module image, so every GPU that loads the library holds
// these 8 MiB until the process exits.
//
// Host code may not use g_noalloc_scratch directly: on the host that name
// is a stand-in symbol, not a device address.  The device address is looked
// up with cudaGetSymbolAddress, with that device current, by each call (a
// lookup allocates nothing; a device reset followed by a new context may
// move the array) and kept per device; the first call on a device does
// this set-up.
// ---------------------------------------------------------------------------
namespace gs {
namespace {

constexpr size_t kNoAllocScratchDoubles = size_t(1) << 20;  // 8 MiB
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

std::mutex g_noalloc_mutex;
double *g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on the current device: looked up
// afresh unless `st` is capturing, then taken from the per-device cache.
int noalloc_scratch(cudaStream_t st, double **out) {
  int dev = 0;
  GS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) return GSYEIG_NOT_SUPPORTED;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  GS_CUDA(cudaStreamIsCapturing(st, &cap));
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (cap == cudaStreamCaptureStatusNone || !g_noalloc_ptr[dev]) {
    void *p = nullptr;
    GS_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[dev] = static_cast<double *>(p);
  }
  *out = g_noalloc_ptr[dev];
  return GSYEIG_SUCCESS;
}

}  // namespace
}  // namespace gs

extern "C" int gsyeig_tridiag_eig_noalloc(const double *d, const double *e, int64_t m, int64_t first, int64_t cnt,
                                          double *lam, double *dZ, int64_t ldz, void *cuda_stream) {
  using namespace gs;
  if (!d) return -1;
  if (!e && m > 1) return -2;
  if (m < 1) return -3;
  if (first < 0 || first >= m) return -4;
  if (cnt < 1 || first + cnt > m) return -5;
  if (!lam) return -6;
  if (dZ && ldz < m) return -8;
  if (dZ && (size_t)5 * (size_t)m * (size_t)cnt > kNoAllocScratchDoubles) return GSYEIG_SCRATCH_TOO_SMALL;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  double *scratch = nullptr;
  if (dZ) GS_TRY(noalloc_scratch(st, &scratch));
  GS_TRY(tri_bisect(st, m, d, e, 0, nullptr, first, cnt, lam));
  // inverse iteration writes every scratch entry before reading it, so the
  // previous call's contents need no clearing
  if (dZ) GS_TRY(tri_invit(st, m, d, e, 0, nullptr, cnt, lam, dZ, ldz, scratch));
  GS_CUDA(cudaStreamSynchronize(st));
  GS_CUDA(cudaGetLastError());
  return GSYEIG_SUCCESS;
}
