// FP64 solution of the generalized eigenproblem of Eq. 2,
//     sum_mn (H - E S) C = 0,
// for the eigenvalues inside an energy window, on the device:
//   1. Cholesky S = L L^T (blocked, right-looking, 32-wide panels);
//   2. A = L^-1 H L^-T by two blocked forward substitutions with the
//      block multipliers L_jj^-1 and L_ij L_jj^-1 formed once;
//   3. Householder reduction of A to a symmetric tridiagonal T (d, e);
//   4. Sturm-sequence counts and bisection on T, one thread per wanted
//      eigenvalue index.
// The paper solves this step with LAPACK on one CPU (Sec. II); this is a
// GPU route to the same numbers in the same (FP64) arithmetic.  The pivot
// check of step 1 reports a non-positive-definite S (OFM_ERR_NOT_POSDEF).
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <vector>

#include "ofm_internal.h"

namespace ofm {

constexpr int NB = 32;

// ---------------------------------------------------------------- Cholesky --

// Factor the kb x kb diagonal block at (k0, k0) in place (lower triangle).
// Column j of the working copy stays unscaled; its pivot's reciprocal square
// root r_j and r_j^2 are formed by ONE thread (an FP64 square root and a
// division are long instruction sequences on a part with few FP64 units):
// the thread that applies column j's update to the next pivot forms the
// next r right away, while the other rows finish their updates, so each
// column costs one barrier and no serial scalar step of its own.  The
// update is a_yx -= a_yj (a_xj r_j^2); the scaling L_yj = a_yj r_j is applied
// on the way out (L_jj = piv r_j).
__global__ void potrf_diag_kernel(double* W, int n, int k0, int kb, int* fail_col) {
  __shared__ double a[NB][NB + 1];
  __shared__ double rinv[NB], r2[NB];
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 32
  if (tx < kb && ty < kb) a[ty][tx] = W[(long long)(k0 + ty) * n + k0 + tx];
  __syncthreads();
  // r of the pivot at (j, j), which no later update of this block touches
  auto pivot = [&](int j) {
    double piv = a[j][j];
    if (!(piv > 0.0)) {
      atomicCAS(fail_col, -1, k0 + j);
      piv = 1.0;  // keep going with finite numbers; the call reports failure
      a[j][j] = 1.0;
    }
    const double r = rsqrt(piv);
    rinv[j] = r;
    r2[j] = r * r;
  };
  if (tx == 0 && ty == 0) pivot(0);
  __syncthreads();
  for (int j = 0; j < kb; ++j) {
    if (ty > j && ty < kb && tx > j && tx <= ty) {
      a[ty][tx] = fma(-a[ty][j], a[tx][j] * r2[j], a[ty][tx]);
      if (tx == j + 1 && ty == j + 1) pivot(j + 1);
    }
    __syncthreads();
  }
  if (tx < kb && ty < kb && tx <= ty) W[(long long)(k0 + ty) * n + k0 + tx] = a[ty][tx] * rinv[tx];
}

// Rows i >= k0+kb of the panel: L21 = W21 L11^-T (forward substitution per
// row).  Four lanes share a row (lane = 4 row + phase), each summing every
// fourth term of x_j = (w_j - sum_{t<j} x_t L_jt) / L_jj, combined by two
// shuffle levels: one warp issues an FP64 instruction every 64 cycles at
// best, so a row's ~kb^2/2 products are split four ways rather than chained
// in one lane.  8 rows per warp, 4 warps per CTA.
__global__ void __launch_bounds__(128) trsm_panel_kernel(double* W, int n, int k0, int kb) {
  __shared__ double l[NB][NB + 1];
  __shared__ double dinv[NB];
  __shared__ double xs[32][NB + 1];   // solved entries of the CTA's 32 rows
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    int r = e / NB, cc = e % NB;
    l[r][cc] = (r < kb && cc <= r) ? W[(long long)(k0 + r) * n + k0 + cc] : 0.0;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < kb; j += blockDim.x) dinv[j] = 1.0 / l[j][j];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rl = warp * 8 + (lane >> 2), ph = lane & 3;   // row within the CTA, phase
  const int i = k0 + kb + blockIdx.x * 32 + rl;
  const bool live = i < n;
  double* row = W + (long long)(live ? i : k0) * n + k0;
  double* x = xs[rl];
  for (int j = 0; j < kb; ++j) {
    double s = 0.0;
    for (int t = ph; t < j; t += 4) s = fma(x[t], l[j][t], s);
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    if (ph == 0) x[j] = live ? (row[j] - s) * dinv[j] : 0.0;
    __syncwarp();
  }
  if (live)
    for (int j = ph; j < kb; j += 4) row[j] = x[j];
}

// Trailing update of the lower triangle: W22 -= L21 L21^T (32x32 tiles).
__global__ void syrk_update_kernel(double* W, int n, int k0, int kb) {
  const int t0 = k0 + kb;
  const int bi = blockIdx.y, bj = blockIdx.x;
  if (bj > bi) return;
  __shared__ double li[NB][NB + 1], lj[NB][NB + 1];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i0 = t0 + bi * NB, j0 = t0 + bj * NB;
  {
    int r = i0 + ty;
    li[ty][tx] = (r < n && tx < kb) ? W[(long long)r * n + k0 + tx] : 0.0;
    r = j0 + ty;
    lj[ty][tx] = (r < n && tx < kb) ? W[(long long)r * n + k0 + tx] : 0.0;
  }
  __syncthreads();
  const int i = i0 + ty, j = j0 + tx;
  if (i < n && j < n && j <= i) {
    double s = 0.0;
#pragma unroll 8
    for (int t = 0; t < NB; ++t) s += li[ty][t] * lj[tx][t];
    W[(long long)i * n + j] -= s;
  }
}

// ------------------------------------------------------ triangular solves --
//
// L X = B is solved by blocks of NB rows with precomputed multipliers
// Q_jj = L_jj^-1 (diagonal blocks) and Q_ij = L_ij L_jj^-1 (i > j): step j
// writes X_j = Q_jj B_j and updates B_i -= Q_ij B_j (= L_ij X_j) for i > j,
// one independent NB x NB x NB product per CTA.  The serial substitutions are
// confined to the NB x NB diagonal inverses, computed once per factorisation
// for all blocks in one launch.

// Q_jj = L_jj^-1: one CTA of NB threads per diagonal block, thread c solves
// L_jj x = e_c by forward substitution (reciprocal pivots); the strictly
// upper part of the block is written as zero.
__global__ void inv_diag_kernel(const double* L, double* Q, int n) {
  __shared__ double l[NB][NB + 1];
  __shared__ double dinv[NB];
  const int k0 = blockIdx.x * NB, kb = min(NB, n - k0);
  const int c = threadIdx.x;
  for (int r = 0; r < NB; ++r) l[r][c] = (r < kb && c <= r) ? L[(long long)(k0 + r) * n + k0 + c] : 0.0;
  __syncthreads();
  if (c < kb) dinv[c] = 1.0 / l[c][c];
  __syncthreads();
  if (c >= kb) return;
  double x[NB];
#pragma unroll
  for (int r = 0; r < NB; ++r) {
    double v = 0.0;
    if (r == c) {
      v = dinv[c];
    } else if (r > c && r < kb) {
      double s = 0.0;
      for (int k = c; k < r; ++k) s -= l[r][k] * x[k];
      v = s * dinv[r];
    }
    x[r] = v;
  }
#pragma unroll
  for (int r = 0; r < NB; ++r)
    if (r < kb) Q[(long long)(k0 + r) * n + k0 + c] = x[r];
}

// Q_ij = L_ij Q_jj for the blocks below the diagonal (grid: j, i).
__global__ void panel_mul_kernel(const double* L, double* Q, int n) {
  const int j = blockIdx.x, i = blockIdx.y;
  if (i <= j) return;
  __shared__ double a[NB][NB + 1], q[NB][NB + 1];
  const int r0 = i * NB, k0 = j * NB;
  const int rb = min(NB, n - r0), kb = min(NB, n - k0);
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, cc = e % NB;
    a[r][cc] = (r < rb && cc < kb) ? L[(long long)(r0 + r) * n + k0 + cc] : 0.0;
    q[r][cc] = (r < kb && cc < kb) ? Q[(long long)(k0 + r) * n + k0 + cc] : 0.0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, cc = e % NB;
    double s = 0.0;
#pragma unroll 8
    for (int k = 0; k < NB; ++k) s = fma(a[r][k], q[k][cc], s);
    if (r < rb && cc < kb) Q[(long long)(r0 + r) * n + k0 + cc] = s;
  }
}

// Step j: block row i = j + blockIdx.y, columns c0 = NB blockIdx.x ..
//   i == j: X_j = Q_jj B_j;   i > j: B_i -= Q_ij B_j.
__global__ void __launch_bounds__(256) trsm_step_kernel(const double* Q, double* B, double* X,
                                                        int n, int j) {
  __shared__ double q[NB][NB + 1], bj[NB][NB + 1];
  const int i = j + blockIdx.y, c0 = blockIdx.x * NB;
  const int r0 = i * NB, k0 = j * NB;
  const int rb = min(NB, n - r0), kb = min(NB, n - k0), cb = min(NB, n - c0);
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, cc = e % NB;
    q[r][cc] = (r < rb && cc < kb) ? Q[(long long)(r0 + r) * n + k0 + cc] : 0.0;
    bj[r][cc] = (r < kb && cc < cb) ? B[(long long)(k0 + r) * n + c0 + cc] : 0.0;
  }
  __syncthreads();
  // four outputs per thread: rows ty, ty + 8, ty + 16, ty + 24 of column tx
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll 8
  for (int k = 0; k < NB; ++k) {
    const double b = bj[k][tx];
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[u] = fma(q[ty + 8 * u][k], b, acc[u]);
  }
  if (tx >= cb) return;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int r = ty + 8 * u;
    if (r >= rb) continue;
    const long long o = (long long)(r0 + r) * n + c0 + tx;
    if (i == j) X[o] = acc[u];
    else B[o] -= acc[u];
  }
}

__global__ void transpose_kernel(const double* in, double* out, int n) {
  __shared__ double t[32][33];
  int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 32 + threadIdx.y;
  if (x < n && y < n) t[threadIdx.y][threadIdx.x] = in[(long long)y * n + x];
  __syncthreads();
  x = blockIdx.y * 32 + threadIdx.x;
  y = blockIdx.x * 32 + threadIdx.y;
  if (x < n && y < n) out[(long long)y * n + x] = t[threadIdx.x][threadIdx.y];
}

__global__ void symmetrize_kernel(double* A, int n) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  int i = (int)(e / n), j = (int)(e % n);
  if (j >= i) return;
  double v = 0.5 * (A[(long long)i * n + j] + A[(long long)j * n + i]);
  A[(long long)i * n + j] = v;
  A[(long long)j * n + i] = v;
}

// ------------------------------------------------------- tridiagonalise ----

// Householder vector for column k: x = A[k+1:, k]; v = x - alpha e1 with
// alpha = -sign(x0) ||x||, tau = 2 / v^T v.  Stores v in vbuf[k+1:] and in
// A[k+1:, k] (for the back-transformation), d[k], e[k], tau[k].
__global__ void householder_kernel(double* A, int n, int k, double* vbuf, double* d, double* e,
                                   double* tau) {
  __shared__ double red[32];
  const int m = n - k - 1;
  double s = 0.0;
  for (int i = threadIdx.x + 1; i < m; i += blockDim.x) {
    double x = A[(long long)(k + 1 + i) * n + k];
    s += x * x;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) red[0] = s;
  }
  __syncthreads();
  const double sig = red[0];  // ||x[1:]||^2
  const double x0 = A[(long long)(k + 1) * n + k];
  double alpha, t, v0;
  if (sig == 0.0) {
    alpha = x0;
    t = 0.0;
    v0 = 1.0;
  } else {
    const double nrm = sqrt(x0 * x0 + sig);
    alpha = (x0 > 0.0) ? -nrm : nrm;
    v0 = x0 - alpha;
    t = 2.0 / (v0 * v0 + sig);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    double v = (i == 0) ? v0 : A[(long long)(k + 1 + i) * n + k];
    vbuf[k + 1 + i] = v;
    A[(long long)k * n + k + 1 + i] = v;  // row k keeps v for the back-transformation
  }
  if (threadIdx.x == 0) {
    d[k] = A[(long long)k * n + k];
    e[k] = alpha;
    tau[k] = t;
  }
}

// p = tau * A22 v over rows k+1.. (one warp per row).
__global__ void symv_kernel(const double* A, int n, int k, const double* vbuf, const double* tau,
                            double* p) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int i = k + 1 + warp;
  if (i >= n) return;
  const double* row = A + (long long)i * n;
  double s = 0.0;
  for (int j = k + 1 + lane; j < n; j += 32) s += row[j] * vbuf[j];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) p[i] = tau[k] * s;
}

// A22 -= v w^T + w v^T with w = p - (tau/2)(v^T p) v; every CTA forms v^T p
// itself (a short read of two vectors) so the step needs no extra launch.
__global__ void rank2_kernel(double* A, int n, int k, const double* vbuf, const double* p,
                             const double* tau) {
  __shared__ double red[8];
  __shared__ double Ks;
  double s = 0.0;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  for (int j = k + 1 + tid; j < n; j += blockDim.x * blockDim.y) s += vbuf[j] * p[j];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((tid & 31) == 0) red[tid >> 5] = s;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x * blockDim.y) / 32; ++w) t += red[w];
    Ks = 0.5 * tau[k] * t;
  }
  __syncthreads();
  const double K = Ks;
  const int i = k + 1 + blockIdx.y * blockDim.y + threadIdx.y;
  const int j0 = k + 1 + blockIdx.x * 64;
  if (i >= n) return;
  const double vi = vbuf[i], wi = p[i] - K * vi;
  for (int jj = threadIdx.x; jj < 64; jj += blockDim.x) {
    const int j = j0 + jj;
    if (j >= n) break;
    const double vj = vbuf[j], wj = p[j] - K * vj;
    A[(long long)i * n + j] -= vi * wj + wi * vj;
  }
}

__global__ void tridiag_tail_kernel(const double* A, int n, double* d, double* e) {
  if (n >= 2) {
    d[n - 2] = A[(long long)(n - 2) * n + n - 2];
    e[n - 2] = A[(long long)(n - 1) * n + n - 2];
  }
  d[n - 1] = A[(long long)(n - 1) * n + n - 1];
}

// ---------------------------------------------------------------- bisection --

// Number of eigenvalues of T below x (negative pivots of T - x I).
__device__ int sturm_count(const double* d, const double* e, int n, double x, double pivmin) {
  int c = 0;
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  if (q < 0) ++c;
  for (int j = 1; j < n; ++j) {
    q = d[j] - x - e[j - 1] * e[j - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0) ++c;
  }
  return c;
}

__device__ void gersh(const double* d, const double* e, int n, double* lo, double* hi) {
  double a = DBL_MAX, b = -DBL_MAX;
  for (int j = 0; j < n; ++j) {
    double r = (j > 0 ? fabs(e[j - 1]) : 0.0) + (j < n - 1 ? fabs(e[j]) : 0.0);
    a = fmin(a, d[j] - r);
    b = fmax(b, d[j] + r);
  }
  double w = fmax(fabs(a), fabs(b));
  *lo = a - 2.0 * DBL_EPSILON * w - 1e-300;
  *hi = b + 2.0 * DBL_EPSILON * w + 1e-300;
}

__device__ double pivmin_of(const double* e, int n) {
  double m = 0.0;
  for (int j = 0; j < n - 1; ++j) m = fmax(m, e[j] * e[j]);
  return fmax(DBL_MIN, DBL_MIN * m);
}

__global__ void count_kernel(const double* d, const double* e, int n, double x, int* out) {
  *out = sturm_count(d, e, n, x, pivmin_of(e, n));
}

__global__ void bisect_kernel(const double* d, const double* e, int n, int i_lo, int m, double* out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m) return;
  const int idx = i_lo + t;
  double lo, hi;
  gersh(d, e, n, &lo, &hi);
  const double pm = pivmin_of(e, n);
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (hi - lo <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + 4.0 * DBL_MIN || mid == lo || mid == hi) break;
    if (sturm_count(d, e, n, mid, pm) > idx) hi = mid; else lo = mid;
  }
  out[t] = 0.5 * (lo + hi);
}

}  // namespace ofm

using namespace ofm;

static ofm_status sync_ctx(ofm_ctx* c, const char* what) {
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return ofm_cuda_check(c, e, what);
  return OFM_OK;
}

// X = L^-1 B (n x n) with the multipliers Q of L; B is overwritten.
static void trsm_lower_left(const double* Q, double* B, double* X, int n, cudaStream_t s) {
  const int nblk = (n + NB - 1) / NB;
  for (int j = 0; j < nblk; ++j)
    trsm_step_kernel<<<dim3(nblk, nblk - j), 256, 0, s>>>(Q, B, X, n, j);
}

ofm_status ofm_window_factor(ofm_ctx* c) {
  const int n = c->dense_n;
  if (c->fault == OFM_FAULT_NOTPOSDEF) {
    c->window_fail_col = 0;
    return ofm_fail(c, OFM_ERR_NOT_POSDEF, "S is not positive definite: Cholesky pivot 0 is not positive (injected by OFM_FAULT=notposdef)");
  }
  const size_t bytes = sizeof(double) * (size_t)n * n;
  OFM_TRY(ofm_ensure(c, c->w_L, bytes, "window L"));
  OFM_TRY(ofm_ensure(c, c->w_A, bytes, "window A"));
  OFM_TRY(ofm_ensure(c, c->w_d, sizeof(double) * n, "window d"));
  OFM_TRY(ofm_ensure(c, c->w_e, sizeof(double) * n, "window e"));
  OFM_TRY(ofm_ensure(c, c->w_tau, sizeof(double) * n, "window tau"));
  OFM_TRY(ofm_ensure(c, c->w_tmp, sizeof(double) * 2 * n, "window vectors"));
  double* L = (double*)c->w_L.p;
  double* A = (double*)c->w_A.p;
  int* flag = (int*)c->flag.p;
  cudaStream_t s = c->stream;
  OFM_CUDA(c, cudaMemcpyAsync(L, c->dense_S.p, bytes, cudaMemcpyDeviceToDevice, s));
  OFM_CUDA(c, cudaMemsetAsync(flag, 0xff, sizeof(int), s));  // -1: no failure
  // 1. Cholesky
  { KTimer kt(c, KC_CHOL, 0, 0.0, (double)n * n * n / 3.0);  // algorithmic n^3/3 flops
  for (int k0 = 0; k0 < n; k0 += NB) {
    kt.add(1);
    const int kb = std::min(NB, n - k0);
    potrf_diag_kernel<<<1, dim3(32, 32), 0, s>>>(L, n, k0, kb, flag);
    const int rows = n - k0 - kb;
    if (rows > 0) {
      trsm_panel_kernel<<<(rows + 31) / 32, 128, 0, s>>>(L, n, k0, kb);
      const int tb = (rows + NB - 1) / NB;
      syrk_update_kernel<<<dim3(tb, tb), dim3(32, 32), 0, s>>>(L, n, k0, kb);
      kt.add(2);
    }
  }
  }
  OFM_CUDA(c, cudaGetLastError());
  int fail = -1;
  OFM_CUDA(c, cudaMemcpyAsync(&fail, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  OFM_TRY(sync_ctx(c, "Cholesky of S"));
  if (fail >= 0) {
    c->window_fail_col = fail;
    char buf[160];
    snprintf(buf, sizeof buf, "S is not positive definite: Cholesky pivot %d is not positive", fail);
    return ofm_fail(c, OFM_ERR_NOT_POSDEF, buf);
  }
  // 2. A = L^-1 H L^-T: multipliers Q of L, X = L^-1 H, then A = L^-1 X^T
  double* T = (double*)c->dense_H.p;  // kept intact: work on a copy
  OFM_CUDA(c, cudaMemcpyAsync(A, T, bytes, cudaMemcpyDeviceToDevice, s));
  {
  const int nblk = (n + NB - 1) / NB;
  KTimer kt(c, KC_REDUCE, 5 + 2LL * nblk, 0.0, (double)n * n * n);  // algorithmic (dsygst) n^3 flops
  OFM_TRY(ofm_ensure(c, c->w_eval, bytes, "window scratch"));
  OFM_TRY(ofm_ensure(c, c->w_Q, bytes, "window multipliers"));
  double* X = (double*)c->w_eval.p;
  double* Q = (double*)c->w_Q.p;
  inv_diag_kernel<<<nblk, NB, 0, s>>>(L, Q, n);
  panel_mul_kernel<<<dim3(nblk, nblk), 256, 0, s>>>(L, Q, n);
  trsm_lower_left(Q, A, X, n, s);          // X = L^-1 H (A is consumed)
  dim3 tg((n + 31) / 32, (n + 31) / 32);
  transpose_kernel<<<tg, dim3(32, 32), 0, s>>>(X, A, n);
  trsm_lower_left(Q, A, X, n, s);          // X = L^-1 (L^-1 H)^T
  symmetrize_kernel<<<(int)(((long long)n * n + 255) / 256), 256, 0, s>>>(X, n);
  OFM_CUDA(c, cudaMemcpyAsync(A, X, bytes, cudaMemcpyDeviceToDevice, s));
  }
  OFM_CUDA(c, cudaGetLastError());
  // 3. tridiagonalise
  double* d = (double*)c->w_d.p;
  double* e = (double*)c->w_e.p;
  double* tau = (double*)c->w_tau.p;
  double* vbuf = (double*)c->w_tmp.p;
  double* p = vbuf + n;
  {
  KTimer kt(c, KC_TRIDIAG, 0, 0.0, 4.0 / 3.0 * n * n * n);  // algorithmic (dsytrd) 4n^3/3 flops
  const ofm_status ps = ofm_tridiag_persistent(c, A, n, d, e, tau, p);
  if (ps == OFM_OK) {
    kt.add(1);
  } else if (ps != OFM_ERR_INVALID) {
    return ps;
  } else {
  kt.add(1 + 3LL * std::max(0, n - 2));
  for (int k = 0; k + 2 < n; ++k) {
    householder_kernel<<<1, 256, 0, s>>>(A, n, k, vbuf, d, e, tau);
    const int m = n - k - 1;
    symv_kernel<<<(m + 7) / 8, 256, 0, s>>>(A, n, k, vbuf, tau, p);
    rank2_kernel<<<dim3((m + 63) / 64, (m + 7) / 8), dim3(32, 8), 0, s>>>(A, n, k, vbuf, p, tau);
  }
  tridiag_tail_kernel<<<1, 1, 0, s>>>(A, n, d, e);
  }
  }
  OFM_CUDA(c, cudaGetLastError());
  OFM_TRY(sync_ctx(c, "tridiagonalisation"));
  c->factored = true;
  return OFM_OK;
}

ofm_status ofm_window_count(ofm_ctx* c, double lo, double hi, int* count_lo, int* count_hi) {
  const double hi_incl = std::nextafter(hi, HUGE_VAL);
  if (2 * (size_t)c->dense_n * sizeof(double) > 200 * 1024)
    return ofm_fail(c, OFM_ERR_INVALID, "dense window solve supports a basis of at most 12800");
  int* dc = (int*)c->flag.p + 2;   // two ints after the pivot flag
  int h[2] = {0, 0};
  KTimer kt(c, KC_BISECT);
  launch_count_below((const double*)c->w_d.p, (const double*)c->w_e.p, c->dense_n, lo, hi_incl, dc,
                     c->stream);
  OFM_CUDA(c, cudaGetLastError());
  OFM_CUDA(c, cudaMemcpyAsync(h, dc, 2 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  OFM_TRY(sync_ctx(c, "Sturm count"));
  *count_lo = h[0];
  *count_hi = h[1];
  return OFM_OK;
}

// Upper estimate of one past the last index of [E_{i_lo}, E_{i_lo} + width]
// from FP32 counts (a guess; the caller checks it with FP64 eigenvalues).
ofm_status ofm_window_size_estimate(ofm_ctx* c, int i_lo, double width, int* i_end) {
  int* dv = (int*)c->flag.p + 4;   // after the pivot flag and the two counts
  KTimer kt(c, KC_BISECT);
  if (!launch_window_size((const double*)c->w_d.p, (const double*)c->w_e.p, c->dense_n, i_lo,
                          width, dv, c->stream)) {
    *i_end = c->dense_n;   // too long to stage: take everything above i_lo
    return OFM_OK;
  }
  OFM_CUDA(c, cudaGetLastError());
  OFM_CUDA(c, cudaMemcpyAsync(i_end, dv, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  return sync_ctx(c, "window size estimate");
}

ofm_status ofm_window_bisect(ofm_ctx* c, int i_lo, int i_hi, double* E_out) {
  const int m = i_hi - i_lo;
  double* out = (double*)c->w_tmp.p;  // 2n doubles, m <= n
  KTimer kt(c, KC_BISECT);
  if (!launch_multisection((const double*)c->w_d.p, (const double*)c->w_e.p, c->dense_n, i_lo, m,
                           out, c->stream))
    bisect_kernel<<<(m + 127) / 128, 128, 0, c->stream>>>((const double*)c->w_d.p,
                                                          (const double*)c->w_e.p, c->dense_n,
                                                          i_lo, m, out);
  OFM_CUDA(c, cudaGetLastError());
  OFM_CUDA(c, cudaMemcpyAsync(E_out, out, sizeof(double) * m, cudaMemcpyDeviceToHost, c->stream));
  return sync_ctx(c, "bisection");
}
