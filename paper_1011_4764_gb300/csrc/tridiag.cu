// Symmetric tridiagonal reduction and spectrum slicing for the window solve
// of Eq. 2 (after the reduction A = L^-1 H L^-T).
//
// 1. Householder reduction of A to tridiagonal form in ONE persistent
//    cooperative kernel: per column k, every CTA forms the Householder
//    vector itself (a short column read), the CTAs compute p = tau A22 v by
//    rows, meet at a grid barrier, apply A22 -= v w^T + w v^T
//    (w = p - (tau/2)(v^T p) v) by rows and meet again.  Two barriers per
//    column instead of three kernel launches.  The barrier spins a bounded
//    number of times and reports a timeout instead of hanging.
// 2. Eigenvalues by index with multisection: one warp per wanted
//    eigenvalue; each lane counts the eigenvalues below one of 32 points of
//    the current interval (Sturm sequence of T - x I written as the
//    three-term recurrence of the leading principal minors, rescaled by
//    powers of two, so a step needs no division), and the interval shrinks
//    33-fold per round.
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cmath>

#include "ofm_internal.h"

namespace ofm {

// Barrier state: a counter that only grows (one arrival per CTA per
// barrier), so the k-th barrier completes when the counter reaches
// k * nblocks; no reset is ever needed.
struct GridBar {
  unsigned int count;
  int err;
  unsigned int pad[30];
};

// All CTAs of a cooperative launch meet here: one release atomic per CTA
// and acquire polls of the counter.  Returns false (and sets bar->err) when
// the wait exceeded its bound or another CTA gave up.
__device__ bool grid_sync(GridBar* bar, unsigned int nblocks) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile int* verr = &bar->err;
    unsigned int old;
    asm volatile("atom.add.release.gpu.global.u32 %0, [%1], 1;" : "=r"(old) : "l"(&bar->count) : "memory");
    const unsigned int target = (old / nblocks + 1u) * nblocks;
    ok = 1;
    unsigned int spins = 0;
    while (true) {
      unsigned int cur;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(&bar->count) : "memory");
      if ((int)(cur - target) >= 0) break;
      if (*verr != 0 || ++spins > (1u << 24)) {
        atomicExch(&bar->err, 1);
        ok = 0;
        break;
      }
      if (spins > 64) __nanosleep(32);
    }
  }
  __syncthreads();
  return ok != 0;
}

__device__ __forceinline__ double block_sum(double s, double* red) {
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) red[32] = s;
  }
  __syncthreads();
  return red[32];
}

__global__ void __launch_bounds__(512) tridiag_persistent_kernel(double* A, int n, double* d,
                                                                 double* e, double* tau,
                                                                 double* pg, GridBar* bar) {
  // matrix entries written by other CTAs since the last barrier are read
  // through L2 (__ldcg): L1 is not coherent across SMs
  extern __shared__ double sv[];
  double* v = sv;        // n: Householder vector at indices k+1..n-1
  double* pw = sv + n;   // n: p at indices k+1..n-1
  __shared__ double red[40];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
  const unsigned int nb = gridDim.x;
  const int gw = blockIdx.x * nwarps + warp, gws = nb * nwarps;
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;
    // Householder vector of column k (every CTA, redundantly)
    double s = 0.0;
    for (int i = tid + 1; i < m; i += nt) {
      const double x = __ldcg(&A[(long long)(k + 1 + i) * n + k]);
      s += x * x;
    }
    const double sig = block_sum(s, red);
    const double x0 = __ldcg(&A[(long long)(k + 1) * n + k]);
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
    for (int i = tid; i < m; i += nt) {
      const double vi = (i == 0) ? v0 : __ldcg(&A[(long long)(k + 1 + i) * n + k]);
      v[k + 1 + i] = vi;
      if (blockIdx.x == 0) A[(long long)k * n + k + 1 + i] = vi;  // kept for back-transformation
    }
    if (blockIdx.x == 0 && tid == 0) {
      d[k] = __ldcg(&A[(long long)k * n + k]);
      e[k] = alpha;
      tau[k] = t;
    }
    __syncthreads();
    // p = t A22 v, one warp per row
    for (int r = gw; r < m; r += gws) {
      const int i = k + 1 + r;
      const double* row = A + (long long)i * n;
      double acc = 0.0;
      int j = k + 1 + lane;
      // eight independent loads in flight per lane
      for (; j + 7 * 32 < n; j += 8 * 32) {
        double a[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) a[u] = __ldcg(&row[j + 32 * u]);
#pragma unroll
        for (int u = 0; u < 8; ++u) acc += a[u] * v[j + 32 * u];
      }
      for (; j < n; j += 32) acc += __ldcg(&row[j]) * v[j];
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
      if (lane == 0) pg[i] = t * acc;
    }
    if (!grid_sync(bar, nb)) return;
    for (int j = tid; j < m; j += nt) pw[k + 1 + j] = __ldcg(&pg[k + 1 + j]);
    __syncthreads();
    double q = 0.0;
    for (int j = tid; j < m; j += nt) q += v[k + 1 + j] * pw[k + 1 + j];
    const double K = 0.5 * t * block_sum(q, red);
    // w = p - K v, once per CTA, so the update costs two FMA per element
    for (int j = tid; j < m; j += nt) pw[k + 1 + j] = fma(-K, v[k + 1 + j], pw[k + 1 + j]);
    __syncthreads();
    for (int r = gw; r < m; r += gws) {
      const int i = k + 1 + r;
      const double vi = v[i], wi = pw[i];
      double* row = A + (long long)i * n;
      int j = k + 1 + lane;
      for (; j + 7 * 32 < n; j += 8 * 32) {
        double a[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) a[u] = __ldcg(&row[j + 32 * u]);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int jj = j + 32 * u;
          row[jj] = fma(-vi, pw[jj], fma(-wi, v[jj], a[u]));
        }
      }
      for (; j < n; j += 32) row[j] = fma(-vi, pw[j], fma(-wi, v[j], __ldcg(&row[j])));
    }
    if (!grid_sync(bar, nb)) return;
  }
  if (blockIdx.x == 0 && tid == 0) {
    if (n >= 2) {
      d[n - 2] = __ldcg(&A[(long long)(n - 2) * n + n - 2]);
      e[n - 2] = __ldcg(&A[(long long)(n - 1) * n + n - 2]);
    }
    d[n - 1] = __ldcg(&A[(long long)(n - 1) * n + n - 1]);
  }
}

// The same reduction with the matrix resident in shared memory: CTA b owns
// the rows i = b, b + nb, b + 2 nb, ... for the whole reduction, so the
// rank-2 updates and the matrix-vector products never leave the SM; only
// the current column (colbuf) and p (pg) travel through L2.
__global__ void __launch_bounds__(512) tridiag_smem_kernel(double* A, int n, double* d, double* e,
                                                           double* tau, double* colbuf,
                                                           double* pg, GridBar* bar) {
  extern __shared__ double sm[];
  const int nb = (int)gridDim.x, b = (int)blockIdx.x;
  const int R = (n - b + nb - 1) / nb;      // rows owned by this CTA
  const int Rmax = (n + nb - 1) / nb;
  double* rows = sm;                        // Rmax x n
  double* v = rows + (size_t)Rmax * n;      // n
  double* pw = v + n;                       // n
  __shared__ double red[40];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
  for (int e2 = tid; e2 < R * n; e2 += nt) {
    const int li = e2 / n, j = e2 - li * n;
    rows[(size_t)li * n + j] = A[(size_t)(b + li * nb) * n + j];
  }
  __syncthreads();
  for (int li = tid; li < R; li += nt) colbuf[b + li * nb] = rows[(size_t)li * n + 0];
  if (!grid_sync(bar, nb)) return;
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;
    // Householder vector of column k from colbuf (rows k+1..n-1)
    // one pass over the column: x into v (shared), its squared norm
    double s = 0.0;
    for (int i = tid; i < m; i += nt) {
      const double x = __ldcg(&colbuf[k + 1 + i]);
      v[k + 1 + i] = x;
      if (i > 0) {
        s += x * x;
        if (b == 0) A[(size_t)k * n + k + 1 + i] = x;  // kept for back-transformation
      }
    }
    const double sig = block_sum(s, red);
    const double x0 = v[k + 1];
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
    __syncthreads();   // every thread has read x0 before it is replaced by v0
    if (tid == 0) {
      v[k + 1] = v0;
      if (b == 0) A[(size_t)k * n + k + 1] = v0;
    }
    if (tid == 0) {
      if (k % nb == b) d[k] = rows[(size_t)(k / nb) * n + k];
      if (b == 0) {
        e[k] = alpha;
        tau[k] = t;
      }
    }
    __syncthreads();
    // p_i = t sum_j A_ij v_j for the owned rows i > k, one warp per row
    const int li0 = (k + 1 - b + nb - 1) / nb;   // first owned row index > k
    for (int li = li0 + warp; li < R; li += nwarps) {
      const double* row = rows + (size_t)li * n;
      double acc = 0.0;
      for (int j = k + 1 + lane; j < n; j += 32) acc += row[j] * v[j];
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
      if (lane == 0) pg[b + li * nb] = t * acc;
    }
    if (!grid_sync(bar, nb)) return;
    for (int j = tid; j < m; j += nt) pw[k + 1 + j] = __ldcg(&pg[k + 1 + j]);
    __syncthreads();
    double q = 0.0;
    for (int j = tid; j < m; j += nt) q += v[k + 1 + j] * pw[k + 1 + j];
    const double K = 0.5 * t * block_sum(q, red);
    for (int j = tid; j < m; j += nt) pw[k + 1 + j] = fma(-K, v[k + 1 + j], pw[k + 1 + j]);
    __syncthreads();
    // rank-2 update of the owned rows; the next column goes to colbuf
    for (int li = li0 + warp; li < R; li += nwarps) {
      const int i = b + li * nb;
      double* row = rows + (size_t)li * n;
      const double vi = v[i], wi = pw[i];
      for (int j = k + 1 + lane; j < n; j += 32) row[j] = fma(-vi, pw[j], fma(-wi, v[j], row[j]));
      __syncwarp();
      if (lane == 0) colbuf[i] = row[k + 1];
    }
    if (!grid_sync(bar, nb)) return;
  }
  if (tid == 0) {
    if (n >= 2) {
      if ((n - 2) % nb == b) d[n - 2] = rows[(size_t)((n - 2) / nb) * n + n - 2];
      if ((n - 1) % nb == b) e[n - 2] = rows[(size_t)((n - 1) / nb) * n + n - 2];
    }
    if ((n - 1) % nb == b) d[n - 1] = rows[(size_t)((n - 1) / nb) * n + n - 1];
  }
}

// Number of eigenvalues of the tridiagonal (d, e) below x: sign changes of
// the leading principal minors p_i of T - x I (p_0 = 1), a zero minor
// counted as a change; both running minors are rescaled by a power of two
// when the newest leaves [2^-400, 2^400].
// SQ: the second array already holds the squared off-diagonals.
template <bool SQ>
__device__ int sturm_count(const double* __restrict__ d, const double* __restrict__ e, int n,
                           double x) {
  // sign and exponent tests on the bit patterns (integer pipe), leaving
  // three FP64 operations per step
  double p0 = 1.0, p1 = d[0] - x;
  if (p1 == 0.0) p1 = -DBL_MIN;
  int c = p1 < 0.0 ? 1 : 0;
  long long s1 = __double_as_longlong(p1);
  for (int i = 1; i < n; ++i) {
    const double ei = e[i - 1];
    double p2 = fma(d[i] - x, p1, -(SQ ? ei : ei * ei) * p0);
    long long s2 = __double_as_longlong(p2);
    if ((s2 << 1) == 0) {  // a zero minor counts as a sign change
      p2 = (s1 < 0) ? DBL_MIN : -DBL_MIN;
      s2 = __double_as_longlong(p2);
    }
    c += (int)((unsigned long long)(s2 ^ s1) >> 63);
    const int ex = (int)((s2 >> 52) & 0x7ff) - 1023;
    if (ex > 400 || ex < -400) {
      p2 = scalbn(p2, -ex);
      p1 = scalbn(p1, -ex);
      s2 = __double_as_longlong(p2);
    }
    p0 = p1;
    p1 = p2;
    s1 = s2;
  }
  return c;
}

__global__ void count_below_kernel(const double* d, const double* e, int n, double x, int* out) {
  *out = sturm_count<false>(d, e, n, x);
}

// One warp per eigenvalue index i_lo + warp; out[warp] = the eigenvalue.
// d and the squared off-diagonals are staged in shared memory (2n doubles).
__global__ void __launch_bounds__(256) multisection_kernel(const double* __restrict__ d,
                                                           const double* __restrict__ e, int n,
                                                           int i_lo, int m, double* out) {
  extern __shared__ double ms_smem[];
  double* ds = ms_smem;
  double* e2s = ms_smem + n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    ds[i] = d[i];
    e2s[i] = (i < n - 1) ? e[i] * e[i] : 0.0;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  // four eigenvalues per warp, eight lanes (eight shifts) each
  const int grp = lane >> 3, sub = lane & 7;
  if (w * 4 >= m) return;
  const int t = w * 4 + grp;                 // output slot of this lane group
  const int idx = i_lo + (t < m ? t : m - 1);
  // Gershgorin interval
  double a = DBL_MAX, b = -DBL_MAX;
  for (int j = lane; j < n; j += 32) {
    const double r = (j > 0 ? fabs(e[j - 1]) : 0.0) + (j < n - 1 ? fabs(e[j]) : 0.0);
    a = fmin(a, d[j] - r);
    b = fmax(b, d[j] + r);
  }
  for (int o = 16; o > 0; o >>= 1) {
    a = fmin(a, __shfl_xor_sync(0xffffffffu, a, o));
    b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
  }
  const double wdt = fmax(fabs(a), fabs(b));
  double lo = a - 2.0 * DBL_EPSILON * wdt - DBL_MIN;
  double hi = b + 2.0 * DBL_EPSILON * wdt + DBL_MIN;
  // every lane group keeps its own [lo, hi]; the warp loops until all four
  // groups have converged (or stopped making progress)
  bool done = false;
  for (int it = 0; it < 128; ++it) {
    done = done || (hi - lo <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + 4.0 * DBL_MIN);
    if (__all_sync(0xffffffffu, done)) break;
    const double x = lo + (hi - lo) * (double)(sub + 1) / 9.0;
    const int cnt = done ? 0 : sturm_count<true>(ds, e2s, n, x);
    const unsigned ball = __ballot_sync(0xffffffffu, cnt > idx);
    const unsigned mask = (ball >> (grp * 8)) & 0xffu;
    const double xprev = __shfl_up_sync(0xffffffffu, x, 1);
    const int l = mask ? __ffs(mask) - 1 : 7;
    const double xl = __shfl_sync(0xffffffffu, x, grp * 8 + l);
    const double xlp = __shfl_sync(0xffffffffu, xprev, grp * 8 + l);
    if (!done) {
      double nlo, nhi;
      if (mask == 0) {
        nlo = xl;        // above all eight shifts
        nhi = hi;
      } else {
        nhi = xl;
        nlo = (l > 0) ? xlp : lo;
      }
      if (nhi == hi && nlo == lo) done = true;  // no progress at this precision
      lo = nlo;
      hi = nhi;
    }
  }
  if (sub == 0 && t < m) out[t] = 0.5 * (lo + hi);
}

}  // namespace ofm

using namespace ofm;

// Returns OFM_OK when the persistent reduction ran; OFM_ERR_INVALID when it
// cannot be used here (the caller then takes the per-column launch path).
ofm_status ofm_tridiag_persistent(ofm_ctx* c, double* A, int n, double* d, double* e, double* tau,
                                  double* pg) {
  const size_t smem = 2 * (size_t)n * sizeof(double);
  if (n < 3 || smem > 200 * 1024) return OFM_ERR_INVALID;
  int dev = 0, coop = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (!coop) return OFM_ERR_INVALID;
  // shared-memory-resident variant when every CTA's rows fit (one CTA per SM)
  {
    const int nbs = sms;
    const size_t rmax = (size_t)(n + nbs - 1) / nbs;
    const size_t smem2 = (rmax * n + 2 * (size_t)n) * sizeof(double);
    int per_sm2 = 0;
    if (smem2 <= 200 * 1024 &&
        cudaFuncSetAttribute(tridiag_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem2) == cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, tridiag_smem_kernel, 512, smem2) ==
            cudaSuccess &&
        per_sm2 >= 1 && c->w_eval.cap >= (size_t)n * sizeof(double)) {
      OFM_TRY(ofm_ensure(c, c->w_bar, sizeof(GridBar), "grid barrier"));
      OFM_CUDA(c, cudaMemsetAsync(c->w_bar.p, 0, sizeof(GridBar), c->stream));
      GridBar* bar = (GridBar*)c->w_bar.p;
      double* colbuf = (double*)c->w_eval.p;
      int nn = n;
      void* args[] = {&A, &nn, &d, &e, &tau, &colbuf, &pg, &bar};
      OFM_CUDA(c, cudaLaunchCooperativeKernel((const void*)tridiag_smem_kernel, dim3(nbs), dim3(512),
                                              args, smem2, c->stream));
      GridBar hb{};
      OFM_CUDA(c, cudaMemcpyAsync(&hb, bar, sizeof(GridBar), cudaMemcpyDeviceToHost, c->stream));
      OFM_CUDA(c, cudaStreamSynchronize(c->stream));
      if (hb.err) return ofm_fail(c, OFM_ERR_TIMEOUT, "tridiagonal reduction: grid barrier wait exceeded its bound");
      return OFM_OK;
    }
    cudaGetLastError();
  }
  OFM_CUDA(c, cudaFuncSetAttribute(tridiag_persistent_kernel,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  OFM_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tridiag_persistent_kernel, 512, smem));
  if (per_sm < 1) return OFM_ERR_INVALID;
  // one CTA per SM: the FP64 pipes of every SM share the rank-2 updates
  // (FP64 issue rate per SM is low on this part), never more than co-resident
  const int nb = std::max(1, std::min(sms * per_sm, sms));
  OFM_TRY(ofm_ensure(c, c->w_bar, sizeof(GridBar), "grid barrier"));
  OFM_CUDA(c, cudaMemsetAsync(c->w_bar.p, 0, sizeof(GridBar), c->stream));
  GridBar* bar = (GridBar*)c->w_bar.p;
  void* args[] = {&A, &n, &d, &e, &tau, &pg, &bar};
  OFM_CUDA(c, cudaLaunchCooperativeKernel((const void*)tridiag_persistent_kernel, dim3(nb),
                                          dim3(512), args, smem, c->stream));
  GridBar hb{};
  OFM_CUDA(c, cudaMemcpyAsync(&hb, bar, sizeof(GridBar), cudaMemcpyDeviceToHost, c->stream));
  OFM_CUDA(c, cudaStreamSynchronize(c->stream));
  if (hb.err) return ofm_fail(c, OFM_ERR_TIMEOUT, "tridiagonal reduction: grid barrier wait exceeded its bound");
  return OFM_OK;
}

void launch_count_below(const double* d, const double* e, int n, double x, int* out, cudaStream_t s) {
  count_below_kernel<<<1, 1, 0, s>>>(d, e, n, x, out);
}

// Returns false when the tridiagonal is too long to stage in shared memory
// (the caller then bisects from global memory).
bool launch_multisection(const double* d, const double* e, int n, int i_lo, int m, double* out,
                         cudaStream_t s) {
  const size_t smem = 2 * (size_t)n * sizeof(double);
  if (smem > 200 * 1024) return false;
  static bool attr_set = false;
  if (!attr_set) {
    if (cudaFuncSetAttribute(multisection_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             200 * 1024) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    attr_set = true;
  }
  // two warps (eight eigenvalues) per CTA so that the work spreads over every SM
  const int per_block = 8;
  multisection_kernel<<<(m + per_block - 1) / per_block, 64, smem, s>>>(d, e, n, i_lo, m, out);
  return true;
}
