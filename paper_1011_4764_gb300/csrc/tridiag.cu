// Symmetric tridiagonal reduction and spectrum slicing for the window solve
// of Eq. 2 (after the reduction A = L^-1 H L^-T).
//
// 1. Householder reduction of A to tridiagonal form in ONE persistent
//    cooperative kernel: per column k, every CTA forms the Householder
//    vector itself, the CTAs compute p = tau A22 v by rows, meet at a grid
//    barrier and apply A22 -= v w^T + w v^T (w = p - (tau/2)(v^T p) v) by
//    rows.  With the matrix rows resident in shared memory one barrier per
//    column suffices (the next column travels with p as a published row);
//    the global-memory fallback meets twice.  The barrier spins a bounded
//    number of times and reports a timeout instead of hanging.
// 2. Eigenvalues by index with multisection: one CTA of one to four warps
//    per wanted eigenvalue; each thread counts the eigenvalues below one of
//    32-128 points of the current interval (Sturm sequence of T - x I
//    written as the three-term recurrence of the leading principal minors,
//    rescaled by powers of two, so a step needs no division), and the
//    interval shrinks 33- to 129-fold per round.
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

// Sum over the first four warps (one per SM sub-partition; their partial
// sums cover the whole range), in a fixed order.  Fewer warps than the whole
// CTA because each FP64 instruction of a warp occupies a sub-partition's
// FP64 pipe for many cycles: sixteen warps' shuffle trees cost more than
// the additions they save.
__device__ __forceinline__ double sum4(double s, double* red, double scale = 1.0) {
  if (threadIdx.x < 128) {
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  }
  __syncthreads();
  // one thread adds the four partials (the SM's FP64 unit is shared: the
  // same three additions in every warp would queue behind each other)
  if (threadIdx.x == 0) red[4] = scale * ((red[0] + red[1]) + (red[2] + red[3]));
  __syncthreads();
  return red[4];
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

// The same reduction with the matrix resident in shared memory and ONE
// grid barrier per column.  CTA b owns the rows i = b, b + nb, b + 2 nb, ...
// for the whole reduction.  At step k every CTA holds the whole column k of
// A_k and forms v itself; it computes p_i = tau (A_k v)_i for its rows, and
// the owner of row k+1 also publishes that row of A_k.  After the barrier
// every CTA has p and row k+1, forms w = p - (tau/2)(v.p) v, updates its own
// rows, and obtains column k+1 of A_{k+1} from row k+1 by symmetry:
//     A_{k+1}[k+1, i] = A_k[k+1, i] - v_{k+1} w_i - w_{k+1} v_i,
// the same expression (same rounding) the owner applies to its copy of the
// row.  So the next Householder vector needs no second exchange.  p and the
// published row are double-buffered by the parity of k: a CTA that runs
// ahead into step k+1 writes the other half while slower CTAs still read.
__global__ void __launch_bounds__(512) tridiag_smem_kernel(double* A, int n, double* d, double* e,
                                                           double* tau, double* xbuf,
                                                           GridBar* bar) {
  extern __shared__ double sm[];
  const int nb = (int)gridDim.x, b = (int)blockIdx.x;
  const int R = (n - b + nb - 1) / nb;      // rows owned by this CTA
  const int Rmax = (n + nb - 1) / nb;
  double* rows = sm;                        // Rmax x n
  double* v = rows + (size_t)Rmax * n;      // n: Householder vector (indices k+1..n-1)
  double* w = v + n;                        // n: p, then w
  double* col = w + n;                      // n: column k of A_k (indices k+1..n-1)
  double* rk = col + n;                     // n: row k+1 of A_k (indices k+1..n-1)
  __shared__ double red[40];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
  for (int e2 = tid; e2 < R * n; e2 += nt) {
    const int li = e2 / n, j = e2 - li * n;
    rows[(size_t)li * n + j] = A[(size_t)(b + li * nb) * n + j];
  }
  for (int j = tid; j < n; j += nt) col[j] = A[j];   // column 0 = row 0 (A is symmetric)
  // nobody reads A after this barrier; CTA 0 then stores the Householder vectors in it
  if (!grid_sync(bar, nb)) return;
  __shared__ double hh[4];   // alpha, tau, v0, tau / 2 of the current column
  for (int k = 0; k + 2 < n; ++k) {
    double s = 0.0;
    if (tid < 128)
      for (int i = k + 2 + tid; i < n; i += 128) s += col[i] * col[i];
    const double sig = sum4(s, red);
    // the scalar part once (FP64 square root and division are long
    // sequences), broadcast through shared memory
    if (tid == 0) {
      const double x0 = col[k + 1];
      if (sig == 0.0) {
        hh[0] = x0;
        hh[1] = 0.0;
        hh[2] = 1.0;
      } else {
        const double nrm = sqrt(x0 * x0 + sig);
        const double al = (x0 > 0.0) ? -nrm : nrm;
        const double vv = x0 - al;
        hh[0] = al;
        hh[1] = 2.0 / (vv * vv + sig);
        hh[2] = vv;
      }
      hh[3] = 0.5 * hh[1];
    }
    __syncthreads();
    const double alpha = hh[0], t = hh[1], v0 = hh[2];
    for (int i = k + 1 + tid; i < n; i += nt) {
      const double vi = (i == k + 1) ? v0 : col[i];
      v[i] = vi;
      if (b == 0) A[(size_t)k * n + i] = vi;   // kept for back-transformation
    }
    if (tid == 0) {
      if (k % nb == b) d[k] = rows[(size_t)(k / nb) * n + k];
      if (b == 0) {
        e[k] = alpha;
        tau[k] = t;
      }
    }
    __syncthreads();
    double* pb = xbuf + (size_t)(k & 1) * n;
    double* rb = xbuf + 2 * (size_t)n + (size_t)(k & 1) * n;
    // p_i = t sum_j A_ij v_j for the owned rows i > k, one warp per row
    const int li0 = (k + 1 - b + nb - 1) / nb;   // first owned row index > k
    for (int li = li0 + warp; li < R; li += nwarps) {
      const double* row = rows + (size_t)li * n;
      double acc = 0.0;
      for (int j = k + 1 + lane; j < n; j += 32) acc += row[j] * v[j];
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
      if (lane == 0) pb[b + li * nb] = t * acc;
    }
    if ((k + 1) % nb == b) {
      const double* row = rows + (size_t)((k + 1) / nb) * n;
      for (int j = k + 1 + tid; j < n; j += nt) rb[j] = row[j];
    }
    if (!grid_sync(bar, nb)) return;
    for (int j = k + 1 + tid; j < n; j += nt) {
      w[j] = __ldcg(&pb[j]);
      rk[j] = __ldcg(&rb[j]);
    }
    __syncthreads();
    double q = 0.0;
    if (tid < 128)
      for (int j = k + 1 + tid; j < n; j += 128) q += v[j] * w[j];
    const double K = sum4(q, red, hh[3]);   // (tau / 2) v.p
    for (int j = k + 1 + tid; j < n; j += nt) w[j] = fma(-K, v[j], w[j]);
    __syncthreads();
    // rank-2 update of the owned rows i > k
    for (int li = li0 + warp; li < R; li += nwarps) {
      const int i = b + li * nb;
      double* row = rows + (size_t)li * n;
      const double vi = v[i], wi = w[i];
      for (int j = k + 1 + lane; j < n; j += 32) row[j] = fma(-vi, w[j], fma(-wi, v[j], row[j]));
    }
    // column k+1 of A_{k+1} from row k+1 (same expression as the owner's update)
    {
      const double vk = v[k + 1], wk = w[k + 1];
      for (int i = k + 2 + tid; i < n; i += nt) col[i] = fma(-vk, w[i], fma(-wk, v[i], rk[i]));
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (n >= 2) {
      if ((n - 2) % nb == b) d[n - 2] = rows[(size_t)((n - 2) / nb) * n + n - 2];
      if ((n - 1) % nb == b) e[n - 2] = rows[(size_t)((n - 1) / nb) * n + n - 2];
    }
    if ((n - 1) % nb == b) d[n - 1] = rows[(size_t)((n - 1) / nb) * n + n - 1];
  }
}

// Number of eigenvalues of the tridiagonal (d, e2 = squared off-diagonals)
// below each of K shifts x[k]: sign changes of the leading principal minors
// p_i of T - x I (p_0 = 1; a minor that is exactly zero counts with the sign
// of its sign bit, which gives the standard count away from exact
// eigenvalues).  The K recurrences are interleaved (independent chains hide
// the FP64 latency); the running pair of minors is rescaled by a power of
// two every 8 steps when it leaves [2^-400, 2^400] (at most a factor 2^40
// of growth per 8 steps for the matrices here, far from overflow).
template <int K>
__device__ __forceinline__ void sturm_counts(const double* __restrict__ d,
                                             const double* __restrict__ e2, int n,
                                             const double* x, int* cnt) {
  double p0[K], p1[K];
  int c[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    p0[k] = 1.0;
    p1[k] = d[0] - x[k];
    c[k] = (int)((unsigned long long)__double_as_longlong(p1[k]) >> 63);
  }
  int i = 1;
  while (i < n) {
    const int stop = min(n, i + 8);
    for (; i < stop; ++i) {
      const double di = d[i], ei = e2[i - 1];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const double p2 = fma(di - x[k], p1[k], -ei * p0[k]);
        c[k] += (int)((unsigned long long)(__double_as_longlong(p2) ^ __double_as_longlong(p1[k])) >> 63);
        p0[k] = p1[k];
        p1[k] = p2;
      }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int ex = (int)((__double_as_longlong(p1[k]) >> 52) & 0x7ff) - 1023;
      if (ex > 400 || ex < -400) {
        p1[k] = scalbn(p1[k], -ex);
        p0[k] = scalbn(p0[k], -ex);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < K; ++k) cnt[k] = c[k];
}

// Counts below two shifts (the window ends) in one pass; e holds the
// off-diagonals themselves.
__global__ void count_below_kernel(const double* d, const double* e, int n, double x0, double x1,
                                   int* out) {
  extern __shared__ double cb_smem[];
  double* ds = cb_smem;
  double* e2s = cb_smem + n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    ds[i] = d[i];
    e2s[i] = (i < n - 1) ? e[i] * e[i] : 0.0;
  }
  __syncthreads();
  // one shift per warp (separate SM sub-partitions)
  if ((threadIdx.x & 31) == 0 && threadIdx.x < 64) {
    const int k = threadIdx.x >> 5;
    double x[1] = {k ? x1 : x0};
    int c[1];
    sturm_counts<1>(ds, e2s, n, x, c);
    out[k] = c[0];
  }
}

// Multisection: one CTA of MS_W warps per wanted eigenvalue index; thread j
// counts the eigenvalues below the shift x_j = lo + (hi - lo)(j + 1)/(S + 1)
// (S = 32 MS_W shifts), and the interval shrinks to the (S + 1)-th part
// holding the eigenvalue.  On this part one warp issues an FP64 instruction
// every 64 cycles at best while an SM retires one warp-wide FP64
// instruction about every 19 cycles: up to four warps per SM cost little
// more time per round than one, beyond that time grows with the warp
// count.  So few wanted eigenvalues take four warps each (129-section,
// fewest rounds); many take one (33-section, least work).  d and e^2 are
// staged in shared memory.
template <int MS_W>
__global__ void __launch_bounds__(32 * MS_W) multisection_kernel(const double* __restrict__ d,
                                                                 const double* __restrict__ e,
                                                                 int n, int i_lo, int m,
                                                                 double* out) {
  constexpr int MS_S = 32 * MS_W;
  extern __shared__ double ms_smem[];
  __shared__ int firstw[MS_W];
  __shared__ double gl[2 * MS_W];
  double* ds = ms_smem;
  double* e2s = ms_smem + n;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int t = blockIdx.x;
  if (t >= m) return;   // uniform over the CTA
  const int idx = i_lo + t;
  // staged d, e^2 and the Gershgorin interval
  double a = DBL_MAX, b = -DBL_MAX;
  for (int i = tid; i < n; i += blockDim.x) {
    ds[i] = d[i];
    e2s[i] = (i < n - 1) ? e[i] * e[i] : 0.0;
    const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i < n - 1 ? fabs(e[i]) : 0.0);
    a = fmin(a, d[i] - r);
    b = fmax(b, d[i] + r);
  }
  for (int o = 16; o > 0; o >>= 1) {
    a = fmin(a, __shfl_xor_sync(0xffffffffu, a, o));
    b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
  }
  if (lane == 0) {
    gl[warp] = a;
    gl[MS_W + warp] = b;
  }
  __syncthreads();
  for (int w = 0; w < MS_W; ++w) {
    a = fmin(a, gl[w]);
    b = fmax(b, gl[MS_W + w]);
  }
  const double wdt = fmax(fabs(a), fabs(b));
  double lo = a - 2.0 * DBL_EPSILON * wdt - DBL_MIN;
  double hi = b + 2.0 * DBL_EPSILON * wdt + DBL_MIN;
  for (int it = 0; it < 64; ++it) {
    if (hi - lo <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + 4.0 * DBL_MIN) break;
    double x[1];
    int cnt[1];
    x[0] = lo + (hi - lo) * (double)(tid + 1) / (MS_S + 1);
    sturm_counts<1>(ds, e2s, n, x, cnt);
    const unsigned ball = __ballot_sync(0xffffffffu, cnt[0] > idx);
    if (lane == 0) firstw[warp] = ball ? __ffs(ball) - 1 : 32;
    __syncthreads();
    int j = MS_S;   // first shift with more than idx eigenvalues below
    for (int w = MS_W - 1; w >= 0; --w)
      if (firstw[w] < 32) j = w * 32 + firstw[w];
    __syncthreads();   // firstw is rewritten next round
    double nlo, nhi;
    if (j == MS_S) {   // above every shift
      nlo = lo + (hi - lo) * (double)MS_S / (MS_S + 1);
      nhi = hi;
    } else {
      nhi = lo + (hi - lo) * (double)(j + 1) / (MS_S + 1);
      nlo = (j > 0) ? lo + (hi - lo) * (double)j / (MS_S + 1) : lo;
    }
    if (nhi == hi && nlo == lo) break;   // no progress at this precision
    lo = nlo;
    hi = nhi;
  }
  if (tid == 0) out[t] = 0.5 * (lo + hi);
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
    const size_t smem2 = (rmax * n + 4 * (size_t)n) * sizeof(double);
    int per_sm2 = 0;
    if (smem2 <= 200 * 1024 &&
        cudaFuncSetAttribute(tridiag_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem2) == cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, tridiag_smem_kernel, 512, smem2) ==
            cudaSuccess &&
        per_sm2 >= 1 && c->w_eval.cap >= 4 * (size_t)n * sizeof(double)) {
      OFM_TRY(ofm_ensure(c, c->w_bar, sizeof(GridBar), "grid barrier"));
      OFM_CUDA(c, cudaMemsetAsync(c->w_bar.p, 0, sizeof(GridBar), c->stream));
      GridBar* bar = (GridBar*)c->w_bar.p;
      double* xbuf = (double*)c->w_eval.p;   // p and the published row, two halves each
      int nn = n;
      void* args[] = {&A, &nn, &d, &e, &tau, &xbuf, &bar};
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

void launch_count_below(const double* d, const double* e, int n, double x0, double x1, int* out,
                        cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(count_below_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  count_below_kernel<<<1, 256, 2 * (size_t)n * sizeof(double), s>>>(d, e, n, x0, x1, out);
}

// Returns false when the tridiagonal is too long to stage in shared memory
// (the caller then bisects from global memory).
bool launch_multisection(const double* d, const double* e, int n, int i_lo, int m, double* out,
                         cudaStream_t s) {
  const size_t smem = 2 * (size_t)n * sizeof(double);
  if (smem > 200 * 1024) return false;
  static bool attr_set = false;
  if (!attr_set) {
    if (cudaFuncSetAttribute(multisection_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             200 * 1024) != cudaSuccess ||
        cudaFuncSetAttribute(multisection_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             200 * 1024) != cudaSuccess ||
        cudaFuncSetAttribute(multisection_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             200 * 1024) != cudaSuccess ||
        cudaFuncSetAttribute(count_below_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             200 * 1024) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    attr_set = true;
  }
  // about four warps per SM of the GB300 (152 SMs) in total
  const long long slots = 4LL * 152;
  if ((long long)m * 4 <= slots)
    multisection_kernel<4><<<m, 128, smem, s>>>(d, e, n, i_lo, m, out);
  else if ((long long)m * 2 <= slots)
    multisection_kernel<2><<<m, 64, smem, s>>>(d, e, n, i_lo, m, out);
  else
    multisection_kernel<1><<<m, 32, smem, s>>>(d, e, n, i_lo, m, out);
  return true;
}
