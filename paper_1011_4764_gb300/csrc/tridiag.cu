// Symmetric tridiagonal reduction and spectrum slicing for the window solve
// of Eq. 2 (after the reduction A = L^-1 H L^-T).
//
// 1. Householder reduction of A to tridiagonal form in ONE persistent
//    cooperative kernel: per column k, every CTA forms the Householder
//    vector itself, the CTAs compute p = tau A22 v by rows, exchange p and
//    apply A22 -= v w^T + w v^T (w = p - (tau/2)(v^T p) v) by rows.  With the
//    matrix rows resident in shared memory the exchange is a set of
//    generation-tagged published values (no barrier; the next column travels
//    as a published row); the global-memory fallback meets at a grid barrier
//    twice per column.  Every wait spins a bounded number of times and
//    reports a timeout instead of hanging.
// 2. Eigenvalues by index with multisection: one CTA of one to four warps
//    per wanted eigenvalue; each thread counts the eigenvalues below one of
//    32-128 points of the current interval, and the interval shrinks 33- to
//    129-fold per round.  FP32 counts (LDL^T pivots) narrow it first; FP64
//    counts (Sturm sequence of T - x I written as the three-term recurrence
//    of the leading principal minors, rescaled by powers of two, so a step
//    needs no division) check the bracket and finish.
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
  unsigned int hold;    // test of the failure detection: CTA 0 withholds its first arrival
  unsigned int limit;   // polls before a wait gives up (0: 2^24)
  unsigned int pad[28];
};

// All CTAs of a cooperative launch meet here: one release atomic per CTA
// and acquire polls of the counter.  Returns false (and sets bar->err) when
// the wait exceeded its bound or another CTA gave up.
__device__ bool grid_sync(GridBar* bar, unsigned int nblocks) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile int* verr = &bar->err;
    // a held arrival (test hook, CTA 0 once): nobody reaches the target, every
    // CTA's wait runs out
    const bool skip = blockIdx.x == 0 && atomicExch(&bar->hold, 0u) != 0u;
    unsigned int old = 0;
    if (!skip)
      asm volatile("atom.add.release.gpu.global.u32 %0, [%1], 1;" : "=r"(old) : "l"(&bar->count) : "memory");
    const unsigned int target = (old / nblocks + 1u) * nblocks;
    const unsigned int lim = *(volatile unsigned int*)&bar->limit ? *(volatile unsigned int*)&bar->limit : (1u << 24);
    ok = 1;
    unsigned int spins = 0;
    while (true) {
      unsigned int cur;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(&bar->count) : "memory");
      if ((int)(cur - target) >= 0) break;
      if (*verr != 0 || ++spins > lim) {
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

// The same reduction with the matrix resident in shared memory and no grid
// barrier inside the column loop.  CTA b owns the rows i = b, b + nb, ... for
// the whole reduction, and every CTA keeps the whole current column k of A_k
// (the Householder vector v is that column with v_{k+1} = x0 - alpha).
//
// Exchange.  The values a CTA needs from the others at column k are p_j =
// tau (A_k v)_j for every j > k and row k+1 of A_k.  Each is published as two
// 64-bit words, each holding 32 bits of the value and the column's generation
// k+1 in the other 32 (an aligned 64-bit store is single-copy atomic), so a
// reader that sees both words with the current generation has the value: no
// counter, no barrier, one L2 round trip between the last writer and the
// readers.  The slots are double-buffered by the parity of k.  A CTA writes
// column k+2's values into a slot only after it has read every p of column
// k+1, and each CTA that still reads column k's values writes some p of
// column k+1 only after that read, so no slot is overwritten while read.
// CTAs whose rows are all done leave the loop.
//
// Work per column, warp-specialised (warps 0-11 own matrix rows, warps 12-15
// the vector work):
//   rows:   p_i = tau (A_k col)_i - tau alpha A_k[i, k+1] (v differs from the
//           column only in entry k+1, so the product starts before alpha and
//           tau exist); after the exchange, pass 1 of the rank-2 update
//           A -= v p^T while the vector warps form K; then pass 2,
//           A -= c v^T with c = p - 2 K v, fused with the next column's
//           product.  Together: A -= v w^T + w v^T with w = p - K v.
//   vector: K = (tau/2) v.p, column k+1 of A_{k+1} from the published row,
//           A_{k+1}[k+1, i] = A_k[k+1, i] - v_{k+1} w_i - w_{k+1} v_i,
//           its norm, and the next alpha, tau (one thread: the FP64 square
//           root and division run while the row warps compute).
namespace {

constexpr int TRI_THREADS = 512;
constexpr int TRI_ROW_WARPS = 12;           // warps 0..11
constexpr int TRI_VEC0 = 32 * TRI_ROW_WARPS;  // threads 384..511
constexpr int TRI_PMAX = 8;                 // published entries polled per thread, at most
constexpr int TRI_RMAX = 16;                // rows per CTA, at most

struct __align__(16) Pub {
  unsigned long long a, b;
};

__device__ __forceinline__ void pub_put(Pub* dst, double x, unsigned int gen) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const unsigned long long g = (unsigned long long)gen << 32;
  const unsigned long long lo = (bits & 0xffffffffull) | g, hi = (bits >> 32) | g;
  asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(dst), "l"(lo), "l"(hi)
               : "memory");
}

__device__ __forceinline__ void pub_get(const Pub* src, unsigned long long& lo,
                                        unsigned long long& hi) {
  asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(lo), "=l"(hi) : "l"(src)
               : "memory");
}

__device__ __forceinline__ void named_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

__device__ __forceinline__ void named_arrive(int id, int count) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}

__device__ __forceinline__ double warp_allsum(double s) {
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// alpha, tau, v0, tau/2 of the reflector that maps (x0, x_rest) to
// (alpha, 0), with sig = |x_rest|^2 (the sign of alpha opposite to x0's).
__device__ __forceinline__ void house_scalars(double x0, double sig, double* hh) {
  if (sig == 0.0) {
    hh[0] = x0;
    hh[1] = 0.0;
    hh[2] = 1.0;
  } else {
    const double nrm = sqrt(fma(x0, x0, sig));
    const double al = (x0 > 0.0) ? -nrm : nrm;
    const double vv = x0 - al;
    hh[0] = al;
    hh[1] = 2.0 / fma(vv, vv, sig);
    hh[2] = vv;
  }
  hh[3] = 0.5 * hh[1];
}

// Polls the published p_j and A_k[k+1, j] (j = k+1 .. n-1) into pw and rk.
// Returns false when the wait exceeded its bound or another CTA gave up.
__device__ __forceinline__ bool poll_column(const Pub* P, const Pub* Rw, int k, int n,
                                            unsigned int gen, double* pw, double* rk,
                                            GridBar* bar) {
  const int m1 = n - k - 1, tot = 2 * m1, tid = threadIdx.x;
  unsigned int pend = 0;
#pragma unroll
  for (int q = 0; q < TRI_PMAX; ++q)
    if (tid + q * TRI_THREADS < tot) pend |= 1u << q;
  unsigned int spins = 0;
  while (pend) {
    unsigned long long lo[TRI_PMAX], hi[TRI_PMAX];
#pragma unroll
    for (int q = 0; q < TRI_PMAX; ++q)
      if ((pend >> q) & 1u) {
        const int e = tid + q * TRI_THREADS;
        pub_get(e < m1 ? P + (k + 1 + e) : Rw + (k + 1 + e - m1), lo[q], hi[q]);
      }
#pragma unroll
    for (int q = 0; q < TRI_PMAX; ++q)
      if (((pend >> q) & 1u) && (unsigned int)(lo[q] >> 32) == gen &&
          (unsigned int)(hi[q] >> 32) == gen) {
        const int e = tid + q * TRI_THREADS;
        const double x =
            __longlong_as_double((long long)(((hi[q] & 0xffffffffull) << 32) | (lo[q] & 0xffffffffull)));
        if (e < m1)
          pw[k + 1 + e] = x;
        else
          rk[k + 1 + e - m1] = x;
        pend &= ~(1u << q);
      }
    if (pend) {
      ++spins;
      if (spins > (1u << 22) || ((spins & 255u) == 0 && *(volatile int*)&bar->err != 0)) {
        atomicExch(&bar->err, 1);
        return false;
      }
      if (spins > 8) __nanosleep(32);
    }
  }
  return true;
}

}  // namespace

__global__ void __launch_bounds__(TRI_THREADS) tridiag_smem_kernel(double* A, int n, double* d,
                                                                   double* e, double* tau,
                                                                   Pub* pub, GridBar* bar) {
  extern __shared__ double sm[];
  const int nb = (int)gridDim.x, b = (int)blockIdx.x;
  const int R = (n - b + nb - 1) / nb;        // rows owned by this CTA (nb < n: R >= 1)
  const int Rmax = (n + nb - 1) / nb;
  const int ilast = b + (R - 1) * nb;         // last owned row
  double* rows = sm;                          // Rmax x n
  double* cb0 = rows + (size_t)Rmax * n;      // columns k (even k) ...
  double* cb1 = cb0 + n;                      // ... and k (odd k)
  double* pw = cb1 + n;                       // p of the current column
  double* rk = pw + n;                        // published row k+1 of A_k
  __shared__ double redq[4], reds[4], us[TRI_RMAX], rs[TRI_RMAX];
  __shared__ double hh[4];   // alpha, tau, v0, tau / 2 of the current column
  __shared__ double Ks;      // (tau / 2) v.p of the last completed column
  __shared__ int s_err;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool vecw = tid >= TRI_VEC0;
  const int vt = tid - TRI_VEC0;
  for (int e2 = tid; e2 < R * n; e2 += TRI_THREADS) {
    const int li = e2 / n, j = e2 - li * n;
    rows[(size_t)li * n + j] = A[(size_t)(b + li * nb) * n + j];
  }
  for (int j = tid; j < n; j += TRI_THREADS) {
    cb0[j] = A[j];   // column 0 = row 0 (A is symmetric)
    cb1[j] = 0.0;    // no update precedes column 0
  }
  if (tid == 0) {
    s_err = 0;
    Ks = 0.0;
    if (b == 0) d[0] = A[0];
  }
  // nobody reads A after this barrier; the Householder vectors go into it
  if (!grid_sync(bar, nb)) return;
  if (vecw) {   // reflector of column 0
    double s = 0.0;
    for (int i = 2 + vt; i < n; i += 128) s = fma(cb0[i], cb0[i], s);
    s = warp_allsum(s);
    if (lane == 0) reds[warp - TRI_ROW_WARPS] = s;
    __syncwarp();
    named_sync(1, 128);
    if (vt == 0) house_scalars(cb0[1], (reds[0] + reds[1]) + (reds[2] + reds[3]), hh);
  }
  for (int k = 0; k + 2 < n; ++k) {
    double* cur = (k & 1) ? cb1 : cb0;   // column k of A_k
    double* prv = (k & 1) ? cb0 : cb1;   // v of column k-1, then column k+1
    Pub* P = pub + (size_t)(k & 1) * 2 * n;
    Pub* Rw = P + n;
    const unsigned int gen = (unsigned int)k + 1u;
    const int la = (k + 1 - b + nb - 1) / nb;   // first owned row > k
    if (!vecw) {
      // pass 2 of column k-1 fused with u_i = (A_k col)_i for the owned rows
      // i > k, one warp per row
      const double K2 = 2.0 * Ks;
      for (int li = la + warp; li < R; li += TRI_ROW_WARPS) {
        const int i = b + li * nb;
        double* row = rows + (size_t)li * n;
        const double ci = (k > 0) ? fma(-K2, prv[i], pw[i]) : 0.0;
        // two independent chains per lane
        double acc0 = 0.0, acc1 = 0.0;
        int j = k + 1 + lane;
        for (; j + 32 < n; j += 64) {
          const double ra = fma(-ci, prv[j], row[j]);
          const double rb = fma(-ci, prv[j + 32], row[j + 32]);
          row[j] = ra;
          row[j + 32] = rb;
          acc0 = fma(ra, cur[j], acc0);
          acc1 = fma(rb, cur[j + 32], acc1);
        }
        if (j < n) {
          const double ra = fma(-ci, prv[j], row[j]);
          row[j] = ra;
          acc0 = fma(ra, cur[j], acc0);
        }
        const double acc = warp_allsum(acc0 + acc1);
        __syncwarp();
        if (i == k + 1)   // row k+1 of A_k for every CTA (each lane its own entries)
          for (int jj = k + 1 + lane; jj < n; jj += 32) pub_put(Rw + jj, row[jj], gen);
        if (lane == 0) {
          us[li] = acc;
          rs[li] = row[k + 1];
        }
      }
    }
    __syncthreads();   // reflector of column k and the row products complete
    {
      const double al = hh[0], t = hh[1];
      for (int li = la + tid; li < R; li += TRI_THREADS)
        pub_put(P + (b + li * nb), t * fma(-al, rs[li], us[li]), gen);
    }
    if (b == (k + 1) % nb && vecw) {   // owner of row k+1 keeps the reflector
      for (int j = k + 1 + vt; j < n; j += 128) A[(size_t)k * n + j] = (j == k + 1) ? hh[2] : cur[j];
      if (vt == 0) {
        e[k] = hh[0];
        tau[k] = hh[1];
      }
    }
    if (ilast < k + 2) break;   // every owned row is finished
    if (!poll_column(P, Rw, k, n, gen, pw, rk, bar)) s_err = 1;
    __syncthreads();   // p and row k+1 of A_k are here
    if (s_err) return;
    if (vecw) {
      // column k+1 of A_{k+1}:  A_k[k+1, i] - v_{k+1} w_i - w_{k+1} v_i
      //   = (A_k[k+1, i] - v0 p_i) + (2 v0 K - p_{k+1}) v_i,
      // the first part formed while K is being reduced
      const double v0 = hh[2], hk = hh[3];
      double q = (vt == 0) ? v0 * pw[k + 1] : 0.0;
      for (int j = k + 2 + vt; j < n; j += 128) {
        q = fma(cur[j], pw[j], q);
        prv[j] = fma(-v0, pw[j], rk[j]);
      }
      q = warp_allsum(q);
      if (lane == 0) redq[warp - TRI_ROW_WARPS] = q;
      __syncwarp();
      named_sync(1, 128);
      const double K = hk * ((redq[0] + redq[1]) + (redq[2] + redq[3]));
      const double wk1 = fma(-K, v0, pw[k + 1]);
      const double beta = fma(2.0 * v0, K, -pw[k + 1]);
      double s = 0.0;
      for (int i = k + 2 + vt; i < n; i += 128) {
        const double x = fma(beta, cur[i], prv[i]);
        prv[i] = x;
        if (i > k + 2) s = fma(x, x, s);
      }
      if (vt == 0) {
        Ks = K;
        if (b == (k + 2) % nb) d[k + 1] = fma(-2.0 * v0, wk1, rk[k + 1]);
      }
      __syncwarp();
      named_arrive(2, TRI_THREADS);   // K and column k+1 are ready
      s = warp_allsum(s);
      if (lane == 0) reds[warp - TRI_ROW_WARPS] = s;
      __syncwarp();
      named_sync(1, 128);
      if (vt == 0) house_scalars(prv[k + 2], (reds[0] + reds[1]) + (reds[2] + reds[3]), hh);
    } else {
      // pass 1 of column k on the owned rows i > k+1: A_ij -= v_i p_j
      const int lb = (k + 2 - b + nb - 1) / nb;
      for (int li = lb + warp; li < R; li += TRI_ROW_WARPS) {
        double* row = rows + (size_t)li * n;
        const double vi = cur[b + li * nb];
        for (int j = k + 2 + lane; j < n; j += 32) row[j] = fma(-vi, pw[j], row[j]);
      }
      named_sync(2, TRI_THREADS);
    }
  }
  __syncthreads();
  if (tid == 0 && b == (n - 1) % nb) {
    // last row: pass 2 of column n-3 on its diagonal, and the last off-diagonal
    const double* v = (((n - 3) & 1) ? cb1 : cb0);
    const double* cl = (((n - 2) & 1) ? cb1 : cb0);
    const double c = fma(-2.0 * Ks, v[n - 1], pw[n - 1]);
    d[n - 1] = fma(-c, v[n - 1], rows[(size_t)((n - 1) / nb) * n + n - 1]);
    e[n - 2] = cl[n - 1];
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

// Number of eigenvalues of the tridiagonal below x in FP32 (pivots of the
// LDL^T factorisation of T - x I: q_0 = d_0 - x, q_i = (d_i - x) -
// e2_{i-1} / q_{i-1}, counted when negative; a pivot below pivmin in
// magnitude becomes -pivmin).  Only used to narrow a bracket that FP64
// counts then check, so the fast division is enough.
__device__ __forceinline__ int sturm_count_f32(const float* __restrict__ d,
                                               const float* __restrict__ e2, int n, float x,
                                               float pivmin) {
  float q = d[0] - x;
  if (fabsf(q) < pivmin) q = -pivmin;
  int c = q < 0.f ? 1 : 0;
  for (int i = 1; i < n; ++i) {
    q = (d[i] - x) - __fdividef(e2[i - 1], q);
    if (fabsf(q) < pivmin) q = -pivmin;
    c += q < 0.f ? 1 : 0;
  }
  return c;
}

// Multisection: one CTA of MS_W warps per wanted eigenvalue index; thread j
// counts the eigenvalues below the shift x_j = lo + (hi - lo)(j + 1)/(S + 1)
// (S = 32 MS_W shifts), and the interval shrinks to the (S + 1)-th part
// holding the eigenvalue.  On this part one warp issues an FP64 instruction
// every 64 cycles at best while an SM retires one warp-wide FP64
// instruction about every 19 cycles: up to four warps per SM cost little
// more time per round than one, beyond that time grows with the warp
// count.  So few wanted eigenvalues take four warps each (129-section,
// fewest rounds); many take one (33-section, least work).
// Two phases: FP32 counts (fast: FP32 issues every cycle) narrow the
// Gershgorin interval to about 2e-5 of the spectrum's scale; the bracket,
// widened by 1e-5 of the scale (far above the FP32 counts' error), is
// checked by the first FP64 round, whose shifts include both ends, and FP64
// rounds finish.  A bracket that misses the eigenvalue sends the search back
// to the Gershgorin interval.  d and e^2 (both precisions) are staged in
// shared memory.
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
  float* dsf = reinterpret_cast<float*>(ms_smem + 2 * (size_t)n);
  float* e2f = dsf + n;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int t = blockIdx.x;
  if (t >= m) return;   // uniform over the CTA
  const int idx = i_lo + t;
  // staged d, e^2 and the Gershgorin interval
  double a = DBL_MAX, b = -DBL_MAX;
  for (int i = tid; i < n; i += blockDim.x) {
    const double e2 = (i < n - 1) ? e[i] * e[i] : 0.0;
    ds[i] = d[i];
    e2s[i] = e2;
    dsf[i] = (float)d[i];
    e2f[i] = (float)e2;
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
  const double lo0 = a - 2.0 * DBL_EPSILON * wdt - DBL_MIN;
  const double hi0 = b + 2.0 * DBL_EPSILON * wdt + DBL_MIN;
  double lo = lo0, hi = hi0;
  // index (0..S) of the first shift with more than idx eigenvalues below
  auto first_above = [&](int cnt) -> int {
    const unsigned ball = __ballot_sync(0xffffffffu, cnt > idx);
    if (lane == 0) firstw[warp] = ball ? __ffs(ball) - 1 : 32;
    __syncthreads();
    int j = MS_S;
    for (int w = MS_W - 1; w >= 0; --w)
      if (firstw[w] < 32) j = w * 32 + firstw[w];
    __syncthreads();   // firstw is rewritten next round
    return j;
  };
  auto shrink = [&](int j) -> bool {   // false: no progress at this precision
    double nlo, nhi;
    if (j == MS_S) {   // above every shift
      nlo = lo + (hi - lo) * (double)MS_S / (MS_S + 1);
      nhi = hi;
    } else {
      nhi = lo + (hi - lo) * (double)(j + 1) / (MS_S + 1);
      nlo = (j > 0) ? lo + (hi - lo) * (double)j / (MS_S + 1) : lo;
    }
    if (nhi == hi && nlo == lo) return false;
    lo = nlo;
    hi = nhi;
    return true;
  };
  // phase 1: FP32 counts
  const float pivmin = 1e-30f;
  bool narrowed = false;
  if (wdt > 0.0 && wdt < 1e30) {
    for (int it = 0; it < 32; ++it) {
      if (hi - lo <= 2e-5 * wdt) break;
      const double x = lo + (hi - lo) * (double)(tid + 1) / (MS_S + 1);
      if (!shrink(first_above(sturm_count_f32(dsf, e2f, n, (float)x, pivmin)))) break;
      narrowed = true;
    }
  }
  if (narrowed) {
    // widen, then one FP64 round whose shifts include both ends
    lo = fmax(lo - 1e-5 * wdt, lo0);
    hi = fmin(hi + 1e-5 * wdt, hi0);
    const double x = (tid == MS_S - 1) ? hi : lo + (hi - lo) * (double)tid / (MS_S - 1);
    double xs[1] = {x};
    int cnt[1];
    sturm_counts<1>(ds, e2s, n, xs, cnt);
    const int j = first_above(cnt[0]);
    if (j == 0 || j == MS_S) {   // the eigenvalue is outside: start over
      lo = lo0;
      hi = hi0;
    } else {
      const double xj = (j == MS_S - 1) ? hi : lo + (hi - lo) * (double)j / (MS_S - 1);
      lo = lo + (hi - lo) * (double)(j - 1) / (MS_S - 1);
      hi = xj;
    }
  }
  // phase 2: FP64 counts to full precision
  for (int it = 0; it < 64; ++it) {
    if (hi - lo <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + 4.0 * DBL_MIN) break;
    double x[1];
    int cnt[1];
    x[0] = lo + (hi - lo) * (double)(tid + 1) / (MS_S + 1);
    sturm_counts<1>(ds, e2s, n, x, cnt);
    if (!shrink(first_above(cnt[0]))) break;
  }
  if (tid == 0) out[t] = 0.5 * (lo + hi);
}
// Size estimate of a window anchored at an index: FP32 multisection (one CTA
// of 4 warps, 129 shifts per round) narrows eigenvalue i_lo to about 2e-5 of
// the spectrum's scale, then one FP32 count at the bracket's top + width +
// 4e-5 scale gives out[0] = an upper estimate of the index one past the
// window.  FP32 counts can be off near eigenvalues, so the caller treats the
// number as a guess and checks it in FP64.
__global__ void __launch_bounds__(128) window_size_kernel(const double* __restrict__ d,
                                                          const double* __restrict__ e, int n,
                                                          int i_lo, double width, int* out) {
  extern __shared__ float ws_smem[];
  float* dsf = ws_smem;
  float* e2f = ws_smem + n;
  __shared__ int firstw[4];
  __shared__ double gl[8];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double a = DBL_MAX, b = -DBL_MAX;
  for (int i = tid; i < n; i += 128) {
    const double e2 = (i < n - 1) ? e[i] * e[i] : 0.0;
    dsf[i] = (float)d[i];
    e2f[i] = (float)e2;
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
    gl[4 + warp] = b;
  }
  __syncthreads();
  a = fmin(fmin(gl[0], gl[1]), fmin(gl[2], gl[3]));
  b = fmax(fmax(gl[4], gl[5]), fmax(gl[6], gl[7]));
  const double wdt = fmax(fabs(a), fabs(b));
  double lo = a - 1e-5 * wdt, hi = b + 1e-5 * wdt;
  const float pivmin = 1e-30f;
  for (int it = 0; it < 32 && hi - lo > 2e-5 * wdt; ++it) {
    const double x = lo + (hi - lo) * (double)(tid + 1) / 129.0;
    const int cnt = sturm_count_f32(dsf, e2f, n, (float)x, pivmin);
    const unsigned ball = __ballot_sync(0xffffffffu, cnt > i_lo);
    if (lane == 0) firstw[warp] = ball ? __ffs(ball) - 1 : 32;
    __syncthreads();
    int j = 128;
    for (int w = 3; w >= 0; --w)
      if (firstw[w] < 32) j = w * 32 + firstw[w];
    __syncthreads();
    const double nhi = (j == 128) ? hi : lo + (hi - lo) * (double)(j + 1) / 129.0;
    const double nlo = (j == 128) ? lo + (hi - lo) * 128.0 / 129.0 : (j > 0 ? lo + (hi - lo) * (double)j / 129.0 : lo);
    if (nlo == lo && nhi == hi) break;
    lo = nlo;
    hi = nhi;
  }
  if (tid == 0) {
    const double top = hi + width + 4e-5 * wdt;
    out[0] = (top >= b) ? n : sturm_count_f32(dsf, e2f, n, (float)top, pivmin);
  }
}

}  // namespace ofm

using namespace ofm;

// The test hook's held arrival for the next reduction (one launch): the
// barrier's hold word and a short poll limit, written after its reset.
static ofm_status arm_hold(ofm_ctx* c) {
  if (!c->hold_tri) return OFM_OK;
  static GridBar h{};   // pageable source of a stream-ordered copy: kept alive
  h = GridBar{};
  h.hold = 1;
  h.limit = c->hold_bound > 0 ? (unsigned int)c->hold_bound : 0u;
  c->hold_tri = 0;
  OFM_CUDA(c, cudaMemcpyAsync(c->w_bar.p, &h, sizeof(GridBar), cudaMemcpyHostToDevice, c->stream));
  return OFM_OK;
}

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
    // nbs < n: every CTA owns a row below row 0
    const int nbs = std::min(sms, n - 1);
    const size_t rmax = (size_t)(n + nbs - 1) / nbs;
    const size_t smem2 = (rmax * n + 4 * (size_t)n) * sizeof(double);
    const size_t pub_bytes = 4 * (size_t)n * sizeof(Pub);   // p and row k+1, two slots each
    int per_sm2 = 0;
    if (smem2 <= 200 * 1024 && rmax <= (size_t)TRI_RMAX &&
        2 * (size_t)n <= (size_t)TRI_PMAX * TRI_THREADS &&
        cudaFuncSetAttribute(tridiag_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem2) == cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, tridiag_smem_kernel, TRI_THREADS,
                                                      smem2) == cudaSuccess &&
        per_sm2 >= 1 && c->w_eval.cap >= pub_bytes) {
      OFM_TRY(ofm_ensure(c, c->w_bar, sizeof(GridBar), "grid barrier"));
      OFM_CUDA(c, cudaMemsetAsync(c->w_bar.p, 0, sizeof(GridBar), c->stream));
      OFM_TRY(arm_hold(c));
      // generation 0 in every slot: no column's value yet
      OFM_CUDA(c, cudaMemsetAsync(c->w_eval.p, 0, pub_bytes, c->stream));
      GridBar* bar = (GridBar*)c->w_bar.p;
      Pub* pub = (Pub*)c->w_eval.p;
      int nn = n;
      void* args[] = {&A, &nn, &d, &e, &tau, &pub, &bar};
      OFM_CUDA(c, cudaLaunchCooperativeKernel((const void*)tridiag_smem_kernel, dim3(nbs),
                                              dim3(TRI_THREADS), args, smem2, c->stream));
      GridBar hb{};
      OFM_CUDA(c, cudaMemcpyAsync(&hb, bar, sizeof(GridBar), cudaMemcpyDeviceToHost, c->stream));
      OFM_CUDA(c, cudaStreamSynchronize(c->stream));
      if (hb.err) return ofm_fail(c, OFM_ERR_TIMEOUT, "tridiagonal reduction: a wait for another CTA exceeded its bound");
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
  OFM_TRY(arm_hold(c));
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
  // d and e^2 in FP64 and in FP32
  const size_t smem = 2 * (size_t)n * (sizeof(double) + sizeof(float));
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

// Estimate (see window_size_kernel) of one past the last index of the window
// [E_{i_lo}, E_{i_lo} + width]; false when the tridiagonal is too long.
bool launch_window_size(const double* d, const double* e, int n, int i_lo, double width, int* out,
                        cudaStream_t s) {
  const size_t smem = 2 * (size_t)n * sizeof(float);
  if (smem > 200 * 1024) return false;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(window_size_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             200 * 1024) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    attr = true;
  }
  window_size_kernel<<<1, 128, smem, s>>>(d, e, n, i_lo, width, out);
  return true;
}
