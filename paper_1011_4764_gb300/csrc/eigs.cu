// Batched fragment eigensolver: the lowest n_a eigenpairs of every fragment
// Hamiltonian (Sec. II, "calculation of basis wave functions"; the paper uses
// a preconditioned conjugate-gradient plane-wave solver per fragment).
//
// All fragments advance together through Chebyshev-filtered subspace
// iteration (Zhou, Saad, Tiago and Chelikowsky, "Self-consistent-field
// calculations using Chebyshev-filtered subspace iteration", J. Comput.
// Phys. 219 (2006)):
//   1. X: a block of m_a = n_a + guard vectors per fragment (random start
//      from a counter-based generator, SplitMix64 of Steele, Lea and Flood);
//   2. Y = p(H_a) X, p the degree-d Chebyshev polynomial of the first kind
//      mapped to the unwanted interval [b_lo, b_up] and scaled at the lowest
//      Ritz value (the scaled three-term recurrence, one fused stencil step
//      per degree, every fragment in one launch);
//   3. Rayleigh-Ritz: G = Y^T Y and K = Y^T H Y (one batched contraction),
//      then per fragment, in the storage precision: diagonal scaling,
//      Cholesky of the scaled G and Jacobi on L^-1 K L^-T when G is well
//      conditioned, else Jacobi eigendecomposition of G, canonical
//      orthogonalisation (directions with relative Gram eigenvalue below a
//      threshold are dropped) and Jacobi on the projected K -> Ritz values
//      and C;
//   4. X <- Y C, and residual norms ||(HY) C_i - theta_i X_i|| with (HY) C
//      formed on the fly (never stored: the next filter starts from X);
//   5. b_lo <- largest Ritz value, repeat until every wanted residual is
//      below tol.
// The Gershgorin bound b_up = 6/h^2 + max V holds for every fragment
// Hamiltonian (principal submatrix of the global one).
// The returned states are the first n_a Ritz vectors with the sign gauge
// "largest |component| positive, ties to the lowest box index".
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <climits>
#include <cmath>
#include <cstdio>
#include <vector>

#include "ofm_internal.h"

using namespace ofm;

struct EigWork {
  std::vector<DevFrag> efr;           // block layout: n = m_a, ld = round4(m_a)
  std::vector<int> cta_start;
  int total_ctas = 0;
  long long elems = 0;
  int mmax = 0;
  std::vector<long long> toff;        // per fragment offset into theta / res (m_a each)
  long long tsum = 0;
  std::vector<DevPair> gpairs;
  std::vector<Piece> gpieces;
  std::vector<WorkItem> gitems;
  long long gpart = 0;
  long long gblk = 0;
  DevBuf d_efr, d_cta, buf[4], coef, theta, res, Cm, work, blocks, partials, d_gpairs, d_gpieces,
      d_gitems, d_toff, d_rank, d_vmax, rpart, xpart;
  double vlim[2] = {0.0, 0.0};        // max V, min V
  size_t rr_smem = 0, rot_smem = 0;   // dynamic shared memory of the two kernels
  int rr_threads = 256;                 // Rayleigh-Ritz CTA size
  int rot_blocks = 1;
  bool rot4 = false;                    // FP32 register-tiled rotation
  size_t cf_smem = 0;                   // on-chip filter: shared memory per CTA (0: off)
  double cf_bytes0 = 0, cf_bytes = 0, cf_flops_step = 0;
  ApplyGrid fgrid;                    // launch shape of the filter steps
  struct TcPlan* gtc = nullptr;       // Gram on tensor cores (TF32 hi+lo), FP32 storage
  bool ready = false;
  // algorithmic traffic / work per launch: a filter step streams the block
  // in, the previous block (three-term steps) and the block out, plus V
  double filter_b2 = 0, filter_b3 = 0, gram_bytes = 0, gram_flops = 0, rot_bytes = 0,
         rot_flops = 0;
};

void ofm_eig_guards(const ofm_ctx* c, std::vector<GuardRef>& out) {
  if (!c->eig) return;
  const EigWork* w = c->eig;
  const struct { const DevBuf* b; const char* n; } bufs[] = {
      {&w->d_efr, "eigensolver fragment table"}, {&w->d_cta, "eigensolver CTA table"},
      {&w->buf[0], "eigensolver block 0"}, {&w->buf[1], "eigensolver block 1"},
      {&w->buf[2], "eigensolver block 2"}, {&w->buf[3], "eigensolver block 3"},
      {&w->coef, "filter coefficients"}, {&w->theta, "Ritz values"}, {&w->res, "residuals"},
      {&w->Cm, "Ritz coefficients"}, {&w->work, "Rayleigh-Ritz work"}, {&w->blocks, "Gram blocks"},
      {&w->partials, "Gram partials"}, {&w->d_gpairs, "Gram pairs"}, {&w->d_gpieces, "Gram pieces"},
      {&w->d_gitems, "Gram items"}, {&w->d_toff, "eigensolver offsets"}, {&w->d_rank, "ranks"},
      {&w->d_vmax, "potential maxima"}, {&w->rpart, "residual partials"}, {&w->xpart, "export partials"}};
  for (const auto& x : bufs)
    if (x.b->p) out.push_back({x.b->p, x.b->cap, x.n});
  ofm_tc_guards(w->gtc, out);
}

void ofm_eig_free(ofm_ctx* c) {
  if (!c->eig) return;
  EigWork* w = c->eig;
  DevBuf* bufs[] = {&w->d_efr, &w->d_cta, &w->buf[0], &w->buf[1], &w->buf[2], &w->buf[3],
                    &w->coef, &w->theta, &w->res, &w->Cm, &w->work, &w->blocks, &w->partials,
                    &w->d_gpairs, &w->d_gpieces, &w->d_gitems, &w->d_toff, &w->d_rank, &w->d_vmax,
                    &w->rpart, &w->xpart};
  for (DevBuf* b : bufs)
    if (b->p) cudaFree(b->p);
  ofm_tc_plan_free(w->gtc);
  delete w;
  c->eig = nullptr;
}

namespace {

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ULL;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
  return x ^ (x >> 31);
}

__device__ __forceinline__ int find_frag(const int* start, int nfrag, int cta) {
  int lo = 0, hi = nfrag - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (start[mid] <= cta) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ bool interior(const DevFrag& F, long long p, int& x, int& y, int& z) {
  x = (int)(p % F.dext[0]);
  y = (int)((p / F.dext[0]) % F.dext[1]);
  z = (int)(p / ((long long)F.dext[0] * F.dext[1]));
  return x >= F.lo[0] && x < F.lo[0] + F.ext[0] && y >= F.lo[1] && y < F.lo[1] + F.ext[1] &&
         z >= F.lo[2] && z < F.lo[2] + F.ext[2];
}

// Uniform(-1, 1) start vectors on interior points; pad columns and halo 0.
template <typename T>
__global__ void init_random_kernel(const DevFrag* fr, const int* cta_start, int nfrag, T* buf,
                                   unsigned long long seed) {
  const int f = find_frag(cta_start, nfrag, blockIdx.x);
  const DevFrag F = fr[f];
  const long long e0 = (long long)(blockIdx.x - cta_start[f]) * blockDim.x + threadIdx.x;
  // the apply launch table covers ld/VN threads per point; here each thread
  // writes ld/VN * VN = ld / (threads per point) columns
  constexpr int VN = sizeof(T) == 8 ? 2 : 4;
  const int qpp = F.ld / VN;
  if (e0 >= F.Pd * qpp) return;
  const long long p = e0 / qpp;
  const int q = (int)(e0 - p * qpp);
  int x, y, z;
  const bool in = interior(F, p, x, y, z);
  const unsigned long long s0 = splitmix64(seed);
  for (int k = 0; k < VN; ++k) {
    const int col = q * VN + k;
    T v = 0;
    if (in && col < F.n) {
      unsigned long long key = ((unsigned long long)f << 44) ^ ((unsigned long long)col << 32) ^
                               (unsigned long long)p;
      unsigned long long r = splitmix64(key + s0);
      // uniform in [-1, 1): 53 random bits for FP64 storage, 24 for FP32
      // (FP32 arithmetic there: the FP64 units of this part are few)
      if (sizeof(T) == 8)
        v = (T)((double)(r >> 11) * (2.0 / 9007199254740992.0) - 1.0);
      else
        v = (T)((float)(r >> 40) * (2.0f / 16777216.0f) - 1.0f);
    }
    buf[F.off + p * F.ld + col] = v;
  }
}

// ---- per-fragment dense Rayleigh-Ritz (one CTA per fragment) -------------
//
// T is the arithmetic of the small dense problems: FP64 for FP64 storage;
// FP32 for FP32 storage, where the states themselves carry FP32 rounding
// (the FP64 pipe of one SM issues about 2 FMA per clock on this part, so
// FP64 here would make the eigensolver bound by a handful of SMs).

// Round-robin schedule (circle method): index ne-1 stays, the others
// rotate; round r pairs (r, ne-1) and ((r+k) mod (ne-1), (r-k) mod (ne-1)).
// Every pair meets once per sweep and the pairs of a round are disjoint.

template <typename T> struct Eps;
template <> struct Eps<float> { static constexpr double v = 6.0e-8; };
template <> struct Eps<double> { static constexpr double v = 1.1e-16; };

// Cyclic parallel Jacobi on the symmetric n x n matrix A (leading dim lda),
// accumulating the rotations into V (which must hold the identity or a
// start basis).  Round-robin pairing: n_even/2 disjoint rotations per round.
// A and V live in shared memory when they fit, so a round costs two CTA
// barriers (after the rows, after the columns) and no global-memory round
// trips.  Stops when the off-diagonal
// mass is at the rounding level of an n x n matrix or a sweep rotated
// nothing (elements below rounding relative to their diagonal pair are
// left alone).
template <typename T>
__device__ void cta_jacobi(T* A, T* V, int n, int lda, int* perm, T* cs, double* red) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int ne = n + (n & 1);
  const int half = ne / 2;
  const double eps = Eps<T>::v;
  const T eps_t = (T)Eps<T>::v;
  // norms, reductions and thresholds in the working precision T: the FP64
  // units of this part are few, and a stopping test needs no more
  for (int sweep = 0; sweep < 40; ++sweep) {
    T off = 0, tot = 0;
    for (int e = tid; e < n * n; e += nt) {
      const int i = e / n, j = e - (e / n) * n;
      const T a = A[i * lda + j];
      tot += a * a;
      if (i != j) off += a * a;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_down_sync(0xffffffffu, off, o);
      tot += __shfl_down_sync(0xffffffffu, tot, o);
    }
    if ((tid & 31) == 0) {
      red[2 * (tid >> 5)] = (double)off;
      red[2 * (tid >> 5) + 1] = (double)tot;
    }
    __syncthreads();
    if (tid == 0) {
      double so = 0.0, st = 0.0;
      for (int w = 0; w < nt / 32; ++w) {
        so += red[2 * w];
        st += red[2 * w + 1];
      }
      const double tol = 4.0 * n * eps;
      red[64] = (so <= tol * tol * st || so == 0.0 || (sweep > 0 && red[65] == 0.0)) ? 1.0 : 0.0;
      red[65] = 0.0;                      // rotations applied in the coming sweep
      red[66] = 2.0 * eps * sqrt(st / n);  // absolute floor: rounding level of an element
    }
    __syncthreads();
    const bool done = red[64] != 0.0;
    const T floor_t = (T)red[66];
    __syncthreads();
    if (done) break;
    const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
    for (int r = 0; r < ne - 1; ++r) {
      // rows p, q: one warp per pair.  The warp forms its pair's angle itself
      // (every lane the same arithmetic) and goes on to the row update, so
      // the angle needs no phase or barrier of its own; perm[] and cs[] carry
      // the pairs and angles to the column phase.  With d = a_qq - a_pp,
      //   t = sgn(d) 2 a_pq / (|d| + sqrt(d^2 + 4 a_pq^2))
      // is the smaller root of t^2 + 2 theta t - 1 = 0, theta = d / (2 a_pq)
      // (the classical cyclic-Jacobi tangent), with one division and one
      // square root fewer than forming theta first.
      for (int k = warp; k < half; k += nwarps) {
        int p, q;
        {   // the round-robin pairing without integer division
          const int M = ne - 1;
          if (k == 0) {
            p = r;
            q = M;
          } else {
            p = r + k;
            if (p >= M) p -= M;
            q = r - k;
            if (q < 0) q += M;
          }
        }
        T c = 1, s = 0;
        if (p < n && q < n) {
          const T apq = A[p * lda + q];
          const T app = A[p * lda + p], aqq = A[q * lda + q];
          const T thr = fmax(T(4) * eps_t * eps_t * fabs(app * aqq), floor_t * floor_t);
          if (apq * apq > thr) {
            if (lane == 0) red[65] = 1.0;
            const T d = aqq - app;
            const T t = (d >= T(0) ? T(2) : T(-2)) * apq / (fabs(d) + sqrt(d * d + T(4) * apq * apq));
            c = T(1) / sqrt(t * t + T(1));
            s = t * c;
          }
        }
        if (lane == 0) {
          perm[k] = p | (q << 16);
          cs[2 * k] = c;
          cs[2 * k + 1] = s;
        }
        __syncwarp();   // every lane has read a_pq, a_pp, a_qq before the rows change
        if (p >= n || q >= n || s == T(0)) continue;   // uniform over the warp
        for (int j = lane; j < n; j += 32) {
          const T ap = A[p * lda + j], aq = A[q * lda + j];
          A[p * lda + j] = c * ap - s * aq;
          A[q * lda + j] = s * ap + c * aq;
        }
      }
      __syncthreads();
      // columns p, q of A and V: one warp per pair, lanes down the column
      for (int k = warp; k < half; k += nwarps) {
        const int pq = perm[k], p = pq & 0xffff, q = pq >> 16;
        const T c = cs[2 * k], s = cs[2 * k + 1];
        if (p >= n || q >= n || s == T(0)) continue;
        for (int i = lane; i < n; i += 32) {
          const T ap = A[i * lda + p], aq = A[i * lda + q];
          A[i * lda + p] = c * ap - s * aq;
          A[i * lda + q] = s * ap + c * aq;
          const T vp = V[i * lda + p], vq = V[i * lda + q];
          V[i * lda + p] = c * vp - s * vq;
          V[i * lda + q] = s * vp + c * vq;
        }
      }
      __syncthreads();
    }
  }
}

// One warp per rotation pair of a Jacobi round (m/2 pairs), so a round's
// row and column phases take one pass; at least 256 and at most
// RR_MAX_THREADS threads (the reduction scratch holds 32 warps' partials).
constexpr int RR_MAX_THREADS = 640;

// Inputs: blocks of the self pair of fragment f, [K | G] with K = Y^T H Y
// and G = Y^T Y (m x m each, symmetrised).  Outputs: C (m x m row-major,
// columns = Ritz vectors in the Y basis, ascending Ritz values; dropped
// directions give zero columns), theta (m; dropped directions repeat the
// largest kept value), rank (number of kept directions).
// Work matrices A, U, W (row stride ld) and vectors D, sig, idx live in
// dynamic shared memory (ld = the odd one of m + 1, m + 2: column walks across
// the warp hit distinct banks) or, for large m, in `work` (ld = m).
template <typename T>
__global__ void __launch_bounds__(RR_MAX_THREADS) rayleigh_ritz_kernel(const DevFrag* efr, const DevPair* gp,
                                                            const double* blocks, T* work,
                                                            long long wstride, double* Cm,
                                                            long long cstride, double* theta,
                                                            const long long* toff, double rank_tol,
                                                            int* rank_out, int use_smem) {
  extern __shared__ __align__(16) unsigned char rr_raw[];
  __shared__ int perm[520];
  __shared__ T cs[520];
  __shared__ double red[80];
  __shared__ int nkeep;
  const int f = blockIdx.x;
  const int m = efr[f].n;
  const int tid = threadIdx.x, nt = blockDim.x;
  const double* Kb = blocks + gp[f].blk_off;
  const double* Gb = Kb + (long long)m * m;
  const int ld = use_smem ? m + 1 + (m & 1) : m;
  T* A = use_smem ? reinterpret_cast<T*>(rr_raw) : work + f * wstride;
  T* U = A + (long long)m * ld;
  T* W = U + (long long)m * ld;
  T* D = W + (long long)m * ld;           // m
  T* sig = D + m;                         // m
  int* idx = reinterpret_cast<int*>(sig + m);   // m
  double* C = Cm + f * cstride;
  double* th = theta + toff[f];

  for (int i = tid; i < m; i += nt) {
    const double g = Gb[(long long)i * m + i];
    D[i] = g > 0.0 ? (T)(1.0 / sqrt(g)) : T(0);
  }
  __syncthreads();
  for (int e = tid; e < m * m; e += nt) {
    const int i = e / m, j = e - (e / m) * m;
    A[i * ld + j] = D[i] * (T)Gb[e] * D[j];
    U[i * ld + j] = (i == j) ? T(1) : T(0);
  }
  __syncthreads();
  // Fast path: when the scaled Gram is well conditioned (every Cholesky
  // pivot above chol_tol, the usual case once the iteration has started to
  // converge), G_s = L L^T, B = L^-1 K_s L^-T, one Jacobi on the nearly
  // diagonal B, C = D L^-T Q.  Otherwise the canonical orthogonalisation
  // below drops the near-dependent directions.
  {
    __shared__ int chol_ok;
    const T chol_tol = sizeof(T) == 8 ? T(1e-8) : T(1e-3);
    if (tid == 0) chol_ok = 1;
    for (int e = tid; e < m * m; e += nt) {
      const int i = e / m, j = e - (e / m) * m;
      W[i * ld + j] = A[i * ld + j];
    }
    __syncthreads();
    for (int j = 0; j < m; ++j) {
      if (tid == 0) {
        T piv = W[j * ld + j];
        if (!(piv > chol_tol)) {
          chol_ok = 0;
          piv = T(1);
        }
        W[j * ld + j] = sqrt(piv);
      }
      __syncthreads();
      for (int i = j + 1 + tid; i < m; i += nt) W[i * ld + j] /= W[j * ld + j];
      __syncthreads();
      // trailing update, one warp per row, lanes along the row (no index division)
      for (int i = j + 1 + (tid >> 5); i < m; i += nt >> 5) {
        const T lij = W[i * ld + j];
        for (int k = j + 1 + (tid & 31); k <= i; k += 32) W[i * ld + k] -= lij * W[k * ld + j];
      }
      __syncthreads();
    }
    if (chol_ok) {
      // U <- L^-1 (D K D), one thread per column
      for (int c = tid; c < m; c += nt)
        for (int i = 0; i < m; ++i) {
          T s = D[i] * (T)Kb[(long long)i * m + c] * D[c];
          for (int k = 0; k < i; ++k) s -= W[i * ld + k] * U[k * ld + c];
          U[i * ld + c] = s / W[i * ld + i];
        }
      __syncthreads();
      // A <- L^-1 U^T = L^-1 (D K D) L^-T
      for (int c = tid; c < m; c += nt)
        for (int i = 0; i < m; ++i) {
          T s = U[c * ld + i];
          for (int k = 0; k < i; ++k) s -= W[i * ld + k] * A[k * ld + c];
          A[i * ld + c] = s / W[i * ld + i];
        }
      __syncthreads();
      for (int e = tid; e < m * m; e += nt) {
        const int i = e / m, j = e - (e / m) * m;
        if (i < j) {
          const T v = T(0.5) * (A[i * ld + j] + A[j * ld + i]);
          A[i * ld + j] = v;
          A[j * ld + i] = v;
        }
      }
      __syncthreads();
      for (int e = tid; e < m * m; e += nt) {
        const int i = e / m, j = e - (e / m) * m;
        U[i * ld + j] = (i == j) ? T(1) : T(0);
      }
      __syncthreads();
      cta_jacobi<T>(A, U, m, ld, perm, cs, red);   // A -> diag(theta), U -> Q
      for (int j = tid; j < m; j += nt) {
        const T t = A[j * ld + j];
        int rk = 0;
        for (int i = 0; i < m; ++i) {
          const T ti = A[i * ld + i];
          rk += (ti < t || (ti == t && i < j)) ? 1 : 0;
        }
        idx[j] = rk;
      }
      // U <- L^-T Q, one thread per column (back substitution in place)
      for (int j = tid; j < m; j += nt)
        for (int i = m - 1; i >= 0; --i) {
          T s = U[i * ld + j];
          for (int k = i + 1; k < m; ++k) s -= W[k * ld + i] * U[k * ld + j];
          U[i * ld + j] = s / W[i * ld + i];
        }
      __syncthreads();
      for (int e = tid; e < m * m; e += nt) {
        const int k = e / m, j = e - (e / m) * m;
        C[(long long)k * m + idx[j]] = (double)(D[k] * U[k * ld + j]);
      }
      for (int j = tid; j < m; j += nt) th[idx[j]] = (double)A[j * ld + j];
      if (tid == 0) rank_out[f] = m;
      return;
    }
  }
  cta_jacobi<T>(A, U, m, ld, perm, cs, red);
  // rank decision on the scaled Gram spectrum
  if (tid == 0) {
    T smax = 0;
    for (int i = 0; i < m; ++i) smax = fmax(smax, A[i * ld + i]);
    int r = 0;
    for (int i = 0; i < m; ++i) {
      const T s = A[i * ld + i];
      if ((double)s > rank_tol * (double)smax) {
        idx[r] = i;
        sig[r] = s;
        ++r;
      }
    }
    nkeep = r;
  }
  __syncthreads();
  const int r = nkeep;
  // W = D U_keep sig^-1/2  (m x r)
  for (int e = tid; e < m * r; e += nt) {
    const int k = e / r, j = e - (e / r) * r;
    W[k * ld + j] = D[k] * U[k * ld + idx[j]] / sqrt(sig[j]);
  }
  __syncthreads();
  // A <- K W (m x r), then U <- W^T (K W) (r x r), symmetrised
  for (int e = tid; e < m * r; e += nt) {
    const int k = e / r, j = e - (e / r) * r;
    T s = 0;
    for (int l = 0; l < m; ++l) s += (T)Kb[(long long)k * m + l] * W[l * ld + j];
    A[k * ld + j] = s;
  }
  __syncthreads();
  for (int e = tid; e < r * r; e += nt) {
    const int i = e / r, j = e - (e / r) * r;
    if (j < i) continue;
    T s = 0, t = 0;
    for (int l = 0; l < m; ++l) {
      s += W[l * ld + i] * A[l * ld + j];
      t += W[l * ld + j] * A[l * ld + i];
    }
    U[i * ld + j] = T(0.5) * (s + t);
    U[j * ld + i] = T(0.5) * (s + t);
  }
  __syncthreads();
  for (int e = tid; e < r * r; e += nt) {
    const int i = e / r, j = e - (e / r) * r;
    A[i * ld + j] = (i == j) ? T(1) : T(0);
  }
  __syncthreads();
  cta_jacobi<T>(U, A, r, ld, perm, cs, red);     // U -> diag(theta), A -> Q
  // ascending order: rank of each Ritz value
  for (int j = tid; j < r; j += nt) {
    const T t = U[j * ld + j];
    int rk = 0;
    for (int i = 0; i < r; ++i) {
      const T ti = U[i * ld + i];
      rk += (ti < t || (ti == t && i < j)) ? 1 : 0;
    }
    idx[j] = rk;
  }
  __syncthreads();
  // C[:, rank(j)] = W Q[:, j]
  for (int e = tid; e < m * m; e += nt) C[e] = 0.0;
  __syncthreads();
  for (int e = tid; e < m * r; e += nt) {
    const int k = e / r, j = e - (e / r) * r;
    T s = 0;
    for (int l = 0; l < r; ++l) s += W[k * ld + l] * A[l * ld + j];
    C[(long long)k * m + idx[j]] = (double)s;
  }
  double tmax = -DBL_MAX;
  for (int j = 0; j < r; ++j) tmax = fmax(tmax, (double)U[j * ld + j]);
  for (int j = tid; j < m; j += nt) {
    if (j < r) th[idx[j]] = (double)U[j * ld + j];
    else th[j] = tmax;
  }
  if (tid == 0) rank_out[f] = r;
}

// X_new = Y C over the interior points (columns >= rank get fresh random
// values), plus per-block partial sums of ((HY) C - theta X_new)^2 per
// column for the residual norms, with (HY) C formed on the fly and not
// stored (a dropped direction's H X counts as zero).
// A CTA takes tiles of RT points: their rows of Y and H Y are staged in
// shared memory (row stride m + 1 or m + 2, whichever is odd: conflict-free
// column reads); thread
// (point lane pl, column group jg) accumulates the columns j = jb + jg + 4 i
// (i < RJ) of its point in registers, so each coefficient read is a warp
// broadcast and feeds two FMAs per point.  Results go back through shared
// memory and leave as whole point rows (coalesced).
constexpr int RT = 64;   // points per tile
constexpr int RJ = 10;   // columns per thread and column block (4 groups x 10 = 40)

template <typename T>
__global__ void __launch_bounds__(256) rotate_kernel(const DevFrag* efr, const T* Y, T* Xo,
                                                     const T* HY, const double* Cm,
                                                     long long cstride, const int* rank,
                                                     const double* theta, const long long* toff,
                                                     double* partial, int mstride,
                                                     unsigned long long salt) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int f = blockIdx.y;
  const DevFrag F = efr[f];
  const int m = F.n, ms = m + 1 + (m & 1);
  const int r = rank[f];
  const int ex = F.ext[0], ey = F.ext[1];
  const int P = F.ext[0] * F.ext[1] * F.ext[2];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int pl = tid & (RT - 1), jg = tid / RT;   // point lane, column group (0..3)
  constexpr int JB = 4 * RJ;                       // columns per block
  int* pds = reinterpret_cast<int*>(smem_raw);                   // RT
  T* rs = reinterpret_cast<T*>(smem_raw + 16 * ((RT * sizeof(int) + 15) / 16));    // JB residual sums
  T* Cs = rs + 4 * RJ;                                           // m * m
  T* ys = Cs + m * m;                                            // RT * ms
  T* hs = ys + RT * ms;                                          // RT * ms
  for (int e = tid; e < m * m; e += blockDim.x) Cs[e] = (T)Cm[f * cstride + e];
  const unsigned long long s0 = splitmix64(salt);
  const T inv_sqrt_p = (T)(1.0 / sqrt((double)P));
  // column blocks of JB columns (one for m <= JB); the tile rows are staged
  // again for each block
  for (int jb = 0; jb < m; jb += JB) {
    const int jn = min(JB, m - jb);
    // residual partial sums of the block's columns, in shared memory
    if (tid < JB) rs[tid] = T(0);
    for (int t0 = blockIdx.x * RT; t0 < P; t0 += gridDim.x * RT) {
      __syncthreads();   // previous tile fully written out
      if (tid < RT) {
        const int t = t0 + tid;
        int pd = -1;
        if (t < P) {
          const int x = t % ex, y = (t / ex) % ey, z = t / (ex * ey);
          pd = ((z + F.lo[2]) * F.dext[1] + (y + F.lo[1])) * F.dext[0] + x + F.lo[0];
        }
        pds[tid] = pd;
      }
      __syncthreads();
      // stage the tile's rows: warp w takes points w, w + 8, ..., lanes along the row
      for (int pp = warp; pp < RT; pp += 8) {
        const int pd = pds[pp];
        const long long a = F.off + (long long)max(pd, 0) * F.ld;
        for (int k = lane; k < m; k += 32) {
          ys[pp * ms + k] = pd >= 0 ? Y[a + k] : T(0);
          hs[pp * ms + k] = pd >= 0 ? HY[a + k] : T(0);
        }
      }
      __syncthreads();
      T x[RJ], hx[RJ];
#pragma unroll
      for (int i = 0; i < RJ; ++i) {
        x[i] = T(0);
        hx[i] = T(0);
      }
      for (int k = 0; k < m; ++k) {
        const T yv = ys[pl * ms + k], hv = hs[pl * ms + k];
        const T* crow = Cs + k * m + jb + jg;
#pragma unroll
        for (int i = 0; i < RJ; ++i) {
          if (jg + 4 * i < jn) {
            const T cc = crow[4 * i];
            x[i] += yv * cc;
            hx[i] += hv * cc;
          }
        }
      }
      __syncthreads();   // every thread has read the staged rows
      const int pd = pds[pl];
      // results of the block into the staged rows' columns jb .. jb + jn - 1
#pragma unroll
      for (int i = 0; i < RJ; ++i) {
        const int c = jg + 4 * i;
        if (c >= jn) continue;
        const int j = jb + c;
        T xv = x[i], hv = hx[i];
        if (j >= r) {   // dropped direction: a fresh random vector, H X left zero
          hv = T(0);
          xv = T(0);
          if (pd >= 0) {
            const unsigned long long key =
                ((unsigned long long)f << 44) ^ ((unsigned long long)j << 32) ^ (unsigned long long)pd;
            const unsigned long long rr = splitmix64(key + s0);
            xv = (T)((double)(rr >> 11) * (2.0 / 9007199254740992.0) - 1.0) * inv_sqrt_p;
          }
        }
        ys[pl * ms + j] = xv;
        // residual of this output, summed over the warp's 32 points by
        // shuffles, then one shared-memory atomic per warp and column
        const T d = pd >= 0 ? hv - (T)theta[toff[f] + j] * xv : T(0);
        T v = d * d;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) atomicAdd(&rs[c], v);
      }
      __syncthreads();
      // coalesced row writes
      for (int pp = warp; pp < RT; pp += 8) {
        const int pdo = pds[pp];
        if (pdo < 0) continue;
        const long long a = F.off + (long long)pdo * F.ld;
        for (int k = jb + lane; k < jb + jn; k += 32) Xo[a + k] = ys[pp * ms + k];
      }
    }
    __syncthreads();
    if (tid < jn) partial[((long long)f * gridDim.x + blockIdx.x) * mstride + jb + tid] = (double)rs[tid];
    __syncthreads();
  }
}

// The same rotation for FP32 blocks with a larger register tile: a CTA takes
// tiles of RT4 = 256 points, staged TRANSPOSED in shared memory (one row per
// column k, the tile's points contiguous), and thread (point group pg,
// column group jg) accumulates 4 points x RJ columns of both products.  Per
// k a thread loads its 4 points of Y and of H Y with one 16-byte load each
// and its RJ coefficients with RJ/2 8-byte loads (warp broadcasts), and
// issues 8 RJ FMAs: the loop is FMA-bound, not shared-memory-bound.  The
// residual partial sums stay in registers across the CTA's tiles.
constexpr int RT4 = 256;   // points per tile (one per thread when staging)
constexpr int RJB = 4 * RJ;  // columns per column block
constexpr int RM4 = 52;      // widest block (m) this form takes

__global__ void __launch_bounds__(256, 2) rotate4_kernel(const DevFrag* efr, const float* Y, float* Xo,
                                                         const float* HY,
                                                         const double* Cm, long long cstride,
                                                         const int* rank, const double* theta,
                                                         const long long* toff, double* partial,
                                                         int mstride, unsigned long long salt) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ float red[8][RJ];
  const int f = blockIdx.y;
  const DevFrag F = efr[f];
  const int m = F.n;
  const int mcs = (m + RJB - 1) / RJB * RJB;   // coefficient row stride (zero-padded)
  const int r = rank[f];
  const int ex = F.ext[0], ey = F.ext[1];
  const int P = F.ext[0] * F.ext[1] * F.ext[2];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int pg = tid & 63, jg = tid >> 6;
  int* pds = reinterpret_cast<int*>(smem_raw);                      // RT4
  float* Cs = reinterpret_cast<float*>(smem_raw + RT4 * sizeof(int));  // m x mcs
  float* ys = Cs + (size_t)m * mcs;                                 // m x RT4, transposed
  float* hs = ys + (size_t)m * RT4;                                 // m x RT4, transposed
  // coefficients: every load of a thread issued before its stores (one
  // round trip, not one per element)
  for (int e0 = 0; e0 < m * mcs; e0 += 8 * 256) {
    double cv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * 256 + tid;
      const int k = e / mcs, j = e - k * mcs;
      cv[u] = (e < m * mcs && j < m) ? Cm[f * cstride + (long long)k * m + j] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * 256 + tid;
      if (e < m * mcs) Cs[e] = (float)cv[u];
    }
  }
  const unsigned long long s0 = splitmix64(salt);
  const float inv_sqrt_p = (float)(1.0 / sqrt((double)P));
  for (int jb = 0; jb < m; jb += RJB) {
    const int jn = min(RJB, m - jb);
    float rsum[RJ];
#pragma unroll
    for (int i = 0; i < RJ; ++i) rsum[i] = 0.f;
    for (int t0 = blockIdx.x * RT4; t0 < P; t0 += gridDim.x * RT4) {
      __syncthreads();   // previous tile written out (and the coefficients staged)
      // stage: thread tid takes point t0 + tid, its row in 16-byte pieces
      int pd = -1;
      {
        const int t = t0 + tid;
        if (t < P) {
          const int x = t % ex, y = (t / ex) % ey, z = t / (ex * ey);
          pd = ((z + F.lo[2]) * F.dext[1] + (y + F.lo[1])) * F.dext[0] + x + F.lo[0];
        }
        pds[tid] = pd;
        const long long a = F.off + (long long)max(pd, 0) * F.ld;
        // the whole row (at most RM4 columns) in flight at once; ld is a
        // multiple of 4, so every 16-byte piece stays inside the row
        float4 yv[RM4 / 4], hv[RM4 / 4];
#pragma unroll
        for (int u = 0; u < RM4 / 4; ++u) {
          yv[u] = make_float4(0.f, 0.f, 0.f, 0.f);
          hv[u] = yv[u];
          if (pd >= 0 && 4 * u < m) {
            yv[u] = *reinterpret_cast<const float4*>(Y + a + 4 * u);
            hv[u] = *reinterpret_cast<const float4*>(HY + a + 4 * u);
          }
        }
#pragma unroll
        for (int u = 0; u < RM4 / 4; ++u) {
          const int k = 4 * u;
          if (k < m) {
            ys[(size_t)k * RT4 + tid] = yv[u].x;
            hs[(size_t)k * RT4 + tid] = hv[u].x;
          }
          if (k + 1 < m) {
            ys[(size_t)(k + 1) * RT4 + tid] = yv[u].y;
            hs[(size_t)(k + 1) * RT4 + tid] = hv[u].y;
          }
          if (k + 2 < m) {
            ys[(size_t)(k + 2) * RT4 + tid] = yv[u].z;
            hs[(size_t)(k + 2) * RT4 + tid] = hv[u].z;
          }
          if (k + 3 < m) {
            ys[(size_t)(k + 3) * RT4 + tid] = yv[u].w;
            hs[(size_t)(k + 3) * RT4 + tid] = hv[u].w;
          }
        }
      }
      __syncthreads();
      float ax[4][RJ], ah[4][RJ];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int i = 0; i < RJ; ++i) {
          ax[q][i] = 0.f;
          ah[q][i] = 0.f;
        }
      const float* cp = Cs + jb + RJ * jg;
      for (int k = 0; k < m; ++k) {
        const float4 y4 = *reinterpret_cast<const float4*>(ys + (size_t)k * RT4 + 4 * pg);
        const float4 h4 = *reinterpret_cast<const float4*>(hs + (size_t)k * RT4 + 4 * pg);
        float cc[RJ];
#pragma unroll
        for (int i = 0; i < RJ / 2; ++i) {
          const float2 c2 = *reinterpret_cast<const float2*>(cp + (size_t)k * mcs + 2 * i);
          cc[2 * i] = c2.x;
          cc[2 * i + 1] = c2.y;
        }
#pragma unroll
        for (int i = 0; i < RJ; ++i) {
          ax[0][i] = fmaf(y4.x, cc[i], ax[0][i]);
          ax[1][i] = fmaf(y4.y, cc[i], ax[1][i]);
          ax[2][i] = fmaf(y4.z, cc[i], ax[2][i]);
          ax[3][i] = fmaf(y4.w, cc[i], ax[3][i]);
          ah[0][i] = fmaf(h4.x, cc[i], ah[0][i]);
          ah[1][i] = fmaf(h4.y, cc[i], ah[1][i]);
          ah[2][i] = fmaf(h4.z, cc[i], ah[2][i]);
          ah[3][i] = fmaf(h4.w, cc[i], ah[3][i]);
        }
      }
      __syncthreads();   // every thread has read the staged tile
      int pq[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) pq[q] = pds[4 * pg + q];
#pragma unroll
      for (int i = 0; i < RJ; ++i) {
        const int c = RJ * jg + i;
        if (c >= jn) continue;
        const int j = jb + c;
        const float th = (float)theta[toff[f] + j];
        float xo[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float xv = ax[q][i], hv = ah[q][i];
          if (j >= r) {   // dropped direction: a fresh random vector, H X left zero
            hv = 0.f;
            xv = 0.f;
            if (pq[q] >= 0) {
              const unsigned long long key = ((unsigned long long)f << 44) ^
                                             ((unsigned long long)j << 32) ^ (unsigned long long)pq[q];
              const unsigned long long rr = splitmix64(key + s0);
              xv = (float)((double)(rr >> 11) * (2.0 / 9007199254740992.0) - 1.0) * inv_sqrt_p;
            }
          }
          if (pq[q] >= 0) {
            const float d = hv - th * xv;
            rsum[i] = fmaf(d, d, rsum[i]);
          }
          xo[q] = xv;
        }
        *reinterpret_cast<float4*>(ys + (size_t)j * RT4 + 4 * pg) = make_float4(xo[0], xo[1], xo[2], xo[3]);
      }
      __syncthreads();
      // write the block's columns of point t0 + tid back, 16 bytes at a time
      if (pd >= 0) {
        const long long a = F.off + (long long)pd * F.ld;
        const int je = jb + jn;
        for (int k = jb; k < je; k += 4) {
          if (k + 3 < je) {
            *reinterpret_cast<float4*>(Xo + a + k) =
                make_float4(ys[(size_t)k * RT4 + tid], ys[(size_t)(k + 1) * RT4 + tid],
                            ys[(size_t)(k + 2) * RT4 + tid], ys[(size_t)(k + 3) * RT4 + tid]);
          } else {
            for (int kk = k; kk < je; ++kk) Xo[a + kk] = ys[(size_t)kk * RT4 + tid];
          }
        }
      }
    }
    // residual partials of the block's columns: over the 64 point groups of
    // column group jg (warps 2 jg and 2 jg + 1)
#pragma unroll
    for (int i = 0; i < RJ; ++i) {
      float v = rsum[i];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[warp][i] = v;
    }
    __syncthreads();
    if (tid < jn) {
      const int g = tid / RJ, i = tid - g * RJ;
      partial[((long long)f * gridDim.x + blockIdx.x) * mstride + jb + tid] =
          (double)red[2 * g][i] + (double)red[2 * g + 1][i];
    }
    __syncthreads();
  }
}

__global__ void residual_reduce_kernel(const DevFrag* efr, const double* partial, int nblocks,
                                       int mstride, const long long* toff, double* res) {
  const int f = blockIdx.x;
  const int m = efr[f].n;
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += partial[((long long)f * nblocks + b) * mstride + j];
    res[toff[f] + j] = sqrt(s);
  }
}

// Export of the first n_a Ritz vectors with the sign gauge (largest
// |component| positive, ties to the lowest point index), in two launches over
// (fragment, 32 columns, EXP_CHUNKS chunks of points): partial maxima per
// chunk, then each CTA combines its columns' partials in chunk order (the
// same winner as one pass over all points) and copies its chunk with the sign.
// Coordinates are stepped without divisions and eight loads are in flight per
// warp.
constexpr int EXP_CHUNKS = 8;

struct PointWalk {   // points t = t0, t0 + nw, ... of an ex x ey x ez box
  int x, y, z, sx, sy, sz, ex, ey;
  __device__ PointWalk(int t0, int nw, int ex_, int ey_) : ex(ex_), ey(ey_) {
    x = t0 % ex;
    y = (t0 / ex) % ey;
    z = t0 / (ex * ey);
    sx = nw % ex;
    sy = (nw / ex) % ey;
    sz = nw / (ex * ey);
  }
  __device__ void step() {
    x += sx;
    int c = 0;
    if (x >= ex) { x -= ex; c = 1; }
    y += sy + c;
    c = 0;
    if (y >= ey) { y -= ey; c = 1; }
    z += sz + c;
  }
  __device__ int at(const DevFrag& D) const {
    return ((z + D.lo[2]) * D.dext[1] + (y + D.lo[1])) * D.dext[0] + x + D.lo[0];
  }
};

template <typename T>
__global__ void __launch_bounds__(256) export_max_kernel(const DevFrag* efr, const DevFrag* fr,
                                                         const T* X, T* pmax, int* pidx, int mstride) {
  // magnitudes compared in the storage type: the same order as in FP64
  __shared__ T bv[8][32];
  __shared__ int bi[8][32];
  const int f = blockIdx.x, chunk = blockIdx.z;
  const DevFrag E = efr[f];
  const DevFrag F = fr[f];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int col = blockIdx.y * 32 + lane;
  const int P = F.ext[0] * F.ext[1] * F.ext[2];
  const int per = (P + EXP_CHUNKS - 1) / EXP_CHUNKS;
  const int p0 = chunk * per, p1 = min(P, p0 + per);
  T best = T(-1);
  int besti = 0x7fffffff;
  if (col < F.n && p0 + warp < p1) {
    constexpr int U = 8;
    PointWalk w(p0 + warp, 8, F.ext[0], F.ext[1]);
    for (int t0 = p0 + warp; t0 < p1; t0 += U * 8) {
      T a[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        a[u] = T(-1);
        if (t0 + u * 8 < p1) {
          a[u] = fabs(X[E.off + (long long)w.at(E) * E.ld + col]);
          w.step();
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (a[u] > best) {  // strictly greater in stream order: the lowest index wins
          best = a[u];
          besti = t0 + u * 8;
        }
    }
  }
  bv[warp][lane] = best;
  bi[warp][lane] = besti;
  __syncthreads();
  if (warp == 0 && col < F.n) {
    T b = bv[0][lane];
    int ib = bi[0][lane];
    for (int v = 1; v < 8; ++v)
      if (bv[v][lane] > b || (bv[v][lane] == b && bi[v][lane] < ib)) {
        b = bv[v][lane];
        ib = bi[v][lane];
      }
    const long long o = ((long long)f * mstride + col) * EXP_CHUNKS + chunk;
    pmax[o] = b;
    pidx[o] = ib;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) export_copy_kernel(const DevFrag* efr, const DevFrag* fr,
                                                          const T* X, const T* pmax,
                                                          const int* pidx, int mstride, T* states) {
  __shared__ T sgn[32];
  const int f = blockIdx.x, chunk = blockIdx.z;
  const DevFrag E = efr[f];
  const DevFrag F = fr[f];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int col = blockIdx.y * 32 + lane;
  const int ex = F.ext[0], ey = F.ext[1];
  const int P = ex * ey * F.ext[2];
  if (warp == 0) {
    T sg = T(1);
    if (col < F.n) {
      const long long o = ((long long)f * mstride + col) * EXP_CHUNKS;
      T b = pmax[o];
      int ib = pidx[o];
      for (int k = 1; k < EXP_CHUNKS; ++k)
        if (pmax[o + k] > b || (pmax[o + k] == b && pidx[o + k] < ib)) {
          b = pmax[o + k];
          ib = pidx[o + k];
        }
      if (ib >= 0 && ib < P) {
        const int x = ib % ex, y = (ib / ex) % ey, z = ib / (ex * ey);
        const int pd = ((z + E.lo[2]) * E.dext[1] + (y + E.lo[1])) * E.dext[0] + x + E.lo[0];
        sg = X[E.off + (long long)pd * E.ld + col] < T(0) ? T(-1) : T(1);
      }
    }
    sgn[lane] = sg;
  }
  __syncthreads();
  if (col >= F.n) return;
  const T s = sgn[lane];
  const int per = (P + EXP_CHUNKS - 1) / EXP_CHUNKS;
  const int p0 = chunk * per, p1 = min(P, p0 + per);
  if (p0 + warp >= p1) return;
  constexpr int U = 8;
  PointWalk w(p0 + warp, 8, ex, ey);
  for (int t0 = p0 + warp; t0 < p1; t0 += U * 8) {
    T v[U];
    int pf[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      pf[u] = -1;
      if (t0 + u * 8 < p1) {
        v[u] = X[E.off + (long long)w.at(E) * E.ld + col];
        pf[u] = w.at(F);
        w.step();
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (pf[u] >= 0) states[F.off + (long long)pf[u] * F.ld + col] = s * v[u];
  }
}

constexpr int VMAX_BLOCKS = 152;

// max and min of V: per-block partials in the storage type (FP32 compares
// are cheap, FP64 ones are not on this part), then one block combines them
// into out[0] = max, out[1] = min; part holds 2 * VMAX_BLOCKS doubles.
template <typename T>
__global__ void __launch_bounds__(256) vmax_partial_kernel(const T* V, long long n, double* part) {
  __shared__ T red[8], redm[8];
  T m = V[0], mn = V[0];
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += 256LL * gridDim.x) {
    m = max(m, V[i]);
    mn = min(mn, V[i]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
  }
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5] = m;
    redm[threadIdx.x >> 5] = mn;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 8; ++w) {
      m = max(m, red[w]);
      mn = min(mn, redm[w]);
    }
    part[2 * blockIdx.x] = (double)m;
    part[2 * blockIdx.x + 1] = (double)mn;
  }
}

__global__ void vmax_final_kernel(const double* part, int nb, double* out) {
  if (threadIdx.x != 0) return;
  double m = part[0], mn = part[1];
  for (int b = 1; b < nb; ++b) {
    m = fmax(m, part[2 * b]);
    mn = fmin(mn, part[2 * b + 1]);
  }
  out[0] = m;
  out[1] = mn;
}

}  // namespace

// Range of V (max, min) for the filter's bounds: taken at every solve,
// since V may change while the fragment layout (and the workspace) stays.
static ofm_status eig_vlim(ofm_ctx* c) {
  EigWork* w = c->eig;
  cudaStream_t s = c->stream;
  const long long npts = (long long)c->grid.n[0] * c->grid.n[1] * c->grid.n[2];
  KTimer kt(c, KC_EIG_INIT);
  double* part = (double*)w->d_vmax.p + 2;
  if (c->storage == OFM_STORE_FP64)
    vmax_partial_kernel<double><<<VMAX_BLOCKS, 256, 0, s>>>((const double*)c->V.p, npts, part);
  else
    vmax_partial_kernel<float><<<VMAX_BLOCKS, 256, 0, s>>>((const float*)c->V.p, npts, part);
  vmax_final_kernel<<<1, 32, 0, s>>>(part, VMAX_BLOCKS, (double*)w->d_vmax.p);
  OFM_CUDA(c, cudaGetLastError());
  OFM_CUDA(c, cudaMemcpyAsync(w->vlim, w->d_vmax.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  OFM_CUDA(c, cudaStreamSynchronize(s));
  return OFM_OK;
}

static ofm_status eig_setup(ofm_ctx* c, int guard_opt) {
  if (!c->eig) c->eig = new EigWork();
  EigWork* w = c->eig;
  const bool fp64 = c->storage == OFM_STORE_FP64;
  const size_t es = fp64 ? 8 : 4;
  const int vn = fp64 ? 2 : 4;
  const int nf = c->nfrag;
  w->efr = c->frags;
  w->elems = 0;
  w->mmax = 0;
  w->toff.resize(nf);
  w->tsum = 0;
  w->cta_start.resize(nf);
  long long ctas = 0;
  // The on-chip filter runs one CTA per (fragment, vector), one CTA per SM
  // (the box takes most of the shared memory), so a filter takes
  // ceil(m_max nfrag / SMs) waves.  With the default guard counts, one or two
  // guard vectors fewer per fragment (never below four) are taken when that
  // saves a whole wave.
  int trim = 0;
  if (guard_opt <= 0 && cheb_filter_smem(c->frags, fp64) > 0) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess || sms < 1) {
      cudaGetLastError();
      sms = 152;
    }
    auto waves = [&](int t) -> long long {
      int mm = 0;
      for (const DevFrag& F : c->frags) {
        const int g = std::max(4, F.n / 4) - t;
        if (g < 4) return LLONG_MAX;
        const long long P = (long long)F.ext[0] * F.ext[1] * F.ext[2];
        mm = std::max(mm, (int)std::min<long long>(std::min<long long>((long long)F.n + g, P - 1), 256));
      }
      return ((long long)mm * nf + sms - 1) / sms;
    };
    const long long w0 = waves(0);
    for (int t = 1; t <= 2 && trim == 0; ++t)
      if (waves(t) < w0) trim = t;
  }
  for (int a = 0; a < nf; ++a) {
    DevFrag& E = w->efr[a];
    const long long P = (long long)E.ext[0] * E.ext[1] * E.ext[2];
    int g = guard_opt > 0 ? guard_opt : std::max(4, E.n / 4) - trim;
    int m = (int)std::min<long long>((long long)E.n + g, P - 1);
    m = std::min(m, 256);
    E.n = m;
    E.ld = (m + 3) / 4 * 4;
    E.off = w->elems;
    w->elems += (E.Pd * E.ld + 63) / 64 * 64;
    w->mmax = std::max(w->mmax, m);
    w->toff[a] = w->tsum;
    w->tsum += m;
    w->cta_start[a] = (int)ctas;
    ctas += (E.Pd * (E.ld / vn) + 255) / 256;
  }
  w->total_ctas = (int)ctas;
  w->fgrid = apply_grid(w->efr, fp64, true);
  // on-chip filter (one launch per filter) where every fragment fits
  w->cf_smem = cheb_filter_smem(w->efr, fp64);
  w->cf_bytes0 = w->cf_bytes = w->cf_flops_step = 0.0;
  for (const DevFrag& E : w->efr) {
    const double P = (double)E.ext[0] * E.ext[1] * E.ext[2];
    // HBM: X in (and V), Y and H Y out; flops: 7-point stencil, shift, scale
    // and the recurrence, ten per point and state per step
    w->cf_bytes0 += P * (2.0 * E.n + 1.0) * es;
    w->cf_bytes += P * (3.0 * E.n + 1.0) * es;
    w->cf_flops_step += 10.0 * P * E.n;
  }
  w->filter_b2 =w->filter_b3 = w->gram_bytes = w->gram_flops = w->rot_bytes = w->rot_flops = 0;
  for (const DevFrag& E : w->efr) {
    const double P = (double)E.ext[0] * E.ext[1] * E.ext[2];
    w->filter_b2 += P * (2.0 * E.n + 1.0) * es;
    w->filter_b3 += P * (3.0 * E.n + 1.0) * es;
    w->gram_bytes += P * 2.0 * E.n * es;
    w->gram_flops += 2.0 * P * E.n * 2.0 * E.n;
    w->rot_bytes += P * 3.0 * E.n * es;   // Y and H Y in, X out
    w->rot_flops += 2.0 * 2.0 * P * E.n * E.n;
  }
  // Gram plan: self pairs over the interior box, chunks of ~1024 points
  std::vector<HostPair> sp(nf);
  for (int a = 0; a < nf; ++a) {
    const DevFrag& E = w->efr[a];
    sp[a].a = sp[a].b = a;
    sp[a].ks = sp[a].kh = (long long)E.ext[0] * E.ext[1] * E.ext[2];
    Piece pc;
    for (int d = 0; d < 3; ++d) {
      pc.la[d] = E.lo[d];
      pc.lb[d] = E.lo[d];
      pc.len[d] = E.ext[d];
    }
    sp[a].pieces.push_back(pc);
  }
  make_items_simt(w->efr, sp, 64, 1024, w->gpairs, w->gpieces, w->gitems, w->gpart);
  w->gblk = 0;
  for (auto& p : w->gpairs) w->gblk = std::max<long long>(w->gblk, p.blk_off + 2LL * w->efr[p.a].n * w->efr[p.b].n);
  // FP32 storage: the same Gram on tensor cores with TF32 hi+lo operands
  // (products to about 2^-22, FP32 accumulation), when the blocks fit
  if (!fp64) {
    std::vector<long long> goff(nf);
    long long gk = 0;
    for (int a = 0; a < nf; ++a) {
      goff[a] = w->gpairs[a].blk_off;
      gk += sp[a].kh;
    }
    OFM_TRY(ofm_tc_plan_build(c, &w->gtc, w->efr, sp, goff, gk, 0));
  }

  for (int i = 0; i < 4; ++i) OFM_TRY(ofm_ensure(c, w->buf[i], w->elems * es, "eigensolver block"));
  for (int i = 0; i < 4; ++i) OFM_CUDA(c, cudaMemsetAsync(w->buf[i].p, 0, w->elems * es, c->stream));
  OFM_TRY(ofm_ensure(c, w->d_efr, sizeof(DevFrag) * nf, "eigensolver table"));
  OFM_TRY(ofm_ensure(c, w->d_cta, sizeof(int) * nf, "eigensolver launch table"));
  OFM_TRY(ofm_ensure(c, w->d_toff, sizeof(long long) * nf, "eigensolver offsets"));
  OFM_TRY(ofm_ensure(c, w->theta, sizeof(double) * w->tsum, "Ritz values"));
  OFM_TRY(ofm_ensure(c, w->res, sizeof(double) * w->tsum, "residuals"));
  OFM_TRY(ofm_ensure(c, w->d_rank, sizeof(int) * nf, "ranks"));
  OFM_TRY(ofm_ensure(c, w->d_vmax, (2 + 2 * VMAX_BLOCKS) * sizeof(double), "max and min V"));
  const long long mm = (long long)w->mmax * w->mmax;
  OFM_TRY(ofm_ensure(c, w->Cm, sizeof(double) * mm * nf, "Ritz coefficients"));
  OFM_TRY(ofm_ensure(c, w->work, sizeof(double) * (3 * mm + 3 * w->mmax + 8) * nf, "Rayleigh-Ritz work"));
  OFM_TRY(ofm_ensure(c, w->blocks, sizeof(double) * w->gblk, "Gram blocks"));
  OFM_TRY(ofm_ensure(c, w->partials, sizeof(double) * w->gpart, "Gram partials"));
  OFM_TRY(ofm_ensure(c, w->d_gpairs, sizeof(DevPair) * w->gpairs.size(), "Gram pairs"));
  OFM_TRY(ofm_ensure(c, w->d_gpieces, sizeof(Piece) * w->gpieces.size(), "Gram pieces"));
  OFM_TRY(ofm_ensure(c, w->d_gitems, sizeof(WorkItem) * w->gitems.size(), "Gram items"));
  cudaStream_t s = c->stream;
  OFM_CUDA(c, cudaMemcpyAsync(w->d_efr.p, w->efr.data(), sizeof(DevFrag) * nf, cudaMemcpyHostToDevice, s));
  OFM_CUDA(c, cudaMemcpyAsync(w->d_cta.p, w->cta_start.data(), sizeof(int) * nf, cudaMemcpyHostToDevice, s));
  OFM_CUDA(c, cudaMemcpyAsync(w->d_toff.p, w->toff.data(), sizeof(long long) * nf, cudaMemcpyHostToDevice, s));
  OFM_CUDA(c, cudaMemcpyAsync(w->d_gpairs.p, w->gpairs.data(), sizeof(DevPair) * w->gpairs.size(), cudaMemcpyHostToDevice, s));
  OFM_CUDA(c, cudaMemcpyAsync(w->d_gpieces.p, w->gpieces.data(), sizeof(Piece) * w->gpieces.size(), cudaMemcpyHostToDevice, s));
  OFM_CUDA(c, cudaMemcpyAsync(w->d_gitems.p, w->gitems.data(), sizeof(WorkItem) * w->gitems.size(), cudaMemcpyHostToDevice, s));
  long long maxP = 0;
  for (auto& E : w->efr) maxP = std::max<long long>(maxP, (long long)E.ext[0] * E.ext[1] * E.ext[2]);
  // FP32 blocks take the 256-point register-tiled rotation when two CTAs fit
  // on an SM; FP64 blocks and very wide ones the 64-point form
  {
    const size_t mcs = (size_t)(w->mmax + RJB - 1) / RJB * RJB;
    const size_t smem4 = RT4 * sizeof(int) + ((size_t)w->mmax * mcs + 2 * (size_t)w->mmax * RT4) * sizeof(float);
    w->rot4 = !fp64 && w->mmax <= RM4 && smem4 <= 110 * 1024;
    if (w->rot4) {
      w->rot_smem = smem4;
      w->rot_blocks = (int)std::min<long long>((maxP + RT4 - 1) / RT4, 64);
    } else {
      w->rot_smem = 16 * ((RT * sizeof(int) + 15) / 16) +
                    (4 * RJ + (size_t)w->mmax * w->mmax + 2 * (size_t)RT * (w->mmax + 1 + (w->mmax & 1))) * es;
      w->rot_blocks = (int)std::min<long long>((maxP + RT - 1) / RT, 64);
    }
  }
  OFM_TRY(ofm_ensure(c, w->rpart, sizeof(double) * (size_t)nf * w->rot_blocks * w->mmax, "residual partials"));
  if (w->rot_smem > 227 * 1024) return ofm_fail(c, OFM_ERR_INVALID, "block size too large for the rotation kernel");
  if (w->rot4) OFM_CUDA(c, cudaFuncSetAttribute(rotate4_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)w->rot_smem));
  else if (fp64) OFM_CUDA(c, cudaFuncSetAttribute(rotate_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)w->rot_smem));
  else OFM_CUDA(c, cudaFuncSetAttribute(rotate_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)w->rot_smem));
  w->rr_threads = std::min(RR_MAX_THREADS, std::max(256, 32 * ((w->mmax + 1) / 2)));
  const size_t rr = (3 * (size_t)w->mmax * (w->mmax + 1 + (w->mmax & 1)) + 3 * (size_t)w->mmax) * es;
  w->rr_smem = rr <= 200 * 1024 ? rr : 0;
  if (w->rr_smem) {
    if (fp64) OFM_CUDA(c, cudaFuncSetAttribute(rayleigh_ritz_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)w->rr_smem));
    else OFM_CUDA(c, cudaFuncSetAttribute(rayleigh_ritz_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)w->rr_smem));
  }
  w->ready = true;
  return OFM_OK;
}

// Gram blocks of (Y, HY), Rayleigh-Ritz, rotation of Y into xo, residuals.
// H X = (H Y) C is formed only for the residual norms, in registers: the
// next filter starts from X alone and the export reads X, so it is never
// stored.
static ofm_status eig_rr(ofm_ctx* c, int y, int hy, int xo, unsigned long long salt) {
  EigWork* w = c->eig;
  const bool fp64 = c->storage == OFM_STORE_FP64;
  const int nf = c->nfrag;
  cudaStream_t s = c->stream;
  if (!fp64 && ofm_tc_plan_ok(w->gtc, OFM_TC_TF32X3)) {
    OFM_TRY(ofm_tc_run(c, w->gtc, OFM_TC_TF32X3, (const DevFrag*)w->d_efr.p, w->buf[y].p,
                       w->buf[hy].p, (double*)w->blocks.p, KC_GRAM, KC_GRAM, w->gram_bytes,
                       w->gram_flops));
  } else {
  KTimer kt(c, KC_GRAM, 2, w->gram_bytes, w->gram_flops);
  launch_contract_simt(fp64 ? OFM_PREC_FP64 : OFM_PREC_FP32, fp64, (const DevFrag*)w->d_efr.p,
                       (const DevPair*)w->d_gpairs.p, (const Piece*)w->d_gpieces.p,
                       (const WorkItem*)w->d_gitems.p, (int)w->gitems.size(), w->buf[y].p,
                       w->buf[hy].p, w->partials.p, 64, s);
  launch_finalize_simt(fp64 ? OFM_PREC_FP64 : OFM_PREC_FP32, (const DevFrag*)w->d_efr.p,
                       (const DevPair*)w->d_gpairs.p, nf, (const WorkItem*)w->d_gitems.p,
                       w->partials.p, 64, (double*)w->blocks.p, s);
  }
  const long long mm = (long long)w->mmax * w->mmax;
  { KTimer kt(c, KC_RR);
  if (fp64)
    rayleigh_ritz_kernel<double><<<nf, w->rr_threads, w->rr_smem, s>>>(
        (const DevFrag*)w->d_efr.p, (const DevPair*)w->d_gpairs.p, (const double*)w->blocks.p,
        (double*)w->work.p, 3 * mm + 3 * w->mmax + 8, (double*)w->Cm.p, mm, (double*)w->theta.p,
        (const long long*)w->d_toff.p, 1e-13, (int*)w->d_rank.p, w->rr_smem > 0 ? 1 : 0);
  else
    rayleigh_ritz_kernel<float><<<nf, w->rr_threads, w->rr_smem, s>>>(
        (const DevFrag*)w->d_efr.p, (const DevPair*)w->d_gpairs.p, (const double*)w->blocks.p,
        (float*)w->work.p, 3 * mm + 3 * w->mmax + 8, (double*)w->Cm.p, mm, (double*)w->theta.p,
        (const long long*)w->d_toff.p, 1e-5, (int*)w->d_rank.p, w->rr_smem > 0 ? 1 : 0);
  }
  dim3 g(w->rot_blocks, nf);
  KTimer kt(c, KC_ROTATE, 2, w->rot_bytes, w->rot_flops);
  if (fp64)
    rotate_kernel<double><<<g, 256, w->rot_smem, s>>>((const DevFrag*)w->d_efr.p, (const double*)w->buf[y].p,
                                               (double*)w->buf[xo].p, (const double*)w->buf[hy].p,
                                               (const double*)w->Cm.p, mm,
                                               (const int*)w->d_rank.p, (const double*)w->theta.p,
                                               (const long long*)w->d_toff.p, (double*)w->rpart.p,
                                               w->mmax, salt);
  else if (w->rot4)
    rotate4_kernel<<<g, 256, w->rot_smem, s>>>((const DevFrag*)w->d_efr.p, (const float*)w->buf[y].p,
                                               (float*)w->buf[xo].p, (const float*)w->buf[hy].p,
                                               (const double*)w->Cm.p, mm,
                                               (const int*)w->d_rank.p, (const double*)w->theta.p,
                                               (const long long*)w->d_toff.p, (double*)w->rpart.p,
                                               w->mmax, salt);
  else
    rotate_kernel<float><<<g, 256, w->rot_smem, s>>>((const DevFrag*)w->d_efr.p, (const float*)w->buf[y].p,
                                              (float*)w->buf[xo].p, (const float*)w->buf[hy].p,
                                              (const double*)w->Cm.p, mm,
                                              (const int*)w->d_rank.p, (const double*)w->theta.p,
                                              (const long long*)w->d_toff.p, (double*)w->rpart.p,
                                              w->mmax, salt);
  residual_reduce_kernel<<<nf, 128, 0, s>>>((const DevFrag*)w->d_efr.p, (const double*)w->rpart.p,
                                            w->rot_blocks, w->mmax, (const long long*)w->d_toff.p,
                                            (double*)w->res.p);
  OFM_CUDA(c, cudaGetLastError());
  return OFM_OK;
}

static void apply_block(ofm_ctx* c, int in, int prev, int out, const double* coef) {
  EigWork* w = c->eig;
  KTimer kt(c, KC_FILTER, 1, prev >= 0 ? w->filter_b3 : w->filter_b2);
  launch_apply_filter((const DevFrag*)w->d_efr.p, c->nfrag, w->fgrid, c->V.p, w->buf[in].p,
                      prev >= 0 ? w->buf[prev].p : nullptr, w->buf[out].p, coef, c->grid.n,
                      c->grid.h, c->storage == OFM_STORE_FP64,
                      (int*)c->flag.p + OFM_FLAG_STENCIL, c->stream);
  c->stencil_check = true;
}

static int other(int a, int b) {
  for (int i = 0; i < 4; ++i)
    if (i != a && i != b) return i;
  return -1;
}

static ofm_status ofm_fragment_eigs_impl(ofm_ctx* c, const ofm_eig_opts* opts, double* eps_out,
                                        double* resid_out) {
  OFM_RANGE("ofm_fragment_eigs");
  if (!c) return OFM_ERR_INVALID;
  if (!c->built) return ofm_fail(c, OFM_ERR_STATE, "ofm_build_fragments must come first");
  if (!eps_out) return ofm_fail(c, OFM_ERR_INVALID, "eps_out must not be NULL");
  ofm_eig_opts o{};
  if (opts) o = *opts;
  const bool fp64 = c->storage == OFM_STORE_FP64;
  const double tol = o.tol > 0 ? o.tol : (fp64 ? 1e-9 : 1e-5);
  // 240: the polymer's FP32 blocks of 32-49 states in 16-24 point boxes need
  // about 200 outer iterations (60 left residuals of 4e-5 against 1e-5);
  // converged blocks stop early, so the bound costs nothing elsewhere
  const int max_iter = o.max_iter > 0 ? o.max_iter : 240;
  const int degree = o.degree > 0 ? o.degree : 32;
  if (o.tol < 0 || o.max_iter < 0 || o.degree < 0 || o.extra_states < 0 || degree > 200)
    return ofm_fail(c, OFM_ERR_INVALID, "bad eigensolver options");
  if (!c->eig || !c->eig->ready || c->eig->efr.size() != (size_t)c->nfrag || o.extra_states > 0) {
    OFM_TRY(eig_setup(c, o.extra_states));
  }
  OFM_TRY(eig_vlim(c));
  EigWork* w = c->eig;
  const int nf = c->nfrag;
  cudaStream_t s = c->stream;
  c->assembled = c->dense_ready = c->factored = false;

  // start block in buffer 0
  { KTimer kt(c, KC_EIG_INIT);
  if (fp64)
    init_random_kernel<double><<<w->total_ctas, 256, 0, s>>>((const DevFrag*)w->d_efr.p, (const int*)w->d_cta.p, nf, (double*)w->buf[0].p, o.seed);
  else
    init_random_kernel<float><<<w->total_ctas, 256, 0, s>>>((const DevFrag*)w->d_efr.p, (const int*)w->d_cta.p, nf, (float*)w->buf[0].p, o.seed); }
  OFM_CUDA(c, cudaGetLastError());
  // coefficient table: degree steps x fragments x (alpha, beta, shift)
  OFM_TRY(ofm_ensure(c, w->coef, sizeof(double) * 3 * nf * (degree + 1), "filter coefficients"));
  std::vector<double> coef(3 * (size_t)nf * (degree + 1));
  // plain H (alpha 1, beta 0, shift 0) sits in slot `degree`
  for (int f = 0; f < nf; ++f) {
    double* cf = &coef[3 * ((size_t)degree * nf + f)];
    cf[0] = 1.0; cf[1] = 0.0; cf[2] = 0.0;
  }
  const double* d_coef = (const double*)w->coef.p;
  const double* d_plain = d_coef + 3 * (size_t)degree * nf;
  OFM_CUDA(c, cudaMemcpyAsync(w->coef.p, coef.data(), sizeof(double) * coef.size(), cudaMemcpyHostToDevice, s));

  // initial Rayleigh-Ritz of the random block
  if (w->cf_smem) {
    KTimer kt(c, KC_FILTER, 1, w->cf_bytes0, w->cf_flops_step);
    launch_cheb_filter((const DevFrag*)w->d_efr.p, nf, w->mmax, w->cf_smem, c->V.p, w->buf[0].p,
                       nullptr, w->buf[3].p, d_coef, 0, c->grid.n, c->grid.h, s);
  } else {
    apply_block(c, 0, -1, 3, d_plain);
  }
  OFM_TRY(eig_rr(c, 0, 3, 1, 0x1234ULL + o.seed));
  int xb = 1;
  std::vector<double> th(w->tsum), rs(w->tsum);
  const double bup = 6.0 / (c->grid.h * c->grid.h) + w->vlim[0];
  // The filter may spread the wanted part of the block by at most a factor
  // s: a component shrunk by s relative to the largest one in its vector
  // carries rounding of unit roundoff u x s.  For a random block every
  // vector mixes every state, so s <= 0.1 tol / u keeps that floor below
  // the tolerance (FP32: 1e2, FP64: 1e6).  Once the block holds Ritz
  // vectors, the lower states enter vector i only through its error,
  // about the largest residual r of the fragment, so the floor is u s r
  // and s may grow to 0.1 tol / (u r), up to 1e6 (FP32) / 1e12 (FP64).
  const double u_round = fp64 ? 1.1e-16 : 6e-8;
  const double s_min = fp64 ? 1e6 : 1e2, s_max = fp64 ? 1e12 : 1e6;
  bool converged = false;
  int it = 0;
  for (; it <= max_iter; ++it) {
    OFM_CUDA(c, cudaMemcpyAsync(th.data(), w->theta.p, sizeof(double) * w->tsum, cudaMemcpyDeviceToHost, s));
    OFM_CUDA(c, cudaMemcpyAsync(rs.data(), w->res.p, sizeof(double) * w->tsum, cudaMemcpyDeviceToHost, s));
    OFM_CUDA(c, cudaStreamSynchronize(s));
    converged = true;
    for (int f = 0; f < nf && converged; ++f)
      for (int i = 0; i < c->frags[f].n; ++i)
        if (!(rs[w->toff[f] + i] <= tol)) {
          converged = false;
          break;
        }
    if (converged || it == max_iter) break;
    // degree of this iteration: T_d grows like exp(d acosh(t)) below the
    // damped interval, so the ratio between the bottom of the spectrum
    // (min V on the first pass, the lowest Ritz value after) and the last
    // wanted Ritz value is about exp(d (acosh(t_low) - acosh(t_want)));
    // keep it within the fragment's spread cap for every fragment
    int deg = degree;
    for (int f = 0; f < nf; ++f) {
      const int m = w->efr[f].n;
      const double* t = &th[w->toff[f]];
      double rmax = 0.0;
      for (int i = 0; i < c->frags[f].n; ++i) rmax = std::max(rmax, rs[w->toff[f] + i]);
      const double smax = (it == 0 || !(rmax > 0.0))
                              ? s_min
                              : std::min(s_max, std::max(s_min, 0.1 * tol / (u_round * rmax)));
      const double spread_max = std::log(smax);
      double blo = t[m - 1], a0 = t[0];
      double bu = std::max(bup, blo + 1e-3);
      if (!(blo > a0)) blo = a0 + 1e-3 * (bu - a0);
      const double e = 0.5 * (bu - blo), cc = 0.5 * (bu + blo);
      const double low = (it == 0) ? std::min(w->vlim[1], a0) : a0;
      const double tl = (cc - low) / e, tw = (cc - t[c->frags[f].n - 1]) / e;
      if (tl > 1.0) {
        const double gap = std::acosh(tl) - (tw > 1.0 ? std::acosh(tw) : 0.0);
        if (gap > 0.0) deg = std::min(deg, std::max(4, (int)(spread_max / gap)));
      }
    }
    // filter coefficients from the current Ritz values
    for (int f = 0; f < nf; ++f) {
      const int m = w->efr[f].n;
      const double* t = &th[w->toff[f]];
      double blo = t[m - 1], a0 = t[0];
      double bu = std::max(bup, blo + 1e-3);
      if (!(blo > a0)) blo = a0 + 1e-3 * (bu - a0);
      const double e = 0.5 * (bu - blo), cc = 0.5 * (bu + blo);
      const double sigma1 = e / (a0 - cc);
      double sigma = sigma1;
      const double tau = 2.0 / sigma1;
      for (int k = 0; k < deg; ++k) {
        double* cf = &coef[3 * ((size_t)k * nf + f)];
        if (k == 0) {
          cf[0] = sigma1 / e;
          cf[1] = 0.0;
        } else {
          const double sn = 1.0 / (tau - sigma);
          cf[0] = 2.0 * sn / e;
          cf[1] = -sigma * sn;
          sigma = sn;
        }
        cf[2] = cc;
      }
    }
    OFM_CUDA(c, cudaMemcpyAsync(w->coef.p, coef.data(), sizeof(double) * 3 * nf * deg, cudaMemcpyHostToDevice, s));
    int cur, hy;
    if (w->cf_smem) {
      // the whole filter and H Y in one launch, on chip
      cur = other(xb, -1);
      hy = other(xb, cur);
      KTimer kt(c, KC_FILTER, 1, w->cf_bytes, (deg + 1) * w->cf_flops_step);
      launch_cheb_filter((const DevFrag*)w->d_efr.p, nf, w->mmax, w->cf_smem, c->V.p, w->buf[xb].p,
                         w->buf[cur].p, w->buf[hy].p, d_coef, deg, c->grid.n, c->grid.h, s);
    } else {
      int prev = -1;
      cur = xb;
      for (int k = 0; k < deg; ++k) {
        const int nxt = other(prev, cur);
        apply_block(c, cur, prev, nxt, d_coef + 3 * (size_t)k * nf);
        prev = cur;
        cur = nxt;
      }
      hy = other(cur, -1);
      apply_block(c, cur, -1, hy, d_plain);
    }
    const int xo = other(cur, hy);
    OFM_TRY(eig_rr(c, cur, hy, xo, 0x9876ULL * (it + 1) + o.seed));
    xb = xo;
  }
  // export the first n_a Ritz vectors with the sign gauge
  dim3 eg(nf, (w->mmax + 31) / 32, EXP_CHUNKS);
  { KTimer kt(c, KC_EXPORT, 2);
  const size_t pe = (size_t)nf * w->mmax * EXP_CHUNKS;
  OFM_TRY(ofm_ensure(c, w->xpart, pe * (sizeof(double) + sizeof(int)), "export partials"));
  int* pidx = (int*)((double*)w->xpart.p + pe);
  const DevFrag* ef = (const DevFrag*)w->d_efr.p;
  const DevFrag* cf = (const DevFrag*)c->d_frags.p;
  if (fp64) {
    double* pm = (double*)w->xpart.p;
    export_max_kernel<double><<<eg, 256, 0, s>>>(ef, cf, (const double*)w->buf[xb].p, pm, pidx, w->mmax);
    export_copy_kernel<double><<<eg, 256, 0, s>>>(ef, cf, (const double*)w->buf[xb].p, pm, pidx,
                                                  w->mmax, (double*)c->states.p);
  } else {
    float* pm = (float*)w->xpart.p;
    export_max_kernel<float><<<eg, 256, 0, s>>>(ef, cf, (const float*)w->buf[xb].p, pm, pidx, w->mmax);
    export_copy_kernel<float><<<eg, 256, 0, s>>>(ef, cf, (const float*)w->buf[xb].p, pm, pidx,
                                                 w->mmax, (float*)c->states.p);
  } }
  OFM_CUDA(c, cudaGetLastError());
  OFM_CUDA(c, cudaStreamSynchronize(s));
  double worst = 0.0;
  for (int f = 0; f < nf; ++f)
    for (int i = 0; i < c->frags[f].n; ++i) {
      eps_out[c->frags[f].basis0 + i] = th[w->toff[f] + i];
      if (resid_out) resid_out[c->frags[f].basis0 + i] = rs[w->toff[f] + i];
      worst = std::max(worst, rs[w->toff[f] + i]);
    }
  OFM_TRY(ofm_wait_status(c));
  std::fill(c->frag_set.begin(), c->frag_set.end(), 1);
  c->have_states = true;
  c->last_eig_iters = it;
  const bool injected = c->fault == OFM_FAULT_NONCONV;
  if (injected) converged = false;
  if (!converged) {
    char buf[192];
    if (injected)
      snprintf(buf, sizeof buf, "fragment eigensolver: not converged (injected by OFM_FAULT=nonconv; "
               "largest residual %.3e after %d iterations)", worst, it);
    else
      snprintf(buf, sizeof buf, "fragment eigensolver: largest residual %.3e > tol %.3e after %d iterations",
               worst, tol, it);
    return ofm_fail(c, OFM_ERR_NOT_CONVERGED, buf);
  }
  return OFM_OK;
}

extern "C" ofm_status ofm_fragment_eigs(ofm_ctx* c, const ofm_eig_opts* opts, double* eps_out, double* resid_out) {
  const ofm_status st = ofm_fragment_eigs_impl(c, opts, eps_out, resid_out);
  if ((st != OFM_OK && st != OFM_ERR_NOT_CONVERGED) || !c || !c->checks) return st;
  const ofm_status g = ofm_check_guards_now(c, "ofm_fragment_eigs");
  return g != OFM_OK ? g : st;
}
