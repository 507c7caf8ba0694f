// Eigenvectors of Eq. 2 for the eigenvalues of an energy window (the
// optional C of the window solve), from the factorisation the eigenvalues
// came from:
//   1. inverse iteration on the tridiagonal T: for each eigenvalue lambda
//      (accurate to a few ulps from the Sturm multisection), solve
//      (T - lambda I) y = b three times from a pseudo-random b, with
//      Gaussian elimination with partial pivoting on the tridiagonal matrix
//      (the row exchanges fill one extra superdiagonal); y grows along the
//      eigenvector by 1/|lambda - lambda_true| per solve.  Eigenvalues
//      closer than 1e-5 ||T||_1 form a cluster, whose vectors are computed
//      in order by one warp and orthogonalised against each other (modified
//      Gram-Schmidt) after every solve; separate clusters run in parallel.
//   2. back-transformation x = Q y with the Householder reflectors of the
//      tridiagonal reduction, Q = H_0 H_1 ... H_{n-3}, H_k = I - tau_k v_k v_k^T
//      (v_k kept in row k of the reduced matrix), applied from k = n-3 down;
//   3. C = L^-T x (back substitution with the Cholesky factor), so that
//      H C = S C diag(E) and C^T S C = I.
// Steps 2 and 3 run in one CTA per eigenvector.
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <vector>

#include "ofm_internal.h"

namespace ofm {

namespace {

__device__ __forceinline__ double warp_sum(double s) {
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// Deterministic start vector entry in [-1, 1): SplitMix64 of (index, row).
__device__ __forceinline__ double start_entry(unsigned long long j, unsigned long long i) {
  unsigned long long z = (j << 32) ^ i ^ 0x5851F42D4C957F2DULL;
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  z ^= z >> 31;
  return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

// One warp per cluster of eigenvalues [cl[c], cl[c+1]).  Scratch per
// cluster: dd, du, du2, dl (n each) and ipiv (n ints).  Lane 0 runs the
// sequential factorisation and solves; the warp does the vector work.
__global__ void __launch_bounds__(32) stein_kernel(const double* __restrict__ d,
                                                    const double* __restrict__ e, int n,
                                                    const double* __restrict__ lam,
                                                    const int* __restrict__ cl, double tnorm,
                                                    double* __restrict__ scratch,
                                                    int* __restrict__ piv_scratch,
                                                    double* __restrict__ Y) {
  const int c = blockIdx.x, lane = threadIdx.x;
  double* dd = scratch + (size_t)c * 4 * n;
  double* du = dd + n;
  double* du2 = du + n;
  double* dl = du2 + n;
  int* ipiv = piv_scratch + (size_t)c * n;
  const double pert = DBL_EPSILON * tnorm;   // replaces an exactly singular pivot
  for (int j = cl[c]; j < cl[c + 1]; ++j) {
    double* y = Y + (size_t)j * n;
    const double shift = lam[j];
    if (lane == 0) {
      // LU of T - shift I with partial pivoting; dd holds U's diagonal as
      // reciprocals afterwards
      for (int i = 0; i < n; ++i) {
        dd[i] = d[i] - shift;
        if (i + 1 < n) {
          dl[i] = e[i];
          du[i] = e[i];
        }
        du2[i] = 0.0;
      }
      for (int i = 0; i + 1 < n; ++i) {
        if (fabs(dd[i]) >= fabs(dl[i])) {
          ipiv[i] = i;
          if (dd[i] == 0.0) dd[i] = pert;
          const double f = dl[i] / dd[i];
          dl[i] = f;
          dd[i + 1] -= f * du[i];
        } else {
          ipiv[i] = i + 1;
          const double f = dd[i] / dl[i];
          dd[i] = dl[i];
          dl[i] = f;
          const double t = du[i];
          du[i] = dd[i + 1];
          dd[i + 1] = t - f * dd[i + 1];
          if (i + 2 < n) {
            du2[i] = du[i + 1];
            du[i + 1] = -f * du[i + 1];
          }
        }
      }
      if (dd[n - 1] == 0.0) dd[n - 1] = pert;
      for (int i = 0; i < n; ++i) dd[i] = 1.0 / dd[i];
    }
    for (int i = lane; i < n; i += 32) y[i] = start_entry((unsigned long long)j, (unsigned long long)i);
    __syncwarp();
    for (int it = 0; it < 3; ++it) {
      if (lane == 0) {
        // forward: apply the row exchanges and L
        for (int i = 0; i + 1 < n; ++i) {
          if (ipiv[i] == i) {
            y[i + 1] -= dl[i] * y[i];
          } else {
            const double t = y[i];
            y[i] = y[i + 1];
            y[i + 1] = t - dl[i] * y[i];
          }
        }
        // back substitution with U (diagonal dd as reciprocals, du, du2)
        y[n - 1] *= dd[n - 1];
        if (n >= 2) y[n - 2] = (y[n - 2] - du[n - 2] * y[n - 1]) * dd[n - 2];
        for (int i = n - 3; i >= 0; --i)
          y[i] = (y[i] - du[i] * y[i + 1] - du2[i] * y[i + 2]) * dd[i];
      }
      __syncwarp();
      // orthogonalise against the cluster's earlier vectors
      for (int q = cl[c]; q < j; ++q) {
        const double* yq = Y + (size_t)q * n;
        double s = 0.0;
        for (int i = lane; i < n; i += 32) s += yq[i] * y[i];
        s = warp_sum(s);
        for (int i = lane; i < n; i += 32) y[i] -= s * yq[i];
        __syncwarp();
      }
      double s = 0.0;
      for (int i = lane; i < n; i += 32) s += y[i] * y[i];
      s = warp_sum(s);
      const double inv = s > 0.0 ? 1.0 / sqrt(s) : 1.0;
      for (int i = lane; i < n; i += 32) y[i] *= inv;
      __syncwarp();
    }
  }
}

__device__ __forceinline__ double cta_sum(double s, double* red) {
  s = warp_sum(s);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  return t;
}

// One CTA per eigenvector: x = Q y, then C(:, j) = L^-T x.
__global__ void __launch_bounds__(256) backtransform_kernel(const double* __restrict__ R,
                                                            const double* __restrict__ tau,
                                                            const double* __restrict__ L, int n,
                                                            const double* __restrict__ Y,
                                                            double* __restrict__ C) {
  extern __shared__ double sx[];
  double* x = sx;        // n
  double* dinv = sx + n; // n
  __shared__ double red[8];
  __shared__ double ci;
  const int j = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < n; i += nt) {
    x[i] = Y[(size_t)j * n + i];
    dinv[i] = 1.0 / L[(size_t)i * n + i];
  }
  __syncthreads();
  // x = H_0 (H_1 (... (H_{n-3} y)))
  for (int k = n - 3; k >= 0; --k) {
    const double t = tau[k];
    if (t == 0.0) continue;   // uniform over the CTA
    const double* v = R + (size_t)k * n;
    double s = 0.0;
    for (int i = k + 1 + tid; i < n; i += nt) s += v[i] * x[i];
    const double f = t * cta_sum(s, red);
    for (int i = k + 1 + tid; i < n; i += nt) x[i] -= f * v[i];
    __syncthreads();
  }
  // L^T c = x, from the last row up: c_i = x_i / L_ii, then x_j -= L_ij c_i (j < i)
  for (int i = n - 1; i >= 0; --i) {
    if (tid == 0) ci = x[i] * dinv[i];
    __syncthreads();
    const double cv = ci;
    const double* Li = L + (size_t)i * n;
    for (int q = tid; q < i; q += nt) x[q] -= Li[q] * cv;
    if (tid == 0) x[i] = cv;
    __syncthreads();
  }
  for (int i = tid; i < n; i += nt) C[(size_t)j * n + i] = x[i];
}

}  // namespace

}  // namespace ofm

using namespace ofm;

// m eigenvectors for the eigenvalues E (host copy, ascending) that the last
// ofm_window_bisect left on the device in w_tmp[0..m).
ofm_status ofm_window_vectors(ofm_ctx* c, int m, const double* E, double* C_out) {
  const int n = c->dense_n;
  cudaStream_t s = c->stream;
  // ||T||_1 from d and e for the cluster threshold and the pivot guard
  std::vector<double> hd(n), he(std::max(1, n - 1));
  OFM_CUDA(c, cudaMemcpyAsync(hd.data(), c->w_d.p, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  if (n > 1)
    OFM_CUDA(c, cudaMemcpyAsync(he.data(), c->w_e.p, sizeof(double) * (n - 1), cudaMemcpyDeviceToHost, s));
  OFM_CUDA(c, cudaStreamSynchronize(s));
  double tnorm = 0.0;
  for (int i = 0; i < n; ++i) {
    const double r = std::fabs(hd[i]) + (i > 0 ? std::fabs(he[i - 1]) : 0.0) +
                     (i + 1 < n ? std::fabs(he[i]) : 0.0);
    tnorm = std::max(tnorm, r);
  }
  if (!(tnorm > 0.0)) tnorm = 1.0;
  std::vector<int> cl{0};
  for (int j = 1; j < m; ++j)
    if (E[j] - E[j - 1] > 1e-5 * tnorm) cl.push_back(j);
  cl.push_back(m);
  const int nc = (int)cl.size() - 1;
  // device scratch: eigenvalues stay in w_tmp; Y, C, LU arrays, cluster table
  const size_t ybytes = sizeof(double) * (size_t)n * m;
  const size_t lubytes = sizeof(double) * 4 * (size_t)n * nc;
  const size_t pivbytes = sizeof(int) * (size_t)n * nc;
  const size_t clbytes = sizeof(int) * (size_t)(nc + 1);
  const size_t total = 2 * ybytes + lubytes + pivbytes + clbytes + 1024;
  OFM_TRY(ofm_ensure(c, c->staging, total, "window eigenvector scratch"));
  unsigned char* base = (unsigned char*)c->staging.p;
  double* Y = (double*)base;
  double* Cd = (double*)(base + ybytes);
  double* lu = (double*)(base + 2 * ybytes);
  int* piv = (int*)(base + 2 * ybytes + lubytes);
  int* dcl = (int*)(base + 2 * ybytes + lubytes + pivbytes);
  OFM_CUDA(c, cudaMemcpyAsync(dcl, cl.data(), clbytes, cudaMemcpyHostToDevice, s));
  {
    KTimer kt(c, KC_VECTORS, 2, 0.0, 4.0 * n * (double)n * m);
    stein_kernel<<<nc, 32, 0, s>>>((const double*)c->w_d.p, (const double*)c->w_e.p, n,
                                   (const double*)c->w_tmp.p, dcl, tnorm, lu, piv, Y);
    const size_t smem = 2 * sizeof(double) * (size_t)n;
    if (smem > 48 * 1024)
      OFM_CUDA(c, cudaFuncSetAttribute(backtransform_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    backtransform_kernel<<<m, 256, smem, s>>>((const double*)c->w_A.p, (const double*)c->w_tau.p,
                                              (const double*)c->w_L.p, n, Y, Cd);
  }
  OFM_CUDA(c, cudaGetLastError());
  OFM_CUDA(c, cudaMemcpyAsync(C_out, Cd, ybytes, cudaMemcpyDeviceToHost, s));
  OFM_CUDA(c, cudaStreamSynchronize(s));
  return OFM_OK;
}
