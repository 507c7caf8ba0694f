// H phi on the dilated fragment boxes (Eq. 1 with the 7-point stencil), and
// the layout conversions between the caller's column-major states and the
// library's point-major storage.
//
// H phi(r) = (3/h^2) phi(r) - (1/(2 h^2)) sum_{6 neighbours} phi + V(r) phi(r)
// with phi zero outside its box (Sec. II: H phi_i^(j) with the whole-system
// H).  It is evaluated on every point of the dilated box, where it can be
// non-zero.  Storage is point-major (the n states of one point are adjacent),
// so one thread owns 16 bytes of states of one point and every neighbour
// access of a warp is a contiguous run: the kernel is a streaming stencil,
// bound by HBM bandwidth.  The launch grid is 2-D: blockIdx.y is the
// fragment, blockIdx.x a chunk of its (point, 16-byte column group)
// elements, each thread handling APPLY_EPT of them.
#include <cuda_runtime.h>

#include <algorithm>

#include "ofm_internal.h"

namespace ofm {

template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int n = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int n = 2; };

__device__ __forceinline__ float4 fma4(float a, float4 x, float4 y) {
  return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}
__device__ __forceinline__ double2 fma4(double a, double2 x, double2 y) {
  return make_double2(fma(a, x.x, y.x), fma(a, x.y, y.y));
}
__device__ __forceinline__ float4 add4(float4 a, float4 b) {
  return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}
__device__ __forceinline__ double2 add4(double2 a, double2 b) {
  return make_double2(a.x + b.x, a.y + b.y);
}
__device__ __forceinline__ float4 zero4(float) { return make_float4(0.f, 0.f, 0.f, 0.f); }
__device__ __forceinline__ double2 zero4(double) { return make_double2(0.0, 0.0); }

// Neighbour index along one dimension in the storage box: +/-1 step of
// `stride` points; in a full-span dimension it wraps, otherwise a step out
// of the storage box reads zero (returns -1).
__device__ __forceinline__ int nb_index(int p, int c, int ext, int full, int dir, int stride) {
  int c2 = c + dir;
  if (c2 < 0 || c2 >= ext) {
    if (!full) return -1;
    c2 = (c2 + ext) % ext;
  }
  return p + (c2 - c) * stride;
}

// Stencil sum over the six neighbours of point p (coordinates x, y, z) for
// the column group q.
template <typename T>
__device__ __forceinline__ typename Vec16<T>::type neighbour_sum(
    const typename Vec16<T>::type* __restrict__ S, const DevFrag& F, int p, int x, int y, int z,
    int q, int qpp) {
  using V16 = typename Vec16<T>::type;
  const int ex = F.dext[0], ey = F.dext[1], ez = F.dext[2];
  // branch-free: a neighbour outside the storage box reads the point itself
  // with weight 0, so all six loads can be in flight at once
  int nb[6];
  nb[0] = nb_index(p, x, ex, F.full[0], +1, 1);
  nb[1] = nb_index(p, x, ex, F.full[0], -1, 1);
  nb[2] = nb_index(p, y, ey, F.full[1], +1, ex);
  nb[3] = nb_index(p, y, ey, F.full[1], -1, ex);
  nb[4] = nb_index(p, z, ez, F.full[2], +1, ex * ey);
  nb[5] = nb_index(p, z, ez, F.full[2], -1, ex * ey);
  V16 v[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) v[i] = S[(nb[i] >= 0 ? nb[i] : p) * qpp + q];
  V16 sum = zero4(T());
#pragma unroll
  for (int i = 0; i < 6; ++i) sum = fma4(nb[i] >= 0 ? T(1) : T(0), v[i], sum);
  return sum;
}

constexpr int APPLY_EPT = 4;   // 16-byte elements per thread

// a1: H phi on every point of the dilated boxes.
template <typename T>
__global__ void __launch_bounds__(256) apply_global_kernel(const DevFrag* __restrict__ fr,
                                                           const T* __restrict__ V,
                                                           const T* __restrict__ states,
                                                           T* __restrict__ hphi, int gx, int gy,
                                                           int gz, T c0, T c1) {
  using V16 = typename Vec16<T>::type;
  constexpr int VN = Vec16<T>::n;
  __shared__ DevFrag Fs;
  if (threadIdx.x == 0) Fs = fr[blockIdx.y];
  __syncthreads();
  const DevFrag& F = Fs;
  const int qpp = F.ld / VN;
  const int total = (int)F.Pd * qpp;   // < 2^31: checked by the planner
  const V16* S = reinterpret_cast<const V16*>(states + F.off);
  V16* O = reinterpret_cast<V16*>(hphi + F.off);
  const int ex = F.dext[0], ey = F.dext[1];
#pragma unroll
  for (int u = 0; u < APPLY_EPT; ++u) {
    const int e = (blockIdx.x * APPLY_EPT + u) * (int)blockDim.x + (int)threadIdx.x;
    if (e >= total) break;
    const int p = e / qpp, q = e - p * qpp;
    const int x = p % ex, yz = p / ex, y = yz % ey, z = yz / ey;
    const int X = (F.doff[0] + x) % gx, Y = (F.doff[1] + y) % gy, Z = (F.doff[2] + z) % gz;
    const T v = V[((long long)Z * gy + Y) * gx + X];
    const V16 ctr = S[e];
    const V16 sum = neighbour_sum<T>(S, F, p, x, y, z, q, qpp);
    V16 out = fma4(c0 + v, ctr, zero4(T()));
    out = fma4(-c1, sum, out);
    O[e] = out;
  }
}

void launch_apply_global(const DevFrag* d_fr, int nfrag, int grid_x, const void* V,
                         const void* states, void* hphi, const int gn[3], double h, bool fp64,
                         cudaStream_t s) {
  const double c0 = 3.0 / (h * h), c1 = 0.5 / (h * h);
  dim3 g(grid_x, nfrag);
  if (fp64)
    apply_global_kernel<double><<<g, 256, 0, s>>>(d_fr, (const double*)V, (const double*)states,
                                                  (double*)hphi, gn[0], gn[1], gn[2], c0, c1);
  else
    apply_global_kernel<float><<<g, 256, 0, s>>>(d_fr, (const float*)V, (const float*)states,
                                                 (float*)hphi, gn[0], gn[1], gn[2], (float)c0,
                                                 (float)c1);
}

// a0, fragment mode: the fragment Hamiltonian is the principal submatrix of
// H on the box, so only interior points are written (the zero halo stays
// zero) and the stencil reads zeros beyond the box.  One fused step of the
// scaled Chebyshev three-term recurrence:
//     out = alpha_f * (H_f in - c_f in) + beta_f * prev
// with per-fragment coefficients coef[f] = (alpha, beta, c); prev may be
// null when beta is zero.
template <typename T>
__global__ void __launch_bounds__(256) apply_filter_kernel(
    const DevFrag* __restrict__ fr, const T* __restrict__ V, const T* __restrict__ in,
    const T* __restrict__ prev, T* __restrict__ out, const double* __restrict__ coef, int gx,
    int gy, int gz, T c0, T c1) {
  using V16 = typename Vec16<T>::type;
  constexpr int VN = Vec16<T>::n;
  __shared__ DevFrag Fs;
  __shared__ T cf[3];
  if (threadIdx.x == 0) Fs = fr[blockIdx.y];
  if (threadIdx.x < 3) cf[threadIdx.x] = (T)coef[3 * blockIdx.y + threadIdx.x];
  __syncthreads();
  const DevFrag& F = Fs;
  const int qpp = F.ld / VN;
  const int total = (int)F.Pd * qpp;
  const V16* S = reinterpret_cast<const V16*>(in + F.off);
  const V16* Pv = prev ? reinterpret_cast<const V16*>(prev + F.off) : nullptr;
  V16* O = reinterpret_cast<V16*>(out + F.off);
  const T alpha = cf[0], beta = cf[1], shift = cf[2];
  const int ex = F.dext[0], ey = F.dext[1];
#pragma unroll
  for (int u = 0; u < APPLY_EPT; ++u) {
    const int e = (blockIdx.x * APPLY_EPT + u) * (int)blockDim.x + (int)threadIdx.x;
    if (e >= total) break;
    const int p = e / qpp, q = e - p * qpp;
    const int x = p % ex, yz = p / ex, y = yz % ey, z = yz / ey;
    if (x < F.lo[0] || x >= F.lo[0] + F.ext[0] || y < F.lo[1] || y >= F.lo[1] + F.ext[1] ||
        z < F.lo[2] || z >= F.lo[2] + F.ext[2])
      continue;
    const int X = (F.doff[0] + x) % gx, Y = (F.doff[1] + y) % gy, Z = (F.doff[2] + z) % gz;
    const T v = V[((long long)Z * gy + Y) * gx + X];
    const V16 ctr = S[e];
    const V16 sum = neighbour_sum<T>(S, F, p, x, y, z, q, qpp);
    V16 hy = fma4(c0 + v - shift, ctr, zero4(T()));
    hy = fma4(-c1, sum, hy);
    V16 o = fma4(alpha, hy, zero4(T()));
    if (Pv != nullptr) o = fma4(beta, Pv[e], o);
    O[e] = o;
  }
}

void launch_apply_filter(const DevFrag* d_fr, int nfrag, int grid_x, const void* V, const void* in,
                         const void* prev, void* out, const double* coef, const int gn[3],
                         double h, bool fp64, cudaStream_t s) {
  const double c0 = 3.0 / (h * h), c1 = 0.5 / (h * h);
  dim3 g(grid_x, nfrag);
  if (fp64)
    apply_filter_kernel<double><<<g, 256, 0, s>>>(d_fr, (const double*)V, (const double*)in,
                                                  (const double*)prev, (double*)out, coef, gn[0],
                                                  gn[1], gn[2], c0, c1);
  else
    apply_filter_kernel<float><<<g, 256, 0, s>>>(d_fr, (const float*)V, (const float*)in,
                                                 (const float*)prev, (float*)out, coef, gn[0],
                                                 gn[1], gn[2], (float)c0, (float)c1);
}

// Grid width for the 2-D stencil launches: enough chunks for the largest
// fragment.
int apply_grid_x(const std::vector<DevFrag>& fr, bool fp64) {
  const int vn = fp64 ? 2 : 4;
  long long mx = 1;
  for (const DevFrag& f : fr) mx = std::max<long long>(mx, f.Pd * (f.ld / vn));
  return (int)((mx + 256LL * APPLY_EPT - 1) / (256LL * APPLY_EPT));
}

// ------------------------------------------------------------ conversions --

template <typename T>
__global__ void convert_V_kernel(const double* __restrict__ src, T* __restrict__ dst, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (T)src[i];
}

void launch_convert_V(const double* src, void* dst, long long n, bool fp64, cudaStream_t s) {
  int blocks = (int)((n + 255) / 256);
  if (fp64) convert_V_kernel<double><<<blocks, 256, 0, s>>>(src, (double*)dst, n);
  else convert_V_kernel<float><<<blocks, 256, 0, s>>>(src, (float*)dst, n);
}

// Column-major box states (P x n, box order) -> point-major dilated storage.
// Writes every interior point and every state column < ld (pad columns get 0).
template <typename T>
__global__ void import_kernel(DevFrag F, const double* __restrict__ src, T* __restrict__ dst) {
  const long long P = (long long)F.ext[0] * F.ext[1] * F.ext[2];
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P * F.ld) return;
  const int s = (int)(i / P);
  const long long p = i - (long long)s * P;
  const int x = (int)(p % F.ext[0]);
  const int y = (int)((p / F.ext[0]) % F.ext[1]);
  const int z = (int)(p / ((long long)F.ext[0] * F.ext[1]));
  const long long pd = ((long long)(z + F.lo[2]) * F.dext[1] + (y + F.lo[1])) * F.dext[0] + (x + F.lo[0]);
  dst[F.off + pd * F.ld + s] = (s < F.n) ? (T)src[(long long)s * P + p] : (T)0;
}

void launch_import_states(const DevFrag* /*d_fr*/, int /*a*/, const DevFrag& fa, const double* src,
                          void* states, bool fp64, cudaStream_t s) {
  const long long P = (long long)fa.ext[0] * fa.ext[1] * fa.ext[2];
  const long long tot = P * fa.ld;
  int blocks = (int)((tot + 255) / 256);
  if (fp64) import_kernel<double><<<blocks, 256, 0, s>>>(fa, src, (double*)states);
  else import_kernel<float><<<blocks, 256, 0, s>>>(fa, src, (float*)states);
}

// Point-major storage -> column-major doubles.  dilated=false: box points
// (P_a x n); dilated=true: every point of the dilated box (Pd x n).
template <typename T>
__global__ void export_kernel(DevFrag F, const T* __restrict__ srcbuf, double* __restrict__ dst,
                              int dilated) {
  const int ex = dilated ? F.dext[0] : F.ext[0];
  const int ey = dilated ? F.dext[1] : F.ext[1];
  const int ez = dilated ? F.dext[2] : F.ext[2];
  const long long P = (long long)ex * ey * ez;
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P * F.n) return;
  const int s = (int)(i / P);
  const long long p = i - (long long)s * P;
  const int x = (int)(p % ex);
  const int y = (int)((p / ex) % ey);
  const int z = (int)(p / ((long long)ex * ey));
  const int ox = dilated ? 0 : F.lo[0], oy = dilated ? 0 : F.lo[1], oz = dilated ? 0 : F.lo[2];
  const long long pd = ((long long)(z + oz) * F.dext[1] + (y + oy)) * F.dext[0] + (x + ox);
  dst[(long long)s * P + p] = (double)srcbuf[F.off + pd * F.ld + s];
}

void launch_export_states(const DevFrag& fa, const void* buf, double* dst, bool fp64,
                          bool dilated, cudaStream_t s) {
  const long long P = dilated ? fa.Pd : (long long)fa.ext[0] * fa.ext[1] * fa.ext[2];
  const long long tot = P * fa.n;
  int blocks = (int)((tot + 255) / 256);
  if (fp64) export_kernel<double><<<blocks, 256, 0, s>>>(fa, (const double*)buf, dst, dilated ? 1 : 0);
  else export_kernel<float><<<blocks, 256, 0, s>>>(fa, (const float*)buf, dst, dilated ? 1 : 0);
}

}  // namespace ofm
