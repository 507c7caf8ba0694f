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
// bound by HBM bandwidth.  The launch grid is 3-D: blockIdx.y is the
// fragment, blockIdx.x a chunk of its (x, y, 16-byte column group) elements
// and blockIdx.z a chunk of z planes that each thread marches through.
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

// z-marching form of both stencils: a thread owns one (x, y, 16-byte column)
// of a fragment and walks along z, keeping the planes z-1, z, z+1 of its
// column in registers; only the plane ahead, the four in-plane neighbours
// (cache hits: the neighbouring threads load them as their own centre),
// V and (filter) the previous block are loaded per output.
// FILTER: fragment mode (interior points only, Chebyshev step);
// otherwise the a1 apply on every point of the dilated box.
template <typename T, bool FILTER>
__global__ void __launch_bounds__(256) apply_zmarch_kernel(
    const DevFrag* __restrict__ fr, const T* __restrict__ V, const T* __restrict__ in,
    const T* __restrict__ prev, T* __restrict__ out, const double* __restrict__ coef, int gx,
    int gy, int gz, T c0, T c1, int zc) {
  using V16 = typename Vec16<T>::type;
  constexpr int VN = Vec16<T>::n;
  __shared__ DevFrag Fs;
  __shared__ T cf[3];
  if (threadIdx.x == 0) Fs = fr[blockIdx.y];
  if (FILTER && threadIdx.x < 3) cf[threadIdx.x] = (T)coef[3 * blockIdx.y + threadIdx.x];
  __syncthreads();
  const DevFrag& F = Fs;
  const int qpp = F.ld / VN;
  const int ex = F.dext[0], ey = F.dext[1], ez = F.dext[2];
  const int e = (int)(blockIdx.x * blockDim.x + threadIdx.x);
  if (e >= ex * ey * qpp) return;
  const int pxy = e / qpp, q = e - pxy * qpp;
  const int x = pxy % ex, y = pxy / ex;
  if (FILTER && (x < F.lo[0] || x >= F.lo[0] + F.ext[0] || y < F.lo[1] || y >= F.lo[1] + F.ext[1]))
    return;
  const int plane = ex * ey;
  // in-plane neighbours (branch-free: outside the storage box -> self, weight 0)
  int nb[4];
  nb[0] = nb_index(pxy, x, ex, F.full[0], +1, 1);
  nb[1] = nb_index(pxy, x, ex, F.full[0], -1, 1);
  nb[2] = nb_index(pxy, y, ey, F.full[1], +1, ex);
  nb[3] = nb_index(pxy, y, ey, F.full[1], -1, ex);
  T w[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    w[i] = nb[i] >= 0 ? T(1) : T(0);
    if (nb[i] < 0) nb[i] = pxy;
  }
  const V16* S = reinterpret_cast<const V16*>(in + F.off);
  const V16* Pv = (FILTER && prev) ? reinterpret_cast<const V16*>(prev + F.off) : nullptr;
  V16* O = reinterpret_cast<V16*>(out + F.off);
  const T alpha = FILTER ? cf[0] : T(1), beta = FILTER ? cf[1] : T(0), shift = FILTER ? cf[2] : T(0);
  // this CTA's chunk of planes (blockIdx.z): zc planes of the marched range
  const int zb = FILTER ? F.lo[2] : 0, ze = FILTER ? F.lo[2] + F.ext[2] : ez;
  const int z0 = zb + (int)blockIdx.z * zc;
  const int z1 = min(ze, z0 + zc);
  if (z0 >= z1) return;
  const int X = (F.doff[0] + x) % gx, Y = (F.doff[1] + y) % gy;
  const T* Vrow = V + (long long)Y * gx + X;
  const long long vstride = (long long)gx * gy;
  // planes below and at the start
  auto plane_val = [&](int z) -> V16 {
    int zz = z;
    if (zz < 0 || zz >= ez) {
      if (!F.full[2]) return zero4(T());
      zz = (zz + ez) % ez;
    }
    return S[(zz * plane + pxy) * qpp + q];
  };
  V16 below = plane_val(z0 - 1);
  V16 ctr = plane_val(z0);
  for (int z = z0; z < z1; ++z) {
    const V16 above = plane_val(z + 1);
    const int base = z * plane;
    V16 sum = add4(below, above);
#pragma unroll
    for (int i = 0; i < 4; ++i) sum = fma4(w[i], S[(base + nb[i]) * qpp + q], sum);
    const T v = Vrow[(long long)((F.doff[2] + z) % gz) * vstride];
    V16 hy = fma4(c0 + v - shift, ctr, zero4(T()));
    hy = fma4(-c1, sum, hy);
    V16 o = fma4(alpha, hy, zero4(T()));
    const int idx = (base + pxy) * qpp + q;
    if (Pv != nullptr) o = fma4(beta, Pv[idx], o);
    O[idx] = o;
    below = ctr;
    ctr = above;
  }
}

// Launch shape of the stencils: x covers the (x, y, column group) elements of
// the largest fragment plane, y the fragments, z chunks of zc planes.  The
// chunk count is chosen so the grid holds about two resident waves of the
// GB300 (152 SMs x 2048 threads); each chunk re-reads only its two boundary
// planes.
ApplyGrid apply_grid(const std::vector<DevFrag>& fr, bool fp64, bool filter) {
  const int vn = fp64 ? 2 : 4;
  long long mx = 1, threads = 0;
  int zmax = 1;
  for (const DevFrag& f : fr) {
    const long long xy = (long long)f.dext[0] * f.dext[1] * (f.ld / vn);
    mx = std::max(mx, xy);
    threads += filter ? (long long)f.ext[0] * f.ext[1] * (f.ld / vn) : xy;
    zmax = std::max(zmax, filter ? f.ext[2] : f.dext[2]);
  }
  ApplyGrid g;
  g.x = (int)((mx + 255) / 256);
  const long long want = 2LL * 152 * 2048;
  const long long nch = std::max(1LL, std::min<long long>(zmax, (want + threads - 1) / std::max(1LL, threads)));
  g.zc = (int)((zmax + nch - 1) / nch);
  g.z = (zmax + g.zc - 1) / g.zc;
  return g;
}

template <typename T, bool FILTER>
static void zmarch(const ApplyGrid& ag, int nfrag, const DevFrag* d_fr, const void* V,
                   const void* in, const void* prev, void* out, const double* coef,
                   const int gn[3], double h, cudaStream_t s) {
  const double c0 = 3.0 / (h * h), c1 = 0.5 / (h * h);
  dim3 g(ag.x, nfrag, ag.z);
  apply_zmarch_kernel<T, FILTER><<<g, 256, 0, s>>>(d_fr, (const T*)V, (const T*)in,
                                                   (const T*)prev, (T*)out, coef, gn[0], gn[1],
                                                   gn[2], (T)c0, (T)c1, ag.zc);
}

void launch_apply_global(const DevFrag* d_fr, int nfrag, const ApplyGrid& g, const void* V,
                         const void* states, void* hphi, const int gn[3], double h, bool fp64,
                         cudaStream_t s) {
  if (fp64) zmarch<double, false>(g, nfrag, d_fr, V, states, nullptr, hphi, nullptr, gn, h, s);
  else zmarch<float, false>(g, nfrag, d_fr, V, states, nullptr, hphi, nullptr, gn, h, s);
}

// a0, fragment mode: the fragment Hamiltonian is the principal submatrix of
// H on the box, so only interior points are written (the zero halo stays
// zero) and the stencil reads zeros beyond the box.  One fused step of the
// scaled Chebyshev three-term recurrence:
//     out = alpha_f * (H_f in - c_f in) + beta_f * prev
// with per-fragment coefficients coef[f] = (alpha, beta, c); prev may be
// null when beta is zero.
void launch_apply_filter(const DevFrag* d_fr, int nfrag, const ApplyGrid& g, const void* V,
                         const void* in, const void* prev, void* out, const double* coef,
                         const int gn[3], double h, bool fp64, cudaStream_t s) {
  if (fp64) zmarch<double, true>(g, nfrag, d_fr, V, in, prev, out, coef, gn, h, s);
  else zmarch<float, true>(g, nfrag, d_fr, V, in, prev, out, coef, gn, h, s);
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
