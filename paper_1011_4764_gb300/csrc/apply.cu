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
#include <cstdlib>
#include <cstring>
#include <vector>

#include "ofm_internal.h"
#include "ptx_util.h"

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

// Shared-memory staged form (the default where a tile fits): a CTA owns
// rows [y0, y1) of one fragment (every x) for a chunk of z planes.  For each
// plane it needs, one thread issues at most three bulk copies (the staged
// rows y0-1 .. y1 are contiguous in storage except where a full-span
// dimension wraps) into a ring of STG_BUF plane buffers, completing on the
// buffer's mbarrier; a slot is refilled as soon as its plane is no longer
// needed, so up to three planes per CTA are in flight while it computes.  All six neighbours then
// come from shared memory; V and (filter) the previous block stream from
// global memory into registers one plane ahead of their use.  Staged rows outside a non-periodic storage box are zeroed
// once; planes outside it complete their barrier phase without a copy and
// are skipped in the sum.
constexpr int STG_BUF = 5;
constexpr int STG_THREADS = 256;
constexpr int STG_EPT = 4;   // tile elements per thread (16 bytes each)

template <typename T, bool FILTER>
__global__ void __launch_bounds__(STG_THREADS) apply_staged_kernel(
    const DevFrag* __restrict__ fr, const T* __restrict__ V, const T* __restrict__ in,
    const T* __restrict__ prev, T* __restrict__ out, const double* __restrict__ coef, int gx,
    int gy, int gz, T c0, T c1, int ty, int zc, int* flag) {
  using namespace ptx;
  using V16 = typename Vec16<T>::type;
  constexpr int VN = Vec16<T>::n;
  extern __shared__ __align__(128) unsigned char stg_smem[];
  __shared__ DevFrag Fs;
  __shared__ T cf[3];
  __shared__ __align__(8) unsigned long long mbar[STG_BUF];
  const int tid = threadIdx.x;
  if (tid == 0) Fs = fr[blockIdx.y];
  if (FILTER && tid < 3) cf[tid] = (T)coef[3 * blockIdx.y + tid];
  __syncthreads();
  const DevFrag& F = Fs;
  const int ex = F.dext[0], ey = F.dext[1], ez = F.dext[2];
  const int yb = FILTER ? F.lo[1] : 0, ye = FILTER ? F.lo[1] + F.ext[1] : ey;
  const int zb = FILTER ? F.lo[2] : 0, ze = FILTER ? F.lo[2] + F.ext[2] : ez;
  const int y0 = yb + (int)blockIdx.x * ty, y1 = min(ye, y0 + ty);
  const int z0 = zb + (int)blockIdx.z * zc, z1 = min(ze, z0 + zc);
  if (y0 >= y1 || z0 >= z1) return;   // uniform over the CTA
  const int qpp = F.ld / VN;
  const int rows = y1 - y0 + 2;                 // staged rows y0-1 .. y1
  const long long rowE = (long long)ex * F.ld;  // elements of one storage row
  const long long planeE = rows * rowE;         // elements of one staged plane
  T* buf = reinterpret_cast<T*>(stg_smem);
  if (tid == 0) {
    for (int i = 0; i < STG_BUF; ++i) mbar_init(smem_u32(&mbar[i]), 1);
    fence_mbar_init();
  }
  // Staged row r holds storage row y0-1+r (wrapped in a full-span dimension);
  // only the first and the last staged row can fall outside the storage box.
  auto srow = [&](int r) { return ((y0 - 1 + r) % ey + ey) % ey; };
  auto zero_row = [&](int r) { return !F.full[1] && (y0 - 1 + r < 0 || y0 - 1 + r >= ey); };
  // those rows read zero: written once, never the target of a copy
  for (int k = 0; k < 2; ++k) {
    const int r = k ? rows - 1 : 0;
    if (zero_row(r))
      for (int i = 0; i < STG_BUF; ++i)
        for (long long e = tid; e < rowE; e += STG_THREADS) buf[i * planeE + r * rowE + e] = T(0);
  }
  fence_async_smem();
  __syncthreads();

  const T* src = in + F.off;
  // end of the run of staged rows from r that is contiguous in storage
  auto run_end = [&](int r) {
    int r2 = r + 1;
    if (zero_row(r)) return r2;
    while (r2 < rows && !zero_row(r2) && srow(r2) == srow(r2 - 1) + 1) ++r2;
    return r2;
  };
  auto plane_ok = [&](int p) { return F.full[2] || (p >= 0 && p < ez); };
  // thread 0: fetch plane p (z0-1 <= p <= z1) into ring slot (p-z0+1) % STG_BUF
  auto issue = [&](int p) {
    const int j = p - (z0 - 1);
    const uint32_t mb = smem_u32(&mbar[j % STG_BUF]);
    if (!plane_ok(p)) {
      mbar_arrive(mb);   // the phase completes without a copy; the plane is skipped
      return;
    }
    const int zz = (p % ez + ez) % ez;
    T* dst = buf + (long long)(j % STG_BUF) * planeE;
    uint32_t bytes = 0;
    for (int r = 0; r < rows; ++r)
      if (!zero_row(r)) bytes += (uint32_t)(rowE * sizeof(T));
    mbar_arrive_expect(mb, bytes);
    for (int r = 0; r < rows;) {
      const int r2 = run_end(r);
      if (!zero_row(r))
        bulk_g2s(smem_u32(dst + r * rowE), src + ((long long)zz * ey + srow(r)) * rowE,
                 (uint32_t)((r2 - r) * rowE * sizeof(T)), mb);
      r = r2;
    }
  };
  auto wait_plane = [&](int p) {
    const int j = p - (z0 - 1);
    return mbar_wait(smem_u32(&mbar[j % STG_BUF]), (uint32_t)((j / STG_BUF) & 1), flag);
  };
  // prologue: fill the ring with planes z0-1 .. z0+STG_BUF-2; afterwards the
  // end of iteration z refills the slot of plane z-1 with plane z+STG_BUF-1
  const int plast = z1;   // last plane needed
  int pnext = min(plast, z0 + STG_BUF - 2) + 1;   // next plane to issue
  if (tid == 0)
    for (int p = z0 - 1; p < pnext; ++p) issue(p);
  int pwait = z0 - 1;     // planes < pwait have been waited for

  const int nx = FILTER ? F.ext[0] : ex, xo = FILTER ? F.lo[0] : 0;
  const int per_row = nx * qpp;
  const int nel = (y1 - y0) * per_row;   // <= STG_THREADS * STG_EPT (host's tile choice)
  const T alpha = FILTER ? cf[0] : T(1), beta = FILTER ? cf[1] : T(0), shift = FILTER ? cf[2] : T(0);
  const V16* Pv = (FILTER && prev) ? reinterpret_cast<const V16*>(prev + F.off) : nullptr;
  V16* O = reinterpret_cast<V16*>(out + F.off);
  const long long vplane = (long long)gx * gy;
  const int rowq = ex * qpp;   // 16-byte elements of one staged row
  // per element of this thread: staged index, global index within a plane, V index within a plane
  int sidx[STG_EPT], xs[STG_EPT], gidx[STG_EPT], vidx[STG_EPT];   // all < 2^31 (planner)
#pragma unroll
  for (int u = 0; u < STG_EPT; ++u) {
    const int e = tid + u * STG_THREADS;
    const int ee = e < nel ? e : 0;
    const int yl = ee / per_row;
    const int rem = ee - yl * per_row;
    const int xl = rem / qpp, q = rem - xl * qpp;
    const int x = xo + xl, y = y0 + yl;
    xs[u] = x;
    sidx[u] = (yl + 1) * rowq + x * qpp + q;
    gidx[u] = (y * ex + x) * qpp + q;
    vidx[u] = ((F.doff[1] + y) % gy) * gx + (F.doff[0] + x) % gx;
  }
  const long long gplane = (long long)ey * ex * qpp;   // 16-byte elements of one storage plane
  // the previous block and V of the plane being computed, loaded one iteration ahead
  V16 pv[STG_EPT];
  T vv[STG_EPT];
  auto prefetch = [&](int z) {
    const long long zo = (long long)z * gplane;
    const long long zv = (long long)((F.doff[2] + z) % gz) * vplane;
#pragma unroll
    for (int u = 0; u < STG_EPT; ++u) {
      if (tid + u * STG_THREADS < nel) {
        vv[u] = V[zv + vidx[u]];
        if (Pv != nullptr) pv[u] = Pv[zo + gidx[u]];
      }
    }
  };
  prefetch(z0);
  bool ok = true;
  for (int z = z0; z < z1; ++z) {
    V16 pvc[STG_EPT];
    T vc[STG_EPT];
#pragma unroll
    for (int u = 0; u < STG_EPT; ++u) {
      pvc[u] = pv[u];
      vc[u] = vv[u];
    }
    if (z + 1 < z1) prefetch(z + 1);
    // planes z-1, z, z+1 must have landed
    while (ok && pwait <= z + 1) {
      ok = wait_plane(pwait);
      if (ok) ++pwait;
    }
    if (!__syncthreads_and(ok)) {
      ok = false;
      break;
    }
    const int jb = z - 1 - (z0 - 1), jc = jb + 1, ja = jb + 2;
    const V16* Bb = reinterpret_cast<const V16*>(buf + (long long)(jb % STG_BUF) * planeE);
    const V16* Bc = reinterpret_cast<const V16*>(buf + (long long)(jc % STG_BUF) * planeE);
    const V16* Ba = reinterpret_cast<const V16*>(buf + (long long)(ja % STG_BUF) * planeE);
    const bool has_b = plane_ok(z - 1), has_a = plane_ok(z + 1);
    const long long zo = (long long)z * gplane;
#pragma unroll
    for (int u = 0; u < STG_EPT; ++u) {
      if (tid + u * STG_THREADS >= nel) continue;
      const int sc = sidx[u], x = xs[u];
      V16 sum = add4(Bc[sc + rowq], Bc[sc - rowq]);
      const int xp = nb_index(x, x, ex, F.full[0], +1, 1), xm = nb_index(x, x, ex, F.full[0], -1, 1);
      if (xp >= 0) sum = add4(sum, Bc[sc + (xp - x) * qpp]);
      if (xm >= 0) sum = add4(sum, Bc[sc + (xm - x) * qpp]);
      if (has_b) sum = add4(sum, Bb[sc]);
      if (has_a) sum = add4(sum, Ba[sc]);
      V16 hy = fma4(c0 + vc[u] - shift, Bc[sc], zero4(T()));
      hy = fma4(-c1, sum, hy);
      if constexpr (FILTER) {
        V16 o = fma4(alpha, hy, zero4(T()));
        if (Pv != nullptr) o = fma4(beta, pvc[u], o);
        O[zo + gidx[u]] = o;
      } else {
        O[zo + gidx[u]] = hy;
      }
    }
    __syncthreads();   // slot of plane z-1 is free
    if (tid == 0 && pnext <= plast) issue(pnext);
    ++pnext;
  }
  if (!ok) {
    // drain: every issued copy must land before the CTA's shared memory is released
    for (; pwait < min(pnext, plast + 1); ++pwait) wait_plane(pwait);
    __syncthreads();
  }
}

// Launch shape of the stencils.  Staged form: x = row tiles of ty rows, y =
// fragments, z = chunks of zc planes; ty minimises the staged rows (tile plus
// two halo rows) per output row within the shared-memory budget (two CTAs per
// SM, else one) and at most STG_EPT elements per thread, and the chunk count
// fills about two resident waves of the GB300 (152 SMs).  Register form (fallback when even one row does not fit):
// x covers the (x, y, column group) elements of the largest plane.
ApplyGrid apply_grid(const std::vector<DevFrag>& fr, bool fp64, bool filter, int form) {
  const int vn = fp64 ? 2 : 4;
  const int es = fp64 ? 8 : 4;
  const int sms = 152;
  long long mx = 1, threads = 0, rowB = 0, rowQ = 0;
  int zmax = 1, ymax = 1;
  for (const DevFrag& f : fr) {
    const long long xy = (long long)f.dext[0] * f.dext[1] * (f.ld / vn);
    mx = std::max(mx, xy);
    threads += filter ? (long long)f.ext[0] * f.ext[1] * (f.ld / vn) : xy;
    zmax = std::max(zmax, filter ? f.ext[2] : f.dext[2]);
    ymax = std::max(ymax, filter ? f.ext[1] : f.dext[1]);
    rowB = std::max(rowB, (long long)f.dext[0] * f.ld * es);
    rowQ = std::max(rowQ, (long long)(filter ? f.ext[0] : f.dext[0]) * (f.ld / vn));
  }
  ApplyGrid g;
  // staged form where the caller (form 2), or with form 0 OFM_STENCIL=staged,
  // asks for it
  const char* env = std::getenv("OFM_STENCIL");
  const bool try_staged =
      form == 2 || (form == 0 && env != nullptr && std::strcmp(env, "staged") == 0);
  const long long budgets[2] = {110 * 1024, 200 * 1024};
  for (int bi = 0; bi < 2 && try_staged && !g.staged; ++bi) {
    int best = 0;
    long long best_cost = 0;
    for (int ty = 1; ty <= ymax; ++ty) {
      if ((long long)STG_BUF * (ty + 2) * rowB > budgets[bi]) break;
      if ((long long)ty * rowQ > (long long)STG_THREADS * STG_EPT) break;
      const long long cost = (long long)((ymax + ty - 1) / ty) * (ty + 2);
      if (best == 0 || cost <= best_cost) {
        best = ty;
        best_cost = cost;
      }
    }
    if (best > 0) {
      g.staged = true;
      g.ty = best;
      g.smem = (int)((long long)STG_BUF * (best + 2) * rowB);
      const int per_sm = bi == 0 ? 2 : 1;
      long long per_chunk = 0;
      for (const DevFrag& f : fr) per_chunk += ((filter ? f.ext[1] : f.dext[1]) + best - 1) / best;
      const long long nch = std::max(1LL, std::min<long long>(zmax, (2LL * sms * per_sm + per_chunk - 1) / per_chunk));
      g.zc = (int)((zmax + nch - 1) / nch);
      g.z = (zmax + g.zc - 1) / g.zc;
      g.x = (ymax + best - 1) / best;
    }
  }
  if (g.staged) {
    // once per plan (the call is not free: kept out of the launch path)
    const void* k = fp64 ? (filter ? (const void*)apply_staged_kernel<double, true>
                                   : (const void*)apply_staged_kernel<double, false>)
                         : (filter ? (const void*)apply_staged_kernel<float, true>
                                   : (const void*)apply_staged_kernel<float, false>);
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, g.smem) == cudaSuccess)
      return g;
    cudaGetLastError();   // not available: the register form below
    g = ApplyGrid();
  }
  // register form
  g.x = (int)((mx + 255) / 256);
  const long long want = 2LL * sms * 2048;
  const long long nch = std::max(1LL, std::min<long long>(zmax, (want + threads - 1) / std::max(1LL, threads)));
  g.zc = (int)((zmax + nch - 1) / nch);
  g.z = (zmax + g.zc - 1) / g.zc;
  return g;
}

template <typename T, bool FILTER>
static void zmarch(const ApplyGrid& ag, int nfrag, const DevFrag* d_fr, const void* V,
                   const void* in, const void* prev, void* out, const double* coef,
                   const int gn[3], double h, int* flag, cudaStream_t s) {
  const double c0 = 3.0 / (h * h), c1 = 0.5 / (h * h);
  dim3 g(ag.x, nfrag, ag.z);
  if (ag.staged) {
    apply_staged_kernel<T, FILTER><<<g, STG_THREADS, ag.smem, s>>>(
        d_fr, (const T*)V, (const T*)in, (const T*)prev, (T*)out, coef, gn[0], gn[1], gn[2],
        (T)c0, (T)c1, ag.ty, ag.zc, flag);
  } else {
    apply_zmarch_kernel<T, FILTER><<<g, 256, 0, s>>>(d_fr, (const T*)V, (const T*)in,
                                                     (const T*)prev, (T*)out, coef, gn[0], gn[1],
                                                     gn[2], (T)c0, (T)c1, ag.zc);
  }
}

void launch_apply_global(const DevFrag* d_fr, int nfrag, const ApplyGrid& g, const void* V,
                         const void* states, void* hphi, const int gn[3], double h, bool fp64,
                         int* flag, cudaStream_t s) {
  if (fp64) zmarch<double, false>(g, nfrag, d_fr, V, states, nullptr, hphi, nullptr, gn, h, flag, s);
  else zmarch<float, false>(g, nfrag, d_fr, V, states, nullptr, hphi, nullptr, gn, h, flag, s);
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
                         const int gn[3], double h, bool fp64, int* flag, cudaStream_t s) {
  if (fp64) zmarch<double, true>(g, nfrag, d_fr, V, in, prev, out, coef, gn, h, flag, s);
  else zmarch<float, true>(g, nfrag, d_fr, V, in, prev, out, coef, gn, h, flag, s);
}

// ------------------------------------------------ whole filter on chip ----
//
// The whole degree-d Chebyshev filter of one fragment and ONE state column
// in one CTA (FP32 storage, interior box EX x EY x EZ fixed at compile
// time): the column's box is loaded once, every step runs between registers
// and shared memory, and the filtered column Y = p(H_f) X and H_f Y leave
// once.  The stencil acts on each state column independently, so the CTAs
// of a fragment's columns share nothing.  Against one launch per degree
// (three blocks through HBM per step) the HBM traffic of a filter drops from
// ~3 d blocks to ~3 blocks; a step is bound by shared memory (four in-plane
// neighbour loads and one store per point) and instruction issue.
//   - two threads own each interior column (x, y), the lower and the upper
//     half of its z range, and keep their half of the current iterate in
//     registers; z neighbours come from registers (the two middle and the
//     wrap-around ones from shared memory), in-plane neighbours from the
//     shared copy of the current iterate;
//   - the shared copy is the interior box ([z][y][x], unpadded: the two rows
//     of 16 points a warp covers are 32 consecutive words, conflict-free) in
//     two buffers: a step reads one and writes the next iterate over the
//     previous one in the other (each point is read and rewritten by its own
//     thread), one barrier per step.  c0 + V of every point sits in a third
//     area;
//   - a missing in-plane neighbour (non-periodic edge) reads the point itself
//     with weight 0 and a periodic one reads the wrapped point, exactly as in
//     apply_zmarch_kernel's filter mode, whose arithmetic and order are kept:
//     both forms give the same values.
template <int EX, int EY, int EZ>
struct CfBox {
  static constexpr int NXY = EX * EY;                 // points per plane (unpadded)
  static constexpr int ZH = EZ / 2, NT = 2 * NXY;     // two threads per z-column
  // two copies of the iterate, then c0 + V of every interior point
  static constexpr size_t smem = 3 * (size_t)EZ * NXY * sizeof(float);
};

// One step for the ZH planes of a thread.  src holds the current iterate
// (also in cur), dst the previous one; the next iterate replaces the
// previous one in dst point by point (only this thread reads those points
// of dst during the step) and replaces cur.  nb[i], w[i]: in-plane
// neighbour offsets and 0/1 weights (x+1, x-1, y+1, y-1; a missing
// neighbour reads the point itself with weight 0, as in the HBM form); ob /
// oa: offsets of the planes just below / above the thread's range (-1:
// zero there).  With write = false (the final H Y) the result goes to cur
// only and dst is untouched.
template <int EX, int EY, int EZ>
__device__ __forceinline__ void cf_step(const float* __restrict__ src, float* __restrict__ dst,
                                        int own, int ob, int oa, const int (&nb)[4],
                                        const float (&w)[4], float (&cur)[CfBox<EX, EY, EZ>::ZH],
                                        const float* __restrict__ vc, float c1, float al, float be,
                                        float sh, bool has_prev, bool write) {
  using B = CfBox<EX, EY, EZ>;
  float below = ob >= 0 ? src[ob] : 0.f;
  const float edge_a = oa >= 0 ? src[oa] : 0.f;
  const float* p0 = src + nb[0];
  const float* p1 = src + nb[1];
  const float* p2 = src + nb[2];
  const float* p3 = src + nb[3];
  float* d = dst + own;
#pragma unroll
  for (int z = 0; z < B::ZH; ++z) {
    const float above = (z + 1 < B::ZH) ? cur[z + 1] : edge_a;
    float sum = below + above;
    sum = fmaf(w[0], p0[z * B::NXY], sum);
    sum = fmaf(w[1], p1[z * B::NXY], sum);
    sum = fmaf(w[2], p2[z * B::NXY], sum);
    sum = fmaf(w[3], p3[z * B::NXY], sum);
    float h = fmaf(vc[z * B::NXY] - sh, cur[z], 0.f);
    h = fmaf(-c1, sum, h);
    float o = fmaf(al, h, 0.f);
    if (has_prev) o = fmaf(be, d[z * B::NXY], o);
    below = cur[z];   // the old value is the next point's lower neighbour
    cur[z] = o;
    if (write) d[z * B::NXY] = o;
  }
}

template <int EX, int EY, int EZ>
__global__ void __launch_bounds__(2 * EX * EY, 1) cheb_filter_kernel(
    const DevFrag* __restrict__ fr, const float* __restrict__ V, const float* __restrict__ X,
    float* __restrict__ Y, float* __restrict__ HY, const double* __restrict__ coef, int nsteps,
    int nfrag, int gx, int gy, int gz, float c0, float c1) {
  using B = CfBox<EX, EY, EZ>;
  constexpr int ZH = B::ZH;
  extern __shared__ float cf_box[];
  const int f = blockIdx.y, j = blockIdx.x;
  const DevFrag F = fr[f];
  if (j >= F.n) return;   // uniform over the CTA
  const int t = threadIdx.x;
  const int c = t % B::NXY, half = t / B::NXY;
  const int x = c % EX, y = c / EX, z0 = half * ZH;
  const bool fz = F.full[2] != 0;
  const int own = z0 * B::NXY + c;
  const int ob = z0 > 0 ? own - B::NXY : (fz ? (EZ - 1) * B::NXY + c : -1);
  const int oa = z0 + ZH < EZ ? own + ZH * B::NXY : (fz ? c : -1);
  // in-plane neighbours within the interior plane (full dimensions wrap)
  int nb[4];
  float w[4];
  {
    const int xp = x + 1 < EX ? c + 1 : (F.full[0] ? c + 1 - EX : -1);
    const int xm = x > 0 ? c - 1 : (F.full[0] ? c - 1 + EX : -1);
    const int yp = y + 1 < EY ? c + EX : (F.full[1] ? c + EX - B::NXY : -1);
    const int ym = y > 0 ? c - EX : (F.full[1] ? c - EX + B::NXY : -1);
    const int q[4] = {xp, xm, yp, ym};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      w[i] = q[i] >= 0 ? 1.f : 0.f;
      nb[i] = (q[i] >= 0 ? q[i] : c) + z0 * B::NXY;
    }
  }
  const long long pstride = (long long)F.dext[0] * F.dext[1];   // storage points per plane
  const long long p0 =
      ((long long)(F.lo[2] + z0) * F.dext[1] + (F.lo[1] + y)) * F.dext[0] + F.lo[0] + x;
  float* vcs = cf_box + 2 * EZ * B::NXY + own;   // c0 + V, plane stride NXY
  {
    const float* Vrow = V + (long long)((F.doff[1] + F.lo[1] + y) % gy) * gx + (F.doff[0] + F.lo[0] + x) % gx;
    const long long vstride = (long long)gx * gy;
#pragma unroll
    for (int z = 0; z < ZH; ++z)
      vcs[z * B::NXY] = c0 + Vrow[(long long)((F.doff[2] + F.lo[2] + z0 + z) % gz) * vstride];
  }
  float cur[ZH];
#pragma unroll
  for (int z = 0; z < ZH; ++z) cur[z] = X[F.off + (p0 + z * pstride) * F.ld + j];
#pragma unroll
  for (int z = 0; z < ZH; ++z) cf_box[own + z * B::NXY] = cur[z];
  __syncthreads();
  float* b0 = cf_box;
  float* b1 = cf_box + EZ * B::NXY;
  const double* cf = coef + 3 * (size_t)f;
  float* src = b0;
  float* dst = b1;
  for (int k = 0; k < nsteps; ++k) {
    const double* ca = cf + 3 * (size_t)k * nfrag;
    cf_step<EX, EY, EZ>(src, dst, own, ob, oa, nb, w, cur, vcs, c1, (float)ca[0], (float)ca[1],
                        (float)ca[2], k > 0, true);
    __syncthreads();
    float* tmp = src;
    src = dst;
    dst = tmp;
  }
  // cur holds the filtered column Y (also in src); H_f Y (alpha 1, beta 0,
  // shift 0) goes to the registers of a second pass, Y straight out first
  if (Y) {
#pragma unroll
    for (int z = 0; z < ZH; ++z) Y[F.off + (p0 + z * pstride) * F.ld + j] = cur[z];
  }
  cf_step<EX, EY, EZ>(src, dst, own, ob, oa, nb, w, cur, vcs, c1, 1.f, 0.f, 0.f, false, false);
#pragma unroll
  for (int z = 0; z < ZH; ++z) HY[F.off + (p0 + z * pstride) * F.ld + j] = cur[z];
}

// Box shapes with an on-chip filter: every fragment must have this interior
// shape, and a full dimension must coincide with the storage box.
static bool cf_shape(const std::vector<DevFrag>& frags, int ex, int ey, int ez) {
  for (const DevFrag& F : frags) {
    if (F.ext[0] != ex || F.ext[1] != ey || F.ext[2] != ez) return false;
    for (int d = 0; d < 3; ++d)
      if (F.full[d] && (F.ext[d] != F.dext[d] || F.lo[d] != 0)) return false;
  }
  return !frags.empty();
}

// Dynamic shared memory of the on-chip filter for these fragments, or 0 when
// it does not apply (FP64 storage, or a box shape without a compiled form).
size_t cheb_filter_smem(const std::vector<DevFrag>& frags, bool fp64) {
  if (fp64) return 0;
  if (cf_shape(frags, 16, 32, 32)) return CfBox<16, 32, 32>::smem;
  return 0;
}

// One launch per filter: CTA (state j, fragment f) for every j < m_f.  Y may
// be null (only H X wanted: nsteps = 0).
void launch_cheb_filter(const DevFrag* d_fr, int nfrag, int mmax, size_t smem, const void* V,
                        const void* X, void* Y, void* HY, const double* coef, int nsteps,
                        const int gn[3], double h, cudaStream_t s) {
  const double c0 = 3.0 / (h * h), c1 = 0.5 / (h * h);
  if (smem == CfBox<16, 32, 32>::smem) {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(cheb_filter_kernel<16, 32, 32>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      attr = true;
    }
    cheb_filter_kernel<16, 32, 32><<<dim3(mmax, nfrag), CfBox<16, 32, 32>::NT, smem, s>>>(
        d_fr, (const float*)V, (const float*)X, (float*)Y, (float*)HY, coef, nsteps, nfrag,
        gn[0], gn[1], gn[2], (float)c0, (float)c1);
  }
}

// ------------------------------------------------------------ conversions --

// Columns [first, first + Fn.n) of one fragment's stored states (every
// storage point, halo included) into the layout Fn; pad columns zero.
template <typename T>
__global__ void select_states_kernel(DevFrag Fo, DevFrag Fn, int first, const T* __restrict__ src,
                                     T* __restrict__ dst) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Fn.Pd * Fn.ld) return;
  const long long p = i / Fn.ld;
  const int j = (int)(i - p * Fn.ld);
  dst[Fn.off + i] = (j < Fn.n) ? src[Fo.off + p * Fo.ld + first + j] : T(0);
}

void launch_select_states(const DevFrag& Fo, const DevFrag& Fn, int first, const void* src,
                          void* dst, bool fp64, cudaStream_t s) {
  const long long n = Fn.Pd * Fn.ld;
  const int blocks = (int)((n + 255) / 256);
  if (fp64)
    select_states_kernel<double><<<blocks, 256, 0, s>>>(Fo, Fn, first, (const double*)src, (double*)dst);
  else
    select_states_kernel<float><<<blocks, 256, 0, s>>>(Fo, Fn, first, (const float*)src, (float*)dst);
}

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
