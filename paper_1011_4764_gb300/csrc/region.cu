// Region-stacked pair contraction on the tcgen05 tensor cores (Sec. II, the
// H_ab / S_ab dot products over the shared grid points).
//
// The grid is cut into coverage regions: per dimension, the boundaries of all
// dilated boxes split the periodic axis into segments, and a region is a
// product of three segments.  Every fragment whose dilated box meets a region
// is in its cover set C(R).  Over one region, the blocks of every pair in
// C(R) come from ONE stacked product
//     D = Phi_C[R]^T [Phi_C[R] | HPhi_C[R]],   Phi_C = [Phi_f0 | Phi_f1 | ...],
// with M = sum of the cover's (padded) state counts, so the 128-row MMA
// tiles are full whatever n_a is, and each fragment's states are read once
// per region instead of once per pair.  The blocks a <= b of D are the
// region's contribution to (H_ab, S_ab); the contributions of the regions
// are summed in region order (deterministic).  Points of a region outside a
// fragment's box carry zeros in that fragment's operands, so each pair's
// sum runs exactly over B_a ∩ B_b+ (Phi_a vanishes outside B_a, H phi_b
// outside B_b+).
//
// Three kernels:
//   pack_kernel      a1: H phi with the whole-system H (7-point stencil + V)
//                    and the operand planes: for each (fragment, region) the
//                    states and H phi of the region's points, already in the
//                    K-major canonical MMA layout (core matrices of 8 rows x
//                    16 bytes) as BF16 hi/lo, BF16 or TF32 -- the contraction
//                    then copies tiles with no conversion;
//   region_kernel    a3/a4: persistent, warp-specialised: a producer warp
//                    issues one bulk copy per (fragment piece, plane, K
//                    chunk) into a ring of stages, one thread issues the
//                    MMAs into two alternating TMEM accumulators, four warps
//                    drain an accumulator into the FP32 partial slot of each
//                    (pair, region part) it covers;
//   rfinalize_kernel a5: FP64 sum of each pair's slots in region order,
//                    symmetrised diagonal blocks.
// The plain forms on the CUDA cores (FP32 and FP64 arithmetic) take the same
// plan: the pack writes FP32 or FP64 operand planes in the same layout (all
// byte offsets doubled for FP64), region_simt_kernel forms the same tiles
// with register-tiled FMAs, and the FP64 form keeps FP64 partial slots.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <unordered_map>
#include <vector>

#include "ofm_internal.h"
#include "ptx_util.h"

using namespace ofm;
using namespace ofm::ptx;

namespace {

// ----------------------------------------------------------- tables -------

// Pack work: one (fragment, region) block of the plane arena.
// The points of a region are ordered plane by plane in z, x fastest within a
// plane, each plane padded to a multiple of 8 points (p8): point (ix, iy, iz)
// has K index iz * p8 + iy * L[0] + ix, so a 16-byte operand unit (8 BF16 or
// 4 TF32 points) never straddles two planes.  K is padded to 64-point tiles.
struct RUnit {
  int frag;
  int s0[3];          // region start (global grid coordinates)
  int L[3];           // region extent
  int p8;             // plane stride in K: L[0] * L[1] rounded up to 8
  int ntiles;         // 64-point tiles: (L[2] * p8) / 64 rounded up
  long long tile0;    // first global tile of this unit
  long long base;     // byte offset of the block in the plane arena
};

// One contraction work item: up to 256 rows (two 128-row halves sharing the
// B operand) x an N tile of one region part.
struct RItem {
  int tile0, ntiles;  // K range of the part in 64-point tiles of the region
  int n_cols;         // MMA N (multiple of 16, <= 256)
  int nh;             // row halves (1 or 2)
  int cskip;          // half 1 skips columns [0, cskip): fragments before its
                      // first one (lower-triangle blocks), a multiple of 16
  int pa0, npa;       // A pieces
  int pb0, npb;       // B pieces
  int rs0, nrs;       // row segments of the epilogue
  int cs0, ncs;       // column segments of the epilogue
  int ncf;            // column fragments (slot-table width)
  long long st0;      // slot table (nrs x ncf)
};

// A run of 8-row groups of one fragment's operand plane for one K chunk.
struct RPiece {
  long long base;     // byte offset of chunk 0 of the hi plane, first group
  long long lo;       // byte offset hi plane -> lo plane (BF16 hi+lo)
  int cb;             // bytes per K chunk of this fragment (rows_pad * 64)
  int bytes;          // groups * 512
  int dst;            // byte offset in the operand tile
  int pad;
};

struct RRowSeg { int r0, nr, i0, na; };              // tile rows [r0, r0+nr) = states i0.. (n_a = na)
struct RColSeg { int c0, nc, j0, nb, part, cf; };    // tile cols [c0, c0+nc) = states j0.. of part
                                                     // (0 phi, 1 H phi) of column fragment cf
// Finalize: one pair's slots.
struct RPair {
  int a, b, na, nb;
  int nslot;
  long long slot0;    // first slot (floats); slot q at slot0 + q * na * 2 nb
  long long blk_off;  // [H_ab | S_ab] in the block arena
};

// operand kinds of the region path (the tensor-core ones numbered as in the
// pair path); RK_F32 and RK_F64 are the plain forms on the CUDA cores
enum { RK_TF32 = 0, RK_BF16 = 1, RK_BF16X3 = 2, RK_F32 = 3, RK_F64 = 4 };

constexpr int RS_THREADS = 192;    // warp 0 copies, 1 MMA, 2-5 epilogue
constexpr int RS_NSTAGE = 3;
constexpr int RS_NQ = 4;           // work-item ring between the roles
constexpr int RS_ACOLS = 256;      // TMEM columns per accumulator (one per row half)
constexpr int RS_ATILE = 256 * 64; // bytes of an A chunk tile (256 rows x 64 B)
constexpr int RS_BTILE = 256 * 64; // bytes of a B chunk tile (256 rows x 64 B)
constexpr int RS_STAGE = 64 * 1024;
constexpr int RS_SMEM = RS_NSTAGE * RS_STAGE;
constexpr int RS_MAXROWS = 128;    // padded states per fragment this path takes
constexpr int PK_THREADS = 256;
constexpr int PK_TPC = 4;          // tiles per pack CTA
constexpr int PK_SEGMAX = 18;      // x and y segments longer than this are split

template <int K> struct KindT;
template <> struct KindT<RK_TF32> {
  static constexpr int esz = 4, KC = 16, CPT = 4, NPL = 1, SC = 2, FMT = 2;
};
template <> struct KindT<RK_BF16> {
  static constexpr int esz = 2, KC = 32, CPT = 2, NPL = 1, SC = 2, FMT = 1;
};
template <> struct KindT<RK_BF16X3> {
  static constexpr int esz = 2, KC = 32, CPT = 2, NPL = 2, SC = 1, FMT = 1;
};
// plain forms: a chunk is 16 points (64 bytes a row in FP32, 128 in FP64)
template <> struct KindT<RK_F32> {
  static constexpr int esz = 4, KC = 16, CPT = 4;
};
template <> struct KindT<RK_F64> {
  static constexpr int esz = 8, KC = 16, CPT = 4;
};
// byte scale of a kind's plane layout against the plan's offsets (FP64: 2)
__host__ __device__ constexpr int kind_scale(int k) { return k == RK_F64 ? 2 : 1; }

__device__ __forceinline__ uint64_t rdesc(uint32_t saddr) {
  // K-major, no swizzle: K-adjacent core matrices 128 bytes apart (LBO),
  // 8-row groups 512 bytes apart (SBO), descriptor version 1
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((128u >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((512u >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

__host__ __device__ constexpr uint32_t ridesc(uint32_t fmt, uint32_t M, uint32_t N) {
  // FP32 accumulator, A/B format, both K-major, N >> 3, M >> 4
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

template <int FMT>
__device__ __forceinline__ void rmma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                     uint32_t accum) {
  if constexpr (FMT == 2) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accum)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accum)
        : "memory");
  }
}

__device__ __forceinline__ void rcommit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ void rtmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t rtf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// ------------------------------------------------------------- a1: pack ---

// One CTA per run of up to PK_TPC consecutive 64-point tiles of one
// (fragment, region) unit (cta[i] = {unit, first tile, tiles}); per tile,
// two phases.
//   1. Threads take (point k, 4-state group q) items with q fastest, so a
//      warp's loads of phi and of each neighbour are contiguous runs of the
//      point-major FP32 storage (zero outside the dilated storage box; a
//      full-span dimension wraps), two items (14 loads) at a time, and form
//          H phi = (3/h^2 + V) phi - (1/(2h^2)) sum_neighbours phi;
//      phi and H phi go to shared memory as [k][state] rows.
//   2. Each thread writes 16-byte units of one (array, K chunk) of the
//      operand planes in the canonical layout (memory order, coalesced):
//      8 (BF16), 4 (TF32, FP32) or 2 (FP64) consecutive points of one
//      state, read down a column of the shared rows, rounded to TF32, BF16,
//      or split into BF16 hi and lo.
// Points of the region outside the fragment's dilated box, the plane and
// tile padding and the state rows beyond n (up to the multiple of 8) are
// zeros.
// Three CTAs per SM (80 registers): measured 20.1 ms against 24.0 ms at two
// CTAs (97 registers) and 31.7 ms at four (64 registers, spills), large lattice.
// CHECK (check mode): every gathered point index is tested against the
// fragment's dilated box and the states arena, every 16-byte store against
// the plane arena; a failing access is skipped and *bounds set.
template <int KIND, bool CHECK = false>
__global__ void __launch_bounds__(PK_THREADS, 3) pack_kernel(
    const RUnit* __restrict__ units, const int4* __restrict__ cta, const DevFrag* __restrict__ fr,
    const float* __restrict__ V, const float* __restrict__ states, unsigned char* __restrict__ planes,
    int gx, int gy, int gz, double c0d, double c1d, long long n_states, long long n_plane_bytes,
    int* bounds) {
  using KT = KindT<KIND>;
  constexpr int ESZ = KT::esz;
  constexpr int KPU = 16 / ESZ;            // points per 16-byte unit
  constexpr int NCORE = KT::KC / KPU;      // 16-byte core columns per chunk
  constexpr int SCL = kind_scale(KIND);
  // the staged values: FP64 for the FP64 form (H phi formed in FP64 from the
  // FP32 states and potential), FP32 otherwise
  using ST = typename std::conditional<KIND == RK_F64, double, float>::type;
  const ST c0 = (ST)c0d, c1 = (ST)c1d;
  extern __shared__ __align__(16) unsigned char pk_raw[];
  ST* pk_smem = reinterpret_cast<ST*>(pk_raw);
  __shared__ RUnit U;
  __shared__ DevFrag F;
  __shared__ int s_p[PK_TPC * 64], s_nb[PK_TPC * 64][6];
  __shared__ float s_v[PK_TPC * 64];
  const int tid = threadIdx.x;
  const int4 job = cta[blockIdx.x];   // unit, first tile, tiles
  if (tid == 0) U = units[job.x];
  __syncthreads();
  if (tid == 0) F = fr[U.frag];
  __syncthreads();
  const int rows = (F.n + 7) / 8 * 8;
  // shared rows [k][state]: FP32 kinds take a row stride of 4 mod 32 words
  // and an XOR swizzle of the state index by the 16-byte core column of k,
  // (k / KPU) % 4, in steps of 8 states, so phase 1 stores 4 states of a
  // point as one 16-byte word and phase 2 reads a column (8 rows x 4 cores
  // per warp) without bank conflicts; FP64 takes an odd stride.
  constexpr bool SWZ = sizeof(ST) == 4;
  const int RS = SWZ ? (rows + 31) / 32 * 32 + 4 : rows + 1;
  auto sw = [](int k, int row) { return SWZ ? row ^ (((k / KPU) & 3) << 3) : row; };
  ST* sPh = pk_smem;
  ST* sHp = pk_smem + 64 * RS;
  const float4* S4 = reinterpret_cast<const float4*>(states + F.off);
  const int qpp = F.ld / 4;
  const int nq = rows / 4;
  const int npl = U.L[0] * U.L[1];
  const long long cb = (long long)rows * 64 * SCL;
  const long long npl2 = (long long)U.ntiles * 128 * rows;   // one 2-byte plane
  const long long half = 2 * npl2 * SCL;                     // phi planes -> H phi planes
  const int upc = rows * NCORE;                              // units per chunk and plane
  unsigned char* blk = planes + U.base * SCL;
  // phase 1 items (k, q): thread tid starts at item tid and steps by two
  // items of PK_THREADS each (incremental division by nq)
  const int k1s = tid / nq, q1s = tid - k1s * nq;
  const int dk = PK_THREADS / nq, dq = PK_THREADS - dk * nq;
  int k2s = k1s + dk, q2s = q1s + dq;
  if (q2s >= nq) { q2s -= nq; ++k2s; }
  const int dk2 = (2 * PK_THREADS) / nq, dq2 = 2 * PK_THREADS - dk2 * nq;
  // phase 2: thread tid writes the units of one (array, chunk) combination
  constexpr int NCOMBO = 2 * KT::CPT;
  constexpr int TPCB = PK_THREADS / NCOMBO;
  const int combo = tid / TPCB, lic = tid % TPCB;
  const int A = combo / KT::CPT, cc = combo % KT::CPT;
  // the coordinates, neighbours and potential of all the CTA's points at
  // once, one point per thread (PK_TPC * 64 = PK_THREADS)
  static_assert(PK_TPC * 64 == PK_THREADS, "one point per thread");
  {
    const int t = job.y + tid / 64;
    const int K = t * 64 + tid % 64;
    const int iz = K / U.p8, r = K - iz * U.p8;
    bool in = t < job.y + job.z && iz < U.L[2] && r < npl;
    int l[3] = {0, 0, 0}, gi[3] = {0, 0, 0};
    if (in) {
      const int ii[3] = {r % U.L[0], r / U.L[0], iz};
      const int gn[3] = {gx, gy, gz};
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        int g = U.s0[d] + ii[d];
        if (g >= gn[d]) g -= gn[d];
        gi[d] = g;
        int ld = g - F.doff[d];
        if (ld < 0) ld += gn[d];
        l[d] = ld;
        in = in && ld < F.dext[d];
      }
    }
    const int ex = F.dext[0], exy = F.dext[0] * F.dext[1];
    const int p = l[0] + ex * l[1] + exy * l[2];
    const int st[3] = {1, ex, exy};
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int sd = 0; sd < 2; ++sd) {
        const int c = l[d] + (sd ? -1 : 1);
        int q = -1;
        if (c >= 0 && c < F.dext[d]) q = p + (c - l[d]) * st[d];
        else if (F.full[d]) q = p + ((c < 0 ? c + F.dext[d] : c - F.dext[d]) - l[d]) * st[d];
        if constexpr (CHECK) {
          if (in && q >= 0 &&
              (q >= F.Pd || F.off + ((long long)q + 1) * F.ld > n_states)) {
            atomicExch(bounds, 1);
            q = -1;
          }
        }
        s_nb[tid][2 * d + sd] = in ? q : -1;
      }
    if constexpr (CHECK) {
      if (in && (p < 0 || p >= F.Pd || F.off + ((long long)p + 1) * F.ld > n_states)) {
        atomicExch(bounds, 1);
        in = false;
      }
    }
    s_p[tid] = in ? p : -1;
    s_v[tid] = in ? V[(long long)gi[0] + (long long)gx * (gi[1] + (long long)gy * gi[2])] : 0.f;
  }
  for (int t = job.y; t < job.y + job.z; ++t) {
    __syncthreads();   // the tables are written / the previous tile's shared rows are consumed
    const int kb = (t - job.y) * 64;   // this tile's points in the tables
    // phase 1: two items per step, their 14 loads issued together (absent
    // points and neighbours load a row of the fragment itself and are
    // masked, so no load depends on a branch)
    for (int k1 = k1s, q1 = q1s, k2 = k2s, q2 = q2s; k1 < 64;) {
      const int kk[2] = {k1, k2 < 64 ? k2 : k1};
      const int qq[2] = {q1, q2};
      float4 w[2][7];
      bool use[2][7];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int p = s_p[kb + kk[h]];
        const bool ok = p >= 0 && qq[h] < qpp;
        const int qc = min(qq[h], qpp - 1);
        const int pc = p >= 0 ? p : 0;
        use[h][0] = ok;
        w[h][0] = S4[(long long)pc * qpp + qc];
#pragma unroll
        for (int j = 0; j < 6; ++j) {
          const int nb = s_nb[kb + kk[h]][j];
          use[h][j + 1] = ok && nb >= 0;
          w[h][j + 1] = S4[(long long)(nb >= 0 ? nb : pc) * qpp + qc];
        }
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (h == 1 && k2 >= 64) break;
        const int k = kk[h], q = qq[h];
        ST pv[4] = {0, 0, 0, 0}, hv[4] = {0, 0, 0, 0};
        if (use[h][0]) {
          ST sum[4] = {0, 0, 0, 0};
#pragma unroll
          for (int j = 1; j < 7; ++j)
            if (use[h][j]) {
              sum[0] += (ST)w[h][j].x; sum[1] += (ST)w[h][j].y;
              sum[2] += (ST)w[h][j].z; sum[3] += (ST)w[h][j].w;
            }
          const ST dv = c0 + (ST)s_v[kb + k];
          pv[0] = w[h][0].x; pv[1] = w[h][0].y; pv[2] = w[h][0].z; pv[3] = w[h][0].w;
#pragma unroll
          for (int i = 0; i < 4; ++i) hv[i] = fma(-c1, sum[i], dv * pv[i]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (4 * q + i >= F.n) pv[i] = hv[i] = (ST)0;
        if constexpr (SWZ) {
          const int o = k * RS + sw(k, 4 * q);
          *reinterpret_cast<float4*>(sPh + o) = make_float4(pv[0], pv[1], pv[2], pv[3]);
          *reinterpret_cast<float4*>(sHp + o) = make_float4(hv[0], hv[1], hv[2], hv[3]);
        } else {
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            sPh[k * RS + 4 * q + i] = pv[i];
            sHp[k * RS + 4 * q + i] = hv[i];
          }
        }
      }
      k1 += dk2; q1 += dq2;
      if (q1 >= nq) { q1 -= nq; ++k1; }
      k2 += dk2; q2 += dq2;
      if (q2 >= nq) { q2 -= nq; ++k2; }
    }
    __syncthreads();
    // phase 2, write-out: 16-byte unit (array A: phi / H phi, chunk cc,
    // 8-row group g, core kc, row r) of plane(A, hi|lo) at
    //   base + part(A) [+ lo] + (t*CPT + cc)*cb + g*(NCORE*128) + kc*128 + r*16
    // (the units of one (A, cc) are consecutive in memory: coalesced)
    const ST* srcA = A ? sHp : sPh;
    // not unrolled: the unrolled loop measured 15 % slower on the large lattice
#pragma unroll 1
    for (int u = lic; u < upc; u += TPCB) {
      const int r = u & 7, kc = (u >> 3) & (NCORE - 1), g = u / (8 * NCORE);
      const int row = 8 * g + r;
      const int k0 = cc * KT::KC + kc * KPU;
      const ST* src = srcA + k0 * RS + sw(k0, row);
      ST x[KPU];
#pragma unroll
      for (int j = 0; j < KPU; ++j) x[j] = src[j * RS];
      const long long off = (long long)(t * KT::CPT + cc) * cb + g * (NCORE * 128) + kc * 128 + r * 16;
      if constexpr (CHECK) {
        const long long last = U.base * SCL + A * half + off + (KIND == RK_BF16X3 ? npl2 : 0) + 16;
        if (last > n_plane_bytes || U.base < 0) {
          atomicExch(bounds, 1);
          continue;
        }
      }
      // streaming stores: the planes are read by the next kernel, long after
      // they would have left L2, and keeping them out of L2 leaves it to the
      // states' neighbour rows
      if constexpr (KIND == RK_TF32) {
        const uint4 v = make_uint4(rtf32(x[0]), rtf32(x[1]), rtf32(x[2]), rtf32(x[3]));
        __stcs(reinterpret_cast<uint4*>(blk + A * half + off), v);
      } else if constexpr (KIND == RK_F32) {
        __stcs(reinterpret_cast<float4*>(blk + A * half + off), make_float4(x[0], x[1], x[2], x[3]));
      } else if constexpr (KIND == RK_F64) {
        __stcs(reinterpret_cast<double2*>(blk + A * half + off), make_double2(x[0], x[1]));
      } else {
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const __nv_bfloat162 h2 = __floats2bfloat162_rn(x[2 * j], x[2 * j + 1]);
          hw[j] = *reinterpret_cast<const uint32_t*>(&h2);
          if constexpr (KIND == RK_BF16X3) {
            const float2 hf = __bfloat1622float2(h2);
            const __nv_bfloat162 l2 = __floats2bfloat162_rn(x[2 * j] - hf.x, x[2 * j + 1] - hf.y);
            lw[j] = *reinterpret_cast<const uint32_t*>(&l2);
          }
        }
        __stcs(reinterpret_cast<uint4*>(blk + A * half + off), make_uint4(hw[0], hw[1], hw[2], hw[3]));
        if constexpr (KIND == RK_BF16X3)
          __stcs(reinterpret_cast<uint4*>(blk + A * half + npl2 + off), make_uint4(lw[0], lw[1], lw[2], lw[3]));
      }
    }
  }   // tiles
}

// -------------------------------------------------------- a3/a4: contract --

// hold (a test of the failure detection): the producer publishes its first
// item and then withholds every copy, so the MMA thread's wait for the first
// stage runs out after wait_iters polls (no copy in flight), the roles give
// up, and the launch reports a timeout through *flag.
// Items are taken in order from a global counter (*next, zero at launch) by
// the producer warp, which passes each index to the MMA thread and the
// epilogue warps through a small ring in shared memory (RS_NQ entries, each
// with a full and an empty mbarrier); an index >= nitems ends the roles.
// Consecutive items -- the M x N tiles of one region -- therefore start
// together on different SMs and read the same operand chunks at about the
// same time, which keeps them in L2.
// An item's two row halves share each B chunk (one accumulator of 256 TMEM
// columns per half): a third less operand traffic from L2 than 128-row
// items.  The accumulators are not double-buffered across items (an item
// runs for milliseconds, its drain for microseconds).
// CHECK (check mode): the producer tests every copy's source range against
// the plane arena and destination against its operand tile, the epilogue
// every slot store against the slot arena; a failing copy ends the launch
// (the roles give up at once), a failing store is skipped; *bounds is set.
template <int KIND, bool CHECK = false>
__global__ void __launch_bounds__(RS_THREADS, 1) region_kernel(
    const RItem* __restrict__ items, int nitems, const RPiece* __restrict__ pieces,
    const RRowSeg* __restrict__ rsegs, const RColSeg* __restrict__ csegs,
    const long long* __restrict__ stab, const unsigned char* __restrict__ planes,
    float* __restrict__ slots, int* flag, int* next, int hold, int wait_iters,
    long long n_plane_bytes, long long n_slots, int* bounds) {
  using KT = KindT<KIND>;
  extern __shared__ __align__(1024) unsigned char rsm[];
  __shared__ __align__(8) unsigned long long full[RS_NSTAGE], empty[RS_NSTAGE], acc_full[1], acc_empty[1];
  __shared__ __align__(8) unsigned long long q_full[RS_NQ], q_empty[RS_NQ];
  __shared__ int q_item[RS_NQ];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_s, issued_s, mma_steps_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // stage s: for chunk cc < SC: A planes then B planes
  auto atile = [&](int s, int cc, int pl) {
    return rsm + (size_t)s * RS_STAGE + (size_t)cc * KT::NPL * (RS_ATILE + RS_BTILE) + (size_t)pl * RS_ATILE;
  };
  auto btile = [&](int s, int cc, int pl) {
    return rsm + (size_t)s * RS_STAGE + (size_t)cc * KT::NPL * (RS_ATILE + RS_BTILE) +
           (size_t)KT::NPL * RS_ATILE + (size_t)pl * RS_BTILE;
  };
  if (tid == 0) {
    for (int i = 0; i < RS_NSTAGE; ++i) {
      mbar_init(smem_u32(&full[i]), 1);
      mbar_init(smem_u32(&empty[i]), 1);
    }
    mbar_init(smem_u32(&acc_full[0]), 1);
    mbar_init(smem_u32(&acc_empty[0]), 4);
    for (int i = 0; i < RS_NQ; ++i) {
      mbar_init(smem_u32(&q_full[i]), 1);
      mbar_init(smem_u32(&q_empty[i]), 5);   // the MMA thread and the four epilogue warps
    }
    fence_mbar_init();
    abort_s = 0;
    issued_s = 0;
    mma_steps_s = 0;
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(2 * RS_ACOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  auto wait = [&](unsigned long long* bar, uint32_t parity) -> bool {
    const uint32_t a = smem_u32(bar);
    for (int i = 0; i < wait_iters; ++i) {
      if (mbar_try(a, parity)) return true;
      if (*(volatile int*)&abort_s) return false;
    }
    atomicExch(flag, 1);
    *(volatile int*)&abort_s = 1;
    return false;
  };

  if (warp == 0) {
    // ---------------------------------------------------------- producer
    int g = 0;
    bool ok = true;
    for (int item_no = 0; ok; ++item_no) {
      // claim the next item and publish it to the other roles
      const int qs = item_no % RS_NQ, qu = item_no / RS_NQ;
      int ii = 0;
      if (lane == 0) {
        bool w = qu == 0 || wait(&q_empty[qs], (uint32_t)((qu - 1) & 1));
        ii = w ? atomicAdd(next, 1) : nitems;
        q_item[qs] = ii;
        mbar_arrive(smem_u32(&q_full[qs]));   // release: the index is visible to the waiters
        ok = w;
      }
      ii = __shfl_sync(0xffffffffu, ii, 0);
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      if (!ok || ii >= nitems || hold) break;
      const RItem it = items[ii];
      const int npc = it.npa + it.npb;   // <= 64 (planner): lane j holds pieces j and j + 32
      RPiece pc[2];
      bool isA[2], has[2];
      uint32_t mine = 0;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int j = lane + 32 * h;
        has[h] = j < npc;
        isA[h] = j < it.npa;
        if (has[h]) {
          pc[h] = pieces[isA[h] ? it.pa0 + j : it.pb0 + j - it.npa];
          mine += (uint32_t)pc[h].bytes;
        }
      }
      const uint32_t sbytes = __reduce_add_sync(0xffffffffu, mine) * (uint32_t)(KT::SC * KT::NPL);
      const int nst = it.ntiles * KT::CPT / KT::SC;
      const long long c00 = (long long)it.tile0 * KT::CPT;
      if constexpr (CHECK) {
        // every chunk of every piece of the item, both planes, inside the
        // arena; every destination inside its tile
        bool bad = false;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (!has[h]) continue;
          const long long first = pc[h].base, last = pc[h].base + (c00 + nst * KT::SC - 1) * pc[h].cb +
                                                     (KT::NPL == 2 ? pc[h].lo : 0) + pc[h].bytes;
          const int tile = isA[h] ? RS_ATILE : RS_BTILE;
          bad = bad || first < 0 || last > n_plane_bytes || pc[h].dst < 0 || pc[h].dst + pc[h].bytes > tile;
        }
        if (__any_sync(0xffffffffu, bad)) {
          if (lane == 0) {
            atomicExch(bounds, 1);
            *(volatile int*)&abort_s = 1;
          }
          break;
        }
      }
      for (int st = 0; st < nst; ++st, ++g) {
        const int s = g % RS_NSTAGE, u = g / RS_NSTAGE;
        if (u > 0) {
          bool w = true;
          if (lane == 0) w = wait(&empty[s], (uint32_t)((u - 1) & 1));
          ok = __shfl_sync(0xffffffffu, w ? 1 : 0, 0) != 0;
          if (!ok) break;
        }
        const uint32_t mb = smem_u32(&full[s]);
        if (lane == 0) mbar_arrive_expect(mb, sbytes);
        __syncwarp();
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (!has[h]) continue;
#pragma unroll
          for (int cc = 0; cc < KT::SC; ++cc) {
            const long long c = c00 + (long long)st * KT::SC + cc;
            const unsigned char* src = planes + pc[h].base + c * pc[h].cb;
#pragma unroll
            for (int pl = 0; pl < KT::NPL; ++pl) {
              unsigned char* dst = (isA[h] ? atile(s, cc, pl) : btile(s, cc, pl)) + pc[h].dst;
              bulk_g2s(smem_u32(dst), src + (pl ? pc[h].lo : 0), (uint32_t)pc[h].bytes, mb);
            }
          }
        }
        if (lane == 0) *(volatile int*)&issued_s = g + 1;
      }
    }
  } else if (warp == 1) {
    // --------------------------------------------------------------- MMA
    if (lane == 0) {
      int g = 0;
      bool ok = true;
      for (int item_no = 0; ok; ++item_no) {
        const int qs = item_no % RS_NQ, qu = item_no / RS_NQ;
        if (!(ok = wait(&q_full[qs], (uint32_t)(qu & 1)))) break;
        const int ii = *(volatile int*)&q_item[qs];
        mbar_arrive(smem_u32(&q_empty[qs]));
        if (ii >= nitems) break;
        const RItem it = items[ii];
        if (item_no > 0 && !(ok = wait(&acc_empty[0], (uint32_t)((item_no - 1) & 1)))) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // half 0: all n_cols columns; half 1: columns [cskip, n_cols)
        const bool two = it.nh > 1 && it.n_cols - it.cskip >= 16;
        const uint32_t id0 = ridesc((uint32_t)KT::FMT, 128, (uint32_t)it.n_cols);
        const uint32_t id1 = ridesc((uint32_t)KT::FMT, 128, (uint32_t)(two ? it.n_cols - it.cskip : 16));
        const uint32_t d0 = tmem, d1 = tmem + (uint32_t)(RS_ACOLS + it.cskip);
        const uint64_t aoff = (uint64_t)((128 * 64) >> 4);             // rows 128.. of the A tile
        const uint64_t boff = (uint64_t)(((it.cskip / 8) * 512) >> 4);  // columns cskip.. of B
        const int nst = it.ntiles * KT::CPT / KT::SC;
        for (int st = 0; st < nst; ++st, ++g) {
          const int s = g % RS_NSTAGE, u = g / RS_NSTAGE;
          if (!(ok = wait(&full[s], (uint32_t)(u & 1)))) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
          for (int cc = 0; cc < KT::SC; ++cc) {
            const uint64_t a0 = rdesc(smem_u32(atile(s, cc, 0)));
            const uint64_t b0 = rdesc(smem_u32(btile(s, cc, 0)));
            uint64_t a1 = 0, b1 = 0;
            if constexpr (KT::NPL == 2) {
              a1 = rdesc(smem_u32(atile(s, cc, 1)));
              b1 = rdesc(smem_u32(btile(s, cc, 1)));
            }
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {   // 32 bytes of K per MMA: two core columns
              const uint64_t o = (uint64_t)((ks * 256) >> 4);
              const uint32_t acc = (st > 0 || cc > 0 || ks > 0) ? 1u : 0u;
              rmma<KT::FMT>(d0, a0 + o, b0 + o, id0, acc);
              if constexpr (KT::NPL == 2) {
                rmma<KT::FMT>(d0, a0 + o, b1 + o, id0, 1u);
                rmma<KT::FMT>(d0, a1 + o, b0 + o, id0, 1u);
              }
              if (two) {
                rmma<KT::FMT>(d1, a0 + aoff + o, b0 + boff + o, id1, acc);
                if constexpr (KT::NPL == 2) {
                  rmma<KT::FMT>(d1, a0 + aoff + o, b1 + boff + o, id1, 1u);
                  rmma<KT::FMT>(d1, a1 + aoff + o, b0 + boff + o, id1, 1u);
                }
              }
            }
          }
          rcommit(smem_u32(&empty[s]));
          *(volatile int*)&mma_steps_s = g + 1;
        }
        if (!ok) break;
        rcommit(smem_u32(&acc_full[0]));
      }
    }
  } else {
    // ---------------------------------------------------------- epilogue
    const int q = warp & 3;   // TMEM lane quadrant
    bool ok = true;
    for (int item_no = 0; ok; ++item_no) {
      const int qs = item_no % RS_NQ, qu = item_no / RS_NQ;
      ok = __all_sync(0xffffffffu, wait(&q_full[qs], (uint32_t)(qu & 1)));
      if (!ok) break;
      const int ii = *(volatile int*)&q_item[qs];
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&q_empty[qs]));
      if (ii >= nitems) break;
      const RItem it = items[ii];
      // the item's segments, one per lane (the planner keeps nrs <= 32 and
      // ncs <= 64), loaded while the accumulators fill
      RRowSeg rsl = {0, 0, 0, 0};
      RColSeg csl[2] = {{0, 0, 0, 0, 0, 0}, {0, 0, 0, 0, 0, 0}};
      if (lane < it.nrs) rsl = rsegs[it.rs0 + lane];
      if (lane < it.ncs) csl[0] = csegs[it.cs0 + lane];
      if (lane + 32 < it.ncs) csl[1] = csegs[it.cs0 + lane + 32];
      ok = __all_sync(0xffffffffu, wait(&acc_full[0], (uint32_t)(item_no & 1)));
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int nh = it.nh > 1 && it.n_cols - it.cskip >= 16 ? 2 : 1;
      for (int hh = 0; hh < nh; ++hh) {
        // this lane's row of half hh and its row segment (half 1's columns
        // below cskip were not formed; they belong to pairs b < a, which
        // have no slot)
        const int row = hh * 128 + q * 32 + lane;
        int rs = -1, i = 0, na = 0;
        for (int r = 0; r < it.nrs; ++r) {
          const int r0 = __shfl_sync(0xffffffffu, rsl.r0, r), nr = __shfl_sync(0xffffffffu, rsl.nr, r);
          const int i0 = __shfl_sync(0xffffffffu, rsl.i0, r), nn = __shfl_sync(0xffffffffu, rsl.na, r);
          if (row >= r0 && row < r0 + nr) {
            rs = r;
            i = i0 + row - r0;
            na = nn;
          }
        }
        const bool rok = rs >= 0 && i < na;
        for (int c = 0; c < it.ncs; ++c) {
          const int h = c >> 5, sl = c & 31;
          const int cc0 = __shfl_sync(0xffffffffu, h ? csl[1].c0 : csl[0].c0, sl);
          const int cnc = __shfl_sync(0xffffffffu, h ? csl[1].nc : csl[0].nc, sl);
          const int cj0 = __shfl_sync(0xffffffffu, h ? csl[1].j0 : csl[0].j0, sl);
          const int cnb = __shfl_sync(0xffffffffu, h ? csl[1].nb : csl[0].nb, sl);
          const int cpart = __shfl_sync(0xffffffffu, h ? csl[1].part : csl[0].part, sl);
          const int ccf = __shfl_sync(0xffffffffu, h ? csl[1].cf : csl[0].cf, sl);
          if (hh == 1 && cc0 + cnc <= it.cskip) continue;   // not formed, no slot
          const long long slot = rok ? stab[it.st0 + (long long)rs * it.ncf + ccf] : -1;
          for (int c0 = cc0; c0 < cc0 + cnc; c0 += 8) {
            float v[8];
            rtmem_ld8(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(hh * RS_ACOLS + c0), v);
            if (slot >= 0) {
              float* o = slots + slot + (long long)i * 2 * cnb + cpart * cnb;
              const int j0 = cj0 + c0 - cc0;
              if constexpr (CHECK) {
                const long long e = slot + (long long)i * 2 * cnb + cpart * cnb + j0;
                if (e < 0 || e + min(8, cnb - j0) > n_slots) {
                  atomicExch(bounds, 1);
                  continue;
                }
              }
              if (j0 + 8 <= cnb && ((reinterpret_cast<uintptr_t>(o + j0) & 15) == 0)) {
                *reinterpret_cast<float4*>(o + j0) = make_float4(v[0], v[1], v[2], v[3]);
                *reinterpret_cast<float4*>(o + j0 + 4) = make_float4(v[4], v[5], v[6], v[7]);
              } else {
#pragma unroll
                for (int jj = 0; jj < 8; ++jj)
                  if (j0 + jj < cnb) o[j0 + jj] = v[jj];
              }
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&acc_empty[0]));
    }
  }

  __syncthreads();
  if (abort_s && tid == 0) {
    // drain the copies of the last issued stages and the MMAs of the last
    // committed stage before shared and tensor memory are released
    auto drain = [&](unsigned long long* bar, uint32_t parity) {
      const uint32_t a = smem_u32(bar);
      for (int i = 0; i < (1 << 24) && !mbar_test(a, parity); ++i)
        if (i > 64) __nanosleep(64);
    };
    const int issued = issued_s;
    for (int g = max(0, issued - RS_NSTAGE); g < issued; ++g)
      drain(&full[g % RS_NSTAGE], (uint32_t)((g / RS_NSTAGE) & 1));
    const int ms = mma_steps_s;
    if (ms > 0) drain(&empty[(ms - 1) % RS_NSTAGE], (uint32_t)(((ms - 1) / RS_NSTAGE) & 1));
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * RS_ACOLS)
                 : "memory");
}


// ------------------------------------------- a3/a4: plain, CUDA cores ----

// The same items, pieces and slots as region_kernel, on the CUDA cores in
// FP32 or FP64 arithmetic: the plain forms the tensor-core precisions are
// measured against.  A persistent CTA takes items from the global counter;
// per item and pass of NP columns it streams the 16-point K chunks of the A
// pieces (128 stacked state rows) and of the B pieces clipped to the pass
// into a ring of shared-memory stages with 16-byte asynchronous copies, and
// each thread accumulates an 8-row x TN-column register tile.  Thread
// (tr, tc) takes rows 8 (2i + tr/8) + tr%8 and columns 8 (2j + tc/8) + tc%8,
// so the eight lanes of a quarter warp read one 16-byte unit of A (a
// broadcast) and eight adjacent units of B (no bank conflict).  Each output
// is a sum in K order with one FMA per point; the FP32 form stores FP32
// partial slots (finalized like the tensor-core ones), the FP64 form FP64
// slots.
constexpr int SR_THREADS = 256;
constexpr int SR_NSTAGE = 3;

template <typename T> struct SimtT;
template <> struct SimtT<float> {
  static constexpr int S = 1, NP = 256, TN = 16, NCORE = 4;
  using V = float4;
};
template <> struct SimtT<double> {
  static constexpr int S = 2, NP = 128, TN = 8, NCORE = 8;
  using V = double2;
};
template <typename T>
constexpr int simt_smem() {
  return SR_NSTAGE * (16 + SimtT<T>::NP / 8) * 512 * SimtT<T>::S;
}

__device__ __forceinline__ void cpa16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst),
               "l"((unsigned long long)__cvta_generic_to_global(src))
               : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cpa_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void fma_unit(float& acc, const float4& a, const float4& b) {
  acc = fmaf(a.x, b.x, acc);
  acc = fmaf(a.y, b.y, acc);
  acc = fmaf(a.z, b.z, acc);
  acc = fmaf(a.w, b.w, acc);
}
__device__ __forceinline__ void fma_unit(double& acc, const double2& a, const double2& b) {
  acc = fma(a.x, b.x, acc);
  acc = fma(a.y, b.y, acc);
}

template <typename T>
__global__ void __launch_bounds__(SR_THREADS, 1) region_simt_kernel(
    const RItem* __restrict__ items, int nitems, const RPiece* __restrict__ pieces,
    const RRowSeg* __restrict__ rsegs, const RColSeg* __restrict__ csegs,
    const long long* __restrict__ stab, const unsigned char* __restrict__ planes,
    T* __restrict__ slots, int* next) {
  using C = SimtT<T>;
  using V = typename C::V;
  constexpr int G = 512 * C::S;   // bytes of one 8-row group of a chunk
  constexpr int ABYTES = 16 * G, STAGE = ABYTES + (C::NP / 8) * G;
  constexpr int HT = C::TN / 2;
  extern __shared__ __align__(16) unsigned char ssm[];
  __shared__ long long s_src[64], s_cb[64];
  __shared__ int s_bytes[64], s_dst[64];
  __shared__ int s_rrs[256], s_ri[256];
  __shared__ int s_ccf[C::NP], s_cpart[C::NP], s_cj[C::NP], s_cnb[C::NP];
  __shared__ int s_item, s_npc, s_aend;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tc = lane & 15, tr = (lane >> 4) + 2 * warp;
  for (;;) {
    __syncthreads();   // the previous item's tables and stages are consumed
    if (tid == 0) s_item = atomicAdd(next, 1);
    __syncthreads();
    const int ii = s_item;
    if (ii >= nitems) break;
    const RItem it = items[ii];
    for (int r = tid; r < 256; r += SR_THREADS) {
      int rs = -1, i = 0;
      for (int q = 0; q < it.nrs; ++q) {
        const RRowSeg g = rsegs[it.rs0 + q];
        if (r >= g.r0 && r < g.r0 + g.nr) {
          i = g.i0 + r - g.r0;
          rs = i < g.na ? q : -1;
        }
      }
      s_rrs[r] = rs;
      s_ri[r] = i;
    }
    const int nch = it.ntiles * 4;   // 16-point chunks of the part
    // passes: row half hh (128 rows; half 1 from column cskip on) x NP columns
    for (int hh = 0; hh < it.nh; ++hh)
    for (int c0 = hh ? it.cskip : 0; c0 < it.n_cols; c0 += C::NP) {
      const int ncp = min(C::NP, it.n_cols - c0);
      __syncthreads();   // the previous pass's tables and stages are consumed
      for (int ci = tid; ci < C::NP; ci += SR_THREADS) {
        int cf = -1, part = 0, j = 0, nb = 0;
        const int col = c0 + ci;
        if (ci < ncp)
          for (int q = 0; q < it.ncs; ++q) {
            const RColSeg g = csegs[it.cs0 + q];
            if (col >= g.c0 && col < g.c0 + g.nc) {
              j = g.j0 + col - g.c0;
              cf = j < g.nb ? g.cf : -1;
              part = g.part;
              nb = g.nb;
            }
          }
        s_ccf[ci] = cf;
        s_cpart[ci] = part;
        s_cj[ci] = j;
        s_cnb[ci] = nb;
      }
      if (tid == 0) {
        // A pieces whole; B pieces clipped to the pass's column groups
        // (plan offsets are those of 4-byte operands: 512 bytes per group)
        int n = 0, aend = 0;
        for (int q = 0; q < it.npa; ++q) {   // clipped to the half's 16 row groups
          const RPiece pc = pieces[it.pa0 + q];
          const int g0 = pc.dst / 512, ng = pc.bytes / 512;
          const int lo = max(g0, 16 * hh), hi = min(g0 + ng, 16 * hh + 16);
          if (hi <= lo) continue;
          s_src[n] = (pc.base + (long long)(lo - g0) * 512) * C::S;
          s_cb[n] = (long long)pc.cb * C::S;
          s_bytes[n] = (hi - lo) * G;
          s_dst[n] = (lo - 16 * hh) * G;
          aend = max(aend, s_dst[n] + s_bytes[n]);
          ++n;
        }
        for (int q = 0; q < it.npb; ++q) {
          const RPiece pc = pieces[it.pb0 + q];
          const int g0 = pc.dst / 512, ng = pc.bytes / 512;
          const int lo = max(g0, c0 / 8), hi = min(g0 + ng, (c0 + C::NP) / 8);
          if (hi <= lo) continue;
          s_src[n] = (pc.base + (long long)(lo - g0) * 512) * C::S;
          s_cb[n] = (long long)pc.cb * C::S;
          s_bytes[n] = (hi - lo) * G;
          s_dst[n] = ABYTES + (lo - c0 / 8) * G;
          ++n;
        }
        s_npc = n;
        s_aend = aend;
      }
      __syncthreads();
      // rows and columns no piece covers read zeros
      {
        const int aend = s_aend, bend = ABYTES + (ncp / 8) * G;
        for (int st = 0; st < SR_NSTAGE; ++st) {
          unsigned char* b = ssm + (size_t)st * STAGE;
          for (int o = aend + 16 * tid; o < ABYTES; o += 16 * SR_THREADS)
            *reinterpret_cast<uint4*>(b + o) = make_uint4(0, 0, 0, 0);
          for (int o = bend + 16 * tid; o < STAGE; o += 16 * SR_THREADS)
            *reinterpret_cast<uint4*>(b + o) = make_uint4(0, 0, 0, 0);
        }
      }
      const int npc = s_npc;
      auto issue = [&](int ch) {
        if (ch < nch) {
          unsigned char* st = ssm + (size_t)(ch % SR_NSTAGE) * STAGE;
          const long long cg = (long long)it.tile0 * 4 + ch;   // chunk index in the unit
          for (int q = 0; q < npc; ++q) {
            const unsigned char* src = planes + s_src[q] + cg * s_cb[q];
            const int nu = s_bytes[q] >> 4;
            const uint32_t dst = smem_u32(st + s_dst[q]);
            for (int u = tid; u < nu; u += SR_THREADS) cpa16(dst + 16 * u, src + 16 * u);
          }
        }
        cpa_commit();
      };
      T acc[8][C::TN];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < C::TN; ++j) acc[i][j] = (T)0;
#pragma unroll
      for (int ch = 0; ch < SR_NSTAGE - 1; ++ch) issue(ch);
      for (int ch = 0; ch < nch; ++ch) {
        issue(ch + SR_NSTAGE - 1);   // into the stage consumed in the previous iteration
        cpa_wait<SR_NSTAGE - 1>();
        __syncthreads();
        const unsigned char* As = ssm + (size_t)(ch % SR_NSTAGE) * STAGE;
        const unsigned char* Bs = As + ABYTES;
#pragma unroll
        for (int kc = 0; kc < C::NCORE; ++kc) {
          V a[8];
#pragma unroll
          for (int i = 0; i < 8; ++i)
            a[i] = *reinterpret_cast<const V*>(As + (2 * i + (tr >> 3)) * G + kc * 128 + (tr & 7) * 16);
#pragma unroll
          for (int jh = 0; jh < 2; ++jh) {
            V b[HT];
#pragma unroll
            for (int j = 0; j < HT; ++j)
              b[j] = *reinterpret_cast<const V*>(Bs + (2 * (jh * HT + j) + (tc >> 3)) * G + kc * 128 +
                                                 (tc & 7) * 16);
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
              for (int j = 0; j < HT; ++j) fma_unit(acc[i][jh * HT + j], a[i], b[j]);
          }
        }
        __syncthreads();
      }
      cpa_wait<0>();
      // epilogue: each valid (row, column) into its pair's slot
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int row = 128 * hh + 8 * (2 * i + (tr >> 3)) + (tr & 7);
        const int rs = s_rrs[row];
        if (rs < 0) continue;
        const int si = s_ri[row];
#pragma unroll
        for (int j = 0; j < C::TN; ++j) {
          const int ci = 8 * (2 * j + (tc >> 3)) + (tc & 7);
          const int cf = s_ccf[ci];
          if (cf < 0) continue;
          const long long slot = stab[it.st0 + (long long)rs * it.ncf + cf];
          if (slot < 0) continue;
          const int nb = s_cnb[ci];
          slots[slot + (long long)si * 2 * nb + s_cpart[ci] * nb + s_cj[ci]] = acc[i][j];
        }
      }
    }
  }
}

// ------------------------------------------------------------ a5: blocks ---

// Pair p = blockIdx.x: S_ab and H_ab as sums of its slots in region order
// ([i][S_j | H_j] rows of 2 n_b floats), accumulated error-free in FP32
// (two-sum: the rounding error of every addition is carried in a second
// FP32 word, so the result is the FP64 value of the FP32 terms' sum to
// about 2^-44 relative, without FP64 arithmetic per term); a diagonal block
// is symmetrised, (X + X^T) / 2.
__device__ __forceinline__ void two_sum(float& s, float& e, float x) {
  const float t = s + x;
  const float bp = t - s;
  e += (s - (t - bp)) + (x - bp);
  s = t;
}

// One CTA per (pair, 32 x 32 tile of the block): thread (ty, tx) sums rows
// ty, ty + 8, ty + 16, ty + 24 of the tile at column tx over the pair's
// slots in region order, S and H; every load is a coalesced row of a slot,
// up to 8 slots in flight.  A diagonal block also sums the mirrored tile
// (rows and columns exchanged, read as rows) into shared memory and writes
// (X + X^T) / 2.  Sums are FP32 two-sum pairs (the rounding error of each
// addition carried in a second word), converted to FP64 at the end.
__device__ __forceinline__ void tile_sums(const float* __restrict__ base, long long ss, int nslot,
                                          int nb, int r0, int c0, int nr, int nc, int ty, int tx,
                                          double S[4], double H[4]) {
  float s1[4], e1[4], s2[4], e2[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) s1[r] = e1[r] = s2[r] = e2[r] = 0.f;
  const int c = c0 + tx;
  for (int k0 = 0; k0 < nslot; k0 += 4) {
    float a[4][4], b[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int i = r0 + ty + 8 * r;
        a[j][r] = 0.f;
        b[j][r] = 0.f;
        if (k0 + j < nslot && i < r0 + nr && c < c0 + nc) {
          const float* p = base + (long long)(k0 + j) * ss + (long long)i * 2 * nb + c;
          a[j][r] = p[0];
          b[j][r] = p[nb];
        }
      }
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (k0 + j < nslot)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          two_sum(s1[r], e1[r], a[j][r]);
          two_sum(s2[r], e2[r], b[j][r]);
        }
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    S[r] = (double)s1[r] + (double)e1[r];
    H[r] = (double)s2[r] + (double)e2[r];
  }
}

// FP64 slots (the FP64 plain form): plain FP64 sums in region order.
__device__ __forceinline__ void tile_sums(const double* __restrict__ base, long long ss, int nslot,
                                          int nb, int r0, int c0, int nr, int nc, int ty, int tx,
                                          double S[4], double H[4]) {
#pragma unroll
  for (int r = 0; r < 4; ++r) S[r] = H[r] = 0.0;
  const int c = c0 + tx;
  for (int k = 0; k < nslot; ++k)
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int i = r0 + ty + 8 * r;
      if (i < r0 + nr && c < c0 + nc) {
        const double* p = base + (long long)k * ss + (long long)i * 2 * nb + c;
        S[r] += p[0];
        H[r] += p[nb];
      }
    }
}

// Four CTAs per SM (64 registers): 2.35 ms against 3.05 ms at two (105
// registers) on the large lattice.
template <typename T>
__global__ void __launch_bounds__(256, 4) rfinalize_kernel(const RPair* __restrict__ prs,
                                                        const T* __restrict__ slots,
                                                        double* __restrict__ blocks) {
  __shared__ double tS[32][33], tH[32][33];
  const RPair pr = prs[blockIdx.x];
  const int na = pr.na, nb = pr.nb;
  const int tcol = (nb + 31) / 32;
  const int ti = blockIdx.y / tcol, tm = blockIdx.y - (blockIdx.y / tcol) * tcol;
  const int r0 = 32 * ti, c0 = 32 * tm;
  if (r0 >= na) return;
  const int nr = min(32, na - r0), nc = min(32, nb - c0);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const long long ss = (long long)na * 2 * nb;
  const T* base = slots + pr.slot0;
  double S[4], H[4];
  tile_sums(base, ss, pr.nslot, nb, r0, c0, nr, nc, ty, tx, S, H);
  if (pr.a == pr.b) {
    // the mirrored tile: rows c0.., columns r0.. (n_a = n_b)
    double St[4], Ht[4];
    tile_sums(base, ss, pr.nslot, nb, c0, r0, nc, nr, ty, tx, St, Ht);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      tS[ty + 8 * r][tx] = St[r];
      tH[ty + 8 * r][tx] = Ht[r];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      S[r] = 0.5 * (S[r] + tS[tx][ty + 8 * r]);
      H[r] = 0.5 * (H[r] + tH[tx][ty + 8 * r]);
    }
  }
  double* Hblk = blocks + pr.blk_off;
  double* Sblk = Hblk + (long long)na * nb;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = r0 + ty + 8 * r, m = c0 + tx;
    if (i < r0 + nr && m < c0 + nc) {
      Sblk[(long long)i * nb + m] = S[r];
      Hblk[(long long)i * nb + m] = H[r];
    }
  }
}

}  // namespace

// ------------------------------------------------------------- planner ----

struct RegionPlan {
  std::vector<RUnit> units;
  std::vector<int4> pack_cta;   // pack CTAs: unit, first tile, tiles
  std::vector<RItem> items;
  std::vector<RPiece> pieces;
  std::vector<RRowSeg> rsegs;
  std::vector<RColSeg> csegs;
  std::vector<long long> stab;
  std::vector<RPair> rpairs;
  long long plane_bytes = 0, slot_elems = 0, total_tiles = 0;
  double mma_flops = 0.0;     // MMA work per 64-point tile summed (M 128 x N), for one product
  int nregions = 0, nparts = 0, w_min = 1;
  DevBuf d_units, d_pcta, d_items, d_pieces, d_rsegs, d_csegs, d_stab, d_rpairs, planes, slots;
  bool ok = false;
  bool uploaded = false;
  std::string why;
};

namespace {

struct Seg { int s0, len; };

// Segments of one periodic dimension cut at every dilated-box boundary;
// segments shorter than w_min are merged into a neighbour.
std::vector<Seg> dim_segments(int n, const std::vector<DevFrag>& fr, int d, int w_min) {
  std::vector<int> bp;
  for (const DevFrag& f : fr)
    if (!f.full[d]) {
      bp.push_back(f.doff[d] % n);
      bp.push_back((f.doff[d] + f.dext[d]) % n);
    }
  std::sort(bp.begin(), bp.end());
  bp.erase(std::unique(bp.begin(), bp.end()), bp.end());
  std::vector<Seg> s;
  const int m = (int)bp.size();
  if (m == 0) s.push_back({0, n});
  for (int i = 0; i < m; ++i) {
    const int a = bp[i], b = i + 1 < m ? bp[i + 1] : bp[0] + n;
    s.push_back({a, b - a});
  }
  // merge short segments into the shorter neighbour (cyclic)
  while (s.size() > 1) {
    int k = -1;
    for (int i = 0; i < (int)s.size(); ++i)
      if (s[i].len < w_min && (k < 0 || s[i].len < s[k].len)) k = i;
    if (k < 0) break;
    const int ns = (int)s.size();
    const int l = (k + ns - 1) % ns, r = (k + 1) % ns;
    if (s[l].len <= s[r].len) {
      s[l].len += s[k].len;
      s.erase(s.begin() + k);
    } else {
      s[r].s0 = s[k].s0;
      s[r].len += s[k].len;
      s.erase(s.begin() + k);
    }
  }
  for (auto& x : s) x.s0 %= n;
  // long x and y segments are split (a region's z plane is staged on chip
  // by the pack); splitting keeps the cover set
  if (d < 2) {
    std::vector<Seg> t;
    for (const Seg& x : s) {
      const int parts = (x.len + PK_SEGMAX - 1) / PK_SEGMAX;
      for (int k = 0; k < parts; ++k) {
        const int a = (int)((long long)x.len * k / parts), b = (int)((long long)x.len * (k + 1) / parts);
        t.push_back({(x.s0 + a) % n, b - a});
      }
    }
    s.swap(t);
  }
  return s;
}

bool meets(int n, int s0, int len, int d0, int dl) {
  if (dl >= n || len >= n) return true;
  const int a = ((s0 - d0) % n + n) % n;   // segment start relative to the interval
  const int b = ((d0 - s0) % n + n) % n;   // interval start relative to the segment
  return a < dl || b < len;
}

}  // namespace

// Builds the region plan: returns OFM_OK with plan->ok false (and why) when
// this path does not apply (more than 128 states, too many slots).
// pair_pts (nullable): per pair, the points of B_a ∩ B_b+ inside the
// regions that hold both fragments, counted point by point (a check of the
// cover sets).
static void region_plan_build(const int gn[3], RegionPlan* P, const std::vector<DevFrag>& fr,
                              const std::vector<HostPair>& prs, const std::vector<long long>& blk_off,
                              int w_min_req, long long slot_budget_bytes,
                              std::vector<long long>* pair_pts = nullptr) {
  P->units.clear(); P->pack_cta.clear(); P->items.clear(); P->pieces.clear(); P->rsegs.clear(); P->csegs.clear();
  P->stab.clear(); P->rpairs.clear();
  P->ok = false;
  P->uploaded = false;
  P->mma_flops = 0.0;
  const int nf = (int)fr.size();
  for (const DevFrag& f : fr)
    if ((f.n + 7) / 8 * 8 > RS_MAXROWS) {
      P->why = "region contraction takes at most 128 states per fragment";
      return;
    }
  // segments, coarsened until the (fragment, region) incidences stay bounded
  std::vector<Seg> seg[3];
  std::vector<std::vector<int>> fseg[3];   // per dim, per fragment: segment indices it meets
  int w_min = std::max(1, w_min_req);
  for (;;) {
    long long inc = 0;
    for (int d = 0; d < 3; ++d) {
      seg[d] = dim_segments(gn[d], fr, d, w_min);
      fseg[d].assign(nf, {});
      for (int a = 0; a < nf; ++a)
        for (int i = 0; i < (int)seg[d].size(); ++i)
          if (fr[a].full[d] || meets(gn[d], seg[d][i].s0, seg[d][i].len, fr[a].doff[d], fr[a].dext[d]))
            fseg[d][a].push_back(i);
    }
    for (int a = 0; a < nf; ++a)
      inc += (long long)fseg[0][a].size() * fseg[1][a].size() * fseg[2][a].size();
    if (inc <= 4000000 || w_min >= 64) break;
    w_min *= 2;
  }
  P->w_min = w_min;
  const long long nsx = seg[0].size(), nsy = seg[1].size(), nsz = seg[2].size();
  // cover sets (fragments in increasing order)
  std::unordered_map<long long, std::vector<int>> cover;
  for (int a = 0; a < nf; ++a)
    for (int k : fseg[2][a])
      for (int j : fseg[1][a])
        for (int i : fseg[0][a]) cover[i + nsx * (j + nsy * (long long)k)].push_back(a);
  std::vector<long long> keys;
  keys.reserve(cover.size());
  for (auto& kv : cover) keys.push_back(kv.first);
  std::sort(keys.begin(), keys.end());
  P->nregions = (int)keys.size();
  std::unordered_map<long long, int> pidx;
  pidx.reserve(prs.size() * 2);
  for (int p = 0; p < (int)prs.size(); ++p) pidx[(long long)prs[p].a * nf + prs[p].b] = p;
  std::vector<int> rows(nf);
  for (int a = 0; a < nf; ++a) rows[a] = (fr[a].n + 7) / 8 * 8;

  // plane arena: one block per (fragment, region), 8 bytes per (point, padded state)
  struct RInfo { long long key; int ix, iy, iz, npts, p8, ntiles; };
  std::vector<RInfo> regs(keys.size());
  std::vector<std::unordered_map<long long, long long>> fbase(nf);
  long long arena = 0, tiles = 0, total_work = 0;
  for (size_t r = 0; r < keys.size(); ++r) {
    const long long key = keys[r];
    RInfo& R = regs[r];
    R.key = key;
    R.ix = (int)(key % nsx);
    R.iy = (int)((key / nsx) % nsy);
    R.iz = (int)(key / (nsx * nsy));
    R.npts = seg[0][R.ix].len * seg[1][R.iy].len * seg[2][R.iz].len;
    R.p8 = (seg[0][R.ix].len * seg[1][R.iy].len + 7) / 8 * 8;
    R.ntiles = (seg[2][R.iz].len * R.p8 + 63) / 64;
    long long M = 0;
    for (int a : cover[key]) {
      RUnit u;
      u.frag = a;
      u.s0[0] = seg[0][R.ix].s0; u.s0[1] = seg[1][R.iy].s0; u.s0[2] = seg[2][R.iz].s0;
      u.L[0] = seg[0][R.ix].len; u.L[1] = seg[1][R.iy].len; u.L[2] = seg[2][R.iz].len;
      u.p8 = R.p8;
      u.ntiles = R.ntiles;
      u.tile0 = tiles;
      u.base = arena;
      fbase[a][key] = arena;
      arena += (long long)R.ntiles * 64 * rows[a] * 8;
      tiles += R.ntiles;

      P->units.push_back(u);
      M += rows[a];
    }
    // work in (tile x N-tile x M-tile) units, for the K split below
    const long long mt = (M + 127) / 128;
    total_work += (long long)R.ntiles * mt * ((2 * M + 255) / 256);
  }
  P->plane_bytes = arena;
  P->total_tiles = tiles;
  for (int ui = 0; ui < (int)P->units.size(); ++ui) {
    const RUnit& u = P->units[ui];
    for (int t0 = 0; t0 < u.ntiles; t0 += PK_TPC)
      P->pack_cta.push_back(make_int4(ui, t0, std::min(PK_TPC, u.ntiles - t0), 0));
  }

  // K split: about two items of equal work per SM, parts of at least 4 tiles
  // (more, shorter parts only multiply the partial slots: six per SM took
  // the alkane chain's assembly from 170 to 204 us, nearly all of it in a5)
  const long long target = std::max<long long>(4, total_work / (2 * 152));

  // slots: count per pair first
  std::vector<int> nslot(prs.size(), 0);
  struct PartInfo { int r, t0, nt; };
  std::vector<PartInfo> parts;
  for (size_t r = 0; r < regs.size(); ++r) {
    const std::vector<int>& C = cover[regs[r].key];
    long long M = 0;
    for (int a : C) M += rows[a];
    const long long per_tile = ((M + 127) / 128) * ((2 * M + 255) / 256);
    const int nt = regs[r].ntiles;
    int nsplit = (int)std::min<long long>(std::max<long long>(1, nt / 4),
                                          std::max<long long>(1, (nt * per_tile + target - 1) / target));
    for (int s = 0; s < nsplit; ++s) {
      const int t0 = (int)((long long)nt * s / nsplit), t1 = (int)((long long)nt * (s + 1) / nsplit);
      if (t1 > t0) parts.push_back({(int)r, t0, t1 - t0});
    }
    for (size_t x = 0; x < C.size(); ++x)
      for (size_t y = x; y < C.size(); ++y) {
        auto it = pidx.find((long long)C[x] * nf + C[y]);
        if (it != pidx.end()) nslot[it->second] += nsplit;
      }
  }
  P->nparts = (int)parts.size();
  P->rpairs.resize(prs.size());
  long long se = 0;
  for (size_t p = 0; p < prs.size(); ++p) {
    RPair& q = P->rpairs[p];
    q.a = prs[p].a;
    q.b = prs[p].b;
    q.na = fr[q.a].n;
    q.nb = fr[q.b].n;
    q.nslot = nslot[p];
    q.slot0 = se;
    q.blk_off = blk_off[p];
    se += (long long)nslot[p] * q.na * 2 * q.nb;
  }
  P->slot_elems = se;
  if (se * 4 > slot_budget_bytes) {
    char buf[160];
    snprintf(buf, sizeof buf, "region contraction needs %.1f GB of partial slots (budget %.1f GB)",
             se * 4e-9, slot_budget_bytes * 1e-9);
    P->why = buf;
    return;
  }
  if (pair_pts) {
    // |R ∩ B_a ∩ B_b+| per dimension by walking the segment's points
    pair_pts->assign(prs.size(), 0);
    auto count = [&](int d, const Seg& sg, const DevFrag& A, const DevFrag& B) {
      long long k = 0;
      for (int t = 0; t < sg.len; ++t) {
        const int g = (sg.s0 + t) % gn[d];
        const int la = ((g - A.doff[d]) % gn[d] + gn[d]) % gn[d];
        const int lb = ((g - B.doff[d]) % gn[d] + gn[d]) % gn[d];
        if (la >= A.lo[d] && la < A.lo[d] + A.ext[d] && lb < B.dext[d]) ++k;
      }
      return k;
    };
    for (const RInfo& R : regs) {
      const std::vector<int>& C = cover[R.key];
      for (size_t x = 0; x < C.size(); ++x)
        for (size_t y = x; y < C.size(); ++y) {
          auto it = pidx.find((long long)C[x] * nf + C[y]);
          if (it == pidx.end()) continue;
          const DevFrag &A = fr[C[x]], &B = fr[C[y]];
          (*pair_pts)[it->second] += count(0, seg[0][R.ix], A, B) * count(1, seg[1][R.iy], A, B) *
                                     count(2, seg[2][R.iz], A, B);
        }
    }
  }
  std::vector<int> used(prs.size(), 0);

  // items
  for (const PartInfo& pt : parts) {
    const RInfo& R = regs[pt.r];
    const std::vector<int>& C = cover[R.key];
    const int nc = (int)C.size();
    std::vector<int> r0(nc + 1, 0);
    for (int x = 0; x < nc; ++x) r0[x + 1] = r0[x] + rows[C[x]];
    const int M = r0[nc];
    // this part's slot of every pair in the cover
    std::vector<long long> slot(nc * nc, -1);
    for (int x = 0; x < nc; ++x)
      for (int y = x; y < nc; ++y) {
        auto it = pidx.find((long long)C[x] * nf + C[y]);
        if (it == pidx.end()) continue;
        const int p = it->second;
        const RPair& q = P->rpairs[p];
        slot[x * nc + y] = q.slot0 + (long long)used[p]++ * q.na * 2 * q.nb;
      }
    for (int m0 = 0; m0 < M; m0 += 256) {
      const int m1 = std::min(M, m0 + 256);
      int xlo = 0;
      while (r0[xlo + 1] <= m0) ++xlo;
      int xlo1 = xlo;   // first fragment of the second half
      while (m1 > m0 + 128 && r0[xlo1 + 1] <= m0 + 128) ++xlo1;
      for (int n0 = 2 * r0[xlo]; n0 < 2 * M; n0 += 256) {
        const int n1 = std::min(2 * M, n0 + 256);
        RItem it;
        it.tile0 = pt.t0;
        it.ntiles = pt.nt;
        it.n_cols = n1 - n0;
        // the second half needs the columns of its own fragments onward
        it.nh = m1 > m0 + 128 ? 2 : 1;
        it.cskip = 0;
        if (it.nh == 2) {
          const int need = std::max(0, 2 * r0[xlo1] - n0);
          if (need >= it.n_cols) it.nh = 1;   // no block of half 1 in this N tile
          else it.cskip = need / 16 * 16;
        }
        it.pa0 = (int)P->pieces.size();
        it.rs0 = (int)P->rsegs.size();
        std::vector<int> rfr;   // cover index of each row segment
        for (int x = xlo; x < nc && r0[x] < m1; ++x) {
          const int lo = std::max(m0, r0[x]), hi = std::min(m1, r0[x + 1]);
          if (hi <= lo) continue;
          const long long base = fbase[C[x]][R.key];
          RPiece pc;
          pc.cb = rows[C[x]] * 64;
          pc.base = base + (long long)((lo - r0[x]) / 8) * 512;
          pc.lo = (long long)R.ntiles * 64 * rows[C[x]] * 2;
          pc.bytes = (hi - lo) / 8 * 512;
          pc.dst = (lo - m0) / 8 * 512;
          pc.pad = 0;
          P->pieces.push_back(pc);
          RRowSeg rs;
          rs.r0 = lo - m0;
          rs.nr = hi - lo;
          rs.i0 = lo - r0[x];
          rs.na = fr[C[x]].n;
          P->rsegs.push_back(rs);
          rfr.push_back(x);
        }
        it.npa = (int)P->pieces.size() - it.pa0;
        it.nrs = (int)P->rsegs.size() - it.rs0;
        it.pb0 = (int)P->pieces.size();
        it.cs0 = (int)P->csegs.size();
        std::vector<int> cfr;   // cover index of each column fragment
        for (int x = 0; x < nc; ++x) {
          for (int part = 0; part < 2; ++part) {
            const int cbeg = 2 * r0[x] + part * rows[C[x]], cend = cbeg + rows[C[x]];
            const int lo = std::max(n0, cbeg), hi = std::min(n1, cend);
            if (hi <= lo) continue;
            const long long base = fbase[C[x]][R.key];
            RPiece pc;
            pc.cb = rows[C[x]] * 64;
            const long long half = (long long)R.ntiles * 64 * rows[C[x]] * 4;
            pc.base = base + part * half + (long long)((lo - cbeg) / 8) * 512;
            pc.lo = (long long)R.ntiles * 64 * rows[C[x]] * 2;
            pc.bytes = (hi - lo) / 8 * 512;
            pc.dst = (lo - n0) / 8 * 512;
            pc.pad = 0;
            P->pieces.push_back(pc);
            if (cfr.empty() || cfr.back() != x) cfr.push_back(x);
            RColSeg cs;
            cs.c0 = lo - n0;
            cs.nc = hi - lo;
            cs.j0 = lo - cbeg;
            cs.nb = fr[C[x]].n;
            cs.part = part;
            cs.cf = (int)cfr.size() - 1;
            P->csegs.push_back(cs);
          }
        }
        it.npb = (int)P->pieces.size() - it.pb0;
        it.ncs = (int)P->csegs.size() - it.cs0;
        if (it.npa + it.npb > 64 || it.nrs > 32 || it.ncs > 64) {
          P->why = "region item with more than 64 copy pieces";
          P->items.clear();
          return;
        }
        it.ncf = (int)cfr.size();
        it.st0 = (long long)P->stab.size();
        for (int x : rfr)
          for (int y : cfr) P->stab.push_back(x <= y ? slot[x * nc + y] : -1);
        P->mma_flops += 2.0 * 128 * (it.n_cols + (it.nh == 2 ? it.n_cols - it.cskip : 0)) * 64.0 * it.ntiles;
        P->items.push_back(it);
      }
    }
  }
  P->ok = true;
}

// ------------------------------------------------------------- runtime ----

template <typename T>
static ofm_status upload(ofm_ctx* c, DevBuf& b, const std::vector<T>& v, const char* what) {
  OFM_TRY(ofm_ensure(c, b, sizeof(T) * std::max<size_t>(1, v.size()), what));
  if (!v.empty())
    OFM_CUDA(c, cudaMemcpyAsync(b.p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, c->stream));
  return OFM_OK;
}

// Test hook of the check mode: the host copy of the first copy piece now
// points just past the plane arena, and the tables are uploaded again at the
// next assembly, whose check-mode producer must refuse it.
ofm_status ofm_region_test_corrupt(ofm_ctx* c) {
  RegionPlan* P = c->region;
  if (!c->checks) return ofm_fail(c, OFM_ERR_STATE, "the corruption hook needs check mode");
  if (!P || !P->ok || P->pieces.empty()) return ofm_fail(c, OFM_ERR_STATE, "no region plan");
  P->pieces[0].base = P->plane_bytes;
  P->uploaded = false;
  return OFM_OK;
}

void ofm_region_guards(const ofm_ctx* c, std::vector<GuardRef>& out) {
  const RegionPlan* P = c->region;
  if (!P) return;
  const struct { const DevBuf* b; const char* n; } bufs[] = {
      {&P->d_units, "region units"}, {&P->d_pcta, "pack launch table"}, {&P->d_items, "region items"},
      {&P->d_pieces, "region pieces"}, {&P->d_rsegs, "region row segments"},
      {&P->d_csegs, "region column segments"}, {&P->d_stab, "region slot table"},
      {&P->d_rpairs, "region pairs"}, {&P->planes, "operand planes"}, {&P->slots, "partial slots"}};
  for (const auto& x : bufs)
    if (x.b->p) out.push_back({x.b->p, x.b->cap, x.n});
}

void ofm_region_free(ofm_ctx* c) {
  RegionPlan* P = c->region;
  if (!P) return;
  DevBuf* bufs[] = {&P->d_units, &P->d_pcta, &P->d_items, &P->d_pieces, &P->d_rsegs, &P->d_csegs,
                    &P->d_stab, &P->d_rpairs, &P->planes, &P->slots};
  for (DevBuf* b : bufs)
    if (b->p) cudaFree(b->p);
  delete P;
  c->region = nullptr;
}

// The region plan of the context's current fragments and pairs (host tables
// only; device buffers on first use).
ofm_status ofm_region_plan(ofm_ctx* c) {
  if (!c->region) c->region = new RegionPlan();
  RegionPlan* P = c->region;
  if (c->storage != OFM_STORE_FP32) {
    P->ok = false;
    P->uploaded = false;
    P->why = "region contraction needs FP32 storage";
    return OFM_OK;
  }
  std::vector<long long> off(c->pairs.size());
  for (size_t p = 0; p < c->pairs.size(); ++p) off[p] = c->simt_pairs[p].blk_off;
  region_plan_build(c->grid.n, P, c->frags, c->pairs, off, c->region_wmin, 16LL << 30);
  return OFM_OK;
}

bool ofm_region_ok(const ofm_ctx* c) { return c->region && c->region->ok; }

// Whether the region plan is the default: its MMA work (one product pass,
// padding and lower-triangle tiles included) stays within 4x the
// algorithmic pair flops.  Irregular boxes cut the grid into many small
// regions whose tiles are mostly padding; there the per-pair GEMMs win.
bool ofm_region_default(const ofm_ctx* c) {
  return ofm_region_ok(c) && c->region->mma_flops <= 4.0 * (double)c->flops;
}

const char* ofm_region_why(const ofm_ctx* c) {
  return c->region ? c->region->why.c_str() : "no region plan";
}

ofm_status ofm_region_prepare(ofm_ctx* c, ofm_precision prec) {
  RegionPlan* P = c->region;
  // the FP64 plain form doubles the planes and keeps FP64 slots
  const int scl = prec == OFM_PREC_FP64 ? 2 : 1;
  if (P->uploaded) {
    OFM_TRY(ofm_ensure_big(c, P->planes, (size_t)P->plane_bytes * scl, "operand planes"));
    return ofm_ensure_big(c, P->slots, 4 * scl * (size_t)std::max<long long>(1, P->slot_elems),
                          "partial slots");
  }
  OFM_TRY(upload(c, P->d_units, P->units, "region units"));
  OFM_TRY(upload(c, P->d_pcta, P->pack_cta, "pack launch table"));
  OFM_TRY(upload(c, P->d_items, P->items, "region items"));
  OFM_TRY(upload(c, P->d_pieces, P->pieces, "region pieces"));
  OFM_TRY(upload(c, P->d_rsegs, P->rsegs, "region row segments"));
  OFM_TRY(upload(c, P->d_csegs, P->csegs, "region column segments"));
  OFM_TRY(upload(c, P->d_stab, P->stab, "region slot table"));
  OFM_TRY(upload(c, P->d_rpairs, P->rpairs, "region pairs"));
  OFM_TRY(ofm_ensure_big(c, P->planes, (size_t)P->plane_bytes * scl, "operand planes"));
  OFM_TRY(ofm_ensure_big(c, P->slots, 4 * scl * (size_t)std::max<long long>(1, P->slot_elems),
                         "partial slots"));
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(region_kernel<RK_TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, RS_SMEM);
    cudaFuncSetAttribute(region_kernel<RK_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, RS_SMEM);
    cudaFuncSetAttribute(region_kernel<RK_BF16X3>, cudaFuncAttributeMaxDynamicSharedMemorySize, RS_SMEM);
    cudaFuncSetAttribute(region_kernel<RK_TF32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, RS_SMEM);
    cudaFuncSetAttribute(region_kernel<RK_BF16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, RS_SMEM);
    cudaFuncSetAttribute(region_kernel<RK_BF16X3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, RS_SMEM);
    const int pk = 2 * 64 * (RS_MAXROWS + 4) * 4;   // phi and H phi, 64 points x (rows + pad) words
    cudaFuncSetAttribute(pack_kernel<RK_TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, pk);
    cudaFuncSetAttribute(pack_kernel<RK_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, pk);
    cudaFuncSetAttribute(pack_kernel<RK_BF16X3>, cudaFuncAttributeMaxDynamicSharedMemorySize, pk);
    cudaFuncSetAttribute(pack_kernel<RK_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, pk);
    cudaFuncSetAttribute(pack_kernel<RK_F64>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * pk);
    cudaFuncSetAttribute(pack_kernel<RK_TF32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, pk);
    cudaFuncSetAttribute(pack_kernel<RK_BF16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, pk);
    cudaFuncSetAttribute(pack_kernel<RK_BF16X3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, pk);
    cudaFuncSetAttribute(pack_kernel<RK_F32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, pk);
    cudaFuncSetAttribute(pack_kernel<RK_F64, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * pk);
    cudaFuncSetAttribute(region_simt_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         simt_smem<float>());
    cudaFuncSetAttribute(region_simt_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         simt_smem<double>());
    OFM_CUDA(c, cudaGetLastError());
    attr = true;
  }
  P->uploaded = true;
  return OFM_OK;
}

// a1 (apply + pack), a3/a4 (region contraction) and a5 (blocks) for one
// precision, enqueued on the context stream.
ofm_status ofm_region_run(ofm_ctx* c, ofm_precision prec) {
  RegionPlan* P = c->region;
  if (!P || !P->ok) return ofm_fail(c, OFM_ERR_INVALID, P ? P->why : "no region plan");
  if (!P->uploaded) return ofm_fail(c, OFM_ERR_STATE, "region plan not prepared");
  const int kind = prec == OFM_PREC_TF32   ? RK_TF32
                   : prec == OFM_PREC_BF16 ? RK_BF16
                   : prec == OFM_PREC_FP32 ? RK_F32
                   : prec == OFM_PREC_FP64 ? RK_F64
                                           : RK_BF16X3;
  const bool f64 = kind == RK_F64;

  const double h = c->grid.h;
  const double c0 = 3.0 / (h * h), c1 = 0.5 / (h * h);
  {
    KTimer t(c, KC_APPLY, 1, c->pack_bytes[kind]);
    const RUnit* u = (const RUnit*)P->d_units.p;
    const DevFrag* f = (const DevFrag*)c->d_frags.p;
    const float* V = (const float*)c->V.p;
    const float* st = (const float*)c->states.p;
    unsigned char* pl = (unsigned char*)P->planes.p;
    int maxrows = 8;
    for (const DevFrag& fq : c->frags) maxrows = std::max(maxrows, (fq.n + 7) / 8 * 8);
    const int sm = f64 ? 2 * 64 * (maxrows + 1) * 8 : 2 * 64 * ((maxrows + 31) / 32 * 32 + 4) * 4;
    const int4* cta = (const int4*)P->d_pcta.p;
    const unsigned grid = (unsigned)P->pack_cta.size();
    if (grid > 0) {
      const long long nst = c->state_elems;
      const long long npb = (long long)P->plane_bytes * (f64 ? 2 : 1);
      int* bd = (int*)c->flag.p + OFM_FLAG_BOUNDS;
#define OFM_PACK(K, CH)                                                                        \
  pack_kernel<K, CH><<<grid, PK_THREADS, sm, c->stream>>>(u, cta, f, V, st, pl, c->grid.n[0],  \
                                                         c->grid.n[1], c->grid.n[2], c0, c1, \
                                                         nst, npb, bd)
      const bool ch = c->checks;
      if (kind == RK_TF32) { if (ch) OFM_PACK(RK_TF32, true); else OFM_PACK(RK_TF32, false); }
      else if (kind == RK_BF16) { if (ch) OFM_PACK(RK_BF16, true); else OFM_PACK(RK_BF16, false); }
      else if (kind == RK_F32) { if (ch) OFM_PACK(RK_F32, true); else OFM_PACK(RK_F32, false); }
      else if (kind == RK_F64) { if (ch) OFM_PACK(RK_F64, true); else OFM_PACK(RK_F64, false); }
      else { if (ch) OFM_PACK(RK_BF16X3, true); else OFM_PACK(RK_BF16X3, false); }
#undef OFM_PACK
    }
    OFM_CUDA(c, cudaGetLastError());
  }
  int* fl = (int*)c->flag.p + OFM_FLAG_TC;
  int* next = (int*)c->flag.p + OFM_FLAG_QUEUE;
  OFM_CUDA(c, cudaMemsetAsync(next, 0, sizeof(int), c->stream));
  {
    KTimer t(c, KC_CONTRACT, 1, c->region_bytes[kind], (double)c->flops);
    const int ni = (int)P->items.size();
    if (ni > 0) {
      const int grid = std::min(ni, 152);
      const RItem* it = (const RItem*)P->d_items.p;
      const RPiece* pc = (const RPiece*)P->d_pieces.p;
      const RRowSeg* rs = (const RRowSeg*)P->d_rsegs.p;
      const RColSeg* cs = (const RColSeg*)P->d_csegs.p;
      const long long* sb = (const long long*)P->d_stab.p;
      const unsigned char* pl = (const unsigned char*)P->planes.p;
      float* sl = (float*)P->slots.p;
      if (kind == RK_F32) {
        region_simt_kernel<float><<<grid, SR_THREADS, simt_smem<float>(), c->stream>>>(
            it, ni, pc, rs, cs, sb, pl, sl, next);
      } else if (kind == RK_F64) {
        region_simt_kernel<double><<<grid, SR_THREADS, simt_smem<double>(), c->stream>>>(
            it, ni, pc, rs, cs, sb, pl, (double*)P->slots.p, next);
      } else {
        const int hold = c->hold_tc;   // armed by the test hook for one launch
        const int wi = hold && c->hold_bound > 0 ? c->hold_bound : (1 << 20);
        c->hold_tc = 0;
        const long long npb = P->plane_bytes, nsl = P->slot_elems;
        int* bd = (int*)c->flag.p + OFM_FLAG_BOUNDS;
#define OFM_REGION(K, CH)                                                                     \
  region_kernel<K, CH><<<grid, RS_THREADS, RS_SMEM, c->stream>>>(it, ni, pc, rs, cs, sb, pl, sl, fl, \
                                                                 next, hold, wi, npb, nsl, bd)
        const bool ch = c->checks;
        if (kind == RK_TF32) { if (ch) OFM_REGION(RK_TF32, true); else OFM_REGION(RK_TF32, false); }
        else if (kind == RK_BF16) { if (ch) OFM_REGION(RK_BF16, true); else OFM_REGION(RK_BF16, false); }
        else { if (ch) OFM_REGION(RK_BF16X3, true); else OFM_REGION(RK_BF16X3, false); }
#undef OFM_REGION
      }
    }
    OFM_CUDA(c, cudaGetLastError());
  }
  {
    KTimer t(c, KC_FINALIZE, 1, (double)P->slot_elems * (f64 ? 8 : 4) + 16.0 * c->blk_elems);
    int nmax = 1, amax = 1;
    for (const RPair& q : P->rpairs) {
      nmax = std::max(nmax, q.nb);
      amax = std::max(amax, q.na);
    }
    const int chunks = ((amax + 31) / 32) * ((nmax + 31) / 32);   // 32 x 32 tiles of the largest block
    const dim3 fg((unsigned)P->rpairs.size(), (unsigned)chunks);
    if (!P->rpairs.empty() && f64)
      rfinalize_kernel<double><<<fg, 256, 0, c->stream>>>((const RPair*)P->d_rpairs.p,
                                                          (const double*)P->slots.p, (double*)c->blocks.p);
    else if (!P->rpairs.empty())
      rfinalize_kernel<float><<<fg, 256, 0, c->stream>>>((const RPair*)P->d_rpairs.p,
                                                         (const float*)P->slots.p, (double*)c->blocks.p);
    OFM_CUDA(c, cudaGetLastError());
  }
  c->tc_check = kind <= RK_BF16X3;
  return OFM_OK;
}

// Host statistics of the region plan (for the planner query).
void ofm_region_stats(const ofm_ctx* c, long long* out) {
  const RegionPlan* P = c->region;
  if (!P) return;
  out[0] = P->ok;
  out[1] = P->nregions;
  out[2] = P->nparts;
  out[3] = (long long)P->items.size();
  out[4] = P->plane_bytes;
  out[5] = P->slot_elems * 4;
  out[6] = (long long)P->mma_flops;
  out[7] = P->w_min;
}

extern "C" ofm_status ofm_plan_regions(const ofm_grid* grid, const ofm_fragment* frags, int n_frag,
                                       int w_min, long long* stats, long long* pair_points,
                                       int max_pairs) {
  if (!grid || !frags) return OFM_ERR_INVALID;
  std::string err;
  if (!validate_geometry(*grid, frags, n_frag, err)) return OFM_ERR_INVALID;
  std::vector<DevFrag> fr;
  long long tot = 0;
  make_frag_table(*grid, frags, n_frag, fr, tot);
  std::vector<HostPair> pairs;
  make_pairs(*grid, fr, pairs);
  std::vector<long long> off(pairs.size());
  long long blk = 0;
  for (size_t p = 0; p < pairs.size(); ++p) {
    off[p] = blk;
    blk += 2LL * fr[pairs[p].a].n * fr[pairs[p].b].n;
  }
  RegionPlan P;
  std::vector<long long> pts;
  region_plan_build(grid->n, &P, fr, pairs, off, w_min, 16LL << 30, pair_points ? &pts : nullptr);
  if (stats) {
    stats[0] = P.ok;
    stats[1] = P.nregions;
    stats[2] = P.nparts;
    stats[3] = (long long)P.items.size();
    stats[4] = P.plane_bytes;
    stats[5] = P.slot_elems * 4;
    stats[6] = (long long)P.mma_flops;
    stats[7] = P.w_min;
  }
  if (pair_points)
    for (int i = 0; i < (int)pts.size() && i < max_pairs; ++i) pair_points[i] = pts[i];
  return OFM_OK;
}
