// Pair-block contraction on the 5th-generation tensor cores (tcgen05):
//     [S_ab | H_ab] = Phi_a[R]^T [Phi_b[R] | HPhi_b[R]]   (Sec. II),
// M = n_a (padded to 128), N = 2 n_b (padded to a multiple of 16), K = |R|.
//
// The work is cut into items (pair, rows of a piece); a persistent CTA per SM
// streams its items through a warp-specialised pipeline (one thread issues
// bulk copies of the K step's point rows into a ring of raw stages; four
// warps convert them into the K-major, no-swizzle canonical operand layout
// of the MMA -- core matrices of 8 rows x 16 bytes, K-adjacent cores 128
// bytes apart, 8-row groups one K-tile apart -- as TF32 (round to nearest),
// BF16 (round to nearest even) or the BF16 pair hi = bf16(x),
// lo = bf16(x - hi); one thread issues tcgen05.mma with FP32 accumulation in
// tensor memory, hi*hi + hi*lo + lo*hi for the split (lo*lo dropped); four
// warps read the accumulator with tcgen05.ld and write the item's FP32
// partial tile).  A finalize kernel sums the partials of each pair in a
// fixed order.  Every wait is bounded: on timeout the CTA sets an error
// flag, drains its copies and MMAs, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <vector>

#include "ofm_internal.h"
#include "ptx_util.h"

using namespace ofm;
using namespace ofm::ptx;

namespace {

struct TcPair {
  int a, b;
  int item0, nitem;
  int N, Npad;          // 2 n_b and its padding to a multiple of 16
  long long blk_off;    // block arena offset (same layout as the CUDA-core path)
};

struct TcItem {
  int pair;
  int piece;
  int r0, r1;
  long long part_off;   // FP32 partial tile of n_a x N
};


// operand kinds: TF32, BF16, BF16 hi+lo, TF32 hi+lo (the last for FP32-class
// Gram matrices: hi = tf32(x), lo = tf32(x - hi), products to about 2^-22)
enum { TC_TF32 = 0, TC_BF16 = 1, TC_BF16X3 = 2, TC_TF32X3 = 3, TC_NKIND = 4 };

template <int KIND> constexpr bool is_tf32() { return KIND == TC_TF32 || KIND == TC_TF32X3; }
template <int KIND> constexpr bool is_split() { return KIND == TC_BF16X3 || KIND == TC_TF32X3; }

// ----------------------------------------------------------- PTX helpers --

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor, no swizzle: start address, leading
// (K-direction core) byte offset, stride (8-row group) byte offset,
// descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor: FP32 accumulator, A/B format (1 = BF16, 2 = TF32),
// both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t instr_desc(uint32_t fmt, uint32_t M, uint32_t N) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

template <int KIND>
__device__ __forceinline__ void mma(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                    uint32_t accum) {
  if constexpr (is_tf32<KIND>()) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
  }
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
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

__device__ __forceinline__ uint32_t f32_to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

// ----------------------------------------------------------- the kernel ---

// Fixed per plan: the largest row strides (floats), operand tile rows,
// ring sizes and tile bytes.
struct SmemLayout {
  int ldA, ldB;        // raw row strides (floats), the largest of the plan
  int Rb;              // B tile rows (largest Npad)
  int kt;              // grid points per K step (operand stage): 64, or 32 where 64 does not fit
  int raw_stage;       // bytes of one raw stage: rsteps x kt points x (ldA + 2 ldB) floats
  int nraw;            // raw stages in the ring
  int nop;             // operand stages in the ring (2..TS_NOP)
  int rsteps;          // K steps per raw stage
  int tileA, tileB;    // bytes of one operand tile
  int ntiles;          // operand tiles per operand (1, or 2 for hi+lo)
  int nitems;          // work items of the plan
};

constexpr int TS_THREADS = 448;  // warp 0 copies, 1 MMA, 2-9 convert, 10-13 epilogue
constexpr int TS_NOP = 4;        // largest operand ring
constexpr int TS_CONV = 8;       // converter warps
constexpr int TS_MAXRAW = 8;
constexpr int TS_ACC_COLS = 256; // columns of one accumulator (N <= 256); two of them

// Persistent, warp-specialised contraction: CTA c takes items c, c + grid,
// c + 2 grid, ...; every role walks the same item sequence, so a global step
// counter g indexes the rings.
//   warp 0   : its lanes issue bulk copies of the K step's point rows (a
//              contiguous x-run of a piece is contiguous in both fragments'
//              storage: one copy per run and operand, one run per lane) into
//              raw stage g % nraw;
//   warps 2-9: convert raw stage -> operand stage g % nop (canonical K-major
//              layout, TF32 / BF16 / BF16 hi+lo), zero past the item's end;
//   warp 1   : one thread issues the MMAs of the stage into the item's
//              accumulator (two in tensor memory, alternating per item) and
//              commits them to the stage's "empty" barrier, and after the
//              item's last stage to the accumulator's "full" barrier;
//   warps 10-13: read the accumulator (warp w owns lanes 32 (w % 4)..), write
//              the item's FP32 partial tile, release the accumulator.
// mbarriers: raw full (copy bytes) / empty (8 converter warps), operand
// full (8 converter warps) / empty (MMA commit), accumulator full (MMA
// commit) / empty (4 epilogue warps).  Every wait is bounded and also stops
// when another role gave up; the CTA then waits (bounded) for its copies and
// MMAs in flight, frees its tensor memory and returns.
template <int KIND, int KT>
__global__ void __launch_bounds__(TS_THREADS, 1) tc_contract_kernel(
    const DevFrag* __restrict__ fr, const TcPair* __restrict__ prs, const Piece* __restrict__ pcs,
    const TcItem* __restrict__ items, const float* __restrict__ states,
    const float* __restrict__ hphi, float* __restrict__ partials, int* flag, SmemLayout L) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) unsigned long long raw_full[TS_MAXRAW], raw_empty[TS_MAXRAW];
  __shared__ __align__(8) unsigned long long op_full[TS_NOP], op_empty[TS_NOP], acc_full[2], acc_empty[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_s, issued_s, mma_steps_s;

  constexpr int ESZ = is_tf32<KIND>() ? 4 : 2;
  constexpr int E = 16 / ESZ;                 // elements per core row
  constexpr uint32_t LBO = 128;               // K-adjacent cores
  constexpr uint32_t SBO = (KT / E) * 128;    // next 8-row group
  constexpr int KSTEPS = (KT * ESZ) / 32;     // MMAs per K step (32 bytes of K each)
  constexpr int NG = KT / E;                  // core groups along K
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nraw = L.nraw, nop = L.nop;
  const int span = L.rsteps * KT;   // points per raw stage
  unsigned char* raw = smem;
  unsigned char* ops = smem + (size_t)nraw * L.raw_stage;
  auto tileA = [&](int o, int t) {
    return ops + (size_t)o * L.ntiles * (L.tileA + L.tileB) + (size_t)t * L.tileA;
  };
  auto tileB = [&](int o, int t) {
    return ops + (size_t)o * L.ntiles * (L.tileA + L.tileB) + (size_t)L.ntiles * L.tileA +
           (size_t)t * L.tileB;
  };

  if (tid == 0) {
    for (int i = 0; i < nraw; ++i) {
      mbar_init(smem_u32(&raw_full[i]), 1);
      mbar_init(smem_u32(&raw_empty[i]), TS_CONV);
    }
    for (int i = 0; i < L.nop; ++i) {
      mbar_init(smem_u32(&op_full[i]), TS_CONV);
      mbar_init(smem_u32(&op_empty[i]), 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(smem_u32(&acc_full[i]), 1);
      mbar_init(smem_u32(&acc_empty[i]), 4);
    }
    fence_mbar_init();
    abort_s = 0;
    issued_s = 0;
    mma_steps_s = 0;
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(2 * TS_ACC_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  // bounded wait that also ends when another role gave up
  auto wait = [&](unsigned long long* bar, uint32_t parity) -> bool {
    const uint32_t a = smem_u32(bar);
    for (int i = 0; i < (1 << 20); ++i) {
      if (mbar_try(a, parity)) return true;
      if (*(volatile int*)&abort_s) return false;
    }
    atomicExch(flag, 1);
    *(volatile int*)&abort_s = 1;
    return false;
  };
  const int nitems = L.nitems;

  if (warp == 0) {
    // ------------------------------------------------------------ copies
    // one raw stage holds `span` points of the item (rsteps K steps); lane j
    // issues the copies of runs j, j + 32, ...: run 0 starts at the stage's
    // first point, run i > 0 at the start of the i-th following row
    int gr = 0;
    bool ok = true;
    for (int ii = blockIdx.x; ii < nitems && ok; ii += gridDim.x) {
      const TcItem it = items[ii];
      const TcPair pr = prs[it.pair];
      const DevFrag A = fr[pr.a], B = fr[pr.b];
      const Piece pc = pcs[it.piece];
      const int lenx = pc.len[0], leny = pc.len[1];
      const int npts = (it.r1 - it.r0) * lenx;
      for (int k0 = 0; k0 < npts; k0 += span, ++gr) {
        const int s = gr % nraw, u = gr / nraw;
        if (u > 0) {   // lane 0 waits; the outcome is the warp's (uniform control flow)
          bool w = true;
          if (lane == 0) w = wait(&raw_empty[s], (uint32_t)((u - 1) & 1));
          ok = __shfl_sync(0xffffffffu, w ? 1 : 0, 0) != 0;
          if (!ok) break;
        }
        const int nk = min(span, npts - k0);
        const uint32_t mb = smem_u32(&raw_full[s]);
        if (lane == 0) mbar_arrive_expect(mb, (uint32_t)(nk * (A.ld + 2 * B.ld) * 4));
        __syncwarp();
        const int row0 = k0 / lenx, x0 = k0 - row0 * lenx;
        const int nruns = (k0 + nk - 1) / lenx - row0 + 1;   // <= span
        unsigned char* rA = raw + (size_t)s * L.raw_stage;
        unsigned char* rB = rA + (size_t)span * L.ldA * 4;
        unsigned char* rH = rB + (size_t)span * L.ldB * 4;
        for (int j = lane; j < nruns; j += 32) {
          const int x = j == 0 ? x0 : 0;
          const int kstart = j == 0 ? k0 : (row0 + j) * lenx;
          const int run = min(lenx - x, k0 + nk - kstart);
          const int r = it.r0 + row0 + j;
          const int y = r % leny, z = r / leny;
          const long long pa =
              ((long long)(pc.la[2] + z) * A.dext[1] + (pc.la[1] + y)) * A.dext[0] + pc.la[0] + x;
          const long long pb =
              ((long long)(pc.lb[2] + z) * B.dext[1] + (pc.lb[1] + y)) * B.dext[0] + pc.lb[0] + x;
          const int kk = kstart - k0;
          bulk_g2s(smem_u32(rA + (size_t)kk * A.ld * 4), states + A.off + pa * A.ld,
                   (uint32_t)(run * A.ld * 4), mb);
          bulk_g2s(smem_u32(rB + (size_t)kk * B.ld * 4), states + B.off + pb * B.ld,
                   (uint32_t)(run * B.ld * 4), mb);
          bulk_g2s(smem_u32(rH + (size_t)kk * B.ld * 4), hphi + B.off + pb * B.ld,
                   (uint32_t)(run * B.ld * 4), mb);
        }
        if (lane == 0) *(volatile int*)&issued_s = gr + 1;
      }
    }
  } else if (warp == 1) {
    // -------------------------------------------------------------- MMAs
    if (lane == 0) {
      constexpr uint32_t FMT = is_tf32<KIND>() ? 2u : 1u;
      int g = 0, item_no = 0;
      bool ok = true;
      for (int ii = blockIdx.x; ii < nitems && ok; ii += gridDim.x, ++item_no) {
        const TcItem it = items[ii];
        const TcPair pr = prs[it.pair];
        const Piece pc = pcs[it.piece];
        const int npts = (it.r1 - it.r0) * pc.len[0];
        const int b = item_no & 1, ub = item_no >> 1;
        if (ub > 0 && !(ok = wait(&acc_empty[b], (uint32_t)((ub - 1) & 1)))) break;
        tc_fence_after();
        const uint32_t idesc = instr_desc(FMT, 128, (uint32_t)pr.Npad);
        const uint32_t dacc = tmem + (uint32_t)(b * TS_ACC_COLS);
        for (int k0 = 0; k0 < npts; k0 += KT, ++g) {
          const int o = g % nop, uo = g / nop;
          if (!(ok = wait(&op_full[o], (uint32_t)(uo & 1)))) break;
          tc_fence_after();
          // descriptors of the stage's tiles; a K sub-step advances the
          // start address by two core matrices (the field holds address >> 4)
          const uint64_t ah0 = smem_desc(smem_u32(tileA(o, 0)), LBO, SBO);
          const uint64_t bh0 = smem_desc(smem_u32(tileB(o, 0)), LBO, SBO);
          uint64_t al0 = 0, bl0 = 0;
          if constexpr (is_split<KIND>()) {
            al0 = smem_desc(smem_u32(tileA(o, 1)), LBO, SBO);
            bl0 = smem_desc(smem_u32(tileB(o, 1)), LBO, SBO);
          }
#pragma unroll
          for (int ks = 0; ks < KSTEPS; ++ks) {
            const uint64_t off = (uint64_t)((ks * 2 * LBO) >> 4);
            mma<KIND>(dacc, ah0 + off, bh0 + off, idesc, (k0 > 0 || ks > 0) ? 1u : 0u);
            if constexpr (is_split<KIND>()) {
              mma<KIND>(dacc, ah0 + off, bl0 + off, idesc, 1u);
              mma<KIND>(dacc, al0 + off, bh0 + off, idesc, 1u);
            }
          }
          mma_commit(smem_u32(&op_empty[o]));
          *(volatile int*)&mma_steps_s = g + 1;
        }
        if (!ok) break;
        mma_commit(smem_u32(&acc_full[b]));
      }
    }
  } else if (warp < 2 + TS_CONV) {
    // -------------------------------------------------------- conversion
    const int ct = tid - 64;   // 0 .. 32 TS_CONV - 1
    int gr = 0, go = 0;
    bool ok = true;
    for (int ii = blockIdx.x; ii < nitems && ok; ii += gridDim.x) {
      const TcItem it = items[ii];
      const TcPair pr = prs[it.pair];
      const DevFrag A = fr[pr.a], B = fr[pr.b];
      const Piece pc = pcs[it.piece];
      const int npts = (it.r1 - it.r0) * pc.len[0];
      const int N = pr.N;
      // e -> (row, k group) without integer division: e / rows from a float
      // reciprocal, corrected by one (exact for e < 2^24)
      const float inv_a = 1.0f / (float)A.n, inv_n = 1.0f / (float)N;
      for (int k0 = 0; k0 < npts && ok; k0 += span, ++gr) {
        const int s = gr % nraw, u = gr / nraw;
        // every lane waits (it reads the copied data); the outcome is the warp's
        ok = __all_sync(0xffffffffu, wait(&raw_full[s], (uint32_t)(u & 1)));
        if (!ok) break;
        const int nkr = min(span, npts - k0);
        const float* rA = reinterpret_cast<const float*>(raw + (size_t)s * L.raw_stage);
        const float* rB = rA + (size_t)span * L.ldA;
        const float* rH = rB + (size_t)span * L.ldB;
        for (int j0 = 0; j0 < nkr; j0 += KT, ++go) {
          const int o = go % nop, uo = go / nop;
          if (uo > 0) {
            ok = __all_sync(0xffffffffu, wait(&op_empty[o], (uint32_t)((uo - 1) & 1)));
            if (!ok) break;
          }
          const int nk = min(KT, nkr - j0);
          // operand rows: A = states of fragment a; B = columns 0..n_b-1 from
          // Phi_b, n_b..2n_b-1 from H Phi_b
          for (int e = ct; e < (A.n + N) * NG; e += 32 * TS_CONV) {
            const bool isA = e < A.n * NG;
            const int e2 = isA ? e : e - A.n * NG;
            const int rows = isA ? A.n : N;
            int gq = (int)((float)e2 * (isA ? inv_a : inv_n));
            if (gq * rows > e2) --gq;
            else if ((gq + 1) * rows <= e2) ++gq;
            const int row = e2 - gq * rows;
            const float* src;
            int col, ld;
            if (isA) {
              src = rA;
              col = row;
              ld = A.ld;
            } else {
              const bool h = row >= B.n;
              src = h ? rH : rB;
              col = h ? row - B.n : row;
              ld = B.ld;
            }
            src += (size_t)j0 * ld + col;
            float v[E];
#pragma unroll
            for (int j = 0; j < E; ++j) {
              const int kk = gq * E + j;
              v[j] = kk < nk ? src[kk * ld] : 0.f;
            }
            const size_t off = (size_t)(row >> 3) * SBO + (size_t)gq * LBO + (size_t)(row & 7) * 16;
            unsigned char* t0 = isA ? tileA(o, 0) : tileB(o, 0);
            if constexpr (is_tf32<KIND>()) {
              uint32_t hi[4];
#pragma unroll
              for (int j = 0; j < 4; ++j) hi[j] = f32_to_tf32(v[j]);
              *reinterpret_cast<uint4*>(t0 + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
              if constexpr (KIND == TC_TF32X3) {
                uint32_t lo[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) lo[j] = f32_to_tf32(v[j] - __uint_as_float(hi[j]));
                unsigned char* t1 = isA ? tileA(o, 1) : tileB(o, 1);
                *reinterpret_cast<uint4*>(t1 + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
              }
            } else {
              uint32_t hi[4], lo[4];
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                hi[j] = pack_bf16(v[2 * j], v[2 * j + 1]);
                if constexpr (KIND == TC_BF16X3) {
                  __nv_bfloat162 hh = *reinterpret_cast<__nv_bfloat162*>(&hi[j]);
                  const float2 hf = __bfloat1622float2(hh);
                  lo[j] = pack_bf16(v[2 * j] - hf.x, v[2 * j + 1] - hf.y);
                }
              }
              *reinterpret_cast<uint4*>(t0 + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
              if constexpr (KIND == TC_BF16X3) {
                unsigned char* t1 = isA ? tileA(o, 1) : tileB(o, 1);
                *reinterpret_cast<uint4*>(t1 + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
              }
            }
          }
          fence_async_smem();   // generic-proxy writes -> tensor-core reads
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_u32(&op_full[o]));
        }
        if (!ok) break;
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&raw_empty[s]));   // every K step of the stage read
      }
    }
  } else {
    // ---------------------------------------------------------- epilogue
    const int q = warp & 3;   // tensor-memory lane quadrant of this warp
    int item_no = 0;
    bool ok = true;
    for (int ii = blockIdx.x; ii < nitems && ok; ii += gridDim.x, ++item_no) {
      const TcItem it = items[ii];
      const TcPair pr = prs[it.pair];
      const int na = fr[pr.a].n, N = pr.N, Npad = pr.Npad;
      const int b = item_no & 1, ub = item_no >> 1;
      ok = __all_sync(0xffffffffu, wait(&acc_full[b], (uint32_t)(ub & 1)));
      if (!ok) break;
      tc_fence_after();
      float* out = partials + it.part_off;
      const int row = q * 32 + lane;
      for (int c0 = 0; c0 < Npad; c0 += 8) {
        float v[8];
        tmem_ld8(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * TS_ACC_COLS + c0), v);
        if (row < na) {
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (c0 + j < N) out[(long long)row * N + c0 + j] = v[j];
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&acc_empty[b]));
    }
  }

  __syncthreads();
  if (abort_s && tid == 0) {
    // drain before the shared and tensor memory are released: the copies of
    // the last issued stages and the MMAs of the last committed stage
    auto drain = [&](unsigned long long* bar, uint32_t parity) {
      const uint32_t a = smem_u32(bar);
      for (int i = 0; i < (1 << 24) && !mbar_test(a, parity); ++i)
        if (i > 64) __nanosleep(64);
    };
    const int issued = issued_s;
    for (int g = max(0, issued - nraw); g < issued; ++g)
      drain(&raw_full[g % nraw], (uint32_t)((g / nraw) & 1));
    const int ms = mma_steps_s;
    if (ms > 0) drain(&op_empty[(ms - 1) % nop], (uint32_t)(((ms - 1) / nop) & 1));
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(2 * TS_ACC_COLS)
                 : "memory");
}

// Sum of the partial tiles of each pair in plan order -> FP64 blocks
// (H_ab then S_ab, n_a x n_b row-major); diagonal blocks symmetrised.
__global__ void tc_finalize_kernel(const DevFrag* __restrict__ fr, const TcPair* __restrict__ prs,
                                   const TcItem* __restrict__ items,
                                   const float* __restrict__ partials, double* __restrict__ blocks) {
  const TcPair pr = prs[blockIdx.x];
  const int na = fr[pr.a].n, nb = fr[pr.b].n, N = pr.N;
  double* Hblk = blocks + pr.blk_off;
  double* Sblk = Hblk + (long long)na * nb;
  auto sum = [&](int i, int c) {
    double s = 0.0;
    for (int k = 0; k < pr.nitem; ++k) s += (double)partials[items[pr.item0 + k].part_off + (long long)i * N + c];
    return s;
  };
  // blockIdx.y: a chunk of outputs (the FP64 sums spread over many SMs)
  for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < na * nb; e += gridDim.y * blockDim.x) {
    const int i = e / nb, m = e % nb;
    double s = sum(i, m), h = sum(i, nb + m);
    if (pr.a == pr.b) {
      s = 0.5 * (s + sum(m, i));
      h = 0.5 * (h + sum(m, nb + i));
    }
    Sblk[e] = s;
    Hblk[e] = h;
  }
}

}  // namespace

struct TcPlan {
  std::vector<TcPair> pairs;
  std::vector<TcItem> items;
  std::vector<Piece> pieces;
  long long part_elems = 0;
  SmemLayout lay[TC_NKIND];
  size_t smem[TC_NKIND] = {0, 0, 0, 0};
  DevBuf d_pairs, d_items, d_pieces, partials;
  bool ok = false;
  std::string why;
};

void ofm_tc_guards(const TcPlan* t, std::vector<GuardRef>& out) {
  if (!t) return;
  const struct { const DevBuf* b; const char* n; } bufs[] = {
      {&t->d_pairs, "tensor-core pairs"}, {&t->d_items, "tensor-core items"},
      {&t->d_pieces, "tensor-core pieces"}, {&t->partials, "tensor-core partials"}};
  for (const auto& x : bufs)
    if (x.b->p) out.push_back({x.b->p, x.b->cap, x.n});
}

void ofm_tc_plan_free(TcPlan* t) {
  if (!t) return;
  DevBuf* bufs[] = {&t->d_pairs, &t->d_items, &t->d_pieces, &t->partials};
  for (DevBuf* b : bufs)
    if (b->p) cudaFree(b->p);
  delete t;
}

void ofm_tc_free(ofm_ctx* c) {
  ofm_tc_plan_free(c->tc);
  c->tc = nullptr;
}

bool ofm_tc_plan_ok(const TcPlan* t, int kind) {
  return t && t->ok && kind >= 0 && kind < TC_NKIND && t->lay[kind].nraw >= 2;
}

template <int KIND, int KTT>
static void set_smem_attr() {
  cudaFuncSetAttribute(tc_contract_kernel<KIND, KTT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       216 * 1024);
}

// Tensor-core plan for the pairs over the fragment table fr (FP32 storage,
// row strides fr[].ld): one item per row chunk of a piece, chunks of about
// `chunk` points (0: sized for about four items per SM); blk_off[p] is pair
// p's offset in the FP64 block
// arena.  The plan is marked not usable (with the reason) when a fragment
// has more than 128 states or the staging does not fit shared memory.
ofm_status ofm_tc_plan_build(ofm_ctx* c, TcPlan** tp, const std::vector<DevFrag>& fr,
                             const std::vector<HostPair>& prs, const std::vector<long long>& blk_off,
                             long long kh, long long chunk) {
  if (!*tp) *tp = new TcPlan();
  TcPlan* t = *tp;
  t->pairs.clear();
  t->items.clear();
  t->pieces.clear();
  t->part_elems = 0;
  t->ok = false;
  int ldA = 4, ldB = 4, Rb = 16;
  for (const HostPair& hp : prs) {
    const DevFrag& A = fr[hp.a];
    const DevFrag& B = fr[hp.b];
    if (A.n > 128 || 2 * B.n > 256) {
      t->why = "tensor-core contraction supports at most 128 states per fragment";
      return OFM_OK;
    }
    ldA = std::max(ldA, A.ld);
    ldB = std::max(ldB, B.ld);
    Rb = std::max(Rb, (2 * B.n + 15) / 16 * 16);
  }
  const long long target = chunk > 0 ? chunk : std::max<long long>(1024, kh / (4 * 152));
  for (size_t p = 0; p < prs.size(); ++p) {
    const HostPair& hp = prs[p];
    const DevFrag& B = fr[hp.b];
    TcPair tq;
    tq.a = hp.a;
    tq.b = hp.b;
    tq.N = 2 * B.n;
    tq.Npad = (tq.N + 15) / 16 * 16;
    tq.blk_off = blk_off[p];
    tq.item0 = (int)t->items.size();
    for (const Piece& pc : hp.pieces) {
      const int pid = (int)t->pieces.size();
      t->pieces.push_back(pc);
      const int rows = pc.len[1] * pc.len[2];
      const int per = (int)std::max<long long>(1, target / pc.len[0]);
      for (int r0 = 0; r0 < rows; r0 += per) {
        TcItem it;
        it.pair = (int)p;
        it.piece = pid;
        it.r0 = r0;
        it.r1 = std::min(rows, r0 + per);
        it.part_off = t->part_elems;
        t->part_elems += (long long)fr[hp.a].n * tq.N;
        t->items.push_back(it);
      }
    }
    tq.nitem = (int)t->items.size() - tq.item0;
    t->pairs.push_back(tq);
  }
  for (int k = 0; k < TC_NKIND; ++k) {
    SmemLayout& L = t->lay[k];
    L.ldA = ldA;
    L.ldB = ldB;
    L.Rb = Rb;
    const int esz = (k == TC_TF32 || k == TC_TF32X3) ? 4 : 2;
    L.ntiles = (k == TC_BF16X3 || k == TC_TF32X3) ? 2 : 1;
    L.nitems = (int)t->items.size();
    // the longest K step, then the largest raw stages (fewest per-stage
    // costs), then the deepest operand ring, that leave two raw stages
    const long long budget = 216 * 1024;
    L.nraw = 0;
    for (L.kt = 64; L.kt >= 32 && L.nraw < 2; L.kt /= 2) {
      L.tileA = (128 * L.kt * esz + 1023) / 1024 * 1024;
      L.tileB = (Rb * L.kt * esz + 1023) / 1024 * 1024;
      for (L.rsteps = 128 / L.kt; L.rsteps >= 1; L.rsteps /= 2) {
        L.raw_stage = (L.rsteps * L.kt * (ldA + 2 * ldB) * 4 + 1023) / 1024 * 1024;
        for (L.nop = TS_NOP; L.nop >= 2; --L.nop) {
          const long long ops = (long long)L.nop * L.ntiles * (L.tileA + L.tileB);
          L.nraw = (int)std::min<long long>(TS_MAXRAW, (budget - ops) / L.raw_stage);
          if (L.nraw >= 2) break;
        }
        if (L.nraw >= 2) break;
      }
      if (L.nraw >= 2) break;
    }
    // a kind whose staging does not fit stays unusable (nraw < 2); the others run
    t->smem[k] = L.nraw >= 2 ? (size_t)L.nraw * L.raw_stage + (size_t)L.nop * L.ntiles * (L.tileA + L.tileB) : 0;
  }
  OFM_TRY(ofm_ensure(c, t->d_pairs, sizeof(TcPair) * std::max<size_t>(1, t->pairs.size()), "tc pairs"));
  OFM_TRY(ofm_ensure(c, t->d_items, sizeof(TcItem) * std::max<size_t>(1, t->items.size()), "tc items"));
  OFM_TRY(ofm_ensure(c, t->d_pieces, sizeof(Piece) * std::max<size_t>(1, t->pieces.size()), "tc pieces"));
  OFM_TRY(ofm_ensure(c, t->partials, sizeof(float) * std::max<long long>(1, t->part_elems), "tc partials"));
  OFM_CUDA(c, cudaMemcpyAsync(t->d_pairs.p, t->pairs.data(), sizeof(TcPair) * t->pairs.size(), cudaMemcpyHostToDevice, c->stream));
  OFM_CUDA(c, cudaMemcpyAsync(t->d_items.p, t->items.data(), sizeof(TcItem) * t->items.size(), cudaMemcpyHostToDevice, c->stream));
  OFM_CUDA(c, cudaMemcpyAsync(t->d_pieces.p, t->pieces.data(), sizeof(Piece) * t->pieces.size(), cudaMemcpyHostToDevice, c->stream));
  static bool attr = false;   // the kernels' shared-memory limit, once per process
  if (!attr) {
    set_smem_attr<TC_TF32, 32>();
    set_smem_attr<TC_BF16, 32>();
    set_smem_attr<TC_BF16X3, 32>();
    set_smem_attr<TC_TF32X3, 32>();
    set_smem_attr<TC_TF32, 64>();
    set_smem_attr<TC_BF16, 64>();
    set_smem_attr<TC_BF16X3, 64>();
    set_smem_attr<TC_TF32X3, 64>();
    OFM_CUDA(c, cudaGetLastError());
    attr = true;
  }
  t->ok = true;
  return OFM_OK;
}

// Plan of the pair contraction after a build.
ofm_status ofm_plan_extra(ofm_ctx* c) {
  if (c->storage != OFM_STORE_FP32) {
    if (!c->tc) c->tc = new TcPlan();
    c->tc->ok = false;
    c->tc->why = "tensor-core contraction needs FP32 storage";
    return OFM_OK;
  }
  std::vector<long long> off(c->pairs.size());
  for (size_t p = 0; p < c->pairs.size(); ++p) off[p] = c->simt_pairs[p].blk_off;
  return ofm_tc_plan_build(c, &c->tc, c->frags, c->pairs, off, c->kh, c->asm_chunk);
}

template <int KIND>
static void launch_kind(const TcPlan* t, int kt, int grid, size_t sm, cudaStream_t s,
                        const DevFrag* fr, const float* st, const float* hp, int* fl) {
  const SmemLayout& L = t->lay[KIND];
  const TcPair* pr = (const TcPair*)t->d_pairs.p;
  const Piece* pc = (const Piece*)t->d_pieces.p;
  const TcItem* itm = (const TcItem*)t->d_items.p;
  float* part = (float*)t->partials.p;
  if (kt == 64)
    tc_contract_kernel<KIND, 64><<<grid, TS_THREADS, sm, s>>>(fr, pr, pc, itm, st, hp, part, fl, L);
  else
    tc_contract_kernel<KIND, 32><<<grid, TS_THREADS, sm, s>>>(fr, pr, pc, itm, st, hp, part, fl, L);
}

// Runs a plan: contraction into FP32 partials, then the fixed-order sum into
// the FP64 block arena.  kind: TC_TF32 .. TC_TF32X3.
ofm_status ofm_tc_run(ofm_ctx* c, TcPlan* t, int kind, const DevFrag* d_frags, const void* states,
                      const void* hphi, double* blocks, int kclass_contract, int kclass_finalize,
                      double bytes, double flops) {
  if (!t || !t->ok) return ofm_fail(c, OFM_ERR_INVALID, t ? t->why : "no tensor-core plan");
  if (!ofm_tc_plan_ok(t, kind))
    return ofm_fail(c, OFM_ERR_INVALID, "tensor-core staging does not fit shared memory for these state counts");
  const int nit = (int)t->items.size();
  int* fl = (int*)c->flag.p + OFM_FLAG_TC;
  {
    KTimer kt(c, kclass_contract, 1, bytes, flops);
    if (nit > 0) {
      const int grid = std::min(nit, 152);   // one persistent CTA per SM
      const int ktl = t->lay[kind].kt;
      const size_t sm = t->smem[kind];
      const float* st = (const float*)states;
      const float* hp = (const float*)hphi;
      if (kind == TC_TF32) launch_kind<TC_TF32>(t, ktl, grid, sm, c->stream, d_frags, st, hp, fl);
      else if (kind == TC_BF16) launch_kind<TC_BF16>(t, ktl, grid, sm, c->stream, d_frags, st, hp, fl);
      else if (kind == TC_BF16X3) launch_kind<TC_BF16X3>(t, ktl, grid, sm, c->stream, d_frags, st, hp, fl);
      else launch_kind<TC_TF32X3>(t, ktl, grid, sm, c->stream, d_frags, st, hp, fl);
    }
    OFM_CUDA(c, cudaGetLastError());
  }
  {
    KTimer kt(c, kclass_finalize, 1, (double)t->part_elems * 4);
    // enough output chunks for the largest block (n_a <= 128, n_b = N / 2)
    int nmax = 1;
    for (const TcPair& q : t->pairs) nmax = std::max(nmax, q.N / 2);
    const int chunks = std::max(1, (128 * nmax + 255) / 256);
    if (!t->pairs.empty())
      tc_finalize_kernel<<<dim3((int)t->pairs.size(), chunks), 256, 0, c->stream>>>(
          d_frags, (const TcPair*)t->d_pairs.p, (const TcItem*)t->d_items.p,
          (const float*)t->partials.p, blocks);
    OFM_CUDA(c, cudaGetLastError());
  }
  c->tc_check = true;
  return OFM_OK;
}

ofm_status ofm_contract_tc(ofm_ctx* c, ofm_precision prec) {
  const int kind = prec == OFM_PREC_TF32 ? TC_TF32 : prec == OFM_PREC_BF16 ? TC_BF16 : TC_BF16X3;
  return ofm_tc_run(c, c->tc, kind, (const DevFrag*)c->d_frags.p, c->states.p, c->hphi.p,
                    (double*)c->blocks.p, KC_CONTRACT, KC_FINALIZE, c->contract_bytes, (double)c->flops);
}

// Reports a bounded-wait timeout of an earlier tensor-core or staged-stencil
// launch (each sets its flag word; the flags are read once and cleared).
ofm_status ofm_wait_status(ofm_ctx* c) {
  if (c->fault_due) {
    c->fault_due = false;
    c->tc_check = c->stencil_check = false;
    return ofm_fail(c, OFM_ERR_TIMEOUT, "a bounded device wait exceeded its bound (injected by OFM_FAULT=timeout)");
  }
  if (c->tc_check) {
    int h = 0;
    int* f = (int*)c->flag.p + OFM_FLAG_TC;
    OFM_CUDA(c, cudaMemcpyAsync(&h, f, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    OFM_CUDA(c, cudaStreamSynchronize(c->stream));
    c->tc_check = false;
    if (h) {
      cudaMemsetAsync(f, 0, sizeof(int), c->stream);
      return ofm_fail(c, OFM_ERR_TIMEOUT, "tensor-core contraction: an mbarrier wait exceeded its bound");
    }
  }
  if (c->stencil_check) {
    int h = 0;
    int* f = (int*)c->flag.p + OFM_FLAG_STENCIL;
    OFM_CUDA(c, cudaMemcpyAsync(&h, f, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    OFM_CUDA(c, cudaStreamSynchronize(c->stream));
    c->stencil_check = false;
    if (h) {
      cudaMemsetAsync(f, 0, sizeof(int), c->stream);
      return ofm_fail(c, OFM_ERR_TIMEOUT, "stencil: a staged-plane wait exceeded its bound");
    }
  }
  return OFM_OK;
}

