// Pair-block contraction on the 5th-generation tensor cores (tcgen05):
//     [S_ab | H_ab] = Phi_a[R]^T [Phi_b[R] | HPhi_b[R]]   (Sec. II),
// M = n_a (padded to 128), N = 2 n_b (padded to a multiple of 16), K = |R|.
//
// One CTA (4 warps) per work item = (pair, rows [r0, r1) of a piece).  Per
// K step of 32 grid points:
//   1. cp.async brings the FP32 rows (states of a point are contiguous) of
//      the 32 points into a raw staging buffer (two stages in flight);
//   2. the CTA converts the raw rows into the operand tiles in the
//      K-major, no-swizzle canonical layout of the MMA (core matrices of
//      8 rows x 16 bytes, K-adjacent cores 128 bytes apart, 8-row groups
//      one K-tile apart): TF32 (round to nearest), BF16 (round to nearest
//      even), or the BF16 pair hi = bf16(x), lo = bf16(x - hi);
//   3. one thread issues tcgen05.mma (kind::tf32 or kind::f16 with bf16
//      operands, FP32 accumulation in tensor memory); the hi+lo split issues
//      hi*hi + hi*lo + lo*hi into the same accumulator (lo*lo dropped);
//      tcgen05.commit arrives on the stage's mbarrier when the MMAs finish,
//      which frees that operand stage for the step after next.
// The epilogue reads the accumulator with tcgen05.ld (warp w owns TMEM
// lanes 32w..32w+31 = rows of the tile) and writes an FP32 partial tile;
// a finalize kernel sums the partials of each pair in a fixed order.
// Every wait is bounded: on timeout the CTA sets an error flag, drains its
// copies, frees its tensor memory and returns.
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

constexpr int KT = 32;          // grid points per K step
constexpr int TC_THREADS = 128;
constexpr int TILE_PAD = 2048;  // slack after every operand tile (bytes)

enum { TC_TF32 = 0, TC_BF16 = 1, TC_BF16X3 = 2 };

// ----------------------------------------------------------- PTX helpers --

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void* g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

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
  if constexpr (KIND == TC_TF32) {
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

struct SmemLayout {
  int ldA, ldB;        // raw row strides (floats), the largest of the plan
  int Rb;              // B tile rows (largest Npad)
  int raw_stage;       // bytes of one raw stage
  int tileA, tileB;    // bytes of one operand tile (+ slack)
  int ntiles;          // operand tiles per operand (1, or 2 for hi+lo)
};

template <int KIND>
__global__ void __launch_bounds__(TC_THREADS) tc_contract_kernel(
    const DevFrag* __restrict__ fr, const TcPair* __restrict__ prs, const Piece* __restrict__ pcs,
    const TcItem* __restrict__ items, const float* __restrict__ states,
    const float* __restrict__ hphi, float* __restrict__ partials, int* flag, SmemLayout L) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) unsigned long long mbar[2];
  __shared__ uint32_t tmem_slot;

  const TcItem it = items[blockIdx.x];
  const TcPair pr = prs[it.pair];
  const DevFrag A = fr[pr.a];
  const DevFrag B = fr[pr.b];
  const Piece pc = pcs[it.piece];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int lenx = pc.len[0], leny = pc.len[1];
  const int npts = (it.r1 - it.r0) * lenx;
  const int niter = (npts + KT - 1) / KT;
  const int N = pr.N, Npad = pr.Npad;
  constexpr int ESZ = (KIND == TC_TF32) ? 4 : 2;
  constexpr int E = 16 / ESZ;                 // elements per core row
  constexpr uint32_t LBO = 128;               // K-adjacent cores
  constexpr uint32_t SBO = (KT / E) * 128;    // next 8-row group
  constexpr int KSTEPS = (KT * ESZ) / 32;     // MMAs per K step (32 bytes of K each)

  float* raw = reinterpret_cast<float*>(smem);
  unsigned char* ops = smem + 2 * L.raw_stage;
  // operand tile t of stage s: A tiles first, then B tiles
  auto tileA = [&](int s, int t) { return ops + (size_t)s * L.ntiles * (L.tileA + L.tileB) + (size_t)t * L.tileA; };
  auto tileB = [&](int s, int t) {
    return ops + (size_t)s * L.ntiles * (L.tileA + L.tileB) + (size_t)L.ntiles * L.tileA + (size_t)t * L.tileB;
  };

  // zero every operand tile once: padding rows stay zero afterwards
  {
    const int total = 2 * L.ntiles * (L.tileA + L.tileB);
    uint4* p = reinterpret_cast<uint4*>(ops);
    for (int i = tid; i < total / 16; i += TC_THREADS) p[i] = make_uint4(0, 0, 0, 0);
  }
  if (tid == 0) {
    mbar_init(smem_u32(&mbar[0]), 1);
    mbar_init(smem_u32(&mbar[1]), 1);
    fence_mbar_init();
  }
  // tensor memory: one column per accumulator column (power of two >= 32)
  uint32_t ncols = 32;
  while ((int)ncols < Npad) ncols <<= 1;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  fence_async_smem();

  const float* Pa = states + A.off;
  const float* Pb = states + B.off;
  const float* Hb = hphi + B.off;
  const int qa = A.ld / 4, qb = B.ld / 4;           // 16-byte chunks per row
  const int per_pt = qa + 2 * qb;
  float* rawA0 = raw;                               // [KT][ldA]
  const int rawAB = KT * L.ldA;                     // floats

  // issue the cp.async copies of K step `step` into raw stage s
  auto load_stage = [&](int step, int s) {
    float* base = raw + (size_t)s * (L.raw_stage / 4);
    float* rA = base;
    float* rB = base + rawAB;
    float* rH = rB + KT * L.ldB;
    for (int c = tid; c < KT * per_pt; c += TC_THREADS) {
      const int kk = c / per_pt, q = c - kk * per_pt;
      const int k = step * KT + kk;
      float* dst;
      const float* src = nullptr;
      if (q < qa) dst = rA + kk * L.ldA + 4 * q;
      else if (q < qa + qb) dst = rB + kk * L.ldB + 4 * (q - qa);
      else dst = rH + kk * L.ldB + 4 * (q - qa - qb);
      if (k < npts) {
        const int r = it.r0 + k / lenx, x = k - (k / lenx) * lenx;
        const int y = r % leny, z = r / leny;
        if (q < qa) {
          const long long pa = ((long long)(pc.la[2] + z) * A.dext[1] + (pc.la[1] + y)) * A.dext[0] + pc.la[0] + x;
          src = Pa + pa * A.ld + 4 * q;
        } else {
          const long long pb = ((long long)(pc.lb[2] + z) * B.dext[1] + (pc.lb[1] + y)) * B.dext[0] + pc.lb[0] + x;
          src = (q < qa + qb) ? (Pb + pb * B.ld + 4 * (q - qa)) : (Hb + pb * B.ld + 4 * (q - qa - qb));
        }
        cp_async16(smem_u32(dst), src);
      } else {
        *reinterpret_cast<float4*>(dst) = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    cp_async_commit();
  };

  // raw stage s -> operand tiles of stage s
  auto convert_stage = [&](int s) {
    const float* base = raw + (size_t)s * (L.raw_stage / 4);
    const float* rA = base;
    const float* rB = base + rawAB;
    const float* rH = rB + KT * L.ldB;
    // A rows = states of fragment a (rows >= n_a stay zero)
    for (int row = tid; row < A.n; row += TC_THREADS) {
      for (int g = 0; g < KT / E; ++g) {
        const size_t off = (size_t)(row >> 3) * SBO + (size_t)g * LBO + (size_t)(row & 7) * 16;
        float v[E];
#pragma unroll
        for (int j = 0; j < E; ++j) v[j] = rA[(g * E + j) * L.ldA + row];
        if constexpr (KIND == TC_TF32) {
          uint4 w = make_uint4(f32_to_tf32(v[0]), f32_to_tf32(v[1]), f32_to_tf32(v[2]), f32_to_tf32(v[3]));
          *reinterpret_cast<uint4*>(tileA(s, 0) + off) = w;
        } else {
          uint32_t hi[4], lo[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            hi[j] = pack_bf16(v[2 * j], v[2 * j + 1]);
            if constexpr (KIND == TC_BF16X3) {
              __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&hi[j]);
              const float2 hf = __bfloat1622float2(h);
              lo[j] = pack_bf16(v[2 * j] - hf.x, v[2 * j + 1] - hf.y);
            }
          }
          *reinterpret_cast<uint4*>(tileA(s, 0) + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
          if constexpr (KIND == TC_BF16X3)
            *reinterpret_cast<uint4*>(tileA(s, 1) + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
      }
    }
    // B rows: columns 0..n_b-1 from Phi_b, n_b..2n_b-1 from H Phi_b
    for (int row = tid; row < N; row += TC_THREADS) {
      const bool h = row >= B.n;
      const float* src = h ? rH : rB;
      const int col = h ? row - B.n : row;
      for (int g = 0; g < KT / E; ++g) {
        const size_t off = (size_t)(row >> 3) * SBO + (size_t)g * LBO + (size_t)(row & 7) * 16;
        float v[E];
#pragma unroll
        for (int j = 0; j < E; ++j) v[j] = src[(g * E + j) * L.ldB + col];
        if constexpr (KIND == TC_TF32) {
          uint4 w = make_uint4(f32_to_tf32(v[0]), f32_to_tf32(v[1]), f32_to_tf32(v[2]), f32_to_tf32(v[3]));
          *reinterpret_cast<uint4*>(tileB(s, 0) + off) = w;
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
          *reinterpret_cast<uint4*>(tileB(s, 0) + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
          if constexpr (KIND == TC_BF16X3)
            *reinterpret_cast<uint4*>(tileB(s, 1) + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
      }
    }
  };

  constexpr uint32_t FMT = (KIND == TC_TF32) ? 2u : 1u;
  const uint32_t idesc = instr_desc(FMT, 128, (uint32_t)Npad);
  bool ok = true;
  if (niter > 0) load_stage(0, 0);
  for (int step = 0; step < niter && ok; ++step) {
    const int s = step & 1;
    if (step + 1 < niter) load_stage(step + 1, s ^ 1);
    else cp_async_commit();                     // keep the group count uniform
    cp_async_wait<1>();
    __syncthreads();                            // raw stage s visible to all threads
    if (step >= 2) ok = mbar_wait(smem_u32(&mbar[s]), (uint32_t)(((step - 2) >> 1) & 1), flag);
    if (!__syncthreads_and(ok)) {
      ok = false;
      break;
    }
    convert_stage(s);
    fence_async_smem();                         // generic-proxy writes -> tensor-core reads
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int ks = 0; ks < KSTEPS; ++ks) {
        const uint32_t aoff = ks * 2 * LBO, boff = ks * 2 * LBO;
        const uint64_t ah = smem_desc(smem_u32(tileA(s, 0)) + aoff, LBO, SBO);
        const uint64_t bh = smem_desc(smem_u32(tileB(s, 0)) + boff, LBO, SBO);
        const uint32_t acc0 = (step > 0 || ks > 0) ? 1u : 0u;
        mma<KIND>(tmem, ah, bh, idesc, acc0);
        if constexpr (KIND == TC_BF16X3) {
          const uint64_t al = smem_desc(smem_u32(tileA(s, 1)) + aoff, LBO, SBO);
          const uint64_t bl = smem_desc(smem_u32(tileB(s, 1)) + boff, LBO, SBO);
          mma<KIND>(tmem, ah, bl, idesc, 1u);
          mma<KIND>(tmem, al, bh, idesc, 1u);
        }
      }
      mma_commit(smem_u32(&mbar[s]));
    }
  }
  cp_async_wait<0>();
  // wait for the last committed MMAs, then read the accumulator
  if (ok && niter > 0) {
    const int last = niter - 1;
    ok = mbar_wait(smem_u32(&mbar[last & 1]), (uint32_t)((last >> 1) & 1), flag);
  }
  ok = __syncthreads_and(ok);
  tc_fence_after();
  if (ok) {
    float* out = partials + it.part_off;
    const int row = warp * 32 + lane;
    for (int c0 = 0; c0 < Npad; c0 += 8) {
      float v[8];
      tmem_ld8(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (row < A.n && niter > 0) {
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (c0 + j < N) out[(long long)row * N + c0 + j] = v[j];
      } else if (row < A.n) {
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (c0 + j < N) out[(long long)row * N + c0 + j] = 0.f;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols)
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
  for (int e = threadIdx.x; e < na * nb; e += blockDim.x) {
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
  SmemLayout lay[3];
  size_t smem[3] = {0, 0, 0};
  DevBuf d_pairs, d_items, d_pieces, partials, flag;
  bool ok = false;
  std::string why;
};

void ofm_tc_free(ofm_ctx* c) {
  if (!c->tc) return;
  DevBuf* bufs[] = {&c->tc->d_pairs, &c->tc->d_items, &c->tc->d_pieces, &c->tc->partials, &c->tc->flag};
  for (DevBuf* b : bufs)
    if (b->p) cudaFree(b->p);
  delete c->tc;
  c->tc = nullptr;
}

// Plan of the tensor-core contraction after a build: one item per row chunk
// of a piece, chunks sized for about four items per SM.
ofm_status ofm_plan_extra(ofm_ctx* c) {
  if (!c->tc) c->tc = new TcPlan();
  TcPlan* t = c->tc;
  t->pairs.clear();
  t->items.clear();
  t->pieces.clear();
  t->part_elems = 0;
  t->ok = false;
  if (c->storage != OFM_STORE_FP32) {
    t->why = "tensor-core contraction needs FP32 storage";
    return OFM_OK;
  }
  int ldA = 4, ldB = 4, Rb = 16;
  for (const HostPair& hp : c->pairs) {
    const DevFrag& A = c->frags[hp.a];
    const DevFrag& B = c->frags[hp.b];
    if (A.n > 128 || 2 * B.n > 256) {
      t->why = "tensor-core contraction supports at most 128 states per fragment";
      return OFM_OK;
    }
    ldA = std::max(ldA, A.ld);
    ldB = std::max(ldB, B.ld);
    Rb = std::max(Rb, (2 * B.n + 15) / 16 * 16);
  }
  const long long target = std::max<long long>(1024, c->kh / (4 * 152));
  for (size_t p = 0; p < c->pairs.size(); ++p) {
    const HostPair& hp = c->pairs[p];
    const DevFrag& B = c->frags[hp.b];
    TcPair tp;
    tp.a = hp.a;
    tp.b = hp.b;
    tp.N = 2 * B.n;
    tp.Npad = (tp.N + 15) / 16 * 16;
    tp.blk_off = c->simt_pairs[p].blk_off;
    tp.item0 = (int)t->items.size();
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
        t->part_elems += (long long)c->frags[hp.a].n * tp.N;
        t->items.push_back(it);
      }
    }
    tp.nitem = (int)t->items.size() - tp.item0;
    t->pairs.push_back(tp);
  }
  for (int k = 0; k < 3; ++k) {
    SmemLayout& L = t->lay[k];
    L.ldA = ldA;
    L.ldB = ldB;
    L.Rb = Rb;
    L.raw_stage = KT * (ldA + 2 * ldB) * 4;
    const int esz = (k == TC_TF32) ? 4 : 2;
    L.tileA = 128 * KT * esz + TILE_PAD;
    L.tileB = Rb * KT * esz + TILE_PAD;
    L.ntiles = (k == TC_BF16X3) ? 2 : 1;
    t->smem[k] = 2 * (size_t)L.raw_stage + 2 * (size_t)L.ntiles * (L.tileA + L.tileB);
  }
  if (t->smem[TC_BF16X3] > 220 * 1024 || t->smem[TC_TF32] > 220 * 1024) {
    t->why = "tensor-core staging does not fit shared memory for these state counts";
    return OFM_OK;
  }
  OFM_TRY(ofm_ensure(c, t->d_pairs, sizeof(TcPair) * std::max<size_t>(1, t->pairs.size()), "tc pairs"));
  OFM_TRY(ofm_ensure(c, t->d_items, sizeof(TcItem) * std::max<size_t>(1, t->items.size()), "tc items"));
  OFM_TRY(ofm_ensure(c, t->d_pieces, sizeof(Piece) * std::max<size_t>(1, t->pieces.size()), "tc pieces"));
  OFM_TRY(ofm_ensure(c, t->partials, sizeof(float) * std::max<long long>(1, t->part_elems), "tc partials"));
  OFM_TRY(ofm_ensure(c, t->flag, sizeof(int), "tc flag"));
  OFM_CUDA(c, cudaMemcpyAsync(t->d_pairs.p, t->pairs.data(), sizeof(TcPair) * t->pairs.size(), cudaMemcpyHostToDevice, c->stream));
  OFM_CUDA(c, cudaMemcpyAsync(t->d_items.p, t->items.data(), sizeof(TcItem) * t->items.size(), cudaMemcpyHostToDevice, c->stream));
  OFM_CUDA(c, cudaMemcpyAsync(t->d_pieces.p, t->pieces.data(), sizeof(Piece) * t->pieces.size(), cudaMemcpyHostToDevice, c->stream));
  OFM_CUDA(c, cudaMemsetAsync(t->flag.p, 0, sizeof(int), c->stream));
  OFM_CUDA(c, cudaFuncSetAttribute(tc_contract_kernel<TC_TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t->smem[TC_TF32]));
  OFM_CUDA(c, cudaFuncSetAttribute(tc_contract_kernel<TC_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t->smem[TC_BF16]));
  OFM_CUDA(c, cudaFuncSetAttribute(tc_contract_kernel<TC_BF16X3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t->smem[TC_BF16X3]));
  t->ok = true;
  return OFM_OK;
}

ofm_status ofm_contract_tc(ofm_ctx* c, ofm_precision prec) {
  TcPlan* t = c->tc;
  if (!t || !t->ok) return ofm_fail(c, OFM_ERR_INVALID, t ? t->why : "no tensor-core plan");
  const int kind = prec == OFM_PREC_TF32 ? TC_TF32 : prec == OFM_PREC_BF16 ? TC_BF16 : TC_BF16X3;
  const int nit = (int)t->items.size();
  {
    KTimer kt(c, KC_CONTRACT, 1, c->contract_bytes, (double)c->flops);
    if (nit > 0) {
      if (kind == TC_TF32)
        tc_contract_kernel<TC_TF32><<<nit, TC_THREADS, t->smem[kind], c->stream>>>(
            (const DevFrag*)c->d_frags.p, (const TcPair*)t->d_pairs.p, (const Piece*)t->d_pieces.p,
            (const TcItem*)t->d_items.p, (const float*)c->states.p, (const float*)c->hphi.p,
            (float*)t->partials.p, (int*)t->flag.p, t->lay[kind]);
      else if (kind == TC_BF16)
        tc_contract_kernel<TC_BF16><<<nit, TC_THREADS, t->smem[kind], c->stream>>>(
            (const DevFrag*)c->d_frags.p, (const TcPair*)t->d_pairs.p, (const Piece*)t->d_pieces.p,
            (const TcItem*)t->d_items.p, (const float*)c->states.p, (const float*)c->hphi.p,
            (float*)t->partials.p, (int*)t->flag.p, t->lay[kind]);
      else
        tc_contract_kernel<TC_BF16X3><<<nit, TC_THREADS, t->smem[kind], c->stream>>>(
            (const DevFrag*)c->d_frags.p, (const TcPair*)t->d_pairs.p, (const Piece*)t->d_pieces.p,
            (const TcItem*)t->d_items.p, (const float*)c->states.p, (const float*)c->hphi.p,
            (float*)t->partials.p, (int*)t->flag.p, t->lay[kind]);
    }
    OFM_CUDA(c, cudaGetLastError());
  }
  {
    KTimer kt(c, KC_FINALIZE, 1, (double)t->part_elems * 4 + 8.0 * c->blk_elems);
    if (!t->pairs.empty())
      tc_finalize_kernel<<<(int)t->pairs.size(), 256, 0, c->stream>>>(
          (const DevFrag*)c->d_frags.p, (const TcPair*)t->d_pairs.p, (const TcItem*)t->d_items.p,
          (const float*)t->partials.p, (double*)c->blocks.p);
    OFM_CUDA(c, cudaGetLastError());
  }
  c->tc_check = true;
  return OFM_OK;
}

// Reports a bounded-wait timeout of an earlier tensor-core or staged-stencil
// launch (each sets its flag word; the flags are read once and cleared).
ofm_status ofm_wait_status(ofm_ctx* c) {
  if (c->tc_check && c->tc && c->tc->flag.p) {
    int h = 0;
    OFM_CUDA(c, cudaMemcpyAsync(&h, c->tc->flag.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    OFM_CUDA(c, cudaStreamSynchronize(c->stream));
    c->tc_check = false;
    if (h) {
      cudaMemsetAsync(c->tc->flag.p, 0, sizeof(int), c->stream);
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

