// Pair-block contraction on CUDA cores (FP64 and FP32 arithmetic), the
// deterministic reduction of K-chunk partials into FP64 blocks, and the
// scatter of blocks into dense basis-ordered H and S.
//
// For a pair a <= b the blocks are (Sec. II)
//     S_ab = Phi_a^T Phi_b       over B_a ∩ B_b,
//     H_ab = Phi_a^T (H Phi_b)   over B_a ∩ B_b+.
// States are stored on dilated boxes with a zero halo, so both sums run over
// the same region R = B_a ∩ B_b+ and become one GEMM
//     [S_ab | H_ab] = Phi_a[R]^T [Phi_b[R] | HPhi_b[R]]
// with M = n_a, N = 2 n_b and K = |R|.  R is cut into pieces (boxes that are
// contiguous in both storages) and each piece into chunks of whole x-rows; a
// CTA gathers the rows of its chunk into shared memory and accumulates one
// TILE x TILE output tile, written as a partial.  The finalize kernel sums
// the partials of each pair in a fixed order, so results are bitwise
// reproducible run to run.
#include <cuda_runtime.h>

#include "ofm_internal.h"

namespace ofm {

constexpr int KT = 16;     // points per shared-memory stage
constexpr int TILE = 64;   // output tile edge
constexpr int NT = 256;    // threads per CTA

template <typename Tin, typename Tacc>
__global__ void __launch_bounds__(NT) contract_simt_kernel(
    const DevFrag* __restrict__ fr, const DevPair* __restrict__ prs, const Piece* __restrict__ pcs,
    const WorkItem* __restrict__ items, const Tin* __restrict__ states,
    const Tin* __restrict__ hphi, Tacc* __restrict__ partials) {
  __shared__ Tacc As[KT][TILE];
  __shared__ Tacc Bs[KT][TILE];
  __shared__ long long pa_s[KT], pb_s[KT];

  const WorkItem it = items[blockIdx.x];
  const DevPair pr = prs[it.pair];
  const DevFrag A = fr[pr.a];
  const DevFrag B = fr[pr.b];
  const Piece pc = pcs[it.piece];
  const int m0 = it.mt * TILE, n0 = it.nt * TILE;
  const Tin* Pa = states + A.off;
  const Tin* Pb = states + B.off;
  const Tin* Hb = hphi + B.off;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int lenx = pc.len[0], leny = pc.len[1];
  const long long npts = (long long)(it.r1 - it.r0) * lenx;

  Tacc acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = Tacc(0);

  for (long long k0 = 0; k0 < npts; k0 += KT) {
    if (tid < KT) {
      long long k = k0 + tid;
      if (k < npts) {
        int r = it.r0 + (int)(k / lenx);
        int x = (int)(k % lenx);
        int y = r % leny, z = r / leny;
        pa_s[tid] = ((long long)(pc.la[2] + z) * A.dext[1] + (pc.la[1] + y)) * A.dext[0] + pc.la[0] + x;
        pb_s[tid] = ((long long)(pc.lb[2] + z) * B.dext[1] + (pc.lb[1] + y)) * B.dext[0] + pc.lb[0] + x;
      } else {
        pa_s[tid] = -1;
        pb_s[tid] = -1;
      }
    }
    __syncthreads();
    for (int e = tid; e < KT * TILE; e += NT) {
      const int kk = e / TILE, c = e % TILE;
      const long long pa = pa_s[kk], pb = pb_s[kk];
      Tacc va = Tacc(0), vb = Tacc(0);
      const int m = m0 + c;
      if (pa >= 0 && m < A.n) va = (Tacc)Pa[pa * A.ld + m];
      const int nn = n0 + c;
      if (pb >= 0) {
        if (nn < B.n) vb = (Tacc)Pb[pb * B.ld + nn];
        else if (nn < 2 * B.n) vb = (Tacc)Hb[pb * B.ld + (nn - B.n)];
      }
      As[kk][c] = va;
      Bs[kk][c] = vb;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KT; ++kk) {
      Tacc a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  Tacc* out = partials + it.part_off;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) out[(ty * 4 + i) * TILE + tx * 4 + j] = acc[i][j];
}

void launch_contract_simt(int prec, bool store_fp64, const DevFrag* d_fr, const DevPair* d_pairs,
                          const Piece* d_pieces, const WorkItem* d_items, int nitems,
                          const void* states, const void* hphi, void* partials, int tile,
                          cudaStream_t s) {
  (void)tile;
  if (nitems <= 0) return;
  if (prec == OFM_PREC_FP64) {
    if (store_fp64)
      contract_simt_kernel<double, double><<<nitems, NT, 0, s>>>(
          d_fr, d_pairs, d_pieces, d_items, (const double*)states, (const double*)hphi,
          (double*)partials);
    else
      contract_simt_kernel<float, double><<<nitems, NT, 0, s>>>(
          d_fr, d_pairs, d_pieces, d_items, (const float*)states, (const float*)hphi,
          (double*)partials);
  } else {
    contract_simt_kernel<float, float><<<nitems, NT, 0, s>>>(
        d_fr, d_pairs, d_pieces, d_items, (const float*)states, (const float*)hphi,
        (float*)partials);
  }
}

// Sum of the partials of output (i, c) of pair pr, chunks in plan order.
template <typename Tacc>
__device__ __forceinline__ double sum_partials(const DevPair& pr, const WorkItem* items,
                                               const Tacc* partials, int i, int c) {
  const int mt = i / TILE, nt = c / TILE;
  const int base = pr.item0 + (mt * pr.ntiles + nt) * pr.nchunk;
  const int off = (i % TILE) * TILE + (c % TILE);
  double s = 0.0;
  for (int k = 0; k < pr.nchunk; ++k) s += (double)partials[items[base + k].part_off + off];
  return s;
}

// One CTA per pair.  Block layout: H_ab then S_ab, each n_a x n_b row-major.
template <typename Tacc>
__global__ void finalize_simt_kernel(const DevFrag* __restrict__ fr, const DevPair* __restrict__ prs,
                                     const WorkItem* __restrict__ items,
                                     const Tacc* __restrict__ partials, double* __restrict__ blocks) {
  const DevPair pr = prs[blockIdx.x];
  const int na = fr[pr.a].n, nb = fr[pr.b].n;
  double* Hblk = blocks + pr.blk_off;
  double* Sblk = Hblk + (long long)na * nb;
  const bool diag = (pr.a == pr.b);
  for (int e = threadIdx.x; e < na * nb; e += blockDim.x) {
    const int i = e / nb, m = e % nb;
    double s = sum_partials(pr, items, partials, i, m);
    double h = sum_partials(pr, items, partials, i, nb + m);
    if (diag) {
      s = 0.5 * (s + sum_partials(pr, items, partials, m, i));
      h = 0.5 * (h + sum_partials(pr, items, partials, m, nb + i));
    }
    Sblk[e] = s;
    Hblk[e] = h;
  }
}

void launch_finalize_simt(int prec, const DevFrag* d_fr, const DevPair* d_pairs, int npairs,
                          const WorkItem* d_items, const void* partials, int tile, double* blocks,
                          cudaStream_t s) {
  (void)tile;
  if (npairs <= 0) return;
  if (prec == OFM_PREC_FP64)
    finalize_simt_kernel<double><<<npairs, 256, 0, s>>>(d_fr, d_pairs, d_items,
                                                        (const double*)partials, blocks);
  else
    finalize_simt_kernel<float><<<npairs, 256, 0, s>>>(d_fr, d_pairs, d_items,
                                                       (const float*)partials, blocks);
}

// Dense basis-ordered matrices from the blocks; the lower block of a pair
// a < b is the transpose of its upper block.  Hd, Sd must be zeroed first.
__global__ void scatter_dense_kernel(const DevFrag* __restrict__ fr, const DevPair* __restrict__ prs,
                                     const double* __restrict__ blocks, int n,
                                     double* __restrict__ Hd, double* __restrict__ Sd) {
  const DevPair pr = prs[blockIdx.x];
  const DevFrag A = fr[pr.a], B = fr[pr.b];
  const double* Hblk = blocks + pr.blk_off;
  const double* Sblk = Hblk + (long long)A.n * B.n;
  for (int e = threadIdx.x; e < A.n * B.n; e += blockDim.x) {
    const int i = e / B.n, m = e % B.n;
    const long long r = A.basis0 + i, c = B.basis0 + m;
    Hd[r * n + c] = Hblk[e];
    Sd[r * n + c] = Sblk[e];
    if (pr.a != pr.b) {
      Hd[c * n + r] = Hblk[e];
      Sd[c * n + r] = Sblk[e];
    }
  }
}

void launch_scatter_dense(const DevFrag* d_fr, const DevPair* d_pairs, int npairs,
                          const double* blocks, int n, double* Hd, double* Sd, cudaStream_t s) {
  if (npairs <= 0) return;
  scatter_dense_kernel<<<npairs, 256, 0, s>>>(d_fr, d_pairs, blocks, n, Hd, Sd);
}

}  // namespace ofm
