// Block-sparse products with the assembled pencil of Eq. 2: Y = H X or
// Y = S X over the pair list, H and S taken from the FP64 pair blocks (the
// block a <= b is stored, the block b > a is its transpose).  This is the
// operation a window solver that never forms the dense n x n matrices is
// built from, for bases too large for the dense FP64 path.
//
// One CTA per (fragment a, 8 columns of X): the outputs (i, c) of block row
// a accumulate in shared memory over the row's blocks in a fixed order (the
// pair list's), so the result is deterministic.  Both block orientations
// read coalesced: for a stored block M_ab (n_a x n_b, row-major) a warp takes
// one output row and its lanes run along j (M_ab[i][j] and x[j] contiguous),
// reduced by shuffles; for a mirrored block (column i of the stored M_ba,
// n_b x n_a row-major) the threads run along i, so a fixed j reads a
// contiguous row of M_ba.  FP64 throughout.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "ofm_internal.h"

namespace ofm {
namespace {

constexpr int SP_KT = 8;         // columns of X per CTA
constexpr int SP_THREADS = 256;

struct SpEnt {
  long long off;   // arena offset of the stored pair's H block (its S block follows)
  int b;           // column fragment
  int tr;          // 1: the stored block is M_ba (the pair is (b, a)), read transposed
};

__global__ void __launch_bounds__(SP_THREADS) pencil_apply_kernel(
    const double* __restrict__ blocks, const DevFrag* __restrict__ fr, const int* __restrict__ rowptr,
    const SpEnt* __restrict__ ents, int which, const double* __restrict__ X, long long ldx,
    double* __restrict__ Y, long long ldy, int k) {
  extern __shared__ double acc[];   // [c][i], n_a x kc
  const int a = blockIdx.x;
  const int c0 = blockIdx.y * SP_KT;
  const int kc = min(SP_KT, k - c0);
  const int na = fr[a].n, ra = fr[a].basis0;
  const int q0 = rowptr[a], q1 = rowptr[a + 1];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int e = tid; e < na * kc; e += blockDim.x) acc[e] = 0.0;
  __syncthreads();
  for (int q = q0; q < q1; ++q) {
    const SpEnt E = ents[q];
    const int nb = fr[E.b].n;
    const double* xb = X + (long long)c0 * ldx + fr[E.b].basis0;
    // the stored block holds n_a n_b entries whichever way it is stored
    const double* m = blocks + E.off + (which ? (long long)na * nb : 0);
    if (!E.tr) {
      for (int r = warp; r < na * kc; r += nw) {
        const int i = r % na, cc = r / na;
        const double* mi = m + (long long)i * nb;
        const double* x = xb + (long long)cc * ldx;
        double s = 0.0;
        for (int j = lane; j < nb; j += 32) s = fma(mi[j], x[j], s);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) acc[cc * na + i] += s;
      }
    } else {
      for (int e = tid; e < na * kc; e += blockDim.x) {
        const int i = e % na, cc = e / na;
        const double* x = xb + (long long)cc * ldx;
        double s = 0.0;
        for (int j = 0; j < nb; ++j) s = fma(m[(long long)j * na + i], x[j], s);
        acc[cc * na + i] += s;
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < na * kc; e += blockDim.x) {
    const int i = e % na, cc = e / na;
    Y[(long long)(c0 + cc) * ldy + ra + i] = acc[e];
  }
}

}  // namespace

// Block rows of the pencil for the current pair list: for every fragment its
// pairs in the pair list's order, the stored block a <= b as is, the mirror
// b > a transposed.  Rebuilt only after the pair list or the plan changes.
static ofm_status pencil_tables(ofm_ctx* c) {
  if (!c->sp_stale) return OFM_OK;
  const int nf = c->nfrag;
  std::vector<std::vector<SpEnt>> rows(nf);
  for (size_t p = 0; p < c->pairs.size(); ++p) {
    const int a = c->pairs[p].a, b = c->pairs[p].b;
    const long long off = c->simt_pairs[p].blk_off;
    rows[a].push_back({off, b, 0});
    if (b != a) rows[b].push_back({off, a, 1});
  }
  std::vector<int> rowptr(nf + 1, 0);
  std::vector<SpEnt> ents;
  for (int a = 0; a < nf; ++a) {
    ents.insert(ents.end(), rows[a].begin(), rows[a].end());
    rowptr[a + 1] = (int)ents.size();
  }
  OFM_TRY(ofm_ensure(c, c->sp_rowptr, sizeof(int) * (nf + 1), "pencil block rows"));
  OFM_TRY(ofm_ensure(c, c->sp_ents, sizeof(SpEnt) * std::max<size_t>(1, ents.size()), "pencil blocks"));
  OFM_CUDA(c, cudaMemcpyAsync(c->sp_rowptr.p, rowptr.data(), sizeof(int) * (nf + 1),
                              cudaMemcpyHostToDevice, c->stream));
  OFM_CUDA(c, cudaMemcpyAsync(c->sp_ents.p, ents.data(), sizeof(SpEnt) * ents.size(),
                              cudaMemcpyHostToDevice, c->stream));
  OFM_CUDA(c, cudaStreamSynchronize(c->stream));   // the host tables are released
  c->sp_flops_per_col = 0.0;
  c->sp_bytes_fixed = 0.0;
  for (size_t p = 0; p < c->pairs.size(); ++p) {
    const double nn = (double)c->frags[c->pairs[p].a].n * c->frags[c->pairs[p].b].n;
    c->sp_flops_per_col += (c->pairs[p].a == c->pairs[p].b ? 2.0 : 4.0) * nn;
    c->sp_bytes_fixed += 8.0 * nn;   // one of the pair's two blocks is read per product
  }
  c->sp_stale = false;
  return OFM_OK;
}

}  // namespace ofm

using namespace ofm;

static ofm_status ofm_pencil_apply_impl(ofm_ctx* c, int which, const double* X, long long ldx,
                                       double* Y, long long ldy, int k) {
  OFM_RANGE("ofm_pencil_apply");
  if (!c) return OFM_ERR_INVALID;
  if (!c->assembled) return ofm_fail(c, OFM_ERR_STATE, "ofm_assemble_HS must come first");
  if (which != 0 && which != 1) return ofm_fail(c, OFM_ERR_INVALID, "which must be 0 (H) or 1 (S)");
  if (!X || !Y) return ofm_fail(c, OFM_ERR_INVALID, "X and Y must not be NULL");
  if (k < 1) return ofm_fail(c, OFM_ERR_INVALID, "k must be >= 1");
  const long long n = c->basis;
  if (ldx < n || ldy < n) return ofm_fail(c, OFM_ERR_INVALID, "leading dimensions must be >= the basis size");
  {   // Y must not overlap X (the kernel reads X while it writes Y)
    const char* x0 = (const char*)X;
    const char* x1 = (const char*)(X + (k - 1) * ldx + n);
    const char* y0 = (const char*)Y;
    const char* y1 = (const char*)(Y + (k - 1) * ldy + n);
    if (x0 < y1 && y0 < x1) return ofm_fail(c, OFM_ERR_INVALID, "X and Y overlap");
  }
  OFM_TRY(ofm_wait_status(c));
  OFM_TRY(pencil_tables(c));
  {
    // algorithmic traffic: every stored block once, X read and Y written once
    KTimer kt(c, KC_PENCIL, 1, c->sp_bytes_fixed + 16.0 * (double)n * k, c->sp_flops_per_col * k);
    int namax = 1;
    for (const DevFrag& f : c->frags) namax = std::max(namax, f.n);
    const size_t sm = sizeof(double) * namax * SP_KT;   // <= 64 KB (n_a <= 1024)
    if (sm > 48 * 1024)
      OFM_CUDA(c, cudaFuncSetAttribute(pencil_apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    pencil_apply_kernel<<<dim3(c->nfrag, (k + SP_KT - 1) / SP_KT), SP_THREADS,
                          sizeof(double) * namax * SP_KT, c->stream>>>(
        (const double*)c->blocks.p, (const DevFrag*)c->d_frags.p, (const int*)c->sp_rowptr.p,
        (const SpEnt*)c->sp_ents.p, which, X, ldx, Y, ldy, k);
  }
  OFM_CUDA(c, cudaGetLastError());
  return OFM_OK;
}

extern "C" ofm_status ofm_pencil_apply(ofm_ctx* c, int which, const double* X, long long ldx, double* Y, long long ldy, int k) {
  const ofm_status st = ofm_pencil_apply_impl(c, which, X, ldx, Y, ldy, k);
  if (st != OFM_OK || !c || !c->checks) return st;
  return ofm_check_guards_now(c, "ofm_pencil_apply");
}
