// Block-sparse products with the assembled pencil of Eq. 2: Y = H X or
// Y = S X over the pair list, H and S taken from the FP64 pair blocks (the
// block a <= b is stored, the block b > a is its transpose).  This is the
// operation a window solver that never forms the dense n x n matrices is
// built from, for bases too large for the dense FP64 path.
//
// One CTA per (fragment a, 32 columns of X): its threads own the outputs
// (i, c) of block row a and sum over the row's blocks in a fixed order (the
// pair list's), so the result is deterministic.  FP64 throughout.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "ofm_internal.h"

namespace ofm {
namespace {

constexpr int SP_KT = 32;        // columns of X per CTA
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
  const int a = blockIdx.x;
  const int c0 = blockIdx.y * SP_KT;
  const int kc = min(SP_KT, k - c0);
  const int na = fr[a].n, ra = fr[a].basis0;
  const int q0 = rowptr[a], q1 = rowptr[a + 1];
  for (int e = threadIdx.x; e < na * kc; e += blockDim.x) {
    const int i = e % na, cc = e / na;
    const double* xc = X + (long long)(c0 + cc) * ldx;
    double acc = 0.0;
    for (int q = q0; q < q1; ++q) {
      const SpEnt E = ents[q];
      const int nb = fr[E.b].n;
      const double* x = xc + fr[E.b].basis0;
      // the stored block holds n_a n_b entries whichever way it is stored
      const double* m = blocks + E.off + (which ? (long long)na * nb : 0);
      if (!E.tr) {
        m += (long long)i * nb;                       // row i of M_ab (n_a x n_b, row-major)
        for (int j = 0; j < nb; ++j) acc = fma(m[j], x[j], acc);
      } else {
        m += i;                                       // column i of M_ba (n_b x n_a, row-major)
        for (int j = 0; j < nb; ++j) acc = fma(m[(long long)j * na], x[j], acc);
      }
    }
    Y[(long long)(c0 + cc) * ldy + ra + i] = acc;
  }
}

}  // namespace
}  // namespace ofm

using namespace ofm;

extern "C" ofm_status ofm_pencil_apply(ofm_ctx* c, int which, const double* X, long long ldx,
                                       double* Y, long long ldy, int k) {
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
  // block rows: for every fragment its pairs in the pair list's order, the
  // stored block a <= b as is, the mirror b > a transposed
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
  // pageable sources: the copies are staged before the calls return
  OFM_CUDA(c, cudaMemcpyAsync(c->sp_rowptr.p, rowptr.data(), sizeof(int) * (nf + 1),
                              cudaMemcpyHostToDevice, c->stream));
  OFM_CUDA(c, cudaMemcpyAsync(c->sp_ents.p, ents.data(), sizeof(SpEnt) * ents.size(),
                              cudaMemcpyHostToDevice, c->stream));
  {
    double flops = 0.0;
    for (size_t p = 0; p < c->pairs.size(); ++p) {
      const double nn = (double)c->frags[c->pairs[p].a].n * c->frags[c->pairs[p].b].n;
      flops += (c->pairs[p].a == c->pairs[p].b ? 2.0 : 4.0) * nn * k;
    }
    KTimer kt(c, KC_PENCIL, 1, 0.0, flops);
    pencil_apply_kernel<<<dim3(nf, (k + SP_KT - 1) / SP_KT), SP_THREADS, 0, c->stream>>>(
        (const double*)c->blocks.p, (const DevFrag*)c->d_frags.p, (const int*)c->sp_rowptr.p,
        (const SpEnt*)c->sp_ents.p, which, X, ldx, Y, ldy, k);
  }
  OFM_CUDA(c, cudaGetLastError());
  return OFM_OK;
}
