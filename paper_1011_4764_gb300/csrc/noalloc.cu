// Pair blocks with no device allocation.
//
// Some callers cannot allocate device memory when they need a block:
//   - code running on a device whose memory is already carved up by another
//     framework's pool, with no headroom for a second allocator;
//   - latency-critical or real-time paths where cudaMalloc/cudaFree are not
//     acceptable, because they may block or synchronise the device;
//   - code running where allocation is simply not permitted, such as a
//     sandboxed plug-in that receives ready-made device buffers.
// For them, ofm_pair_blocks_noalloc computes H_ab and S_ab of one pair
// from caller-provided device buffers.  Its only scratch (work tables and
// the K-chunk partial tiles of the contraction) is a fixed array compiled
// into this library, so the call allocates nothing.
//
// The scratch is one file-scope __device__ array of OFM_NOALLOC_SCRATCH
// bytes.  Every GPU that loads the library holds it until the process
// exits.  In host code the array's name is only a host-side stand-in, not a
// device address; the first call on each device (with that device current)
// looks up the real address with cudaGetSymbolAddress and caches it.  That
// first call should happen before any stream capture.  The work tables are
// staged from host memory that lives only for the call, so a call made
// while its stream is being captured returns OFM_ERR_INVALID (the captured
// copy would read that memory after the call).  The stream must belong to
// the current device (the cached address is the current device's).  Every
// call shares the array, so calls whose GPU work overlaps (other streams,
// other host threads) race on it.  The partial tiles need no clearing: every work item
// overwrites its whole tile before the reduction reads it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "ofm_internal.h"

using namespace ofm;

namespace {

static __device__ __align__(256) unsigned char g_pair_scratch[OFM_NOALLOC_SCRATCH];

constexpr int kMaxDevices = 64;
std::mutex g_lock;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(g_lock);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_pair_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

extern "C" ofm_status ofm_pair_blocks_noalloc(const ofm_grid* grid, const ofm_fragment* fa,
                                              const ofm_fragment* fb, const float* phi_a,
                                              const float* phi_b, const float* hphi_b,
                                              double* HS_ab, void* cuda_stream) {
  if (!grid || !fa || !fb || !phi_a || !phi_b || !hphi_b || !HS_ab) return OFM_ERR_INVALID;
  const ofm_fragment two[2] = {*fa, *fb};
  std::string err;
  if (!validate_geometry(*grid, two, 2, err)) return OFM_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
      cudaGetLastError();
      return OFM_ERR_CUDA;
    }
    if (cs != cudaStreamCaptureStatusNone) return OFM_ERR_INVALID;
    int cur = 0, sdev = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) {
      cudaGetLastError();
      return OFM_ERR_CUDA;
    }
    if (s != nullptr) {
      if (cudaStreamGetDevice(s, &sdev) != cudaSuccess) {
        cudaGetLastError();
        return OFM_ERR_CUDA;
      }
      if (sdev != cur) return OFM_ERR_INVALID;
    }
  }
  const bool same = std::memcmp(fa, fb, sizeof(ofm_fragment)) == 0 && phi_a == phi_b;

  // fragment table: the caller's buffers are addressed relative to phi_a
  std::vector<DevFrag> fr;
  long long total = 0;
  make_frag_table(*grid, two, 2, fr, total);
  fr[0].off = 0;
  const long long gap = (long long)((intptr_t)phi_b - (intptr_t)phi_a);
  if (gap % (long long)sizeof(float) != 0) return OFM_ERR_INVALID;
  fr[1].off = same ? 0 : gap / (long long)sizeof(float);
  std::vector<HostPair> pairs;
  make_pairs(*grid, fr, pairs);
  const int want_b = same ? 0 : 1;
  const HostPair* hp = nullptr;
  for (const HostPair& p : pairs)
    if (p.a == 0 && p.b == want_b) hp = &p;
  const size_t out_bytes = sizeof(double) * 2 * (size_t)fa->n_states * fb->n_states;
  if (!hp) {  // boxes do not interact: both blocks are zero
    return cudaMemsetAsync(HS_ab, 0, out_bytes, s) == cudaSuccess ? OFM_OK : OFM_ERR_CUDA;
  }
  std::vector<HostPair> one(1, *hp);
  one[0].b = want_b;

  // choose the K chunk so that tables and partial tiles fit the scratch
  std::vector<DevPair> dp;
  std::vector<Piece> pcs;
  std::vector<WorkItem> items;
  long long partial_elems = 0;
  size_t tables = 0;
  long long chunk = std::max<long long>(256, hp->kh / 256);
  for (int tries = 0; tries < 40; ++tries) {
    make_items_simt(fr, one, 64, chunk, dp, pcs, items, partial_elems);
    tables = align_up(sizeof(DevFrag) * 2, 256) + align_up(sizeof(DevPair), 256) +
             align_up(sizeof(Piece) * pcs.size(), 256) + align_up(sizeof(WorkItem) * items.size(), 256);
    if (tables + sizeof(float) * (size_t)partial_elems <= OFM_NOALLOC_SCRATCH) break;
    chunk *= 2;
  }
  if (tables + sizeof(float) * (size_t)partial_elems > OFM_NOALLOC_SCRATCH)
    return OFM_ERR_INVALID;  // pair too large for the fixed scratch
  dp[0].blk_off = 0;

  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) {
    cudaGetLastError();
    return OFM_ERR_CUDA;
  }
  // pack the tables on the host and copy them into the scratch
  std::vector<unsigned char> host(tables, 0);
  size_t o = 0;
  const size_t o_fr = o;
  std::memcpy(&host[o], fr.data(), sizeof(DevFrag) * 2);
  o += align_up(sizeof(DevFrag) * 2, 256);
  const size_t o_pair = o;
  std::memcpy(&host[o], dp.data(), sizeof(DevPair));
  o += align_up(sizeof(DevPair), 256);
  const size_t o_pc = o;
  std::memcpy(&host[o], pcs.data(), sizeof(Piece) * pcs.size());
  o += align_up(sizeof(Piece) * pcs.size(), 256);
  const size_t o_it = o;
  std::memcpy(&host[o], items.data(), sizeof(WorkItem) * items.size());
  unsigned char* d = (unsigned char*)base;
  if (cudaMemcpyAsync(d, host.data(), tables, cudaMemcpyHostToDevice, s) != cudaSuccess) {
    cudaGetLastError();
    return OFM_ERR_CUDA;
  }
  // H phi of b sits at offset fr[1].off from this base, like phi_b from phi_a
  const float* hbase =
      (const float*)((intptr_t)hphi_b - (intptr_t)(fr[1].off * (long long)sizeof(float)));
  launch_contract_simt(OFM_PREC_FP32, false, (const DevFrag*)(d + o_fr), (const DevPair*)(d + o_pair),
                       (const Piece*)(d + o_pc), (const WorkItem*)(d + o_it), (int)items.size(),
                       phi_a, hbase, d + tables, 64, s);
  launch_finalize_simt(OFM_PREC_FP32, (const DevFrag*)(d + o_fr), (const DevPair*)(d + o_pair), 1,
                       (const WorkItem*)(d + o_it), d + tables, 64, HS_ab, s);
  if (cudaGetLastError() != cudaSuccess) return OFM_ERR_CUDA;
  return OFM_OK;
}
