// Per-kernel-class launch counting and CUDA-event timing on the context
// stream (tracing support for the benchmark and the profiles).
#include <cuda_runtime.h>

#include <cstring>

#include "ofm_internal.h"

namespace ofm {

const char* kclass_name(int k) {
  static const char* names[KC_COUNT] = {
      "convert",  "apply",  "contract", "finalize", "scatter", "eig_init", "filter", "gram",
      "rayleigh_ritz", "rotate", "eig_export", "cholesky", "reduce", "tridiag", "bisect",
      "vectors", "pencil"};
  return (k >= 0 && k < KC_COUNT) ? names[k] : "?";
}

const char* kclass_row(int k) {
  static const char* rows[KC_COUNT] = {"a2", "a1", "a4", "a5", "a5", "a0", "a0", "a0",
                                       "a0", "a0", "a0", "a6", "a6", "a6", "a6", "a6", "a6"};
  return (k >= 0 && k < KC_COUNT) ? rows[k] : "?";
}

}  // namespace ofm

using namespace ofm;

static cudaEvent_t take_event(ofm_ctx* c) {
  auto& pool = c->prof.pool;
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

static void resolve(ofm_ctx* c) {
  auto& pr = c->prof;
  if (pr.pending.empty()) return;
  cudaStreamSynchronize(c->stream);
  for (auto& p : pr.pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) pr.st[p.k].ms += ms;
    else cudaGetLastError();
    pr.pool.push_back(p.a);
    pr.pool.push_back(p.b);
  }
  pr.pending.clear();
}

KTimer::KTimer(ofm_ctx* c_, int k_, long long nlaunch, double bytes, double flops) : c(c_), k(k_) {
  c->prof.st[k].launches += nlaunch;
  c->prof.st[k].bytes += bytes;
  c->prof.st[k].flops += flops;
  if (c->prof.on) {
    a = take_event(c);
    if (a) cudaEventRecord(a, c->stream);
  }
}

void KTimer::add(long long n) { c->prof.st[k].launches += n; }

KTimer::~KTimer() {
  if (!a) return;
  cudaEvent_t b = take_event(c);
  if (!b) {
    c->prof.pool.push_back(a);
    return;
  }
  cudaEventRecord(b, c->stream);
  c->prof.pending.push_back({k, a, b});
  if (c->prof.pending.size() > 4096) resolve(c);
}

void ofm_prof_release(ofm_ctx* c) {
  resolve(c);
  for (cudaEvent_t e : c->prof.pool) cudaEventDestroy(e);
  c->prof.pool.clear();
}

extern "C" ofm_status ofm_set_profiling(ofm_ctx* c, int on) {
  if (!c) return OFM_ERR_INVALID;
  resolve(c);
  for (auto& s : c->prof.st) s = KStat{};
  c->prof.on = on != 0;
  return OFM_OK;
}

extern "C" ofm_status ofm_get_kernel_stats(ofm_ctx* c, ofm_kernel_stat* out, int max, int* n) {
  if (!c) return OFM_ERR_INVALID;
  if (!n || (max > 0 && !out)) return ofm_fail(c, OFM_ERR_INVALID, "bad arguments");
  resolve(c);
  int w = 0;
  for (int k = 0; k < KC_COUNT && w < max; ++k) {
    if (c->prof.st[k].launches == 0) continue;
    std::memset(&out[w], 0, sizeof(ofm_kernel_stat));
    std::strncpy(out[w].name, kclass_name(k), sizeof(out[w].name) - 1);
    std::strncpy(out[w].row, kclass_row(k), sizeof(out[w].row) - 1);
    out[w].launches = c->prof.st[k].launches;
    out[w].total_ms = c->prof.st[k].ms;
    out[w].bytes = c->prof.st[k].bytes;
    out[w].flops = c->prof.st[k].flops;
    ++w;
  }
  *n = w;
  return OFM_OK;
}
