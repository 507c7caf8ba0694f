// C ABI entry points of the OFM library (include/ofm.h): context handling,
// argument validation, buffer management and the order of device work.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <string>
#include <new>

#include "ofm_internal.h"

using namespace ofm;

// ------------------------------------------------------------- helpers -----

ofm_status ofm_fail(ofm_ctx* c, ofm_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

ofm_status ofm_cuda_check(ofm_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return OFM_OK;
  std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  if (e == cudaErrorMemoryAllocation) return ofm_fail(c, OFM_ERR_OOM, m);
  return ofm_fail(c, OFM_ERR_CUDA, m);
}

ofm_status ofm_ensure(ofm_ctx* c, DevBuf& b, size_t bytes, const char* what) {
  if (bytes == 0) bytes = 16;
  if (b.cap >= bytes) return OFM_OK;
  if (c && c->fault == OFM_FAULT_OOM && bytes >= 4096) {
    char buf[160];
    snprintf(buf, sizeof buf, "cudaMalloc of %zu bytes for %s failed (injected by OFM_FAULT=oom)", bytes, what);
    return ofm_fail(c, OFM_ERR_OOM, buf);
  }
  if (b.p) {
    cudaError_t e = cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
    if (e != cudaSuccess) return ofm_cuda_check(c, e, "cudaFree");
  }
  // the buffer and its guard band (OFM_GUARD_BYTES of 0xA5 after the end)
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes + OFM_GUARD_BYTES);
  if (e == cudaSuccess) {
    b.p = p;
    e = cudaMemsetAsync((char*)p + bytes, 0xA5, OFM_GUARD_BYTES, c ? c->stream : nullptr);
  }
  if (e != cudaSuccess) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    cudaGetLastError();
    char buf[160];
    snprintf(buf, sizeof buf, "cudaMalloc of %zu bytes for %s failed", bytes, what);
    return ofm_fail(c, e == cudaErrorMemoryAllocation ? OFM_ERR_OOM : OFM_ERR_CUDA, buf);
  }
  b.cap = bytes;
  return OFM_OK;
}

ofm_status ofm_ensure_big(ofm_ctx* c, DevBuf& b, size_t bytes, const char* what) {
  const ofm_status st = ofm_ensure(c, b, bytes, what);
  if (st != OFM_ERR_OOM || !c->eig) return st;
  ofm_eig_free(c);   // the largest reclaimable buffers; the next eigensolve re-makes them
  return ofm_ensure(c, b, bytes, what);
}

static void free_buf(DevBuf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
}

static ofm_status check_launch(ofm_ctx* c, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return ofm_cuda_check(c, e, what);
  return OFM_OK;
}

static ofm_status sync(ofm_ctx* c, const char* what) {
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return ofm_cuda_check(c, e, what);
  return OFM_OK;
}

static size_t elem_size(const ofm_ctx* c) { return c->storage == OFM_STORE_FP64 ? 8 : 4; }

// Captured assembly graphs refer to the plans and buffers of the moment.
static void drop_graphs(ofm_ctx* c) {
  for (auto& g : c->asm_exec)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
}


static int find_pair(const ofm_ctx* c, int a, int b) {
  // pairs are sorted by (a, b) with a <= b
  int lo = 0, hi = (int)c->pairs.size() - 1;
  while (lo <= hi) {
    int mid = (lo + hi) / 2;
    const HostPair& p = c->pairs[mid];
    if (p.a == a && p.b == b) return mid;
    if (p.a < a || (p.a == a && p.b < b)) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

// ----------------------------------------------------- guard bands -------

namespace {
// One CTA per buffer: thread t reads byte t of the guard band; the smallest
// index of a buffer with a byte other than 0xA5 goes to *bad.
__global__ void guard_check_kernel(const GuardRef* tab, int* bad) {
  const GuardRef g = tab[blockIdx.x];
  const unsigned char v = static_cast<const unsigned char*>(g.p)[g.cap + threadIdx.x];
  if (v != 0xA5) atomicMin(bad, (int)blockIdx.x);
}
}  // namespace

static void ctx_guards(const ofm_ctx* c, std::vector<GuardRef>& out) {
  const struct { const DevBuf* b; const char* n; } own[] = {
      {&c->V, "V"}, {&c->states, "fragment states"}, {&c->hphi, "H phi"},
      {&c->d_frags, "fragment table"}, {&c->d_pairs, "pair table"}, {&c->d_pieces, "piece table"},
      {&c->d_items, "work items"}, {&c->partials, "partials"}, {&c->blocks, "blocks"},
      {&c->dense_H, "dense H"}, {&c->dense_S, "dense S"}, {&c->staging, "staging"},
      {&c->flag, "error flags"}, {&c->w_A, "window A"}, {&c->w_L, "window L"},
      {&c->w_d, "window d"}, {&c->w_e, "window e"}, {&c->w_tau, "window tau"},
      {&c->w_tmp, "window tmp"}, {&c->w_eval, "window eigenvalues"}, {&c->w_bar, "window barrier"},
      {&c->w_Q, "window Q"}, {&c->sp_rowptr, "pencil rows"}, {&c->sp_ents, "pencil entries"},
      {&c->blk_stage, "block staging"}};
  for (const auto& o : own)
    if (o.b->p) out.push_back({o.b->p, o.b->cap, o.n});
  ofm_tc_guards(c->tc, out);
  ofm_eig_guards(c, out);
  ofm_region_guards(c, out);
}

// Reads every guard band (and the check-mode kernels' refusal flag):
// OFM_ERR_CORRUPT naming the first overwritten buffer.  Synchronises.
ofm_status ofm_check_guards_now(ofm_ctx* c, const char* after) {
  std::vector<GuardRef> g;
  ctx_guards(c, g);
  OFM_TRY(ofm_ensure(c, c->guard_tab, sizeof(GuardRef) * (g.size() + 1), "guard table"));
  g.push_back({c->guard_tab.p, c->guard_tab.cap, "guard table"});
  OFM_CUDA(c, cudaMemcpyAsync(c->guard_tab.p, g.data(), sizeof(GuardRef) * g.size(),
                              cudaMemcpyHostToDevice, c->stream));
  int* flags = (int*)c->flag.p;
  const int none = INT_MAX;
  OFM_CUDA(c, cudaMemcpyAsync(flags + OFM_FLAG_GUARD, &none, sizeof(int), cudaMemcpyHostToDevice,
                              c->stream));
  guard_check_kernel<<<(unsigned)g.size(), (unsigned)OFM_GUARD_BYTES, 0, c->stream>>>(
      (const GuardRef*)c->guard_tab.p, flags + OFM_FLAG_GUARD);
  OFM_CUDA(c, cudaGetLastError());
  int res[2] = {0, 0};
  OFM_CUDA(c, cudaMemcpyAsync(res, flags + OFM_FLAG_GUARD, 2 * sizeof(int), cudaMemcpyDeviceToHost,
                              c->stream));
  OFM_CUDA(c, cudaStreamSynchronize(c->stream));
  if (res[1]) {
    cudaMemsetAsync(flags + OFM_FLAG_BOUNDS, 0, sizeof(int), c->stream);
    return ofm_fail(c, OFM_ERR_CORRUPT, std::string("a check-mode kernel refused an access outside its buffer (after ") + after + ")");
  }
  if (res[0] != none)
    return ofm_fail(c, OFM_ERR_CORRUPT, std::string("the guard band of ") + g[res[0]].name +
                                            " was overwritten (found after " + after + ")");
  return OFM_OK;
}

extern "C" ofm_status ofm_set_checks(ofm_ctx* c, int on) {
  if (!c) return OFM_ERR_INVALID;
  c->checks = on != 0;
  drop_graphs(c);          // the captured assemblies use the other kernel forms
  c->region_stale = true;  // and a fresh region plan drops anything a test hook changed
  return OFM_OK;
}

extern "C" ofm_status ofm_check_guards(ofm_ctx* c) {
  if (!c) return OFM_ERR_INVALID;
  OFM_RANGE("ofm_check_guards");
  return ofm_check_guards_now(c, "ofm_check_guards");
}

void ofm_free_extra(ofm_ctx* c) {
  ofm_eig_free(c);
  ofm_tc_free(c);
  ofm_region_free(c);
}

// ------------------------------------------------------------- lifecycle ---

extern "C" const char* ofm_status_string(ofm_status s) {
  switch (s) {
    case OFM_OK: return "OFM_OK";
    case OFM_ERR_INVALID: return "OFM_ERR_INVALID";
    case OFM_ERR_OOM: return "OFM_ERR_OOM";
    case OFM_ERR_CUDA: return "OFM_ERR_CUDA";
    case OFM_ERR_NOT_CONVERGED: return "OFM_ERR_NOT_CONVERGED";
    case OFM_ERR_NOT_POSDEF: return "OFM_ERR_NOT_POSDEF";
    case OFM_ERR_TIMEOUT: return "OFM_ERR_TIMEOUT";
    case OFM_ERR_STATE: return "OFM_ERR_STATE";
    case OFM_ERR_CORRUPT: return "OFM_ERR_CORRUPT";
  }
  return "OFM_ERR_UNKNOWN";
}

extern "C" ofm_status ofm_create(ofm_ctx** out, void* cuda_stream) {
  if (!out) return OFM_ERR_INVALID;
  *out = nullptr;
  ofm_ctx* c = new (std::nothrow) ofm_ctx();
  if (!c) return OFM_ERR_OOM;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e != cudaSuccess) {
    delete c;
    cudaGetLastError();
    return OFM_ERR_CUDA;
  }
  if (const char* f = std::getenv("OFM_FAULT")) {
    const std::string k(f);
    c->fault = k == "oom" ? OFM_FAULT_OOM : k == "timeout" ? OFM_FAULT_TIMEOUT
             : k == "nonconv" ? OFM_FAULT_NONCONV : k == "notposdef" ? OFM_FAULT_NOTPOSDEF : OFM_FAULT_NONE;
  }
  if (const char* k = std::getenv("OFM_CHECK")) c->checks = std::string(k) == "1";
  if (cuda_stream) {
    c->stream = (cudaStream_t)cuda_stream;
  } else {
    e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete c;
      cudaGetLastError();
      return OFM_ERR_CUDA;
    }
    c->own_stream = true;
  }
  if (ofm_ensure(c, c->flag, 64, "error flags") != OFM_OK ||
      cudaMemsetAsync(c->flag.p, 0, 64, c->stream) != cudaSuccess) {
    if (c->flag.p) cudaFree(c->flag.p);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    cudaGetLastError();
    return OFM_ERR_OOM;
  }
  *out = c;
  return OFM_OK;
}

extern "C" void ofm_destroy(ofm_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  drop_graphs(c);
  ofm_prof_release(c);
  if (c->copy_stream) cudaStreamSynchronize(c->copy_stream);
  DevBuf* bufs[] = {&c->V, &c->states, &c->hphi, &c->d_frags, &c->d_pairs,
                    &c->d_pieces, &c->d_items, &c->partials, &c->blocks, &c->dense_H,
                    &c->dense_S, &c->staging, &c->flag, &c->w_A, &c->w_L, &c->w_d, &c->w_e,
                    &c->w_tau, &c->w_tmp, &c->w_eval, &c->w_bar, &c->w_Q, &c->sp_rowptr, &c->sp_ents,
                    &c->blk_stage};
  for (DevBuf* b : bufs) free_buf(*b);
  ofm_free_extra(c);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  if (c->stage_ready) cudaEventDestroy(c->stage_ready);
  if (c->copy_done) cudaEventDestroy(c->copy_done);
  delete c;
}

extern "C" const char* ofm_last_error(const ofm_ctx* c) {
  if (!c) return "null context";
  return c->err.c_str();
}

// ------------------------------------------------------------- build -------

// Contraction plans (CUDA-core and tensor-core) for the current fragments,
// with work items of about c->asm_chunk points (0: the planner's choice,
// about 8 items per SM on CUDA cores, 4 per SM on tensor cores).  Any
// captured assembly graph refers to the old plan and is dropped.
static long long planner_chunk(const ofm_ctx* c) {
  return std::min<long long>(std::max<long long>(256, c->kh / (8 * 152)), 16384);
}

static ofm_status plan_contraction(ofm_ctx* c) {
  drop_graphs(c);
  const size_t es = elem_size(c);
  const long long chunk = c->asm_chunk > 0 ? c->asm_chunk : planner_chunk(c);
  c->simt_chunk = chunk;
  make_items_simt(c->frags, c->pairs, c->simt_tile, chunk, c->simt_pairs, c->simt_pieces,
                  c->simt_items, c->simt_partial_elems);
  const int np = (int)c->simt_pairs.size();
  OFM_TRY(ofm_ensure(c, c->d_pairs, sizeof(DevPair) * std::max(1, np), "pair table"));
  OFM_TRY(ofm_ensure(c, c->d_pieces, sizeof(Piece) * std::max<size_t>(1, c->simt_pieces.size()), "piece table"));
  OFM_TRY(ofm_ensure(c, c->d_items, sizeof(WorkItem) * std::max<size_t>(1, c->simt_items.size()), "work items"));
  OFM_CUDA(c, cudaMemcpyAsync(c->d_pairs.p, c->simt_pairs.data(), sizeof(DevPair) * np,
                              cudaMemcpyHostToDevice, c->stream));
  OFM_CUDA(c, cudaMemcpyAsync(c->d_pieces.p, c->simt_pieces.data(),
                              sizeof(Piece) * c->simt_pieces.size(), cudaMemcpyHostToDevice, c->stream));
  OFM_CUDA(c, cudaMemcpyAsync(c->d_items.p, c->simt_items.data(),
                              sizeof(WorkItem) * c->simt_items.size(), cudaMemcpyHostToDevice, c->stream));
  c->blk_elems = 0;
  for (auto& p : c->simt_pairs) c->blk_elems = std::max<long long>(c->blk_elems, p.blk_off + 2LL * c->frags[p.a].n * c->frags[p.b].n);
  OFM_TRY(ofm_ensure(c, c->blocks, sizeof(double) * c->blk_elems, "blocks"));
  c->finalize_bytes = (double)c->simt_partial_elems * (es == 8 ? 8 : 4) + 8.0 * c->blk_elems;
  c->region_stale = true;
  c->sp_stale = true;
  return ofm_plan_extra(c);
}

// Overlap counts and flops of the current pair list.
static void pair_totals(ofm_ctx* c) {
  c->flops = c->ks = c->kh = 0;
  for (auto& p : c->pairs) {
    c->ks += p.ks;
    c->kh += p.kh;
    c->flops += 2LL * c->frags[p.a].n * c->frags[p.b].n * (p.ks + p.kh);
  }
}

// The pair list of the current fragments: boxes that meet, then (when a
// distance cutoff is set, Sec. III.C) only the pairs whose fragments have
// atoms closer than d_cut; self pairs always stay.
static void plan_pairs(ofm_ctx* c) {
  make_pairs(c->grid, c->frags, c->pairs);
  if (!(c->cut_d > 0.0)) return;
  const std::vector<int>& off = c->cut_off;
  const std::vector<double>& xyz = c->cut_xyz;
  double L[3];
  for (int d = 0; d < 3; ++d) L[d] = c->grid.n[d] * c->grid.h;
  const double dc2 = c->cut_d * c->cut_d;
  auto near = [&](int a, int b) {
    for (int i = off[a]; i < off[a + 1]; ++i)
      for (int j = off[b]; j < off[b + 1]; ++j) {
        double r2 = 0.0;
        for (int d = 0; d < 3; ++d) {
          double x = xyz[3 * i + d] - xyz[3 * j + d];
          x -= L[d] * std::nearbyint(x / L[d]);   // minimum image
          r2 += x * x;
        }
        if (r2 < dc2) return true;
      }
    return false;
  };
  std::vector<HostPair> kept;
  for (auto& p : c->pairs)
    if (p.a == p.b || near(p.a, p.b)) kept.push_back(std::move(p));
  c->pairs.swap(kept);
}

// Everything that follows from the fragment list c->in_frags (geometry and
// state counts): fragment table, pairs, traffic figures, zeroed state and
// H phi storage, the device fragment table, launch shapes and contraction
// plans.  The eigensolver's workspace, sized for the old table, is dropped.
static ofm_status layout_fragments(ofm_ctx* c) {
  const int n_frag = c->nfrag;
  // the eigensolver's workspace is kept while the layout it was made for
  // (grid, storage, boxes and state counts) stays
  bool same = c->laid_storage == (int)c->storage && c->laid_frags.size() == c->in_frags.size() &&
              c->laid_grid.h == c->grid.h;
  for (int d = 0; d < 3; ++d) same = same && c->laid_grid.n[d] == c->grid.n[d];
  for (size_t a = 0; same && a < c->in_frags.size(); ++a)
    same = std::memcmp(&c->laid_frags[a], &c->in_frags[a], sizeof(ofm_fragment)) == 0;
  if (!same) {
    ofm_eig_free(c);
    c->stencil_form = 0;
    c->tuned_chunk = 0;
    c->schedule = 0;
  }
  c->laid_frags = c->in_frags;
  c->laid_grid = c->grid;
  c->laid_storage = (int)c->storage;
  make_frag_table(c->grid, c->in_frags.data(), n_frag, c->frags, c->state_elems);
  plan_pairs(c);
  c->basis = 0;
  c->apply_points = 0;
  for (auto& f : c->frags) {
    c->basis += f.n;
    c->apply_points += f.Pd * f.n;
  }
  pair_totals(c);
  c->frag_set.assign(n_frag, 0);
  const size_t es = elem_size(c);
  // algorithmic traffic: the H apply reads every state and V once and writes
  // H phi once on the dilated boxes; the contraction at its minimum reads
  // states and H phi once.
  c->apply_bytes = 0;
  for (auto& f : c->frags) c->apply_bytes += (double)f.Pd * (2.0 * f.n + 1.0) * es;
  c->contract_bytes = 0;
  for (auto& f : c->frags) c->contract_bytes += (double)f.Pd * 2.0 * f.n * es;
  // the region path's traffic: the apply + pack reads the states once and
  // writes phi and H phi as operands (8 bytes per point-state for BF16 hi+lo
  // and TF32, 4 for BF16); the contraction reads those operands once
  for (int k = 0; k < 5; ++k) {   // TF32, BF16, BF16 hi+lo, FP32, FP64 operands
    const double ob = k == 1 ? 2.0 : k == 4 ? 8.0 : 4.0;
    c->pack_bytes[k] = 0;
    c->region_bytes[k] = 0;
    for (auto& f : c->frags) {
      c->pack_bytes[k] += (double)f.Pd * f.n * (4.0 + 2.0 * ob) + (double)f.Pd * 4.0;
      c->region_bytes[k] += (double)f.Pd * f.n * 2.0 * ob;
    }
  }
  OFM_TRY(ofm_ensure(c, c->states, c->state_elems * es, "fragment states"));
  OFM_CUDA(c, cudaMemsetAsync(c->states.p, 0, c->state_elems * es, c->stream));
  // H phi (every element written by the apply) is allocated on first use
  c->hphi_ready = c->hphi.cap >= (size_t)(c->state_elems * es);
  OFM_TRY(ofm_ensure(c, c->d_frags, sizeof(DevFrag) * n_frag, "fragment table"));
  OFM_CUDA(c, cudaMemcpyAsync(c->d_frags.p, c->frags.data(), sizeof(DevFrag) * n_frag,
                              cudaMemcpyHostToDevice, c->stream));
  // H-apply launch: 2-D grid (chunks of the largest fragment x fragments)
  c->agrid = apply_grid(c->frags, es == 8, false, c->stencil_form);
  c->asm_chunk = c->tuned_chunk;
  OFM_TRY(plan_contraction(c));
  // host copies of tables are read back by later calls: wait for the uploads
  return sync(c, "fragment layout");
}

extern "C" ofm_status ofm_build_fragments(ofm_ctx* c, const ofm_grid* grid, const double* V,
                                          ofm_location v_loc, const ofm_fragment* frags,
                                          int n_frag, ofm_storage storage) {
  OFM_RANGE("ofm_build_fragments");
  if (!c) return OFM_ERR_INVALID;
  if (!grid || !V) return ofm_fail(c, OFM_ERR_INVALID, "grid and V must not be NULL");
  if (storage != OFM_STORE_FP32 && storage != OFM_STORE_FP64)
    return ofm_fail(c, OFM_ERR_INVALID, "unknown storage type");
  if (v_loc != OFM_HOST && v_loc != OFM_DEVICE)
    return ofm_fail(c, OFM_ERR_INVALID, "unknown V location");
  std::string msg;
  if (!validate_geometry(*grid, frags, n_frag, msg)) return ofm_fail(c, OFM_ERR_INVALID, msg);
  if (n_frag > 65535) return ofm_fail(c, OFM_ERR_INVALID, "at most 65535 fragments");

  c->built = c->have_states = c->assembled = c->dense_ready = c->factored = false;
  c->grid = *grid;
  c->storage = storage;
  c->nfrag = n_frag;
  c->in_frags.assign(frags, frags + n_frag);
  c->cut_d = 0.0;   // a distance cutoff belongs to the previous fragments
  c->cut_xyz.clear();
  c->cut_off.clear();

  const size_t es = elem_size(c);
  const long long npts = (long long)grid->n[0] * grid->n[1] * grid->n[2];
  OFM_TRY(ofm_ensure(c, c->V, npts * es, "potential"));
  if (v_loc == OFM_HOST) {
    OFM_TRY(ofm_ensure(c, c->staging, npts * sizeof(double), "staging"));
    OFM_CUDA(c, cudaMemcpyAsync(c->staging.p, V, npts * sizeof(double), cudaMemcpyHostToDevice,
                                c->stream));
    KTimer t(c, KC_CONVERT);
    launch_convert_V((const double*)c->staging.p, c->V.p, npts, es == 8, c->stream);
  } else {
    KTimer t(c, KC_CONVERT);
    launch_convert_V(V, c->V.p, npts, es == 8, c->stream);
  }
  OFM_TRY(check_launch(c, "convert V"));
  OFM_TRY(layout_fragments(c));
  c->built = true;
  return OFM_OK;
}

// A new potential on the same grid and fragments (Eq. 1): the states stay
// (they remain the basis), the pair list and plans stay, the blocks are
// discarded.
extern "C" ofm_status ofm_set_potential(ofm_ctx* c, const double* V, ofm_location v_loc) {
  OFM_RANGE("ofm_set_potential");
  if (!c) return OFM_ERR_INVALID;
  if (!c->built) return ofm_fail(c, OFM_ERR_STATE, "ofm_build_fragments must come first");
  if (!V) return ofm_fail(c, OFM_ERR_INVALID, "V must not be NULL");
  if (v_loc != OFM_HOST && v_loc != OFM_DEVICE) return ofm_fail(c, OFM_ERR_INVALID, "unknown V location");
  const size_t es = elem_size(c);
  const long long npts = (long long)c->grid.n[0] * c->grid.n[1] * c->grid.n[2];
  const double* src = V;
  if (v_loc == OFM_HOST) {
    OFM_TRY(ofm_ensure(c, c->staging, npts * sizeof(double), "staging"));
    OFM_CUDA(c, cudaMemcpyAsync(c->staging.p, V, npts * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    src = (const double*)c->staging.p;
  }
  {
    KTimer t(c, KC_CONVERT, 1, (double)npts * (8 + es));
    launch_convert_V(src, c->V.p, npts, es == 8, c->stream);
  }
  OFM_TRY(check_launch(c, "convert V"));
  c->assembled = c->dense_ready = c->factored = false;
  // host V: the staging buffer is reused by later calls
  return v_loc == OFM_HOST ? sync(c, "set_potential") : OFM_OK;
}

// Every assembled block in pair-list order: [H_ab | S_ab], n_a x n_b
// row-major FP64 each.
static ofm_status ofm_get_blocks_impl(ofm_ctx* c, double* HS, ofm_location loc, long long* n_elems) {
  OFM_RANGE("ofm_get_blocks");
  if (!c) return OFM_ERR_INVALID;
  if (!c->assembled) return ofm_fail(c, OFM_ERR_STATE, "ofm_assemble_HS must come first");
  if (loc != OFM_HOST && loc != OFM_DEVICE) return ofm_fail(c, OFM_ERR_INVALID, "unknown location");
  long long n = 0;
  for (const HostPair& p : c->pairs) n += 2LL * c->frags[p.a].n * c->frags[p.b].n;
  if (n_elems) *n_elems = n;
  if (!HS) return OFM_OK;
  OFM_TRY(ofm_wait_status(c));
  OFM_CUDA(c, cudaMemcpyAsync(HS, c->blocks.p, sizeof(double) * n,
                              loc == OFM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                              c->stream));
  return sync(c, "get_blocks");
}

extern "C" ofm_status ofm_get_blocks(ofm_ctx* c, double* HS, ofm_location loc, long long* n_elems) {
  const ofm_status st = ofm_get_blocks_impl(c, HS, loc, n_elems);
  if (st != OFM_OK || !c || !c->checks) return st;
  return ofm_check_guards_now(c, "ofm_get_blocks");
}

// Asynchronous read-back: the blocks are copied device-to-device into a
// staging buffer on the context stream (after the assembly), then to HS on
// the copy stream, so the next assembly runs while they travel.  Before the
// staging buffer is overwritten by a later call, the context stream waits
// for the previous transfer.
extern "C" ofm_status ofm_get_blocks_async(ofm_ctx* c, double* HS, long long* n_elems) {
  OFM_RANGE("ofm_get_blocks_async");
  if (!c) return OFM_ERR_INVALID;
  if (!c->assembled) return ofm_fail(c, OFM_ERR_STATE, "ofm_assemble_HS must come first");
  long long n = 0;
  for (const HostPair& p : c->pairs) n += 2LL * c->frags[p.a].n * c->frags[p.b].n;
  if (n_elems) *n_elems = n;
  if (!HS) return OFM_OK;
  if (!c->copy_stream) {
    OFM_CUDA(c, cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
    OFM_CUDA(c, cudaEventCreateWithFlags(&c->stage_ready, cudaEventDisableTiming));
    OFM_CUDA(c, cudaEventCreateWithFlags(&c->copy_done, cudaEventDisableTiming));
  }
  if (c->copy_pending) OFM_CUDA(c, cudaStreamWaitEvent(c->stream, c->copy_done, 0));
  OFM_TRY(ofm_ensure_big(c, c->blk_stage, sizeof(double) * (size_t)std::max<long long>(1, n),
                         "block staging"));
  OFM_CUDA(c, cudaMemcpyAsync(c->blk_stage.p, c->blocks.p, sizeof(double) * n,
                              cudaMemcpyDeviceToDevice, c->stream));
  OFM_CUDA(c, cudaEventRecord(c->stage_ready, c->stream));
  OFM_CUDA(c, cudaStreamWaitEvent(c->copy_stream, c->stage_ready, 0));
  OFM_CUDA(c, cudaMemcpyAsync(HS, c->blk_stage.p, sizeof(double) * n, cudaMemcpyDefault,
                              c->copy_stream));
  OFM_CUDA(c, cudaEventRecord(c->copy_done, c->copy_stream));
  c->copy_pending = true;
  return OFM_OK;
}

extern "C" ofm_status ofm_sync_blocks(ofm_ctx* c) {
  OFM_RANGE("ofm_sync_blocks");
  if (!c) return OFM_ERR_INVALID;
  if (c->copy_pending) {
    OFM_CUDA(c, cudaEventSynchronize(c->copy_done));
    c->copy_pending = false;
  }
  return ofm_wait_status(c);
}

// Test hook of the failure detection: the next launch of the chosen bounded
// device wait runs out (its producer withholds what it waits for), nothing
// faults or hangs, and the status reports OFM_ERR_TIMEOUT.
extern "C" ofm_status ofm_test_hold_wait(ofm_ctx* c, int what, int bound) {
  if (!c) return OFM_ERR_INVALID;
  if (what < 0 || what > 4 || bound < 0) return ofm_fail(c, OFM_ERR_INVALID, "what must be 0..4 and bound >= 0");
  if (what == 3) {
    // one byte of the block arena's guard band overwritten from the host
    if (!c->blocks.p) return ofm_fail(c, OFM_ERR_STATE, "no block arena yet");
    OFM_CUDA(c, cudaMemsetAsync((char*)c->blocks.p + c->blocks.cap + 7, 0x5A, 1, c->stream));
    return sync(c, "test_hold_wait");
  }
  if (what == 4) return ofm_region_test_corrupt(c);
  c->hold_tc = what == 1;
  c->hold_tri = what == 2;
  c->hold_bound = bound;
  return OFM_OK;
}

// Sec. III.C: pairs whose fragments' atoms are all at least d_cut apart are
// left out.  The cutoff and the atoms are kept for later re-plans (a state
// selection); a new ofm_build_fragments clears them.
extern "C" ofm_status ofm_set_pair_cutoff(ofm_ctx* c, const double* atom_xyz,
                                          const int* frag_atom_off, double d_cut) {
  if (!c) return OFM_ERR_INVALID;
  if (!c->built) return ofm_fail(c, OFM_ERR_STATE, "ofm_build_fragments must come first");
  const bool cut = atom_xyz != nullptr && d_cut > 0.0;
  if (cut) {
    if (!frag_atom_off || frag_atom_off[0] != 0)
      return ofm_fail(c, OFM_ERR_INVALID, "frag_atom_off must start at 0");
    for (int a = 0; a < c->nfrag; ++a)
      if (frag_atom_off[a + 1] < frag_atom_off[a])
        return ofm_fail(c, OFM_ERR_INVALID, "frag_atom_off must not decrease");
    c->cut_off.assign(frag_atom_off, frag_atom_off + c->nfrag + 1);
    c->cut_xyz.assign(atom_xyz, atom_xyz + 3 * (size_t)frag_atom_off[c->nfrag]);
    c->cut_d = d_cut;
  } else {
    c->cut_d = 0.0;
    c->cut_xyz.clear();
    c->cut_off.clear();
  }
  plan_pairs(c);
  pair_totals(c);
  c->assembled = c->dense_ready = c->factored = false;
  OFM_TRY(plan_contraction(c));
  return sync(c, "set_pair_cutoff");
}

// Sec. III, "Choice of the number of basis states per fragment": a sub-range
// of each fragment's states (e.g. its highest occupied ones) as the basis.
// The selected columns are copied on the device into the layout for the new
// state counts.
extern "C" ofm_status ofm_select_states(ofm_ctx* c, const int* first, const int* count) {
  OFM_RANGE("ofm_select_states");
  if (!c) return OFM_ERR_INVALID;
  if (!c->built || !c->have_states)
    return ofm_fail(c, OFM_ERR_STATE, "fragment states are not set (ofm_fragment_eigs or ofm_set_fragment_states)");
  if (!first || !count) return ofm_fail(c, OFM_ERR_INVALID, "first and count must not be NULL");
  for (int a = 0; a < c->nfrag; ++a)
    if (first[a] < 0 || count[a] < 1 || first[a] + count[a] > c->frags[a].n) {
      char buf[128];
      snprintf(buf, sizeof buf, "fragment %d: states [%d, %d) outside its %d states", a, first[a],
               first[a] + count[a], c->frags[a].n);
      return ofm_fail(c, OFM_ERR_INVALID, buf);
    }
  const size_t es = elem_size(c);
  const std::vector<DevFrag> old = c->frags;
  OFM_TRY(ofm_ensure(c, c->staging, c->state_elems * es, "staging"));
  OFM_CUDA(c, cudaMemcpyAsync(c->staging.p, c->states.p, c->state_elems * es,
                              cudaMemcpyDeviceToDevice, c->stream));
  for (int a = 0; a < c->nfrag; ++a) c->in_frags[a].n_states = count[a];
  OFM_TRY(layout_fragments(c));   // zeroed storage, new plans; the cutoff stays
  {
    KTimer t(c, KC_CONVERT);
    for (int a = 0; a < c->nfrag; ++a)
      launch_select_states(old[a], c->frags[a], first[a], c->staging.p, c->states.p, es == 8,
                           c->stream);
  }
  OFM_TRY(check_launch(c, "select states"));
  c->frag_set.assign(c->nfrag, 1);
  c->have_states = true;
  c->assembled = c->dense_ready = c->factored = false;
  return sync(c, "select_states");
}

// The H phi buffer of the current layout (outside any stream capture).
static ofm_status ensure_hphi(ofm_ctx* c) {
  if (c->hphi_ready) return OFM_OK;
  OFM_TRY(ofm_ensure_big(c, c->hphi, c->state_elems * elem_size(c), "H phi"));
  c->hphi_ready = true;
  return OFM_OK;
}

// ------------------------------------------------------------- states ------

extern "C" ofm_status ofm_set_fragment_states(ofm_ctx* c, int a, const double* phi, ofm_location loc) {
  OFM_RANGE("ofm_set_fragment_states");
  if (!c) return OFM_ERR_INVALID;
  if (!c->built) return ofm_fail(c, OFM_ERR_STATE, "ofm_build_fragments must come first");
  if (a < 0 || a >= c->nfrag || !phi) return ofm_fail(c, OFM_ERR_INVALID, "bad fragment index or NULL states");
  const DevFrag& F = c->frags[a];
  const long long P = (long long)F.ext[0] * F.ext[1] * F.ext[2];
  const double* src = phi;
  if (loc == OFM_HOST) {
    OFM_TRY(ofm_ensure(c, c->staging, P * F.n * sizeof(double), "staging"));
    OFM_CUDA(c, cudaMemcpyAsync(c->staging.p, phi, P * F.n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    src = (const double*)c->staging.p;
  } else if (loc != OFM_DEVICE) {
    return ofm_fail(c, OFM_ERR_INVALID, "unknown location");
  }
  { KTimer t(c, KC_CONVERT);
  launch_import_states((const DevFrag*)c->d_frags.p, a, F, src, c->states.p, c->storage == OFM_STORE_FP64, c->stream); }
  OFM_TRY(check_launch(c, "import states"));
  if (loc == OFM_HOST) OFM_TRY(sync(c, "set_fragment_states"));  // staging is reused
  c->frag_set[a] = 1;
  c->have_states = std::all_of(c->frag_set.begin(), c->frag_set.end(), [](char v) { return v != 0; });
  c->assembled = c->dense_ready = c->factored = false;
  return OFM_OK;
}

extern "C" ofm_status ofm_get_fragment_states(ofm_ctx* c, int a, double* out, ofm_location loc) {
  OFM_RANGE("ofm_get_fragment_states");
  if (!c) return OFM_ERR_INVALID;
  if (!c->built || !c->frag_set.size() || !c->frag_set[a < 0 || a >= c->nfrag ? 0 : a])
    return ofm_fail(c, OFM_ERR_STATE, "states of this fragment are not set");
  if (a < 0 || a >= c->nfrag || !out) return ofm_fail(c, OFM_ERR_INVALID, "bad fragment index or NULL output");
  const DevFrag& F = c->frags[a];
  const long long cnt = (long long)F.ext[0] * F.ext[1] * F.ext[2] * F.n;
  double* dst = out;
  if (loc == OFM_HOST) {
    OFM_TRY(ofm_ensure(c, c->staging, cnt * sizeof(double), "staging"));
    dst = (double*)c->staging.p;
  }
  launch_export_states(F, c->states.p, dst, c->storage == OFM_STORE_FP64, false, c->stream);
  OFM_TRY(check_launch(c, "export states"));
  if (loc == OFM_HOST)
    OFM_CUDA(c, cudaMemcpyAsync(out, dst, cnt * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  return sync(c, "get_fragment_states");
}

extern "C" ofm_status ofm_get_hphi(ofm_ctx* c, int b, double* out) {
  OFM_RANGE("ofm_get_hphi");
  if (!c) return OFM_ERR_INVALID;
  if (!c->assembled) return ofm_fail(c, OFM_ERR_STATE, "ofm_assemble_HS must come first");
  if (b < 0 || b >= c->nfrag || !out) return ofm_fail(c, OFM_ERR_INVALID, "bad fragment index or NULL output");
  const DevFrag& F = c->frags[b];
  const long long cnt = F.Pd * F.n;
  OFM_TRY(ofm_ensure(c, c->staging, cnt * sizeof(double), "staging"));
  // the region path never stores H phi in the states' layout: apply H here
  OFM_TRY(ensure_hphi(c));
  OFM_TRY(ofm_apply_h(c));
  launch_export_states(F, c->hphi.p, (double*)c->staging.p, c->storage == OFM_STORE_FP64, true, c->stream);
  OFM_TRY(check_launch(c, "export H phi"));
  OFM_CUDA(c, cudaMemcpyAsync(out, c->staging.p, cnt * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  return sync(c, "get_hphi");
}

// ------------------------------------------------------------- assembly ----

ofm_status ofm_apply_h(ofm_ctx* c) {
  if (!c->hphi_ready) return ofm_fail(c, OFM_ERR_STATE, "H phi buffer not allocated");
  KTimer t(c, KC_APPLY, 1, c->apply_bytes);
  launch_apply_global((const DevFrag*)c->d_frags.p, c->nfrag, c->agrid, c->V.p,
                      c->states.p, c->hphi.p, c->grid.n, c->grid.h,
                      c->storage == OFM_STORE_FP64, (int*)c->flag.p + OFM_FLAG_STENCIL, c->stream);
  c->stencil_check = true;
  return check_launch(c, "apply H");
}

// Whether an assembly takes the region-stacked schedule: requested (2), or
// by default (0) wherever its plan applies (FP32 storage; the CUDA-core
// precisions then run the plain region form).
static bool region_schedule(const ofm_ctx* c, ofm_precision prec, int sched) {
  (void)prec;
  if (sched == 1) return false;
  return sched == 2 ? ofm_region_ok(c) : ofm_region_default(c);
}

// Plans and buffers an assembly needs, made before any capture: the region
// plan (host tables after a re-plan), or the H phi buffer and the CUDA-core
// partial sums.
static ofm_status prepare_assembly(ofm_ctx* c, ofm_precision prec, int sched) {
  if (sched != 1 && c->region_stale) {
    OFM_TRY(ofm_region_plan(c));
    c->region_stale = false;
  }
  if (sched == 2 && !region_schedule(c, prec, sched))
    return ofm_fail(c, OFM_ERR_INVALID, std::string("region schedule unavailable: ") + ofm_region_why(c));
  if (region_schedule(c, prec, sched)) return ofm_region_prepare(c, prec);   // tables and buffers
  OFM_TRY(ensure_hphi(c));
  if (prec == OFM_PREC_FP64 || prec == OFM_PREC_FP32)
    OFM_TRY(ofm_ensure_big(c, c->partials, sizeof(double) * c->simt_partial_elems, "partials"));
  return OFM_OK;
}

// The launches of one assembly (a1 apply, a3/a4 contraction, a5 blocks) on
// the context stream; no host synchronisation, so it can be captured.
static ofm_status enqueue_assembly(ofm_ctx* c, ofm_precision prec, int sched) {
  if (region_schedule(c, prec, sched)) {
    c->last_schedule = 2;
    return ofm_region_run(c, prec);
  }
  OFM_TRY(ofm_apply_h(c));
  c->last_schedule = 1;
  if (prec == OFM_PREC_FP64 || prec == OFM_PREC_FP32) {
    { KTimer t(c, KC_CONTRACT, 1, c->contract_bytes, (double)c->flops);
    launch_contract_simt(prec, c->storage == OFM_STORE_FP64, (const DevFrag*)c->d_frags.p,
                         (const DevPair*)c->d_pairs.p, (const Piece*)c->d_pieces.p,
                         (const WorkItem*)c->d_items.p, (int)c->simt_items.size(), c->states.p,
                         c->hphi.p, c->partials.p, c->simt_tile, c->stream); }
    OFM_TRY(check_launch(c, "contract (CUDA cores)"));
    { KTimer t(c, KC_FINALIZE, 1, c->finalize_bytes);
    launch_finalize_simt(prec, (const DevFrag*)c->d_frags.p, (const DevPair*)c->d_pairs.p,
                         (int)c->simt_pairs.size(), (const WorkItem*)c->d_items.p, c->partials.p,
                         c->simt_tile, (double*)c->blocks.p, c->stream); }
    OFM_TRY(check_launch(c, "finalize blocks"));
  } else {
    OFM_TRY(ofm_contract_tc(c, prec));
  }
  return OFM_OK;
}

// Captures enqueue_assembly for `prec` as a CUDA graph.  A stream that cannot
// be captured (the legacy default stream, for one) turns graphs off for the
// context; the assembly is then launched directly.
static ofm_status capture_assembly(ofm_ctx* c, ofm_precision prec, int sched) {
  ofm::KStat before[KC_COUNT];
  for (int k = 0; k < KC_COUNT; ++k) before[k] = c->prof.st[k];
  if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    c->graphs_off = true;
    return OFM_OK;
  }
  const ofm_status st = enqueue_assembly(c, prec, sched);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(c->stream, &g);
  // nothing ran yet: the counters take what one replay adds
  for (int k = 0; k < KC_COUNT; ++k) {
    c->asm_cost[prec][k].launches = c->prof.st[k].launches - before[k].launches;
    c->asm_cost[prec][k].bytes = c->prof.st[k].bytes - before[k].bytes;
    c->asm_cost[prec][k].flops = c->prof.st[k].flops - before[k].flops;
    c->prof.st[k] = before[k];
  }
  c->asm_tc[prec] = c->tc_check;
  c->asm_sched[prec] = sched;
  c->tc_check = false;
  c->stencil_check = false;
  if (st != OFM_OK || e != cudaSuccess || !g ||
      cudaGraphInstantiate(&c->asm_exec[prec], g, 0) != cudaSuccess) {
    cudaGetLastError();
    c->asm_exec[prec] = nullptr;
    c->graphs_off = true;
  }
  if (g) cudaGraphDestroy(g);
  return OFM_OK;
}

static ofm_status ofm_assemble_HS_impl(ofm_ctx* c, ofm_precision prec, const ofm_assemble_opts* opts) {
  OFM_RANGE("ofm_assemble_HS");
  if (!c) return OFM_ERR_INVALID;
  c->fault_due = c->fault == OFM_FAULT_TIMEOUT;   // host-side injection: the next status read
  if (!c->built) return ofm_fail(c, OFM_ERR_STATE, "ofm_build_fragments must come first");
  if (!c->have_states) return ofm_fail(c, OFM_ERR_STATE, "fragment states are not set (ofm_fragment_eigs or ofm_set_fragment_states)");
  if (prec < OFM_PREC_FP64 || prec > OFM_PREC_BF16X3) return ofm_fail(c, OFM_ERR_INVALID, "unknown precision");
  if (prec != OFM_PREC_FP64 && c->storage == OFM_STORE_FP64)
    return ofm_fail(c, OFM_ERR_INVALID, "FP32 and tensor-core contractions need FP32 storage");
  long long chunk = opts ? opts->chunk_points : 0;
  const bool use_graph = opts ? opts->use_graph != 0 : true;
  int sched = opts ? opts->schedule : 0;
  if (chunk < 0) return ofm_fail(c, OFM_ERR_INVALID, "chunk_points must be >= 0");
  if (sched < 0 || sched > 2) return ofm_fail(c, OFM_ERR_INVALID, "schedule must be 0, 1 or 2");
  // the autotuned schedule is the tensor-core one; the CUDA-core precisions
  // take the plan's default unless one is requested
  if (sched == 0 && prec != OFM_PREC_FP64 && prec != OFM_PREC_FP32) sched = c->schedule;
  if (chunk == 0) chunk = c->tuned_chunk;
  if (chunk != c->asm_chunk) {
    c->asm_chunk = chunk;
    OFM_TRY(plan_contraction(c));
  }
  c->assembled = c->dense_ready = c->factored = false;
  OFM_TRY(prepare_assembly(c, prec, sched));
  const bool held = c->hold_tc && region_schedule(c, prec, sched) && prec != OFM_PREC_FP64 &&
                    prec != OFM_PREC_FP32;   // one direct launch
  if (c->asm_exec[prec] && c->asm_sched[prec] != sched) {
    cudaGraphExecDestroy(c->asm_exec[prec]);
    c->asm_exec[prec] = nullptr;
  }
  if (use_graph && !c->prof.on && !c->graphs_off && !held) {
    if (!c->asm_exec[prec]) OFM_TRY(capture_assembly(c, prec, sched));
    if (c->asm_exec[prec]) {
      OFM_CUDA(c, cudaGraphLaunch(c->asm_exec[prec], c->stream));
      for (int k = 0; k < KC_COUNT; ++k) {
        c->prof.st[k].launches += c->asm_cost[prec][k].launches;
        c->prof.st[k].bytes += c->asm_cost[prec][k].bytes;
        c->prof.st[k].flops += c->asm_cost[prec][k].flops;
      }
      c->stencil_check = !region_schedule(c, prec, sched);
      if (c->asm_tc[prec]) c->tc_check = true;
      c->last_schedule = region_schedule(c, prec, sched) ? 2 : 1;
      c->assembled = true;
      return OFM_OK;
    }
  }
  OFM_TRY(enqueue_assembly(c, prec, sched));
  c->assembled = true;
  return OFM_OK;
}

extern "C" ofm_status ofm_assemble_HS(ofm_ctx* c, ofm_precision prec, const ofm_assemble_opts* opts) {
  const ofm_status st = ofm_assemble_HS_impl(c, prec, opts);
  if (st != OFM_OK || !c || !c->checks) return st;
  return ofm_check_guards_now(c, "ofm_assemble_HS");
}

// Measuring autotuner of the assembly schedule: every (stencil form, points
// per work item) candidate is planned, run once (which captures its graph)
// and then timed over `reps` runs with CUDA events on the ctx stream; the
// fastest becomes the ctx's schedule.  The blocks are recomputed with it at
// the end, so the ctx holds an assembly of the chosen plan.
extern "C" ofm_status ofm_autotune_assembly(ofm_ctx* c, ofm_precision prec, const int* chunks,
                                            int n_chunks, int reps, double* times_ms,
                                            ofm_tune_result* out) {
  OFM_RANGE("ofm_autotune_assembly");
  if (!c) return OFM_ERR_INVALID;
  if (!c->built) return ofm_fail(c, OFM_ERR_STATE, "ofm_build_fragments must come first");
  if (!c->have_states) return ofm_fail(c, OFM_ERR_STATE, "fragment states are not set (ofm_fragment_eigs or ofm_set_fragment_states)");
  if (c->prof.on) return ofm_fail(c, OFM_ERR_STATE, "turn profiling off while tuning");
  if (reps < 1) return ofm_fail(c, OFM_ERR_INVALID, "reps must be >= 1");
  if (chunks && n_chunks < 1) return ofm_fail(c, OFM_ERR_INVALID, "n_chunks must be >= 1");
  std::vector<long long> cand;
  if (chunks) {
    for (int i = 0; i < n_chunks; ++i) {
      if (chunks[i] <= 0) return ofm_fail(c, OFM_ERR_INVALID, "chunk candidates must be > 0");
      cand.push_back(chunks[i]);
    }
  } else {
    // the planner's own size for this contraction, and 1/4 .. 4 times it
    const bool tc = prec >= OFM_PREC_TF32;
    const long long base = tc ? std::max<long long>(1024, c->kh / (4 * 152)) : planner_chunk(c);
    for (int m = -2; m <= 2; ++m)
      cand.push_back(std::max<long long>(64, m < 0 ? base >> -m : base << m));
  }
  const int nc = (int)cand.size();
  const size_t es = elem_size(c);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  OFM_CUDA(c, cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return ofm_cuda_check(c, cudaGetLastError(), "cudaEventCreate");
  }
  double best = -1.0;
  int best_form = 1;
  long long best_chunk = cand[0];
  int tried = 0;
  ofm_status st = OFM_OK;
  ofm_assemble_opts o{};
  o.use_graph = 1;
  o.schedule = 1;
  const bool tcp = prec >= OFM_PREC_TF32;
  for (int form = 1; form <= 2 && st == OFM_OK; ++form) {
    const ApplyGrid g = apply_grid(c->frags, es == 8, false, form);
    const bool fits = form == 1 || g.staged;
    for (int i = 0; i < nc && st == OFM_OK; ++i) {
      if (times_ms) times_ms[(form - 1) * nc + i] = -1.0;
      if (!fits) continue;
      drop_graphs(c);
      c->agrid = g;
      c->stencil_form = form;
      o.chunk_points = (int)cand[i];
      st = ofm_assemble_HS(c, prec, &o);   // plans, captures and runs once
      if (st != OFM_OK) break;
      if ((st = ofm_wait_status(c)) != OFM_OK) break;
      if (cudaEventRecord(e0, c->stream) != cudaSuccess) { st = ofm_cuda_check(c, cudaGetLastError(), "event"); break; }
      for (int r = 0; r < reps && st == OFM_OK; ++r) st = ofm_assemble_HS(c, prec, &o);
      if (st != OFM_OK) break;
      if (cudaEventRecord(e1, c->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
        st = ofm_cuda_check(c, cudaGetLastError(), "autotune timing");
        break;
      }
      if ((st = ofm_wait_status(c)) != OFM_OK) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      const double t = (double)ms / reps;
      if (times_ms) times_ms[(form - 1) * nc + i] = t;
      ++tried;
      if (best < 0.0 || t < best) {
        best = t;
        best_form = form;
        best_chunk = cand[i];
      }
    }
  }
  // the region schedule (tensor-core precisions, where its plan applies)
  double region_ms = -1.0;
  int best_sched = 1;
  if (st == OFM_OK && tcp) {
    if (c->region_stale) {
      st = ofm_region_plan(c);
      c->region_stale = false;
    }
    if (st == OFM_OK && ofm_region_ok(c)) {
      o.schedule = 2;
      st = ofm_assemble_HS(c, prec, &o);
      if (st == OFM_OK) st = ofm_wait_status(c);
      if (st == OFM_OK && cudaEventRecord(e0, c->stream) != cudaSuccess) st = ofm_cuda_check(c, cudaGetLastError(), "event");
      for (int r = 0; r < reps && st == OFM_OK; ++r) st = ofm_assemble_HS(c, prec, &o);
      if (st == OFM_OK && (cudaEventRecord(e1, c->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
        st = ofm_cuda_check(c, cudaGetLastError(), "autotune timing");
      if (st == OFM_OK) st = ofm_wait_status(c);
      if (st == OFM_OK) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        region_ms = (double)ms / reps;
        ++tried;
        if (best < 0.0 || region_ms < best) {
          best = region_ms;
          best_sched = 2;
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // the chosen schedule (the default one after a failure), then one assembly
  // with it
  drop_graphs(c);
  c->stencil_form = st == OFM_OK ? best_form : 0;
  c->tuned_chunk = st == OFM_OK ? best_chunk : 0;
  c->schedule = st == OFM_OK && tcp ? best_sched : 0;
  c->agrid = apply_grid(c->frags, es == 8, false, c->stencil_form);
  c->asm_chunk = -1;   // re-plan at the next assembly
  if (st != OFM_OK) return st;
  OFM_TRY(ofm_assemble_HS(c, prec, nullptr));
  OFM_TRY(ofm_wait_status(c));
  if (out) {
    out->chunk_points = (int)best_chunk;
    out->stencil_form = best_form;
    out->ms = best;
    out->n_tried = tried;
    out->schedule = best_sched;
    out->region_ms = region_ms;
  }
  return sync(c, "autotuned assembly");
}

extern "C" ofm_status ofm_get_pairs(ofm_ctx* c, int* n_pairs, int* pair_ab) {
  if (!c) return OFM_ERR_INVALID;
  if (!c->built) return ofm_fail(c, OFM_ERR_STATE, "ofm_build_fragments must come first");
  if (!n_pairs) return ofm_fail(c, OFM_ERR_INVALID, "n_pairs must not be NULL");
  *n_pairs = (int)c->pairs.size();
  if (pair_ab)
    for (size_t i = 0; i < c->pairs.size(); ++i) {
      pair_ab[2 * i] = c->pairs[i].a;
      pair_ab[2 * i + 1] = c->pairs[i].b;
    }
  return OFM_OK;
}

extern "C" ofm_status ofm_get_plan_info(ofm_ctx* c, ofm_plan_info* info) {
  if (!c) return OFM_ERR_INVALID;
  if (!c->built) return ofm_fail(c, OFM_ERR_STATE, "ofm_build_fragments must come first");
  if (!info) return ofm_fail(c, OFM_ERR_INVALID, "info must not be NULL");
  info->n_frag = c->nfrag;
  info->n_pairs = (int)c->pairs.size();
  info->basis_size = c->basis;
  info->n_work_items = (int)c->simt_items.size();
  info->pair_flops = c->flops;
  info->overlap_points_s = c->ks;
  info->overlap_points_h = c->kh;
  info->state_bytes = c->state_elems * (long long)elem_size(c);
  info->hphi_bytes = c->state_elems * (long long)elem_size(c);
  info->apply_points = c->apply_points;
  info->last_schedule = c->last_schedule;
  info->pad_ = 0;
  return OFM_OK;
}

extern "C" ofm_status ofm_get_block(ofm_ctx* c, int a, int b, double* H_ab, double* S_ab) {
  OFM_RANGE("ofm_get_block");
  if (!c) return OFM_ERR_INVALID;
  if (!c->assembled) return ofm_fail(c, OFM_ERR_STATE, "ofm_assemble_HS must come first");
  if (a < 0 || b < 0 || a >= c->nfrag || b >= c->nfrag) return ofm_fail(c, OFM_ERR_INVALID, "bad fragment index");
  OFM_TRY(ofm_wait_status(c));
  const bool swap = a > b;
  const int lo = swap ? b : a, hi = swap ? a : b;
  const int na = c->frags[a].n, nb = c->frags[b].n;
  const int p = find_pair(c, lo, hi);
  if (p < 0) {
    if (H_ab) std::memset(H_ab, 0, sizeof(double) * na * nb);
    if (S_ab) std::memset(S_ab, 0, sizeof(double) * na * nb);
    return OFM_OK;
  }
  const int nlo = c->frags[lo].n, nhi = c->frags[hi].n;
  std::vector<double> tmp(2LL * nlo * nhi);
  OFM_CUDA(c, cudaMemcpyAsync(tmp.data(), (const double*)c->blocks.p + c->simt_pairs[p].blk_off,
                              sizeof(double) * tmp.size(), cudaMemcpyDeviceToHost, c->stream));
  OFM_TRY(sync(c, "get_block"));
  const double* Hs = tmp.data();
  const double* Ss = tmp.data() + (long long)nlo * nhi;
  for (int i = 0; i < na; ++i)
    for (int m = 0; m < nb; ++m) {
      const long long src = swap ? (long long)m * nhi + i : (long long)i * nhi + m;
      if (H_ab) H_ab[(long long)i * nb + m] = Hs[src];
      if (S_ab) S_ab[(long long)i * nb + m] = Ss[src];
    }
  return OFM_OK;
}

ofm_status ofm_make_dense(ofm_ctx* c) {
  if (c->dense_ready) return OFM_OK;
  if (!c->assembled) return ofm_fail(c, OFM_ERR_STATE, "ofm_assemble_HS must come first");
  OFM_TRY(ofm_wait_status(c));
  const long long n = c->basis;
  OFM_TRY(ofm_ensure(c, c->dense_H, sizeof(double) * n * n, "dense H"));
  OFM_TRY(ofm_ensure(c, c->dense_S, sizeof(double) * n * n, "dense S"));
  OFM_CUDA(c, cudaMemsetAsync(c->dense_H.p, 0, sizeof(double) * n * n, c->stream));
  OFM_CUDA(c, cudaMemsetAsync(c->dense_S.p, 0, sizeof(double) * n * n, c->stream));
  { KTimer t(c, KC_SCATTER);
  launch_scatter_dense((const DevFrag*)c->d_frags.p, (const DevPair*)c->d_pairs.p,
                       (int)c->simt_pairs.size(), (const double*)c->blocks.p, (int)n,
                       (double*)c->dense_H.p, (double*)c->dense_S.p, c->stream); }
  OFM_TRY(check_launch(c, "scatter dense"));
  c->dense_n = (int)n;
  c->dense_ready = true;
  c->factored = false;
  return OFM_OK;
}

extern "C" ofm_status ofm_get_dense_HS(ofm_ctx* c, double* H, double* S, ofm_location loc) {
  OFM_RANGE("ofm_get_dense_HS");
  if (!c) return OFM_ERR_INVALID;
  if (!c->dense_ready) OFM_TRY(ofm_make_dense(c));
  const size_t bytes = sizeof(double) * (size_t)c->dense_n * c->dense_n;
  const cudaMemcpyKind k = loc == OFM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (H) OFM_CUDA(c, cudaMemcpyAsync(H, c->dense_H.p, bytes, k, c->stream));
  if (S) OFM_CUDA(c, cudaMemcpyAsync(S, c->dense_S.p, bytes, k, c->stream));
  return sync(c, "get_dense_HS");
}

extern "C" ofm_status ofm_set_dense_HS(ofm_ctx* c, int n, const double* H, const double* S) {
  OFM_RANGE("ofm_set_dense_HS");
  if (!c) return OFM_ERR_INVALID;
  if (n < 1 || !H || !S) return ofm_fail(c, OFM_ERR_INVALID, "need n >= 1 and non-NULL H, S");
  const size_t bytes = sizeof(double) * (size_t)n * n;
  OFM_TRY(ofm_ensure(c, c->dense_H, bytes, "dense H"));
  OFM_TRY(ofm_ensure(c, c->dense_S, bytes, "dense S"));
  OFM_CUDA(c, cudaMemcpyAsync(c->dense_H.p, H, bytes, cudaMemcpyHostToDevice, c->stream));
  OFM_CUDA(c, cudaMemcpyAsync(c->dense_S.p, S, bytes, cudaMemcpyHostToDevice, c->stream));
  OFM_TRY(sync(c, "set_dense_HS"));
  c->dense_n = n;
  c->dense_ready = true;
  c->factored = false;
  c->assembled = false;  // the dense pencil no longer comes from the blocks
  return OFM_OK;
}

// ------------------------------------------------------------- Eq. 2 -------

static ofm_status ofm_window_eigs_impl(ofm_ctx* c, double E_lo, double E_hi, int max_out,
                                      double* E_out, int* n_out, double* C_out) {
  OFM_RANGE("ofm_window_eigs");
  if (!c) return OFM_ERR_INVALID;
  if (!n_out || (max_out > 0 && !E_out) || max_out < 0 || !(E_lo <= E_hi))
    return ofm_fail(c, OFM_ERR_INVALID, "bad window arguments");
  if (!c->dense_ready) OFM_TRY(ofm_make_dense(c));
  if (!c->factored) OFM_TRY(ofm_window_factor(c));
  int i_lo = 0, i_hi = 0;
  OFM_TRY(ofm_window_count(c, E_lo, E_hi, &i_lo, &i_hi));
  *n_out = i_hi - i_lo;
  const int m = std::min(*n_out, max_out);
  if (m > 0) OFM_TRY(ofm_window_bisect(c, i_lo, i_lo + m, E_out));
  if (C_out && m > 0) OFM_TRY(ofm_window_vectors(c, m, E_out, C_out));
  return OFM_OK;
}

extern "C" ofm_status ofm_window_eigs(ofm_ctx* c, double E_lo, double E_hi, int max_out, double* E_out, int* n_out, double* C_out) {
  const ofm_status st = ofm_window_eigs_impl(c, E_lo, E_hi, max_out, E_out, n_out, C_out);
  if (st != OFM_OK || !c || !c->checks) return st;
  return ofm_check_guards_now(c, "ofm_window_eigs");
}

static ofm_status ofm_eigs_by_index_impl(ofm_ctx* c, int i_lo, int i_hi, double* E_out) {
  OFM_RANGE("ofm_eigs_by_index");
  if (!c) return OFM_ERR_INVALID;
  if (!c->dense_ready) OFM_TRY(ofm_make_dense(c));
  if (i_lo < 0 || i_hi > c->dense_n || i_lo > i_hi || (!E_out && i_hi > i_lo))
    return ofm_fail(c, OFM_ERR_INVALID, "bad index range");
  if (!c->factored) OFM_TRY(ofm_window_factor(c));
  if (i_hi > i_lo) OFM_TRY(ofm_window_bisect(c, i_lo, i_hi, E_out));
  return OFM_OK;
}

extern "C" ofm_status ofm_eigs_by_index(ofm_ctx* c, int i_lo, int i_hi, double* E_out) {
  const ofm_status st = ofm_eigs_by_index_impl(c, i_lo, i_hi, E_out);
  if (st != OFM_OK || !c || !c->checks) return st;
  return ofm_check_guards_now(c, "ofm_eigs_by_index");
}

// A window anchored at an index: E_{i_lo} and every later eigenvalue up to
// E_{i_lo} + width.  An FP32 estimate of the window's size sizes ONE
// multisection launch over [i_lo, i_lo + estimate + pad); the FP64
// eigenvalues then decide the window exactly (more are computed when the
// last one is still inside).
static ofm_status ofm_window_from_index_impl(ofm_ctx* c, int i_lo, double width, int max_out,
                                            double* E_out, int* n_out) {
  OFM_RANGE("ofm_window_from_index");
  if (!c) return OFM_ERR_INVALID;
  if (!n_out || (max_out > 0 && !E_out) || max_out < 0 || !(width >= 0.0))
    return ofm_fail(c, OFM_ERR_INVALID, "bad window arguments");
  if (!c->dense_ready) OFM_TRY(ofm_make_dense(c));
  if (!c->factored) OFM_TRY(ofm_window_factor(c));
  const int n = c->dense_n;
  if (i_lo < 0 || i_lo >= n) return ofm_fail(c, OFM_ERR_INVALID, "i_lo outside the spectrum");
  int est = n;
  OFM_TRY(ofm_window_size_estimate(c, i_lo, width, &est));
  int i_hi = std::min(n, std::max(i_lo + 1, est + 8));
  std::vector<double> E(i_hi - i_lo);
  OFM_TRY(ofm_window_bisect(c, i_lo, i_hi, E.data()));
  const double top = E[0] + width;
  while (E.back() <= top && i_hi < n) {   // the estimate fell short: extend
    const int more = std::min(n, i_hi + std::max(64, i_hi - i_lo)) - i_hi;
    E.resize(E.size() + more);
    OFM_TRY(ofm_window_bisect(c, i_hi, i_hi + more, E.data() + (i_hi - i_lo)));
    i_hi += more;
  }
  int cnt = 0;
  while (cnt < (int)E.size() && E[cnt] <= top) ++cnt;
  *n_out = cnt;
  if (max_out > 0) std::copy(E.begin(), E.begin() + std::min(cnt, max_out), E_out);
  return OFM_OK;
}

extern "C" ofm_status ofm_window_from_index(ofm_ctx* c, int i_lo, double width, int max_out, double* E_out, int* n_out) {
  const ofm_status st = ofm_window_from_index_impl(c, i_lo, width, max_out, E_out, n_out);
  if (st != OFM_OK || !c || !c->checks) return st;
  return ofm_check_guards_now(c, "ofm_window_from_index");
}

// Sec. III, occupation with a HOMO basis: e_a = <HOMO_a|H|HOMO_a> with the
// whole-system H (the last diagonal entry of the assembled H_aa: the
// fragment's highest basis state), e_ref = max_a e_a, then the first spacing
// wider than gap_min between consecutive eigenvalues of Eq. 2, scanning up
// from the largest eigenvalue <= e_ref (the spacing that holds e_ref counts).
extern "C" ofm_status ofm_homo_lumo_gap(ofm_ctx* c, double gap_min, double* e_ref_out,
                                        double* E_homo, double* E_lumo, int* n_occ) {
  OFM_RANGE("ofm_homo_lumo_gap");
  if (!c) return OFM_ERR_INVALID;
  if (!c->assembled) return ofm_fail(c, OFM_ERR_STATE, "ofm_assemble_HS must come first");
  if (!(gap_min > 0.0) || !E_homo || !E_lumo || !n_occ)
    return ofm_fail(c, OFM_ERR_INVALID, "gap_min must be positive and the outputs not NULL");
  OFM_TRY(ofm_wait_status(c));
  std::vector<double> e(c->nfrag);
  for (int a = 0; a < c->nfrag; ++a) {
    const int p = find_pair(c, a, a);
    const long long n = c->frags[a].n;
    if (p < 0) return ofm_fail(c, OFM_ERR_STATE, "a self pair is missing");
    OFM_CUDA(c, cudaMemcpyAsync(&e[a], (const double*)c->blocks.p + c->simt_pairs[p].blk_off + n * n - 1,
                                sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  }
  OFM_TRY(sync(c, "homo_lumo_gap"));
  const double e_ref = *std::max_element(e.begin(), e.end());
  if (e_ref_out) *e_ref_out = e_ref;
  if (!c->dense_ready) OFM_TRY(ofm_make_dense(c));
  if (!c->factored) OFM_TRY(ofm_window_factor(c));
  int below = 0, upto = 0;
  OFM_TRY(ofm_window_count(c, e_ref, e_ref, &below, &upto));   // upto: eigenvalues <= e_ref
  const int n = c->dense_n;
  int k = std::max(upto - 1, 0);
  const int chunk = 64;
  std::vector<double> E(chunk + 1);
  while (k + 1 < n) {
    const int m = std::min(chunk + 1, n - k);   // E_k .. E_{k+m-1}
    OFM_TRY(ofm_window_bisect(c, k, k + m, E.data()));
    for (int i = 0; i + 1 < m; ++i)
      if (E[i + 1] - E[i] > gap_min) {
        *E_homo = E[i];
        *E_lumo = E[i + 1];
        *n_occ = k + i + 1;
        return OFM_OK;
      }
    k += m - 1;
  }
  return ofm_fail(c, OFM_ERR_INVALID, "no spacing wider than gap_min at or above e_ref");
}
