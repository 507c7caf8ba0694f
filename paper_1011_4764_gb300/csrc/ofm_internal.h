// Internal declarations of the OFM library: context, plan tables, kernel
// launchers.  Not part of the public ABI (see include/ofm.h).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "ofm.h"

namespace ofm {

// An NVTX range for the lifetime of a C-ABI call (visible in nsys/ncu
// timelines; a no-op without a tool attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
#define OFM_RANGE(name) ::ofm::NvtxRange ofm_nvtx_range_(name)

// ---------------------------------------------------------------- geometry --

// One fragment as the kernels see it.  States and H phi are stored
// point-major on the dilated box: element (p, s) at off + p * ld + s, where p
// is the dilated-local linear index (x fastest) and s the state.  Halo points
// of the states are zero.
struct DevFrag {
  int doff[3];     // global coordinate of dilated-local 0
  int dext[3];     // dilated extent (storage box)
  int lo[3];       // first interior (box) coordinate, dilated-local
  int ext[3];      // box extent
  int full[3];     // 1 when the box spans the whole grid in that dimension
  int n;           // states
  int ld;          // row stride in elements (n rounded up to 4)
  int basis0;      // first basis index of this fragment
  long long Pd;    // points of the dilated box
  long long off;   // element offset of this fragment in the state / H phi arenas
};

// A product of per-dimension runs: a sub-box of B_a ∩ B_b+ that is a
// contiguous box in both fragments' dilated-local coordinates.
struct Piece {
  int la[3];       // start, dilated-local coordinates of fragment a
  int lb[3];       // start, dilated-local coordinates of fragment b
  int len[3];      // extent
};

struct DevPair {
  int a, b;
  int item0, nitem;     // work items of this pair (contiguous)
  int nchunk;           // K chunks per output tile
  int mtiles, ntiles;   // output tiles (SIMT path)
  long long blk_off;    // element offset of [H_ab | S_ab] in the block arena
};

// One unit of contraction work: rows [r0, r1) of a piece (a row is one
// x-run of len[0] points at fixed y, z), for one output tile.
struct WorkItem {
  int pair;
  int piece;
  int r0, r1;
  int mt, nt;
  long long part_off;   // element offset of this item's partial tile
};

struct HostPair {
  int a, b;
  long long ks, kh;           // |B_a ∩ B_b|, |B_a ∩ B_b+|
  std::vector<Piece> pieces;  // cover B_a ∩ B_b+
};

// ------------------------------------------------------------ device buffer --

struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
};

// ---------------------------------------------------------------- planner --

// Runs of one dimension: positions t of box a (0 <= t < ext_a) that lie in
// the (dilated) box b, grouped into maximal runs that are contiguous in both
// fragments' local coordinates.  Returns (t_start, lb_start, len) triples.
struct Run { int ta, lb, len; };
std::vector<Run> dim_runs(int n, int offa, int exta, int offb, int extb);
bool validate_geometry(const ofm_grid& g, const ofm_fragment* f, int nf, std::string& err);
void make_frag_table(const ofm_grid& g, const ofm_fragment* f, int nf, std::vector<DevFrag>& out,
                     long long& total_elems);
void make_pairs(const ofm_grid& g, const std::vector<DevFrag>& fr, std::vector<HostPair>& pairs);
// SIMT plan: items for output tiles of TILE x TILE, K chunks of ~chunk points.
void make_items_simt(const std::vector<DevFrag>& fr, const std::vector<HostPair>& pairs,
                     int tile, long long chunk, std::vector<DevPair>& dpairs,
                     std::vector<Piece>& pieces, std::vector<WorkItem>& items,
                     long long& partial_elems);

// ------------------------------------------------------------ kernels ------

// launch shape of the stencils: shared-memory staged (row tiles of ty rows,
// smem bytes per CTA) or register z-marching; z = chunks of zc planes
struct ApplyGrid {
  bool staged = false;
  int x = 1, z = 1, zc = 1, ty = 1, smem = 0;
};
// form: 0 register form unless OFM_STENCIL=staged, 1 register form, 2 staged
// form where it fits (else the register form)
ApplyGrid apply_grid(const std::vector<DevFrag>& fr, bool fp64, bool filter, int form = 0);
// flag: set to 1 when a bounded wait of the staged form gives up
void launch_apply_global(const DevFrag* d_fr, int nfrag, const ApplyGrid& g, const void* V,
                         const void* states, void* hphi, const int gn[3], double h, bool fp64,
                         int* flag, cudaStream_t s);
void launch_import_states(const DevFrag* d_fr, int a, const DevFrag& fa, const double* src,
                          void* states, bool fp64, cudaStream_t s);
void launch_export_states(const DevFrag& fa, const void* states, double* dst, bool fp64,
                          bool dilated_hphi, cudaStream_t s);
size_t cheb_filter_smem(const std::vector<DevFrag>& frags, bool fp64);
void launch_select_states(const DevFrag& Fo, const DevFrag& Fn, int first, const void* src,
                          void* dst, bool fp64, cudaStream_t s);
void launch_cheb_filter(const DevFrag* d_fr, int nfrag, int mmax, size_t smem, const void* V,
                        const void* X, void* Y, void* HY, const double* coef, int nsteps,
                        const int gn[3], double h, cudaStream_t s);
void launch_apply_filter(const DevFrag* d_fr, int nfrag, const ApplyGrid& g, const void* V,
                         const void* in, const void* prev, void* out, const double* coef,
                         const int gn[3], double h, bool fp64, int* flag, cudaStream_t s);
void launch_convert_V(const double* src, void* dst, long long n, bool fp64, cudaStream_t s);
void launch_contract_simt(int prec, bool store_fp64, const DevFrag* d_fr, const DevPair* d_pairs,
                          const Piece* d_pieces, const WorkItem* d_items, int nitems,
                          const void* states, const void* hphi, void* partials, int tile,
                          cudaStream_t s);
void launch_finalize_simt(int prec, const DevFrag* d_fr, const DevPair* d_pairs, int npairs,
                          const WorkItem* d_items, const void* partials, int tile,
                          double* blocks, cudaStream_t s);
void launch_scatter_dense(const DevFrag* d_fr, const DevPair* d_pairs, int npairs,
                          const double* blocks, int n, double* Hd, double* Sd, cudaStream_t s);

}  // namespace ofm

// ------------------------------------------------------------- profiling ----

namespace ofm {
enum KClass {
  KC_CONVERT, KC_APPLY, KC_CONTRACT, KC_FINALIZE, KC_SCATTER, KC_EIG_INIT, KC_FILTER, KC_GRAM,
  KC_RR, KC_ROTATE, KC_EXPORT, KC_CHOL, KC_REDUCE, KC_TRIDIAG, KC_BISECT, KC_VECTORS, KC_PENCIL,
  KC_COUNT
};
struct KStat {
  long long launches = 0;
  double ms = 0.0;
  double bytes = 0.0;
  double flops = 0.0;
};
const char* kclass_name(int k);
const char* kclass_row(int k);
}  // namespace ofm

struct ofm_prof {
  bool on = false;
  ofm::KStat st[ofm::KC_COUNT];
  std::vector<cudaEvent_t> pool;
  struct Pending { int k; cudaEvent_t a, b; };
  std::vector<Pending> pending;
};

// ------------------------------------------------------------- context ------

struct ofm_ctx {
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;
  std::string err;

  // state machine
  bool built = false;
  bool have_states = false;
  bool assembled = false;
  bool dense_ready = false;   // dense H, S hold the matrices to solve
  bool factored = false;      // tridiagonal form of the current dense pencil is ready

  ofm_grid grid{};
  ofm_storage storage = OFM_STORE_FP32;
  int nfrag = 0;
  int basis = 0;
  std::vector<ofm_fragment> in_frags;
  // layout the eigensolver's workspace was made for
  std::vector<ofm_fragment> laid_frags;
  ofm_grid laid_grid{};
  int laid_storage = -1;
  std::vector<ofm::DevFrag> frags;
  std::vector<ofm::HostPair> pairs;
  // distance cutoff on the pair list (Sec. III.C); cut_d <= 0: none
  double cut_d = 0.0;
  std::vector<double> cut_xyz;   // atom positions, 3 per atom, grouped by fragment
  std::vector<int> cut_off;      // nfrag + 1 offsets into the atoms
  long long state_elems = 0;
  long long flops = 0, ks = 0, kh = 0, apply_points = 0;

  // SIMT plan
  std::vector<ofm::DevPair> simt_pairs;
  std::vector<ofm::Piece> simt_pieces;
  std::vector<ofm::WorkItem> simt_items;
  long long simt_partial_elems = 0;
  int simt_tile = 64;
  long long simt_chunk = 0;

  std::vector<long long> blk_off;   // per pair
  long long blk_elems = 0;
  ofm::ApplyGrid agrid;                // launch shape of the a1 stencil
  // assembly schedule chosen by ofm_autotune_assembly (kept while the layout
  // stays): stencil form (0: default) and points per work item (0: planner)
  int stencil_form = 0;
  long long tuned_chunk = 0;

  // device buffers
  ofm::DevBuf V, states, hphi, d_frags, d_pairs, d_pieces, d_items, partials,
      blocks, dense_H, dense_S, staging, flag;
  ofm::DevBuf w_A, w_L, w_d, w_e, w_tau, w_tmp, w_eval, w_bar, w_Q;   // window-solver workspaces
  ofm::DevBuf sp_rowptr, sp_ents;   // block rows of the pencil for ofm_pencil_apply
  // asynchronous read-back of the blocks (ofm_get_blocks_async): a device
  // staging copy, and the device-to-host copy on a stream of its own
  ofm::DevBuf blk_stage;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t stage_ready = nullptr, copy_done = nullptr;
  bool copy_pending = false;
  bool sp_stale = true;             // rebuilt after the pair list or the plan changes
  double sp_flops_per_col = 0.0, sp_bytes_fixed = 0.0;
  int dense_n = 0;
  int window_fail_col = -1;
  std::vector<char> frag_set;       // per fragment: states imported or computed
  int last_eig_iters = 0;           // filter iterations of the last fragment eigensolve
  // algorithmic traffic of one launch, set by the planner
  double apply_bytes = 0, contract_bytes = 0, finalize_bytes = 0;
  ofm_prof prof;                    // per-kernel-class launch counts and event timing
  // assembly as CUDA graphs (one per precision, captured on first use with
  // profiling off); what one replay adds to the per-class counters
  long long asm_chunk = 0;          // contraction work-item points of the current plans (0: planner)
  cudaGraphExec_t asm_exec[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  ofm::KStat asm_cost[5][ofm::KC_COUNT];
  bool asm_tc[5] = {false, false, false, false, false};
  int asm_sched[5] = {0, 0, 0, 0, 0};   // schedule each graph was captured with
  bool graphs_off = false;          // capture failed once on this stream: launch directly
  bool tc_check = false;            // a tensor-core launch's timeout flag is unread
  bool stencil_check = false;       // a stencil launch's timeout flag is unread
  struct EigWork* eig = nullptr;    // fragment-eigensolver buffers and plan
  struct TcPlan* tc = nullptr;      // tensor-core contraction plan (one GEMM per pair)
  // region-stacked tensor-core contraction: plan (built on first use after a
  // re-plan), its segment coarsening, and the schedule of the tensor-core
  // assembly (0: region where its plan applies, else per pair; 1: per pair;
  // 2: region)
  struct RegionPlan* region = nullptr;
  bool region_stale = true;
  int region_wmin = 1;
  int schedule = 0;                 // the tuned or caller-set default schedule
  int last_schedule = 0;            // schedule of the last assembly (1 pair, 2 region)
  bool hphi_ready = false;          // the FP32/FP64 H phi buffer is allocated
  // failure injection: host-side (OFM_FAULT at ofm_create; never touches the
  // device) and the test hook that makes one bounded device wait run out
  int fault = 0;                    // OFM_FAULT_*
  bool fault_due = false;           // an injected timeout waits for the next status read
  int hold_tc = 0, hold_tri = 0;    // armed for the next launch
  int hold_bound = 0;               // polls before the held wait gives up (0: usual bound)
  double pack_bytes[5] = {0, 0, 0, 0, 0};     // algorithmic bytes of the apply + pack, per kind
  double region_bytes[5] = {0, 0, 0, 0, 0};   // algorithmic bytes of the region contraction, per kind
  // check mode (ofm_set_checks / OFM_CHECK): guard bands read after the
  // calls, bounds-checking kernel forms on the region schedule
  bool checks = false;
  bool bounds_check = false;        // a check-mode launch may have set OFM_FLAG_BOUNDS
  ofm::DevBuf guard_tab;            // device copy of the guard table
};

// words of the context's 16-int flag buffer: 0 pivot flag and 2..3 window
// counts (window solver), 8 staged-stencil wait timeout, 9 tensor-core wait
// timeout, 12 next work item of the region contraction, 13 the guard check's
// result, 14 a refused access of a check-mode kernel
constexpr int OFM_FLAG_STENCIL = 8;
constexpr int OFM_FLAG_TC = 9;
constexpr int OFM_FLAG_QUEUE = 12;   // work counter of the region contraction
constexpr int OFM_FLAG_GUARD = 13;   // first overwritten guard band (INT_MAX: none)
constexpr int OFM_FLAG_BOUNDS = 14;  // a check-mode kernel refused an access
constexpr size_t OFM_GUARD_BYTES = 256;   // guard band after every device buffer

// A device buffer whose guard band the check reads.
struct GuardRef {
  const void* p;
  size_t cap;
  const char* name;
};
void ofm_eig_guards(const ofm_ctx* c, std::vector<GuardRef>& out);
void ofm_region_guards(const ofm_ctx* c, std::vector<GuardRef>& out);
void ofm_tc_guards(const struct TcPlan* t, std::vector<GuardRef>& out);
ofm_status ofm_check_guards_now(ofm_ctx* c, const char* after);
ofm_status ofm_region_test_corrupt(ofm_ctx* c);

// host-side fault injection (environment variable OFM_FAULT read by ofm_create)
enum { OFM_FAULT_NONE = 0, OFM_FAULT_OOM = 1, OFM_FAULT_TIMEOUT = 2, OFM_FAULT_NONCONV = 3,
       OFM_FAULT_NOTPOSDEF = 4 };

// helpers used by every translation unit
ofm_status ofm_fail(ofm_ctx* c, ofm_status s, const std::string& msg);
ofm_status ofm_cuda_check(ofm_ctx* c, cudaError_t e, const char* what);
ofm_status ofm_ensure(ofm_ctx* c, ofm::DevBuf& b, size_t bytes, const char* what);
// ofm_ensure for the large lazily-sized buffers: when the device is out of
// memory it releases the fragment eigensolver's workspace (re-made by the next
// ofm_fragment_eigs) and tries once more
ofm_status ofm_ensure_big(ofm_ctx* c, ofm::DevBuf& b, size_t bytes, const char* what);

// cross-translation-unit steps
ofm_status ofm_apply_h(ofm_ctx* c);
ofm_status ofm_make_dense(ofm_ctx* c);
ofm_status ofm_plan_extra(ofm_ctx* c);        // tensor-core plan after a build
void ofm_free_extra(ofm_ctx* c);              // frees eig and tc
void ofm_eig_free(ofm_ctx* c);
void ofm_prof_release(ofm_ctx* c);            // waits for and frees timing events
void ofm_tc_free(ofm_ctx* c);
ofm_status ofm_contract_tc(ofm_ctx* c, ofm_precision prec);
// tensor-core plans over any fragment table (assembly, eigensolver Gram)
enum { OFM_TC_TF32 = 0, OFM_TC_BF16 = 1, OFM_TC_BF16X3 = 2, OFM_TC_TF32X3 = 3 };
ofm_status ofm_tc_plan_build(ofm_ctx* c, struct TcPlan** tp, const std::vector<ofm::DevFrag>& fr,
                             const std::vector<ofm::HostPair>& pairs,
                             const std::vector<long long>& blk_off, long long kh, long long chunk);
ofm_status ofm_tc_run(ofm_ctx* c, struct TcPlan* t, int kind, const ofm::DevFrag* d_frags,
                      const void* states, const void* hphi, double* blocks, int kclass_contract,
                      int kclass_finalize, double bytes, double flops);
bool ofm_tc_plan_ok(const struct TcPlan* t, int kind);   // the kind's staging fits
void ofm_tc_plan_free(struct TcPlan* t);
ofm_status ofm_wait_status(ofm_ctx* c);
// region-stacked contraction (region.cu)
ofm_status ofm_region_plan(ofm_ctx* c);
bool ofm_region_ok(const ofm_ctx* c);
bool ofm_region_default(const ofm_ctx* c);   // the plan applies and is not mostly padding
const char* ofm_region_why(const ofm_ctx* c);
ofm_status ofm_region_prepare(ofm_ctx* c, ofm_precision prec);   // device tables and buffers
ofm_status ofm_region_run(ofm_ctx* c, ofm_precision prec);
void ofm_region_free(ofm_ctx* c);
void ofm_region_stats(const ofm_ctx* c, long long* out);       // OFM_ERR_TIMEOUT if a bounded wait gave up
ofm_status ofm_window_factor(ofm_ctx* c);
// eigenvalues below lo and below-or-at hi of the factored pencil
ofm_status ofm_window_count(ofm_ctx* c, double lo, double hi, int* count_lo, int* count_hi);
ofm_status ofm_window_bisect(ofm_ctx* c, int i_lo, int i_hi, double* E_out);
ofm_status ofm_window_size_estimate(ofm_ctx* c, int i_lo, double width, int* i_end);
// eigenvectors for the m eigenvalues E (host, ascending) of the last bisection
ofm_status ofm_window_vectors(ofm_ctx* c, int m, const double* E, double* C_out);
ofm_status ofm_tridiag_persistent(ofm_ctx* c, double* A, int n, double* d, double* e, double* tau,
                                  double* pg);
void launch_count_below(const double* d, const double* e, int n, double x0, double x1, int* out,
                        cudaStream_t s);
bool launch_window_size(const double* d, const double* e, int n, int i_lo, double width, int* out,
                        cudaStream_t s);
bool launch_multisection(const double* d, const double* e, int n, int i_lo, int m, double* out,
                         cudaStream_t s);

// Counts the launches of one kernel class and, while profiling is on,
// brackets them with CUDA events on the context stream.
struct KTimer {
  ofm_ctx* c;
  int k;
  cudaEvent_t a = nullptr;
  // bytes / flops: algorithmic traffic and work of the launches (for the
  // roofline figures), not measured counters
  KTimer(ofm_ctx* c_, int k_, long long nlaunch = 1, double bytes = 0.0, double flops = 0.0);
  ~KTimer();
  void add(long long n);
};

#define OFM_CUDA(ctx, expr)                                             \
  do {                                                                  \
    cudaError_t _e = (expr);                                            \
    if (_e != cudaSuccess) return ofm_cuda_check((ctx), _e, #expr);     \
  } while (0)

#define OFM_TRY(expr)                           \
  do {                                          \
    ofm_status _s = (expr);                     \
    if (_s != OFM_OK) return _s;                \
  } while (0)
