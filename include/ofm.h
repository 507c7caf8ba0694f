/*
 * ofm.h -- C ABI of the GB300 overlapping-fragments-method (OFM) library.
 *
 * The method (Vukmirovic & Wang, "Overlapping fragments method for
 * electronic structure calculation of large systems", Sec. II): the system is
 * divided into mutually overlapping fragments; the lowest eigenstates of each
 * fragment form a basis; the whole-system Hamiltonian H and the overlap S are
 * represented in that basis,
 *     H_{ij,mn} = <phi_i^(j)| H |phi_m^(n)>,   S_{ij,mn} = <phi_i^(j)|phi_m^(n)>,
 * and the generalized eigenproblem sum_mn (H - E S) C = 0 (Eq. 2) is solved for
 * the states in an energy window.
 *
 * Discretisation used by every entry point:
 *   - periodic grid of n[0] x n[1] x n[2] points, spacing h (bohr); point
 *     (x,y,z) has linear index x + n0*(y + n1*z) (x fastest);
 *   - H = -1/2 Laplacian + V (Eq. 1 in atomic units), Laplacian = 7-point
 *     finite difference (sum of the six neighbours - 6 phi) / h^2;
 *   - fragment a is the box off + [0, ext) (mod n); its Hamiltonian is the
 *     principal submatrix of H on the box (zero outside; periodic wrap kept
 *     in a dimension that the box spans completely);
 *   - the dilated box B_a+ grows the box by one point on each side in every
 *     dimension with ext < n; H phi_a is non-zero only there;
 *   - states are unit-norm in the plain Euclidean grid sum; basis order is
 *     fragment-major, states ascending in fragment energy;
 *   - a pair a <= b is kept when box a meets the dilated box of b.
 *
 * Conventions:
 *   - Every call returns an ofm_status.  On failure a message is kept in the
 *     context (ofm_last_error) and the context stays valid for ofm_destroy.
 *     Calls out of order return OFM_ERR_STATE.  No exception crosses the ABI.
 *   - The context owns every device buffer it allocates.  The caller owns all
 *     pointers it passes; inputs are copied before the call returns (or, for
 *     device inputs, before work enqueued on the context stream reads them).
 *   - All device work is ordered on the context's CUDA stream.  Calls that
 *     return host data synchronise that stream before returning.
 *   - A "device" pointer is a CUDA global-memory address on the context's
 *     current device; a "host" pointer is ordinary (pageable or pinned) memory.
 */
#ifndef OFM_H
#define OFM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  OFM_OK = 0,
  OFM_ERR_INVALID = 1,        /* bad argument or geometry */
  OFM_ERR_OOM = 2,            /* device allocation failed */
  OFM_ERR_CUDA = 3,           /* a CUDA runtime call failed */
  OFM_ERR_NOT_CONVERGED = 4,  /* iteration cap reached (residuals reported) */
  OFM_ERR_NOT_POSDEF = 5,     /* Cholesky of S met a non-positive pivot */
  OFM_ERR_TIMEOUT = 6,        /* a bounded device-side wait gave up */
  OFM_ERR_STATE = 7,          /* call out of order */
  OFM_ERR_CORRUPT = 8         /* check mode: a guard band was overwritten or a device
                                 bounds check refused an access */
} ofm_status;

/* Arithmetic of the pair contraction (Sec. II, the H_ab / S_ab dot products). */
typedef enum {
  OFM_PREC_FP64 = 0,    /* FP64 products and sums (CUDA cores) */
  OFM_PREC_FP32 = 1,    /* FP32 products and sums (CUDA cores) */
  OFM_PREC_TF32 = 2,    /* tcgen05 kind::tf32, FP32 accumulation in TMEM */
  OFM_PREC_BF16 = 3,    /* tcgen05 kind::f16 (bf16 operands), FP32 accumulation */
  OFM_PREC_BF16X3 = 4   /* bf16 hi+lo split: hi*hi + hi*lo + lo*hi, FP32 accumulation */
} ofm_precision;

/* Storage type of the fragment states and of H phi in device memory. */
typedef enum { OFM_STORE_FP64 = 0, OFM_STORE_FP32 = 1 } ofm_storage;

typedef enum { OFM_HOST = 0, OFM_DEVICE = 1 } ofm_location;

typedef struct { int n[3]; double h; } ofm_grid;
typedef struct { int off[3]; int ext[3]; int n_states; } ofm_fragment;

/* Options of the batched fragment eigensolver (Chebyshev-filtered subspace
 * iteration with Rayleigh-Ritz).  Zero fields take the defaults in brackets. */
typedef struct {
  double tol;            /* stop when every max_i ||H phi_i - eps_i phi_i|| <= tol [1e-5 FP32, 1e-9 FP64] */
  int max_iter;          /* outer iterations [240] */
  int degree;            /* Chebyshev degree per iteration [32] */
  int extra_states;      /* guard vectors beyond n_states [max(4, n/4), or one or two fewer
                            (at least 4) when that saves a wave of the on-chip filter] */
  uint64_t seed;         /* start vectors from a counter-based generator [0] */
} ofm_eig_opts;

/* Options of the assembly.  NULL means defaults. */
typedef struct {
  int chunk_points;      /* target points per contraction work item [0 = planner's choice];
                            a value different from the current plan's re-plans */
  int use_graph;         /* [1] capture the assembly's launches for this precision as a
                            CUDA graph on first use and replay it; used only while
                            profiling is off (per-launch timing needs separate launches)
                            and on a stream that can be captured (not the legacy default
                            stream); 0 launches the kernels one by one */
  int schedule;          /* [0] the default: for the tensor-core precisions the context's
                            schedule (the one ofm_autotune_assembly chose), else, and for
                            FP32 / FP64, "region" where its plan applies and its MMA
                            work, padding included, stays within 4x the algorithmic
                            flops, else "pair"; 1 "pair": H phi in the states' layout,
                            then one GEMM per pair (M = n_a padded to 128); 2 "region":
                            the grid is cut into coverage regions (products of the
                            segments between dilated-box boundaries) and every region's
                            fragments are stacked into one GEMM (M = sum of their
                            n_a), with the H apply writing the operands (OFM_ERR_INVALID
                            where that plan does not apply: FP64 storage, more than
                            128 states per fragment, or partial sums beyond 16 GB).
                            FP32 and FP64 run both schedules on the CUDA cores; the
                            FP64 region form forms H phi in FP64 from the FP32 states
                            and needs twice the operand and partial-sum memory */
} ofm_assemble_opts;

/* Counts describing the planned work (after ofm_build_fragments). */
typedef struct {
  int n_frag;
  int n_pairs;
  int basis_size;                 /* sum of n_states */
  int n_work_items;               /* contraction work items of the current plan */
  long long pair_flops;           /* sum_{a<=b} 2 n_a n_b (|B_a ∩ B_b| + |B_a ∩ B_b+|) */
  long long overlap_points_s;     /* sum_{a<=b} |B_a ∩ B_b| */
  long long overlap_points_h;     /* sum_{a<=b} |B_a ∩ B_b+| */
  long long state_bytes;          /* device bytes of the fragment states (one copy) */
  long long hphi_bytes;           /* device bytes of H phi */
  long long apply_points;         /* sum_a |B_a+| * n_a (point-states written by the H apply) */
  int last_schedule;              /* schedule of the last ofm_assemble_HS: 1 pair, 2 region,
                                     0 none yet */
  int pad_;
} ofm_plan_info;

typedef struct ofm_ctx ofm_ctx;

/* Create a context on the current CUDA device.  stream: a cudaStream_t to
 * order all work on, or NULL for a context-owned non-blocking stream. */
ofm_status ofm_create(ofm_ctx** ctx, void* cuda_stream);
void ofm_destroy(ofm_ctx* ctx);
const char* ofm_last_error(const ofm_ctx* ctx);
const char* ofm_status_string(ofm_status s);

/* Sec. II (input: the potential on a real-space grid, and fragments = boxes).
 * Validates the grid and boxes, copies V (n0*n1*n2 doubles, x fastest; host
 * or device per v_loc) into the context in the storage type, plans the pair
 * list and the per-pair overlap geometry, and allocates every device buffer
 * the later calls use (re-using them when a new geometry fits).
 * Returns OFM_ERR_INVALID for: h <= 0; any n < 1; ext_d < 1 or ext_d > n_d;
 * ext_d == n_d - 1 (the dilated box would wrap onto itself);
 * n_states < 1 or n_states > P_a - 1. */
ofm_status ofm_build_fragments(ofm_ctx* ctx, const ofm_grid* grid, const double* V,
                               ofm_location v_loc, const ofm_fragment* frags, int n_frag,
                               ofm_storage storage);

/* Sec. II, "calculation of basis wave functions": the lowest n_a eigenpairs
 * of every fragment Hamiltonian, all fragments in one batch.  eps_out: host,
 * basis_size doubles (fragment-major, ascending); resid_out: host, basis_size
 * residual norms ||H phi - eps phi|| or NULL.  OFM_ERR_NOT_CONVERGED leaves
 * the best states found in place (usable) and fills both outputs. */
ofm_status ofm_fragment_eigs(ofm_ctx* ctx, const ofm_eig_opts* opts,
                             double* eps_out, double* resid_out);

/* Import / export the states of fragment a: phi is P_a x n_a, column-major
 * (state i is phi[i*P_a .. (i+1)*P_a), box points x fastest), doubles, on the
 * host or device per loc.  Import marks the states as the current basis. */
ofm_status ofm_set_fragment_states(ofm_ctx* ctx, int a, const double* phi, ofm_location loc);
ofm_status ofm_get_fragment_states(ofm_ctx* ctx, int a, double* phi_out, ofm_location loc);

/* Checkpoint of the basis: every fragment's states written to <path>.bin
 * (raw little-endian values in the storage precision, fragment after
 * fragment, each laid out as ofm_get_fragment_states returns it) with a
 * JSON header <path>.json (format, grid, h, storage, the boxes and state
 * counts).  ofm_load_basis reads them into a context built with the same
 * grid, boxes, state counts and storage (OFM_ERR_INVALID otherwise, or for
 * a file that cannot be read or has the wrong length) and marks them as the
 * current basis: a run resumes after the eigensolve.  Both synchronise. */
ofm_status ofm_save_basis(ofm_ctx* ctx, const char* path);
ofm_status ofm_load_basis(ofm_ctx* ctx, const char* path);

/* Sec. II, the main part of the calculation: H phi_b on every dilated box
 * (whole-system H), then for every pair a <= b
 *     S_ab = Phi_a^T Phi_b  over B_a ∩ B_b,   H_ab = Phi_a^T (H Phi_b) over B_a ∩ B_b+,
 * in the requested arithmetic, summed in a fixed order (deterministic), and
 * stored as FP64 blocks; a diagonal block is symmetrised as (X + X^T)/2.
 * FP64 arithmetic is allowed with either storage; the others need FP32
 * storage.  The tensor-core precisions (TF32, BF16, BF16 hi+lo) take at most
 * 128 states per fragment (OFM_ERR_INVALID beyond; FP32 and FP64 have no
 * such limit).  Enqueued on the context stream; does not synchronise. */
ofm_status ofm_assemble_HS(ofm_ctx* ctx, ofm_precision prec, const ofm_assemble_opts* opts);

/* Result of ofm_autotune_assembly. */
typedef struct {
  int chunk_points;      /* chosen points per contraction work item (pair schedule) */
  int stencil_form;      /* chosen form of the H apply: 1 register, 2 staged (shared-memory planes) */
  double ms;             /* its mean assembly time over the timed runs, milliseconds */
  int n_tried;           /* candidates timed */
  int schedule;          /* chosen schedule: 1 pair, 2 region */
  double region_ms;      /* mean time of the region schedule, -1 where it does not apply
                            or for the CUDA-core precisions */
} ofm_tune_result;

/* Measuring autotuner of the assembly schedule of ofm_assemble_HS (the same
 * computation in every candidate: the schedule moves work between launches
 * and changes the order of the FP32/FP64 partial sums, nothing else).  Each
 * candidate (stencil form 1 or 2) x (points per work item) is planned, run
 * once, then run `reps` times between two CUDA events on the context stream;
 * the fastest becomes the context's schedule, used by later ofm_assemble_HS
 * calls whose chunk_points is 0, until ofm_build_fragments changes the layout
 * (boxes, state counts, grid or storage).  For the tensor-core precisions
 * the region schedule (ofm_assemble_opts.schedule) is timed too and kept
 * when it is the fastest.  chunks: n_chunks candidate sizes
 * (> 0), or NULL for five: the planner's own size for this precision's
 * contraction times 1/4, 1/2, 1, 2 and 4.  times_ms (host, nullable) gets
 * 2 x n_cand mean times, form-major, -1 where the staged form does not fit.
 * out (nullable) gets the choice.  Ends with one assembly of the chosen
 * schedule and synchronises the stream.  Needs states; profiling must be off
 * (OFM_ERR_STATE); reps >= 1 (OFM_ERR_INVALID). */
ofm_status ofm_autotune_assembly(ofm_ctx* ctx, ofm_precision prec, const int* chunks, int n_chunks,
                                 int reps, double* times_ms, ofm_tune_result* out);

/* Eq. 1 with a new potential on the same grid: V (n0*n1*n2 doubles, x
 * fastest; host or device per v_loc) replaces the current one.  The
 * fragments, pair list, plans and states stay -- the states remain the basis
 * (Sec. II: the basis is fixed once the fragment eigenstates are computed;
 * the whole-system H is then represented in it) -- and the assembled blocks
 * are discarded, so the next ofm_assemble_HS represents the new H in the
 * same basis.  A host V is copied before the call returns.  OFM_ERR_STATE
 * before ofm_build_fragments. */
ofm_status ofm_set_potential(ofm_ctx* ctx, const double* V, ofm_location v_loc);

/* Distance cutoff on the pair list (Sec. III.C, "Choice of the distance
 * cutoff": a pair of fragments is included when the minimal distance between
 * an atom of one and an atom of the other is below d_cut).  The atoms of
 * fragment a are atom_xyz[3*i .. 3*i+2] for frag_atom_off[a] <= i <
 * frag_atom_off[a+1] (host arrays: n_frag + 1 non-decreasing offsets from 0;
 * positions in bohr, in the periodic box of n[d] * h; distances are minimum
 * image).  A pair (a, b), a != b, whose boxes meet is kept when that
 * distance is below d_cut; a self pair is always kept; a fragment without
 * atoms keeps only its self pair.  Dropped pairs give zero blocks (in
 * ofm_get_block and in the dense pencil).  atom_xyz == NULL or d_cut <= 0
 * restores the geometric pair list.  Needs ofm_build_fragments first; the
 * arrays are read during the call only.  Re-plans the contraction and
 * discards any assembled blocks; synchronises the context stream.
 * OFM_ERR_INVALID: bad offsets; OFM_ERR_STATE: no fragments built. */
ofm_status ofm_set_pair_cutoff(ofm_ctx* ctx, const double* atom_xyz, const int* frag_atom_off,
                               double d_cut);

/* Basis selection (Sec. III, "Choice of the number of basis states per
 * fragment": e.g. only the n highest occupied states of every fragment, its
 * HOMOs): keep states first[a] .. first[a] + count[a] - 1 (0-based, in the
 * ascending order of the stored states) of every fragment a as its basis.
 * The selected columns are copied on the device; the fragment table, the
 * pair plans and the state and H phi storage are laid out again for the new
 * state counts; the geometry, V and a distance cutoff stay.  Needs every
 * fragment's states (ofm_fragment_eigs or ofm_set_fragment_states); first
 * and count are host arrays of n_frag ints, read during the call only.
 * Discards assembled blocks and the eigensolver's workspace (a later
 * ofm_fragment_eigs computes count[a] states).  Synchronises the context
 * stream.  OFM_ERR_INVALID: a range outside a fragment's states, NULL
 * arrays; OFM_ERR_STATE: states not set. */
ofm_status ofm_select_states(ofm_ctx* ctx, const int* first, const int* count);

/* Occupation with a HOMO basis (Sec. III, end of "Choice of the number of
 * basis states per fragment"): e_a = <HOMO_a|H|HOMO_a> with the whole-system
 * H for every fragment (the last diagonal entry of the assembled H_aa, i.e.
 * of the fragment's highest basis state), e_ref = max_a e_a, then the first
 * spacing wider than gap_min (Ha) between consecutive eigenvalues of Eq. 2,
 * scanning upward from the largest eigenvalue <= e_ref.  Outputs: *e_ref
 * (may be NULL), the eigenvalues *E_homo < *E_lumo bounding that spacing and
 * *n_occ, the number of eigenvalues <= *E_homo (the occupied states).  Needs
 * ofm_assemble_HS; solves Eq. 2 like ofm_eigs_by_index.  OFM_ERR_INVALID:
 * gap_min <= 0, NULL outputs, or no such spacing; OFM_ERR_STATE: nothing
 * assembled. */
ofm_status ofm_homo_lumo_gap(ofm_ctx* ctx, double gap_min, double* e_ref, double* E_homo,
                             double* E_lumo, int* n_occ);

/* The pair list: *n_pairs always; pair_ab (2*n_pairs ints, a then b, a<=b,
 * sorted by a then b) when not NULL. */
ofm_status ofm_get_pairs(ofm_ctx* ctx, int* n_pairs, int* pair_ab);
ofm_status ofm_get_plan_info(ofm_ctx* ctx, ofm_plan_info* info);

/* Block of the pair (a, b) (either order): n_a x n_b row-major doubles,
 * host.  A pair not in the list yields zeros.  H_ab / S_ab may be NULL. */
ofm_status ofm_get_block(ofm_ctx* ctx, int a, int b, double* H_ab, double* S_ab);

/* Every assembled block at once, in the order of the pair list
 * (ofm_get_pairs): for each pair a <= b, H_ab then S_ab, each n_a x n_b
 * row-major doubles, concatenated -- the block-sparse form of the pencil of
 * Eq. 2 that a sparse or distributed eigensolver takes (Sec. II points to
 * ScaLAPACK / PARPACK for large systems).  *n_elems (nullable) receives the
 * element count; HS (host or device per loc; NULL only queries the count)
 * receives the blocks.  Synchronises the context stream. */
ofm_status ofm_get_blocks(ofm_ctx* ctx, double* HS, ofm_location loc, long long* n_elems);

/* The same blocks, read back without synchronising: the call enqueues a
 * device copy of the blocks into a staging buffer on the context stream
 * (ordered after the assembly) and their transfer to HS (host memory,
 * pinned for the transfer to overlap; or device memory) on a stream of the
 * context's own, and returns.  A later ofm_assemble_HS on the context stream
 * runs while the blocks travel.  HS holds the blocks once ofm_sync_blocks
 * returns OFM_OK; until then the caller must neither read nor free it.  A
 * second call waits (on the device, not the host) for the first transfer
 * before it overwrites the staging buffer.  *n_elems (nullable) receives the
 * element count; HS NULL only queries it.  Device errors of the assembly are
 * reported by ofm_sync_blocks. */
ofm_status ofm_get_blocks_async(ofm_ctx* ctx, double* HS, long long* n_elems);
ofm_status ofm_sync_blocks(ofm_ctx* ctx);

/* Dense n x n (n = basis_size) row-major H and S in basis order, host or
 * device per loc.  Either pointer may be NULL. */
ofm_status ofm_get_dense_HS(ofm_ctx* ctx, double* H, double* S, ofm_location loc);

/* H phi_b of fragment b on its dilated box as |B_b+| x n_b column-major
 * doubles (host), available after ofm_assemble_HS. */
ofm_status ofm_get_hphi(ofm_ctx* ctx, int b, double* hphi_out);

/* Block-sparse product with the assembled pencil of Eq. 2, without forming
 * the dense matrices: Y = M X with M = H (which = 0) or M = S (which = 1),
 * summed over the pair blocks (the stored block a <= b, its transpose for
 * b > a; blocks of pairs outside the pair list are zero), FP64, in basis
 * order.  X and Y are DEVICE arrays of k columns, column-major: column c of
 * X starts at X + c * ldx, ldx and ldy >= basis_size; Y is written, X only
 * read, and the two must not overlap.  The caller owns both.  Enqueued on
 * the context stream (X must be ready there); does not synchronise.  Each
 * output is summed in a fixed order (deterministic).
 * OFM_ERR_STATE before ofm_assemble_HS; OFM_ERR_INVALID for which not 0/1,
 * NULL pointers, k < 1, leading dimensions < basis_size, or X and Y
 * overlapping. */
ofm_status ofm_pencil_apply(ofm_ctx* ctx, int which, const double* X, long long ldx, double* Y,
                            long long ldy, int k);

/* Eq. 2 restricted to an energy window, FP64 on the device: Cholesky
 * S = L L^T, A = L^-1 H L^-T, Householder tridiagonalisation, Sturm-count
 * bisection for the eigenvalues in [E_lo, E_hi] (inclusive).  E_out: host,
 * max_out doubles, ascending; *n_out = number found (may exceed max_out, in
 * which case only max_out are written).  C_out: host, n x min(n_out,max_out)
 * column-major S-orthonormal eigenvectors, or NULL.
 * OFM_ERR_NOT_POSDEF when S is not positive definite. */
ofm_status ofm_window_eigs(ofm_ctx* ctx, double E_lo, double E_hi, int max_out,
                           double* E_out, int* n_out, double* C_out);

/* Eigenvalues with 0-based ascending indices [i_lo, i_hi) of Eq. 2 (host
 * output), from the same factorisation as ofm_window_eigs.  Used to place
 * an energy window relative to a gap. */
ofm_status ofm_eigs_by_index(ofm_ctx* ctx, int i_lo, int i_hi, double* E_out);

/* A window of Eq. 2 anchored at an index: E_{i_lo} and every later
 * eigenvalue E_j <= E_{i_lo} + width (width in Ha, >= 0), ascending, e.g.
 * the levels within 0.3 Ha above the first empty one.  *n_out is the window
 * size; E_out (host) receives min(*n_out, max_out) values.  The same set as
 * ofm_eigs_by_index for E_{i_lo} followed by ofm_window_eigs on
 * [E_{i_lo}, E_{i_lo} + width], in one multisection launch sized by an FP32
 * estimate (extended when short), so the anchor's own search is not a
 * separate serial step.  OFM_ERR_INVALID: i_lo outside the spectrum, width <
 * 0, NULL outputs. */
ofm_status ofm_window_from_index(ofm_ctx* ctx, int i_lo, double width, int max_out, double* E_out,
                                 int* n_out);

/* Eq. 2 for caller-supplied dense n x n row-major H (symmetric) and S
 * (symmetric positive definite), host pointers, solved by the same device
 * path as ofm_window_eigs (replaces the assembled matrices). */
ofm_status ofm_set_dense_HS(ofm_ctx* ctx, int n, const double* H, const double* S);

/* Per-kernel-class launch counts and device time.  Counting is always on;
 * device time is measured with CUDA events recorded on the context stream
 * around each launch (or launch sequence) while profiling is on.
 * ofm_set_profiling clears the statistics.  ofm_get_kernel_stats
 * synchronises the stream, writes up to max entries (one per class that has
 * launched) and sets *n to the number written. */
typedef struct {
  char name[32];          /* kernel class, e.g. "filter", "contract" */
  char row[8];            /* method step: "a0".."a6" */
  long long launches;
  double total_ms;        /* 0 when profiling was off */
  double bytes;           /* algorithmic bytes moved by these launches (model, not counters) */
  double flops;           /* algorithmic flops of these launches */
} ofm_kernel_stat;

ofm_status ofm_set_profiling(ofm_ctx* ctx, int on);
ofm_status ofm_get_kernel_stats(ofm_ctx* ctx, ofm_kernel_stat* out, int max, int* n);

/* Test hook of the failure detection (for tests, not for production use).
 * Every device-side wait of the library is bounded: when it runs out, the
 * kernel records the failure, waits (bounded) for its own copies in flight,
 * frees what it holds and returns, and the call returns OFM_ERR_TIMEOUT with
 * the context still usable.  This hook makes one such wait run out, on
 * purpose and without any fault: what = 1 arms the next region-schedule
 * contraction launch of ofm_assemble_HS, whose producer then withholds every
 * operand copy (the tensor cores' first wait gives up; that assembly is
 * launched directly, not from a captured graph); what = 2 arms the next
 * tridiagonal reduction of Eq. 2, one of whose CTAs withholds its first
 * grid-barrier arrival.  bound: polls before the held wait gives up (0: the
 * usual bound, about a second).  what = 0 disarms.  The timeout is reported
 * by the call that reads the device status (ofm_get_block etc. after an
 * assembly; the window call itself for Eq. 2).
 * Host-side injection, which never touches the device: the environment
 * variable OFM_FAULT, read by ofm_create, makes that context report
 * OFM_ERR_OOM for its allocations of 4 KiB or more (oom), OFM_ERR_TIMEOUT when
 * it reads the device status after an assembly (timeout),
 * OFM_ERR_NOT_CONVERGED from ofm_fragment_eigs with every output filled
 * (nonconv), or OFM_ERR_NOT_POSDEF from the factorisation of Eq. 2
 * (notposdef). */
ofm_status ofm_test_hold_wait(ofm_ctx* ctx, int what, int bound);
/* The same hook tests the check mode below, again from the host and without
 * any device fault: what = 3 overwrites one byte of the block arena's guard
 * band (the next guard check reports it); what = 4 (check mode only) points
 * the region plan's first copy piece just past its plane arena, for the next
 * region-schedule assembly, whose checking producer refuses it. */

/* Check mode (also on when the environment variable OFM_CHECK is set to 1
 * when the context is created).  Every device buffer of the library carries
 * a 256-byte guard band of the byte 0xA5 after its end, written when it is
 * allocated.  With checks on:
 *  - ofm_fragment_eigs, ofm_assemble_HS, the window calls, ofm_pencil_apply
 *    and ofm_get_blocks end with ofm_check_guards (which synchronises);
 *  - the region schedule's pack and contraction run forms that check every
 *    gathered point index and every copied byte range against their buffers
 *    and refuse (skip) an access outside them.
 * A failure returns OFM_ERR_CORRUPT naming the buffer or the kernel.
 * Checks cost time (a synchronisation per call, a bounds test per access);
 * results are the same bit for bit. */
ofm_status ofm_set_checks(ofm_ctx* ctx, int on);
/* Reads every guard band of the context's buffers now: OFM_ERR_CORRUPT
 * (naming the first overwritten buffer) or OFM_OK.  Synchronises. */
ofm_status ofm_check_guards(ofm_ctx* ctx);

/* Host-only planner query (needs no GPU and no context): validates the
 * geometry like ofm_build_fragments and returns the pair list (Sec. II,
 * pairs of fragments that share grid points through the stencil) with the
 * overlap sizes.  *n_pairs always; when pair_ab is not NULL, up to
 * max_pairs pairs (a, b) with a <= b; when counts is not NULL, 2 per written
 * pair: |B_a ∩ B_b| then |B_a ∩ B_b+|.  *pair_flops (nullable) receives the
 * algorithmic flop count sum 2 n_a n_b (|B_a ∩ B_b| + |B_a ∩ B_b+|). */
ofm_status ofm_plan_pairs(const ofm_grid* grid, const ofm_fragment* frags, int n_frag,
                          int* n_pairs, int* pair_ab, long long* counts, int max_pairs,
                          long long* pair_flops);

/* Host-only query of the region plan of the tensor-core assembly (needs no
 * GPU and no context), for the pair list of ofm_plan_pairs.  Sec. II sums
 * H_ab and S_ab over the grid points two fragments share; the region plan
 * cuts the grid into coverage regions (per dimension, the segments between
 * dilated-box boundaries, merged while shorter than w_min points; products
 * of three segments) and sums every pair over the regions whose cover set
 * holds both fragments.  stats (8 long longs, nullable): plan applies (0/1),
 * regions, region parts (K splits), work items, operand-plane bytes,
 * partial-slot bytes, MMA flops of one product pass, the segment width
 * used.  pair_points (nullable, max_pairs entries, pair-list order): for
 * each pair, the points of B_a ∩ B_b+ that the regions holding both
 * fragments cover, counted point by point (equal to |B_a ∩ B_b+| when the
 * plan is right).  OFM_ERR_INVALID for a bad geometry. */
ofm_status ofm_plan_regions(const ofm_grid* grid, const ofm_fragment* frags, int n_frag,
                            int w_min, long long* stats, long long* pair_points, int max_pairs);

/* Allocation-free pair blocks.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory when they need
 * a block -- code whose device memory is owned by another framework's pool,
 * latency-critical paths where cudaMalloc/cudaFree may block or synchronise
 * the device, or sandboxed code that is handed ready-made device buffers.
 * It computes, for one pair of fragments on the grid, in FP32 arithmetic,
 *     HS_ab[0 .. n_a*n_b)        = H_ab = Phi_a^T (H Phi_b), row-major n_a x n_b,
 *     HS_ab[n_a*n_b .. 2 n_a n_b) = S_ab = Phi_a^T Phi_b,
 * symmetrised when fa and fb describe the same fragment with the same
 * buffer, and zeros when the boxes do not interact.
 * Inputs (device, FP32): phi_a, phi_b, hphi_b in the library's storage
 * layout -- point-major on the fragment's dilated box (the box grown by one
 * point on each side in every dimension it does not span), element
 * (p, s) at p * ld + s with ld = n_states rounded up to a multiple of 4, p
 * the dilated-box point index (x fastest), halo rows of phi zero.  hphi_b
 * is H phi_b with the whole-system H on the dilated box, same layout.
 * The work uses only the caller's buffers and one fixed device array of
 * OFM_NOALLOC_SCRATCH bytes inside the library (held by every GPU that
 * loads it until exit); no cudaMalloc, cudaFree or allocating library call
 * is made.  The first call on a device looks up that array's address and
 * should come before any stream capture.  Calls share the array: calls
 * whose GPU work overlaps race.  Work is enqueued on cuda_stream (NULL =
 * legacy default stream; otherwise a stream of the current device) and not
 * synchronised.  Returns OFM_ERR_INVALID for bad geometry or pointers, when
 * the pair's work tables and partial tiles do not fit the scratch, when
 * cuda_stream belongs to another device, or when cuda_stream is being
 * captured (the work tables are staged from host memory that lives only
 * for the call); OFM_ERR_CUDA when a runtime call fails. */
#define OFM_NOALLOC_SCRATCH (32u * 1024u * 1024u)
ofm_status ofm_pair_blocks_noalloc(const ofm_grid* grid, const ofm_fragment* fa,
                                   const ofm_fragment* fb, const float* phi_a,
                                   const float* phi_b, const float* hphi_b, double* HS_ab,
                                   void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* OFM_H */
