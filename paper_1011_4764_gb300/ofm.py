"""Thin ctypes binding of libofm.so (include/ofm.h).

Every function marshals arguments and calls the C ABI of the same name; all
computation runs in the library's CUDA kernels.  There is no fallback: if
the library is missing or fails to load, the import of the entry points
raises.  PyTorch is used only to hand device pointers and streams across.
"""
from __future__ import annotations

import collections
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libofm.so")

OFM_OK, OFM_ERR_INVALID, OFM_ERR_OOM, OFM_ERR_CUDA = 0, 1, 2, 3
OFM_ERR_NOT_CONVERGED, OFM_ERR_NOT_POSDEF, OFM_ERR_TIMEOUT, OFM_ERR_STATE = 4, 5, 6, 7
OFM_ERR_CORRUPT = 8
PREC = {"fp64": 0, "fp32": 1, "tf32": 2, "bf16": 3, "bf16x3": 4}
STORE = {"fp64": 0, "fp32": 1}
HOST, DEVICE = 0, 1

# every symbol the header declares (checked by the CPU tests)
EXPORTS = [
    "ofm_create", "ofm_destroy", "ofm_last_error", "ofm_status_string", "ofm_build_fragments",
    "ofm_fragment_eigs", "ofm_set_fragment_states", "ofm_get_fragment_states",
    "ofm_assemble_HS", "ofm_get_pairs", "ofm_get_plan_info", "ofm_get_block",
    "ofm_get_dense_HS", "ofm_get_hphi", "ofm_window_eigs", "ofm_eigs_by_index",
    "ofm_set_dense_HS", "ofm_plan_pairs", "ofm_set_profiling", "ofm_get_kernel_stats",
    "ofm_pair_blocks_noalloc", "ofm_set_pair_cutoff", "ofm_select_states", "ofm_homo_lumo_gap",
    "ofm_window_from_index", "ofm_autotune_assembly", "ofm_pencil_apply", "ofm_plan_regions",
    "ofm_set_potential", "ofm_get_blocks", "ofm_get_blocks_async", "ofm_sync_blocks",
    "ofm_test_hold_wait", "ofm_set_checks", "ofm_check_guards", "ofm_save_basis",
    "ofm_load_basis",
]
SCHEDULE = {"auto": 0, "pair": 1, "region": 2}


# fragment geometry with the state count of the current basis
_Frag = collections.namedtuple("_Frag", "off ext n_states")


class ofm_grid(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("h", C.c_double)]


class ofm_fragment(C.Structure):
    _fields_ = [("off", C.c_int * 3), ("ext", C.c_int * 3), ("n_states", C.c_int)]


class ofm_eig_opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int), ("degree", C.c_int),
                ("extra_states", C.c_int), ("seed", C.c_uint64)]


class ofm_assemble_opts(C.Structure):
    _fields_ = [("chunk_points", C.c_int), ("use_graph", C.c_int), ("schedule", C.c_int)]


class ofm_tune_result(C.Structure):
    _fields_ = [("chunk_points", C.c_int), ("stencil_form", C.c_int), ("ms", C.c_double),
                ("n_tried", C.c_int), ("schedule", C.c_int), ("region_ms", C.c_double)]


class ofm_plan_info(C.Structure):
    _fields_ = [("n_frag", C.c_int), ("n_pairs", C.c_int), ("basis_size", C.c_int),
                ("n_work_items", C.c_int), ("pair_flops", C.c_longlong),
                ("overlap_points_s", C.c_longlong), ("overlap_points_h", C.c_longlong),
                ("state_bytes", C.c_longlong), ("hphi_bytes", C.c_longlong),
                ("apply_points", C.c_longlong), ("last_schedule", C.c_int), ("pad_", C.c_int)]


class ofm_kernel_stat(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("row", C.c_char * 8), ("launches", C.c_longlong),
                ("total_ms", C.c_double), ("bytes", C.c_double), ("flops", C.c_double)]


_LIB = None


def load_library(path: str = LIB_PATH):
    """Load libofm.so once and declare the signatures.  Raises when absent."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libofm.so not found at {path}; build it with "
                           "paper_1011_4764_gb300.build.build() (no CPU fallback exists)")
    lib = C.CDLL(path)
    P, I, D = C.c_void_p, C.c_int, C.c_double
    DP, IP = C.POINTER(C.c_double), C.POINTER(C.c_int)
    sig = {
        "ofm_create": ([C.POINTER(C.c_void_p), P], I),
        "ofm_destroy": ([P], None),
        "ofm_last_error": ([P], C.c_char_p),
        "ofm_status_string": ([I], C.c_char_p),
        "ofm_build_fragments": ([P, C.POINTER(ofm_grid), P, I, C.POINTER(ofm_fragment), I, I], I),
        "ofm_fragment_eigs": ([P, C.POINTER(ofm_eig_opts), DP, DP], I),
        "ofm_set_fragment_states": ([P, I, P, I], I),
        "ofm_get_fragment_states": ([P, I, P, I], I),
        "ofm_assemble_HS": ([P, I, C.POINTER(ofm_assemble_opts)], I),
        "ofm_get_pairs": ([P, IP, IP], I),
        "ofm_get_plan_info": ([P, C.POINTER(ofm_plan_info)], I),
        "ofm_get_block": ([P, I, I, DP, DP], I),
        "ofm_get_blocks_async": ([P, P, C.POINTER(C.c_longlong)], I),
        "ofm_sync_blocks": ([P], I),
        "ofm_get_dense_HS": ([P, P, P, I], I),
        "ofm_get_hphi": ([P, I, DP], I),
        "ofm_window_eigs": ([P, D, D, I, DP, IP, DP], I),
        "ofm_eigs_by_index": ([P, I, I, DP], I),
        "ofm_set_dense_HS": ([P, I, DP, DP], I),
        "ofm_plan_pairs": ([C.POINTER(ofm_grid), C.POINTER(ofm_fragment), I, IP, IP,
                            C.POINTER(C.c_longlong), I, C.POINTER(C.c_longlong)], I),
        "ofm_set_profiling": ([P, I], I),
        "ofm_pair_blocks_noalloc": ([C.POINTER(ofm_grid), C.POINTER(ofm_fragment),
                                     C.POINTER(ofm_fragment), P, P, P, P, P], I),
        "ofm_get_kernel_stats": ([P, C.POINTER(ofm_kernel_stat), I, IP], I),
        "ofm_set_pair_cutoff": ([P, DP, IP, D], I),
        "ofm_select_states": ([P, IP, IP], I),
        "ofm_homo_lumo_gap": ([P, D, DP, DP, DP, IP], I),
        "ofm_window_from_index": ([P, I, D, I, DP, IP], I),
        "ofm_autotune_assembly": ([P, I, IP, I, I, DP, C.POINTER(ofm_tune_result)], I),
        "ofm_pencil_apply": ([P, I, P, C.c_longlong, P, C.c_longlong, I], I),
        "ofm_plan_regions": ([C.POINTER(ofm_grid), C.POINTER(ofm_fragment), I, I,
                              C.POINTER(C.c_longlong), C.POINTER(C.c_longlong), I], I),
        "ofm_set_potential": ([P, P, I], I),
        "ofm_get_blocks": ([P, P, I, C.POINTER(C.c_longlong)], I),
        "ofm_test_hold_wait": ([P, I, I], I),
        "ofm_set_checks": ([P, I], I),
        "ofm_save_basis": ([P, C.c_char_p], I),
        "ofm_load_basis": ([P, C.c_char_p], I),
        "ofm_check_guards": ([P], I),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _LIB = lib
    return lib


class OFMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{status_name(status)}: {msg}")
        self.status = status


def status_name(s: int) -> str:
    return load_library().ofm_status_string(s).decode()


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _iptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _c_geometry(grid, frags):
    g = ofm_grid((C.c_int * 3)(*grid.n), float(grid.h))
    fa = (ofm_fragment * len(frags))()
    for i, f in enumerate(frags):
        fa[i].off = (C.c_int * 3)(*f.off)
        fa[i].ext = (C.c_int * 3)(*f.ext)
        fa[i].n_states = int(f.n_states)
    return g, fa


def plan_pairs(grid, frags):
    """Host-only planner query: (pairs, counts (P, 2): |B_a∩B_b|, |B_a∩B_b+|, flops)."""
    lib = load_library()
    g, fa = _c_geometry(grid, frags)
    n = C.c_int()
    s = lib.ofm_plan_pairs(C.byref(g), fa, len(frags), C.byref(n), None, None, 0, None)
    if s != OFM_OK:
        raise OFMError(s, "invalid geometry")
    ab = np.zeros(2 * n.value, dtype=np.int32)
    cnt = np.zeros(2 * n.value, dtype=np.int64)
    F = C.c_longlong()
    lib.ofm_plan_pairs(C.byref(g), fa, len(frags), C.byref(n), _iptr(ab),
                       cnt.ctypes.data_as(C.POINTER(C.c_longlong)), n.value, C.byref(F))
    return [tuple(map(int, ab[2 * i:2 * i + 2])) for i in range(n.value)], cnt.reshape(-1, 2), F.value


def plan_regions(grid, frags, w_min=1):
    """Host-only query of the region plan: (stats dict, per-pair points of
    B_a ∩ B_b+ covered by the regions holding both fragments)."""
    lib = load_library()
    g, fa = _c_geometry(grid, frags)
    pairs, _, _ = plan_pairs(grid, frags)
    st = np.zeros(8, dtype=np.int64)
    pts = np.zeros(max(1, len(pairs)), dtype=np.int64)
    LP = C.POINTER(C.c_longlong)
    s = lib.ofm_plan_regions(C.byref(g), fa, len(frags), int(w_min), st.ctypes.data_as(LP),
                             pts.ctypes.data_as(LP), len(pairs))
    if s != OFM_OK:
        raise OFMError(s, "invalid geometry")
    keys = ("ok", "regions", "parts", "items", "plane_bytes", "slot_bytes", "mma_flops", "w_min")
    return dict(zip(keys, map(int, st))), pts[:len(pairs)]


def pair_blocks_noalloc(grid, fa, fb, phi_a, phi_b, hphi_b, out, stream=0):
    """ofm_pair_blocks_noalloc: for callers that cannot allocate device
    memory.  phi_a, phi_b, hphi_b: CUDA float32 tensors in the storage layout
    (point-major on the dilated box, row stride n rounded up to 4); out: CUDA
    float64 tensor of 2 n_a n_b (H_ab then S_ab).  Enqueued on `stream` (a
    cudaStream_t handle, 0 = legacy default); not synchronised."""
    lib = load_library()
    g, fab = _c_geometry(grid, [fa, fb])
    for t in (phi_a, phi_b, hphi_b):
        assert t.is_cuda and str(t.dtype) == "torch.float32" and t.is_contiguous()
    assert out.is_cuda and str(out.dtype) == "torch.float64" and out.is_contiguous()

    def stored(f):   # floats of the storage layout: dilated-box points x ld
        Pd = 1
        for d in range(3):
            Pd *= f.ext[d] + 2 if f.ext[d] < grid.n[d] else f.ext[d]
        return Pd * ((f.n_states + 3) // 4 * 4)
    assert phi_a.numel() >= stored(fa), "phi_a is shorter than fragment a's storage layout"
    assert phi_b.numel() >= stored(fb) and hphi_b.numel() >= stored(fb), \
        "phi_b / hphi_b are shorter than fragment b's storage layout"
    assert out.numel() == 2 * fa.n_states * fb.n_states, "out must hold 2 n_a n_b doubles"
    s = lib.ofm_pair_blocks_noalloc(C.byref(g), C.byref(fab[0]), C.byref(fab[1]),
                                    C.c_void_p(phi_a.data_ptr()), C.c_void_p(phi_b.data_ptr()),
                                    C.c_void_p(hphi_b.data_ptr()), C.c_void_p(out.data_ptr()),
                                    C.c_void_p(stream) if stream else None)
    if s != OFM_OK:
        raise OFMError(s, "ofm_pair_blocks_noalloc failed")


class Context:
    """One library context (ofm_ctx) bound to a CUDA stream."""

    def __init__(self, stream=None):
        self.lib = load_library()
        h = C.c_void_p()
        st = None
        if stream is not None:
            st = C.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
        s = self.lib.ofm_create(C.byref(h), st)
        if s != OFM_OK:
            raise OFMError(s, "ofm_create failed")
        self.h = h
        self.frags = []
        self.grid = None
        self._dense_n = 0
        self.stream_obj = stream if (stream is not None and not isinstance(stream, int)) else None

    def close(self):
        if getattr(self, "h", None):
            self.lib.ofm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, s, allow=()):
        if s != OFM_OK and s not in allow:
            raise OFMError(s, self.lib.ofm_last_error(self.h).decode())
        return s

    # -- ofm_build_fragments
    def build_fragments(self, grid, V, frags, storage="fp32"):
        """grid: object with .n (nx, ny, nz) and .h; V: float64 array (nz, ny, nx)
        as numpy (host) or a CUDA torch tensor (device); frags: objects with
        .off, .ext, .n_states."""
        g, fa = _c_geometry(grid, frags)
        if _is_torch(V):
            assert str(V.dtype) == "torch.float64" and V.is_contiguous()
            ptr, loc = C.c_void_p(V.data_ptr()), (DEVICE if V.is_cuda else HOST)
            keep = V
        else:
            keep = np.ascontiguousarray(V, dtype=np.float64)
            ptr, loc = C.c_void_p(keep.ctypes.data), HOST
        self._check(self.lib.ofm_build_fragments(self.h, C.byref(g), ptr, loc, fa, len(frags),
                                                 STORE[storage]))
        del keep
        self.frags = list(frags)
        self.grid = grid
        return self

    # -- ofm_test_hold_wait (failure-detection tests)
    def test_hold_wait(self, what, bound=0):
        """Arm one bounded device wait to run out: "contract" (the next region
        contraction) or "tridiag" (the next reduction of Eq. 2); None disarms.
        Check-mode tests: "guard" overwrites a byte of the block arena's guard
        band, "piece" points the region plan's first copy piece past its
        arena (check mode only)."""
        self._check(self.lib.ofm_test_hold_wait(
            self.h, {None: 0, "contract": 1, "tridiag": 2, "guard": 3, "piece": 4}[what], int(bound)))

    # -- ofm_save_basis / ofm_load_basis
    def save_basis(self, path):
        """Writes <path>.bin and <path>.json (the basis checkpoint)."""
        self._check(self.lib.ofm_save_basis(self.h, os.fsencode(str(path))))

    def load_basis(self, path):
        """Reads a checkpoint written by save_basis for the same geometry."""
        self._check(self.lib.ofm_load_basis(self.h, os.fsencode(str(path))))

    # -- ofm_set_checks / ofm_check_guards
    def set_checks(self, on=True):
        self._check(self.lib.ofm_set_checks(self.h, 1 if on else 0))

    def check_guards(self):
        self._check(self.lib.ofm_check_guards(self.h))

    # -- ofm_set_potential
    def set_potential(self, V):
        """V: float64 (nz, ny, nx) numpy array (host) or CUDA/pinned torch tensor."""
        if _is_torch(V):
            assert str(V.dtype) == "torch.float64" and V.is_contiguous()
            self._check(self.lib.ofm_set_potential(self.h, C.c_void_p(V.data_ptr()),
                                                   DEVICE if V.is_cuda else HOST))
            return
        keep = np.ascontiguousarray(V, dtype=np.float64)
        self._check(self.lib.ofm_set_potential(self.h, C.c_void_p(keep.ctypes.data), HOST))

    # -- ofm_get_blocks
    def blocks_count(self):
        n = C.c_longlong()
        self._check(self.lib.ofm_get_blocks(self.h, None, HOST, C.byref(n)))
        return n.value

    def get_blocks(self, out=None):
        """Every block [H_ab | S_ab] in pair-list order, as one float64 array:
        numpy (host) by default, or into `out` (a float64 torch tensor, CUDA
        or pinned host, of blocks_count() elements)."""
        if out is None:
            out = np.zeros(self.blocks_count())
            self._check(self.lib.ofm_get_blocks(self.h, C.c_void_p(out.ctypes.data), HOST, None))
            return out
        assert _is_torch(out) and str(out.dtype) == "torch.float64" and out.is_contiguous()
        assert out.numel() >= self.blocks_count()
        self._check(self.lib.ofm_get_blocks(self.h, C.c_void_p(out.data_ptr()),
                                            DEVICE if out.is_cuda else HOST, None))
        return out

    def get_blocks_async(self, out):
        """Starts the read-back of every block into `out` (a float64 torch
        tensor, pinned host or CUDA, of blocks_count() elements) and returns;
        `out` holds the blocks after sync_blocks()."""
        assert _is_torch(out) and str(out.dtype) == "torch.float64" and out.is_contiguous()
        assert out.numel() >= self.blocks_count()
        self._check(self.lib.ofm_get_blocks_async(self.h, C.c_void_p(out.data_ptr()), None))
        return out

    def sync_blocks(self):
        self._check(self.lib.ofm_sync_blocks(self.h))

    # -- ofm_fragment_eigs
    def fragment_eigs(self, tol=0.0, max_iter=0, degree=0, extra_states=0, seed=0,
                      allow_not_converged=False):
        n = sum(f.n_states for f in self.frags)
        eps = np.zeros(n)
        res = np.zeros(n)
        o = ofm_eig_opts(tol, max_iter, degree, extra_states, seed)
        s = self._check(self.lib.ofm_fragment_eigs(self.h, C.byref(o), _dptr(eps), _dptr(res)),
                        allow=(OFM_ERR_NOT_CONVERGED,) if allow_not_converged else ())
        return eps, res, s

    # -- ofm_set_fragment_states / ofm_get_fragment_states
    def set_fragment_states(self, a, phi):
        """phi: numpy (P_a, n_a) float64 array of box states (column j = state
        j), or a CUDA float64 torch tensor of shape (n_a, P_a), contiguous
        (the same column-major memory)."""
        if _is_torch(phi):
            assert phi.is_cuda and phi.is_contiguous() and str(phi.dtype) == "torch.float64"
            self._check(self.lib.ofm_set_fragment_states(self.h, a, C.c_void_p(phi.data_ptr()), DEVICE))
            return
        arr = np.asfortranarray(phi, dtype=np.float64)
        self._check(self.lib.ofm_set_fragment_states(self.h, a, C.c_void_p(arr.ctypes.data), HOST))

    def get_fragment_states(self, a):
        f = self.frags[a]
        P = f.ext[0] * f.ext[1] * f.ext[2]
        out = np.zeros((f.n_states, P))
        self._check(self.lib.ofm_get_fragment_states(self.h, a, C.c_void_p(out.ctypes.data), HOST))
        return out.T

    # -- ofm_assemble_HS
    def assemble(self, precision="fp32", chunk_points=0, use_graph=True, schedule="auto"):
        """schedule: "auto" (the context's choice; for FP32 / FP64 the plan's
        default), "pair" (one GEMM per pair) or "region" (coverage regions
        stacked); FP32 and FP64 run either on the CUDA cores."""
        o = ofm_assemble_opts(chunk_points, 1 if use_graph else 0, SCHEDULE[schedule])
        self._check(self.lib.ofm_assemble_HS(self.h, PREC[precision], C.byref(o)))

    # -- ofm_autotune_assembly
    def autotune_assembly(self, precision="fp32", chunks=None, reps=3):
        """Times every (stencil form, chunk) candidate of the pair schedule and,
        for the tensor-core precisions, the region schedule, and keeps the
        fastest.  Returns (chunk_points, stencil_form, ms, times) with times a
        (2, n_candidates) array of mean milliseconds (-1: form does not fit);
        self.tuned holds the schedule chosen and the region time."""
        cand = None if chunks is None else np.ascontiguousarray(chunks, dtype=np.int32)
        nc = 5 if cand is None else len(cand)
        times = np.full(2 * nc, -1.0)
        r = ofm_tune_result()
        self._check(self.lib.ofm_autotune_assembly(
            self.h, PREC[precision], None if cand is None else _iptr(cand), nc, int(reps),
            _dptr(times), C.byref(r)))
        self.tuned = {"schedule": {1: "pair", 2: "region"}.get(r.schedule, "pair"),
                      "region_ms": r.region_ms}
        return r.chunk_points, r.stencil_form, r.ms, times.reshape(2, nc)

    # -- ofm_pencil_apply
    def pencil_apply(self, which, X, out=None):
        """Y = H X (which "H") or S X (which "S") with the assembled blocks.
        X: CUDA float64 torch tensor of shape (k, basis), contiguous (its rows
        are the k columns), ready on the context stream; returns Y of the
        same shape, written on the context stream (use it there, or
        synchronise)."""
        assert _is_torch(X) and X.is_cuda and str(X.dtype) == "torch.float64" and X.is_contiguous()
        k, n = X.shape
        assert n == self.plan_info()["basis_size"], "X must have basis_size columns per row"
        if out is not None:
            assert (_is_torch(out) and out.is_cuda and out.device == X.device and out.is_contiguous()
                    and str(out.dtype) == "torch.float64" and tuple(out.shape) == (k, n)), \
                "out must be a contiguous CUDA float64 tensor of X's shape on X's device"
        Y = out if out is not None else X.new_empty((k, n))
        if self.stream_obj is not None and hasattr(Y, "record_stream"):
            Y.record_stream(self.stream_obj)   # written on the context stream
        self._check(self.lib.ofm_pencil_apply(self.h, {"H": 0, "S": 1}[which], C.c_void_p(X.data_ptr()),
                                              n, C.c_void_p(Y.data_ptr()), n, k))
        return Y

    # -- ofm_set_pair_cutoff
    def set_pair_cutoff(self, atoms, d_cut):
        """atoms: one (k_a, 3) array of positions (bohr) per fragment, or
        None (with any d_cut) to restore the geometric pair list."""
        if atoms is None or d_cut is None or d_cut <= 0:
            self._check(self.lib.ofm_set_pair_cutoff(self.h, None, None, 0.0))
            return
        if len(atoms) != len(self.frags):
            raise ValueError("one atom array per fragment")
        xyz = np.ascontiguousarray(np.concatenate(
            [np.asarray(a, dtype=np.float64).reshape(-1, 3) for a in atoms]), dtype=np.float64)
        off = np.zeros(len(atoms) + 1, dtype=np.int32)
        off[1:] = np.cumsum([np.asarray(a).reshape(-1, 3).shape[0] for a in atoms])
        if xyz.size == 0:
            xyz = np.zeros(3)
        self._check(self.lib.ofm_set_pair_cutoff(self.h, _dptr(xyz), _iptr(off), float(d_cut)))

    # -- ofm_window_from_index
    def window_from_index(self, i_lo, width, max_out=None):
        """(E, n): E_{i_lo} and the later eigenvalues up to E_{i_lo} + width."""
        if max_out is None:
            max_out = sum(f.n_states for f in self.frags) or self._dense_n or 1
        out = np.zeros(max(1, max_out))
        n = C.c_int()
        self._check(self.lib.ofm_window_from_index(self.h, int(i_lo), float(width), int(max_out),
                                                   _dptr(out), C.byref(n)))
        return out[:min(n.value, max_out)].copy(), n.value

    # -- ofm_select_states
    def select_states(self, first, count):
        """Keep states first[a] .. first[a] + count[a] - 1 of every fragment
        (ints or per-fragment sequences) as the basis."""
        nf = len(self.frags)
        f = np.ascontiguousarray(np.broadcast_to(np.asarray(first, dtype=np.int32), (nf,)))
        n = np.ascontiguousarray(np.broadcast_to(np.asarray(count, dtype=np.int32), (nf,)))
        self._check(self.lib.ofm_select_states(self.h, _iptr(f), _iptr(n)))
        self.frags = [_Frag(tuple(fr.off), tuple(fr.ext), int(n[a])) for a, fr in enumerate(self.frags)]

    # -- ofm_homo_lumo_gap
    def homo_lumo_gap(self, gap_min):
        """(e_ref, E_homo, E_lumo, n_occ) of the HOMO-basis occupation rule."""
        e_ref, eh, el, n = C.c_double(), C.c_double(), C.c_double(), C.c_int()
        self._check(self.lib.ofm_homo_lumo_gap(self.h, float(gap_min), C.byref(e_ref), C.byref(eh),
                                               C.byref(el), C.byref(n)))
        return e_ref.value, eh.value, el.value, n.value

    def pairs(self):
        n = C.c_int()
        self._check(self.lib.ofm_get_pairs(self.h, C.byref(n), None))
        out = np.zeros(2 * n.value, dtype=np.int32)
        self._check(self.lib.ofm_get_pairs(self.h, C.byref(n), _iptr(out)))
        return [tuple(map(int, out[2 * i:2 * i + 2])) for i in range(n.value)]

    def plan_info(self):
        info = ofm_plan_info()
        self._check(self.lib.ofm_get_plan_info(self.h, C.byref(info)))
        return {k: getattr(info, k) for k, _ in ofm_plan_info._fields_}

    def last_schedule(self):
        """Schedule of the last assembly: "pair", "region" or None."""
        return {1: "pair", 2: "region"}.get(self.plan_info()["last_schedule"])

    def block(self, a, b):
        na, nb = self.frags[a].n_states, self.frags[b].n_states
        H = np.zeros((na, nb))
        S = np.zeros((na, nb))
        self._check(self.lib.ofm_get_block(self.h, a, b, _dptr(H), _dptr(S)))
        return H, S

    def dense_HS(self, out_H=None, out_S=None):
        """Host numpy arrays, or CUDA torch tensors when out_H/out_S are given."""
        if out_H is not None or out_S is not None:
            pH = C.c_void_p(out_H.data_ptr()) if out_H is not None else None
            pS = C.c_void_p(out_S.data_ptr()) if out_S is not None else None
            self._check(self.lib.ofm_get_dense_HS(self.h, pH, pS, DEVICE))
            return out_H, out_S
        n = sum(f.n_states for f in self.frags)
        H = np.zeros((n, n))
        S = np.zeros((n, n))
        self._check(self.lib.ofm_get_dense_HS(self.h, C.c_void_p(H.ctypes.data),
                                              C.c_void_p(S.ctypes.data), HOST))
        return H, S

    def hphi(self, b):
        f = self.frags[b]
        Pd = 1
        for d in range(3):
            Pd *= f.ext[d] + 2 if f.ext[d] < self.grid.n[d] else f.ext[d]
        out = np.zeros((f.n_states, Pd))
        self._check(self.lib.ofm_get_hphi(self.h, b, _dptr(out)))
        return out.T

    # -- ofm_window_eigs / ofm_eigs_by_index / ofm_set_dense_HS
    def window_eigs(self, E_lo, E_hi, max_out=None, vectors=False, n_basis=None):
        if max_out is None:
            max_out = n_basis or sum(f.n_states for f in self.frags) or self._dense_n or 1
        E = np.zeros(max(1, max_out))
        nout = C.c_int()
        Cv = None
        if vectors:
            n = n_basis or sum(f.n_states for f in self.frags)
            Cv = np.zeros((max_out, n))
        self._check(self.lib.ofm_window_eigs(self.h, float(E_lo), float(E_hi), max_out, _dptr(E),
                                             C.byref(nout), _dptr(Cv) if vectors else None))
        m = min(nout.value, max_out)
        if vectors:
            return E[:m], Cv[:m].T, nout.value
        return E[:m], nout.value

    def eigs_by_index(self, i_lo, i_hi):
        E = np.zeros(max(1, i_hi - i_lo))
        self._check(self.lib.ofm_eigs_by_index(self.h, i_lo, i_hi, _dptr(E)))
        return E[:i_hi - i_lo]

    # -- ofm_set_profiling / ofm_get_kernel_stats
    def set_profiling(self, on=True):
        self._check(self.lib.ofm_set_profiling(self.h, 1 if on else 0))

    def kernel_stats(self):
        """{class name: dict(row, launches, ms, bytes, flops)}; synchronises."""
        out = (ofm_kernel_stat * 64)()
        n = C.c_int()
        self._check(self.lib.ofm_get_kernel_stats(self.h, out, 64, C.byref(n)))
        return {out[i].name.decode(): dict(row=out[i].row.decode(), launches=out[i].launches,
                                           ms=out[i].total_ms, bytes=out[i].bytes,
                                           flops=out[i].flops)
                for i in range(n.value)}

    def set_dense_HS(self, H, S):
        H = np.ascontiguousarray(H, dtype=np.float64)
        S = np.ascontiguousarray(S, dtype=np.float64)
        self._check(self.lib.ofm_set_dense_HS(self.h, H.shape[0], _dptr(H), _dptr(S)))
        self._dense_n = H.shape[0]
