"""Measuring autotuner of the assembly schedule (stencil form x points per
contraction work item).  Every candidate is a schedule of the same sums
(Sec. II, the pair blocks S_ab and H_ab), so the tuned assembly still meets
the oracle's per-entry bounds; the choice is the fastest reported time, later
default assemblies keep it, and a new layout drops it."""
import numpy as np
import pytest

from ofm_inputs import Fragment, Grid, random_states, small_workload
from oracle import ofm_oracle as O

from gpu_util import U32, gpu_lib

pytestmark = pytest.mark.gpu

# unit roundoff of the operands (Higham's inner-product bound, FP32 sums)
U_IN = {"fp32": 0.0, "bf16x3": 2.0 ** -16}

GRID = Grid((48, 10, 10), 0.5)
FRAGS = [Fragment((6 * a, 0, 0), (12, 10, 10), 6 + a % 3) for a in range(8)]


@pytest.fixture(scope="module")
def ofm():
    return gpu_lib()


@pytest.fixture(scope="module")
def chain():
    wl = small_workload(grid_n=GRID.n, h=GRID.h, frags=FRAGS, seed=5)
    Phis = [random_states(GRID, f, seed=300 + a).astype(np.float32).astype(np.float64)
            for a, f in enumerate(FRAGS)]
    return wl, Phis, O.hamiltonian(wl.grid, wl.V)


def _ctx(ofm, wl, Phis):
    ctx = ofm.Context()
    ctx.build_fragments(wl.grid, wl.V, wl.frags, storage="fp32")
    for a, P in enumerate(Phis):
        ctx.set_fragment_states(a, P)
    return ctx


def _check_bounds(ctx, wl, Phis, H, prec):
    for a, b in O.pair_list(wl.grid, wl.frags):
        fa, fb = wl.frags[a], wl.frags[b]
        Hab, Sab = O.pair_block(H, wl.grid, fa, Phis[a], fb, Phis[b])
        if a == b:
            Hab, Sab = 0.5 * (Hab + Hab.T), 0.5 * (Sab + Sab.T)
        Hg, Sg = ctx.block(a, b)
        Ea = O.zero_extend(wl.grid, fa, Phis[a])
        Eb = O.zero_extend(wl.grid, fb, Phis[b])
        absS = (abs(Ea).T @ abs(Eb)).toarray()
        absH = (abs(Ea).T @ (abs(H) @ abs(Eb))).toarray()
        K = int(np.prod(fa.ext))
        cS = (2 * U_IN[prec] + 2 * K * U32) * absS + 1e-30
        cH = (2 * U_IN[prec] + (2 * K + 8) * U32) * absH + 1e-30
        assert np.all(np.abs(Sg - Sab) <= cS), (prec, a, b)
        assert np.all(np.abs(Hg - Hab) <= cH), (prec, a, b)


def test_autotune_default_candidates_fp32(ofm, chain):
    wl, Phis, H = chain
    ctx = _ctx(ofm, wl, Phis)
    ctx.assemble("fp32")
    chunk, form, ms, times = ctx.autotune_assembly("fp32", reps=2)
    assert times.shape == (2, 5)
    assert np.all(times[0] > 0)                       # the register form always fits
    ok = times[times > 0]
    assert form in (1, 2) and ms > 0 and ms == ok.min()
    assert times[form - 1][times[form - 1] == ms].size >= 1
    _check_bounds(ctx, wl, Phis, H, "fp32")
    # later default assemblies keep the tuned plan
    items = ctx.plan_info()["n_work_items"]
    ctx.assemble("fp32")
    assert ctx.plan_info()["n_work_items"] == items
    _check_bounds(ctx, wl, Phis, H, "fp32")
    # the same layout again keeps it; other state counts drop it
    ctx.build_fragments(wl.grid, wl.V, wl.frags, storage="fp32")
    assert ctx.plan_info()["n_work_items"] == items
    fewer = [Fragment(f.off, f.ext, 4) for f in wl.frags]
    ctx.build_fragments(wl.grid, wl.V, fewer, storage="fp32")
    ref = ofm.Context()
    ref.build_fragments(wl.grid, wl.V, fewer, storage="fp32")
    assert ctx.plan_info()["n_work_items"] == ref.plan_info()["n_work_items"]


def test_autotune_given_candidates_bf16x3(ofm, chain):
    wl, Phis, H = chain
    ctx = _ctx(ofm, wl, Phis)
    cand = [256, 1024, 4096]
    chunk, form, ms, times = ctx.autotune_assembly("bf16x3", chunks=cand, reps=2)
    assert times.shape == (2, 3)
    assert chunk in cand and form in (1, 2)
    assert ms == times[times > 0].min()
    _check_bounds(ctx, wl, Phis, H, "bf16x3")


def test_autotune_errors(ofm, chain):
    wl, Phis, H = chain
    ctx = ofm.Context()
    with pytest.raises(ofm.OFMError):
        ctx.autotune_assembly("fp32")                 # nothing built
    ctx = _ctx(ofm, wl, Phis)
    with pytest.raises(ofm.OFMError):
        ctx.autotune_assembly("fp32", reps=0)
    with pytest.raises(ofm.OFMError):
        ctx.autotune_assembly("fp32", chunks=[512, 0])
    ctx.set_profiling(True)
    with pytest.raises(ofm.OFMError):
        ctx.autotune_assembly("fp32")
    ctx.set_profiling(False)
    ctx.autotune_assembly("fp32", chunks=[512], reps=1)
    _check_bounds(ctx, wl, Phis, H, "fp32")
