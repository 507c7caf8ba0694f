"""Edge cases of the assembly against the FP64 oracle on the same FP32 states:

- the largest state count the tensor-core contractions take (128 per
  fragment: a full 128-row half of a region item, a full M tile of a pair)
  and one more (129: both schedules refuse the tensor-core precisions; FP32
  on the CUDA cores takes the per-pair schedule);
- degenerate boxes: one point thick, one state, a fragment with a single
  point row, a box spanning the whole grid, next to ordinary ones.

Per-entry bounds as in test_gpu_tensorcore.py (Higham's inner-product bound
with the operand rounding of each arithmetic)."""
import numpy as np
import pytest

from ofm_inputs import Fragment, Grid, small_workload
from oracle import ofm_oracle as O

from gpu_util import gpu_lib
from test_gpu_tensorcore import check_blocks, fp32_states

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ofm():
    return gpu_lib()


def _run(ofm, grid, frags, prec, sched, seed=7):
    wl = small_workload(grid_n=grid.n, h=grid.h, frags=frags, seed=seed)
    Phis = fp32_states(grid, frags, 800)
    ctx = ofm.Context()
    ctx.build_fragments(grid, wl.V, frags, storage="fp32")
    for a, P in enumerate(Phis):
        ctx.set_fragment_states(a, P)
    ctx.assemble(prec, schedule=sched)
    return ctx, wl, Phis


@pytest.mark.parametrize("sched", ["pair", "region"])
def test_128_states_per_fragment(ofm, sched):
    grid = Grid((24, 12, 12), 0.5)
    frags = [Fragment((0, 0, 0), (16, 12, 12), 128), Fragment((8, 0, 0), (16, 12, 12), 128)]
    ctx, wl, Phis = _run(ofm, grid, frags, "bf16x3", sched)
    assert ctx.last_schedule() == sched
    check_blocks(ctx, wl, Phis, O.hamiltonian(grid, wl.V), O.pair_list(grid, frags), "bf16x3")
    ctx.close()


def test_129_states_take_the_cuda_cores(ofm):
    """Beyond 128 states per fragment the tensor-core contractions refuse
    (OFM_ERR_INVALID, both schedules); FP32 on the CUDA cores takes the
    per-pair schedule (the region plan does not apply either)."""
    grid = Grid((24, 12, 12), 0.5)
    frags = [Fragment((0, 0, 0), (16, 12, 12), 129), Fragment((8, 0, 0), (16, 12, 12), 40)]
    wl = small_workload(grid_n=grid.n, h=grid.h, frags=frags, seed=7)
    ctx = ofm.Context()
    ctx.build_fragments(grid, wl.V, frags, storage="fp32")
    Phis = fp32_states(grid, frags, 800)
    for a, P in enumerate(Phis):
        ctx.set_fragment_states(a, P)
    for sched in ("region", "pair", "auto"):
        with pytest.raises(ofm.OFMError) as e:
            ctx.assemble("bf16x3", schedule=sched)
        assert e.value.status == ofm.OFM_ERR_INVALID and "128 states" in str(e.value)
    ctx.assemble("fp32")
    assert ctx.last_schedule() == "pair"
    H = O.hamiltonian(grid, wl.V)
    for a, b in O.pair_list(grid, frags):
        Hab, Sab = O.pair_block(H, grid, frags[a], Phis[a], frags[b], Phis[b])
        if a == b:
            Hab, Sab = 0.5 * (Hab + Hab.T), 0.5 * (Sab + Sab.T)
        Hg, Sg = ctx.block(a, b)
        Ea = O.zero_extend(grid, frags[a], Phis[a])
        Eb = O.zero_extend(grid, frags[b], Phis[b])
        K = int(np.prod(frags[a].ext))
        cS = 2 * K * 2.0 ** -24 * (abs(Ea).T @ abs(Eb)).toarray() + 1e-30
        cH = (2 * K + 8) * 2.0 ** -24 * (abs(Ea).T @ (abs(H) @ abs(Eb))).toarray() + 1e-30
        assert np.all(np.abs(Sg - Sab) <= cS) and np.all(np.abs(Hg - Hab) <= cH), (a, b)
    ctx.close()


DEGENERATE = [
    Fragment((0, 0, 0), (1, 10, 9), 1),      # one point thick, one state
    Fragment((1, 2, 3), (5, 1, 1), 2),       # a single point row
    Fragment((3, 0, 0), (6, 10, 9), 11),     # ordinary
    Fragment((0, 0, 0), (14, 10, 9), 3),     # the whole grid
    Fragment((9, 4, 0), (3, 3, 9), 1),       # full span in z only
]


@pytest.mark.parametrize("prec,sched", [("bf16x3", "region"), ("bf16x3", "pair"),
                                        ("tf32", "region"), ("fp32", "region"),
                                        ("fp64", "region"), ("fp32", "pair")])
def test_degenerate_boxes(ofm, prec, sched):
    grid = Grid((14, 10, 9), 0.5)
    ctx, wl, Phis = _run(ofm, grid, DEGENERATE, prec, sched)
    pairs = O.pair_list(grid, DEGENERATE)
    assert len(pairs) == len(ctx.pairs())
    H = O.hamiltonian(grid, wl.V)
    if prec in ("bf16x3", "tf32"):
        check_blocks(ctx, wl, Phis, H, pairs, prec)
    else:
        # CUDA-core arithmetic: the FP32 bound (FP64 sits far inside it)
        for a, b in pairs:
            Hab, Sab = O.pair_block(H, grid, DEGENERATE[a], Phis[a], DEGENERATE[b], Phis[b])
            if a == b:
                Hab, Sab = 0.5 * (Hab + Hab.T), 0.5 * (Sab + Sab.T)
            Hg, Sg = ctx.block(a, b)
            Ea = O.zero_extend(grid, DEGENERATE[a], Phis[a])
            Eb = O.zero_extend(grid, DEGENERATE[b], Phis[b])
            K = int(np.prod(DEGENERATE[a].ext))
            cS = 2 * K * 2.0 ** -24 * (abs(Ea).T @ abs(Eb)).toarray() + 1e-30
            cH = (2 * K + 8) * 2.0 ** -24 * (abs(Ea).T @ (abs(H) @ abs(Eb))).toarray() + 1e-30
            assert np.all(np.abs(Sg - Sab) <= cS) and np.all(np.abs(Hg - Hab) <= cH), (a, b)
    ctx.close()
