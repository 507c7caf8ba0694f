"""The assembly as a captured CUDA graph (replayed on later calls) gives the
same blocks as launching the kernels one by one, follows new states, counts
its launches, and re-plans when the work-item size changes."""
import numpy as np
import pytest

from ofm_inputs import make_workload, random_states, small_workload
from oracle import ofm_oracle as O

from gpu_util import gpu_lib
from test_gpu_assembly import GEOMS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ofm():
    return gpu_lib()


def blocks_of(ctx, pairs):
    return {p: ctx.block(*p) for p in pairs}


@pytest.mark.parametrize("storage,prec", [("fp64", "fp64"), ("fp32", "fp32"), ("fp32", "tf32"),
                                          ("fp32", "bf16"), ("fp32", "bf16x3")])
def test_graph_replay_matches_direct_launches(ofm, storage, prec):
    grid, frags = GEOMS["chain"]
    wl = small_workload(grid_n=grid.n, h=grid.h, frags=frags, seed=9)
    ctx = ofm.Context()
    ctx.build_fragments(grid, wl.V, frags, storage=storage)
    for a, f in enumerate(frags):
        ctx.set_fragment_states(a, random_states(grid, f, seed=500 + a))
    pairs = ctx.pairs()
    ctx.assemble(prec, use_graph=False)
    direct = blocks_of(ctx, pairs)
    before = ctx.kernel_stats()
    ctx.assemble(prec, use_graph=True)     # capture + replay
    first = blocks_of(ctx, pairs)
    mid = ctx.kernel_stats()
    ctx.assemble(prec, use_graph=True)     # replay
    second = blocks_of(ctx, pairs)
    after = ctx.kernel_stats()
    for p in pairs:
        for k in range(2):
            assert np.array_equal(direct[p][k], first[p][k]), p
            assert np.array_equal(direct[p][k], second[p][k]), p
    # one replay adds the same per-class launch counts as one direct assembly
    for name in ("apply", "contract", "finalize"):
        assert after[name]["launches"] - mid[name]["launches"] == mid[name]["launches"] - before[name]["launches"] >= 1


def test_graph_replay_follows_new_states(ofm):
    grid, frags = GEOMS["wrap"]
    wl = small_workload(grid_n=grid.n, h=grid.h, frags=frags, seed=10)
    ctx = ofm.Context()
    ctx.build_fragments(grid, wl.V, frags, storage="fp64")
    for a, f in enumerate(frags):
        ctx.set_fragment_states(a, random_states(grid, f, seed=600 + a))
    ctx.assemble("fp64", use_graph=True)
    Phis = [random_states(grid, f, seed=700 + a) for a, f in enumerate(frags)]
    for a, P in enumerate(Phis):
        ctx.set_fragment_states(a, P)
    ctx.assemble("fp64", use_graph=True)   # replay with the new states
    H = O.hamiltonian(wl.grid, wl.V)
    for (a, b), (Hab, Sab) in O.pair_blocks(H, grid, frags, Phis, ctx.pairs()).items():
        Hg, Sg = ctx.block(a, b)
        assert np.max(np.abs(Sg - Sab)) < 1e-12 * max(1.0, np.abs(Sab).max()), (a, b)
        assert np.max(np.abs(Hg - Hab)) < 1e-11 * max(1.0, np.abs(Hab).max()), (a, b)


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_chunk_points_replans(ofm, prec):
    """Other work-item sizes change only the order of the sums."""
    wl = make_workload("tiny")
    storage = "fp64" if prec == "fp64" else "fp32"
    ctx = ofm.Context()
    ctx.build_fragments(wl.grid, wl.V, wl.frags, storage=storage)
    for a, f in enumerate(wl.frags):
        ctx.set_fragment_states(a, random_states(wl.grid, f, seed=800 + a))
    pairs = ctx.pairs()
    ctx.assemble(prec)
    ref = blocks_of(ctx, pairs)
    items_default = ctx.plan_info()["n_work_items"]
    for chunk in (64, 4000):
        ctx.assemble(prec, chunk_points=chunk)
        got = blocks_of(ctx, pairs)
        tol = 1e-12 if prec == "fp64" else 1e-5
        for p in pairs:
            for k in range(2):
                scale = max(1.0, np.abs(ref[p][k]).max())
                assert np.max(np.abs(got[p][k] - ref[p][k])) < tol * scale, (chunk, p)
    ctx.assemble(prec, chunk_points=64)
    assert ctx.plan_info()["n_work_items"] > items_default
