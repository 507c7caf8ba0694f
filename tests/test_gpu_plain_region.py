"""The plain forms of the region schedule on the CUDA cores (FP32 and FP64
arithmetic) against the FP64 oracle on the same FP32 states.

FP32: the per-entry bound of an FP32 inner product of the exact (FP32) states,
    |err| <= 2 K u_32 sum_r |phi_a(r)| |phi_b(r)|
(K the points of box a; the H block adds the FP32 H-apply error).

FP64: the region form forms H phi in FP64 from the context's FP32 states and
FP32 potential, so the oracle takes the potential rounded to FP32 too, and
the bound is the FP64 one,
    |err| <= 2 (K + 64) u_64 sum_r |phi_a(r)| |(|H| |phi_b|)(r)|.
The pair schedule (FP32 H phi, FP64 sums) is checked against the FP32 bound.
"""
import numpy as np
import pytest

from ofm_inputs import make_workload, small_workload
from oracle import ofm_oracle as O

from gpu_util import U32, U64, gpu_lib
from test_gpu_tensorcore import GEOMS, fp32_states

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ofm():
    return gpu_lib()


def bounds(wl, H, Phis, a, b, prec, sched):
    fa, fb = wl.frags[a], wl.frags[b]
    Ea = O.zero_extend(wl.grid, fa, Phis[a])
    Eb = O.zero_extend(wl.grid, fb, Phis[b])
    absS = (abs(Ea).T @ abs(Eb)).toarray()
    absH = (abs(Ea).T @ (abs(H) @ abs(Eb))).toarray()
    K = int(np.prod(fa.ext))
    if prec == "fp64" and sched == "region":
        c = 2 * (K + 64) * U64
        return c * absS + 1e-300, c * absH + 1e-300
    return 2 * K * U32 * absS + 1e-30, (2 * K + 8) * U32 * absH + 1e-30


def check(ctx, wl, Phis, H, pairs, prec, sched):
    worst = 0.0
    for a, b in pairs:
        Hab, Sab = O.pair_block(H, wl.grid, wl.frags[a], Phis[a], wl.frags[b], Phis[b])
        if a == b:
            Hab, Sab = 0.5 * (Hab + Hab.T), 0.5 * (Sab + Sab.T)
        Hg, Sg = ctx.block(a, b)
        cS, cH = bounds(wl, H, Phis, a, b, prec, sched)
        eS, eH = np.abs(Sg - Sab), np.abs(Hg - Hab)
        assert np.all(np.isfinite(Sg)) and np.all(np.isfinite(Hg)), (a, b)
        assert np.all(eS <= cS), (prec, sched, a, b, float((eS / cS).max()))
        assert np.all(eH <= cH), (prec, sched, a, b, float((eH / cH).max()))
        worst = max(worst, float((eS / cS).max()), float((eH / cH).max()))
    return worst


def v32(V):
    return np.asarray(V, dtype=np.float64).astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("sched", ["pair", "region"])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("geom", sorted(GEOMS))
def test_plain_blocks_within_bounds(ofm, geom, prec, sched):
    grid, frags = GEOMS[geom]
    wl = small_workload(grid_n=grid.n, h=grid.h, frags=frags, seed=3)
    Phis = fp32_states(grid, frags, 500)
    H = O.hamiltonian(grid, v32(wl.V) if (prec, sched) == ("fp64", "region") else wl.V)
    ctx = ofm.Context()
    ctx.build_fragments(grid, wl.V, frags, storage="fp32")
    for a, P in enumerate(Phis):
        ctx.set_fragment_states(a, P)
    ctx.assemble(prec, schedule=sched)
    check(ctx, wl, Phis, H, O.pair_list(grid, frags), prec, sched)
    first = ctx.block(0, 1)
    ctx.assemble(prec, schedule=sched)   # graph replay: the same blocks bit for bit
    again = ctx.block(0, 1)
    assert np.array_equal(first[0], again[0]) and np.array_equal(first[1], again[1])


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_plain_region_alkane_sampled(ofm, prec):
    """Full-size alkane chain (31 boxes 16x32x32, 32 states), the plain
    region form by default, sampled pairs including the halo-only ones."""
    wl = make_workload("alkane")
    Phis = fp32_states(wl.grid, wl.frags, 900)
    H = O.hamiltonian(wl.grid, v32(wl.V) if prec == "fp64" else wl.V)
    ctx = ofm.Context()
    ctx.build_fragments(wl.grid, wl.V, wl.frags, storage="fp32")
    for a, P in enumerate(Phis):
        ctx.set_fragment_states(a, P)
    ctx.assemble(prec)
    assert ctx.last_schedule() == "region"
    check(ctx, wl, Phis, H, [(0, 0), (0, 1), (0, 2), (0, 30), (14, 15), (15, 17), (30, 30)],
          prec, "region")


def test_plain_region_fp64_window_on_shared_states(ofm):
    """Tiny workload, the oracle's eigenstates rounded to FP32: the FP64
    region form's window against the oracle's pencil on the same states and
    the potential rounded to FP32, to 1e-9 Ha."""
    wl = make_workload("tiny")
    r = O.run_ofm(wl)
    Phis32 = [P.astype(np.float32).astype(np.float64) for P in r["Phis"]]
    H32 = O.hamiltonian(wl.grid, v32(wl.V))
    blocks = O.pair_blocks(H32, wl.grid, wl.frags, Phis32, r["pairs"])
    Hd, Sd = O.assemble_dense(wl.frags, blocks)
    E = O.generalized_eigs(Hd, Sd)
    lo, hi = O.window_bounds(E, wl.window)
    ctx = ofm.Context()
    ctx.build_fragments(wl.grid, wl.V, wl.frags, storage="fp32")
    for a, P in enumerate(Phis32):
        ctx.set_fragment_states(a, P)
    ctx.assemble("fp64", schedule="region")
    m = int(np.sum((E >= lo) & (E <= hi)))
    got = ctx.eigs_by_index(0, m)
    assert np.max(np.abs(got - E[:m])) < 1e-9, np.max(np.abs(got - E[:m]))
