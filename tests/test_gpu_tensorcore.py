"""Tensor-core (tcgen05) pair contraction in TF32, BF16 and BF16 hi+lo
against the FP64 oracle on the same FP32 states, in both schedules: one GEMM
per pair, and coverage regions with their fragments stacked into one GEMM
(the region sums are FP32 over each region's points, FP64 across regions).

Per-entry bound (Higham's inner-product bound with rounded inputs):
    |err| <= (2 u_in + 2 K u_32) sum_r |phi_a(r)| |phi_b(r)|
with u_in the unit roundoff of the operand type (2^-11 for TF32 rounded to
nearest, 2^-9 for BF16, 2^-16 for the hi+lo pair, whose dropped lo*lo term
and split rounding sit below 2^-16), K the points of box a and u_32 = 2^-24
for the FP32 accumulation; the H block adds the FP32 H-apply error.
"""
import math

import numpy as np
import pytest

from ofm_inputs import Fragment, Grid, make_workload, random_states, small_workload
from oracle import ofm_oracle as O

from gpu_util import U32, gpu_lib

pytestmark = pytest.mark.gpu

U_IN = {"tf32": 2.0 ** -11, "bf16": 2.0 ** -9, "bf16x3": 2.0 ** -16}


@pytest.fixture(scope="module")
def ofm():
    return gpu_lib()


GEOMS = {
    "wrap": (Grid((20, 9, 8), 0.45), [
        Fragment((15, 0, 0), (9, 9, 5), 5), Fragment((3, 2, 4), (7, 5, 8), 7),
        Fragment((9, 7, 6), (6, 4, 6), 3), Fragment((0, 0, 0), (20, 9, 8), 9),
        Fragment((18, 5, 2), (4, 9, 3), 2)]),
    "chain": (Grid((48, 10, 10), 0.5), [Fragment((6 * a, 0, 0), (12, 10, 10), 6 + a % 3)
                                         for a in range(8)]),
    "wide": (Grid((40, 12, 12), 0.5), [Fragment((10 * a, 0, 0), (16, 12, 12), 37 + 23 * a)
                                        for a in range(4)]),
}


def fp32_states(grid, frags, seed0):
    return [random_states(grid, f, seed=seed0 + a).astype(np.float32).astype(np.float64)
            for a, f in enumerate(frags)]


def check_blocks(ctx, wl, Phis, H, pairs, prec):
    worst = 0.0
    for a, b in pairs:
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
        eS, eH = np.abs(Sg - Sab), np.abs(Hg - Hab)
        assert np.all(np.isfinite(Sg)) and np.all(np.isfinite(Hg)), (a, b)
        assert np.all(eS <= cS), (prec, a, b, float((eS / cS).max()))
        assert np.all(eH <= cH), (prec, a, b, float((eH / cH).max()))
        worst = max(worst, float((eS / cS).max()), float((eH / cH).max()))
    return worst


@pytest.mark.parametrize("sched", ["pair", "region"])
@pytest.mark.parametrize("prec", ["tf32", "bf16", "bf16x3"])
@pytest.mark.parametrize("geom", sorted(GEOMS))
def test_tensor_core_blocks_within_bounds(ofm, geom, prec, sched):
    grid, frags = GEOMS[geom]
    wl = small_workload(grid_n=grid.n, h=grid.h, frags=frags, seed=3)
    Phis = fp32_states(grid, frags, 500)
    H = O.hamiltonian(grid, wl.V)
    ctx = ofm.Context()
    ctx.build_fragments(grid, wl.V, frags, storage="fp32")
    for a, P in enumerate(Phis):
        ctx.set_fragment_states(a, P)
    ctx.assemble(prec, schedule=sched)
    check_blocks(ctx, wl, Phis, H, O.pair_list(grid, frags), prec)
    # a second assembly (captured graph replay) gives the same blocks bit for bit
    H01 = ctx.block(0, 1)
    ctx.assemble(prec, schedule=sched)
    H01b = ctx.block(0, 1)
    assert np.array_equal(H01[0], H01b[0]) and np.array_equal(H01[1], H01b[1])


@pytest.mark.parametrize("sched", ["pair", "region"])
@pytest.mark.parametrize("prec", ["tf32", "bf16x3"])
def test_tensor_core_alkane_full_size_sampled(ofm, prec, sched):
    wl = make_workload("alkane")
    Phis = fp32_states(wl.grid, wl.frags, 900)
    H = O.hamiltonian(wl.grid, wl.V)
    ctx = ofm.Context()
    ctx.build_fragments(wl.grid, wl.V, wl.frags, storage="fp32")
    for a, P in enumerate(Phis):
        ctx.set_fragment_states(a, P)
    ctx.assemble(prec, schedule=sched)
    check_blocks(ctx, wl, Phis, H, [(0, 0), (0, 1), (0, 2), (0, 30), (14, 15), (15, 17), (30, 30)],
                 prec)


@pytest.mark.parametrize("sched", ["pair", "region"])
@pytest.mark.parametrize("prec,tol", [("tf32", 1e-4), ("bf16x3", 1e-5), ("bf16", 5e-3)])
def test_tensor_core_window_on_shared_states(ofm, prec, tol, sched):
    """Tiny workload, the oracle's eigenstates (rounded to FP32) imported:
    window eigenvalues of the mixed-precision path against the oracle's."""
    wl = make_workload("tiny")
    r = O.run_ofm(wl)
    Phis32 = [P.astype(np.float32).astype(np.float64) for P in r["Phis"]]
    blocks = O.pair_blocks(r["H"], wl.grid, wl.frags, Phis32, r["pairs"])
    Hd, Sd = O.assemble_dense(wl.frags, blocks)
    E = O.generalized_eigs(Hd, Sd)
    lo, hi = O.window_bounds(E, wl.window)
    ctx = ofm.Context()
    ctx.build_fragments(wl.grid, wl.V, wl.frags, storage="fp32")
    for a, P in enumerate(Phis32):
        ctx.set_fragment_states(a, P)
    ctx.assemble(prec, schedule=sched)
    m = int(np.sum((E >= lo) & (E <= hi)))
    got = ctx.eigs_by_index(0, m)
    assert np.max(np.abs(got - E[:m])) < tol, (prec, np.max(np.abs(got - E[:m])))
