"""GPU parity of the assembly path (H apply, pair contraction, symmetrise,
dense export) and of the window solver, against the FP64 oracle on the same
seeded inputs, through the C ABI."""
import math

import numpy as np
import pytest

from ofm_inputs import Fragment, Grid, make_workload, random_states, small_workload
from oracle import ofm_oracle as O

from gpu_util import U32, gpu_lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ofm():
    return gpu_lib()


def abs_overlap(grid, fa, Pa, fb, Pb):
    """sum_r |phi_a(r)| |phi_b(r)| with zero-extended states."""
    Ea = O.zero_extend(grid, fa, Pa)
    Eb = O.zero_extend(grid, fb, Pb)
    return (abs(Ea).T @ abs(Eb)).toarray()


def oracle_with_states(wl, Phis):
    H = O.hamiltonian(wl.grid, wl.V)
    pairs = O.pair_list(wl.grid, wl.frags)
    blocks = O.pair_blocks(H, wl.grid, wl.frags, Phis, pairs)
    return H, pairs, blocks


def run_gpu(ofm, wl, Phis, storage, prec):
    ctx = ofm.Context()
    ctx.build_fragments(wl.grid, wl.V, wl.frags, storage=storage)
    for a, P in enumerate(Phis):
        ctx.set_fragment_states(a, P)
    ctx.assemble(prec)
    return ctx


# ---------------------------------------------------------------- FP64 -----

def test_tiny_fp64_shared_states_blocks_hphi_window(ofm):
    """Tiny workload, oracle eigenstates imported: every block, every H phi
    and the window eigenvalues agree with the oracle to FP64 rounding."""
    wl = make_workload("tiny")
    r = O.run_ofm(wl)
    ctx = run_gpu(ofm, wl, r["Phis"], "fp64", "fp64")
    assert ctx.pairs() == r["pairs"]
    for (a, b), (Hab, Sab) in r["blocks"].items():
        Hg, Sg = ctx.block(a, b)
        scale = max(1.0, np.abs(Hab).max())
        assert np.max(np.abs(Hg - Hab)) < 1e-12 * scale, (a, b)
        assert np.max(np.abs(Sg - Sab)) < 1e-12, (a, b)
        Hg2, Sg2 = ctx.block(b, a)
        assert np.array_equal(Hg2, Hg.T) and np.array_equal(Sg2, Sg.T)
    for b, f in enumerate(wl.frags):
        want = O.apply_h(r["H"], wl.grid, f, r["Phis"][b])
        got = ctx.hphi(b)
        assert got.shape == want.shape
        assert np.max(np.abs(got - want)) < 1e-12 * np.abs(want).max()
    Hd, Sd = ctx.dense_HS()
    assert np.max(np.abs(Hd - r["Hd"])) < 1e-12 * np.abs(r["Hd"]).max()
    assert np.max(np.abs(Sd - r["Sd"])) < 1e-12
    lo, hi = O.window_bounds(r["E"], wl.window)
    want = r["E"][(r["E"] >= lo - 1e-9) & (r["E"] <= hi + 1e-9)]
    got, n = ctx.window_eigs(lo - 1e-9, hi + 1e-9)
    assert n == len(want)
    assert np.max(np.abs(got - want)) < 1e-10
    allE = ctx.eigs_by_index(0, len(r["E"]))
    assert np.max(np.abs(allE - r["E"])) < 1e-10


GEOMS = {
    # boxes wrapping through the periodic boundary, mixed full-span dims,
    # halo-only pairs, uneven state counts (not multiples of 4)
    "wrap": (Grid((20, 9, 8), 0.45), [
        Fragment((15, 0, 0), (9, 9, 5), 5), Fragment((3, 2, 4), (7, 5, 8), 7),
        Fragment((9, 7, 6), (6, 4, 6), 3), Fragment((0, 0, 0), (20, 9, 8), 9),
        Fragment((18, 5, 2), (4, 9, 3), 2)]),
    "chain": (Grid((48, 10, 10), 0.5), [Fragment((6 * a, 0, 0), (12, 10, 10), 6 + a % 3)
                                         for a in range(8)]),
}


@pytest.mark.parametrize("geom", sorted(GEOMS))
def test_random_states_fp64_blocks_exact(ofm, geom):
    grid, frags = GEOMS[geom]
    wl = small_workload(grid_n=grid.n, h=grid.h, frags=frags, seed=3)
    Phis = [random_states(grid, f, seed=100 + a) for a, f in enumerate(frags)]
    H, pairs, blocks = oracle_with_states(wl, Phis)
    ctx = run_gpu(ofm, wl, Phis, "fp64", "fp64")
    assert ctx.pairs() == pairs
    for (a, b), (Hab, Sab) in blocks.items():
        Hg, Sg = ctx.block(a, b)
        bound_s = 1e-13 * max(1.0, abs_overlap(wl.grid, frags[a], Phis[a], frags[b], Phis[b]).max())
        assert np.max(np.abs(Sg - Sab)) < bound_s, (a, b)
        assert np.max(np.abs(Hg - Hab)) < 1e-12 * max(1.0, np.abs(Hab).max()), (a, b)
    for b, f in enumerate(frags):
        want = O.apply_h(H, grid, f, Phis[b])
        assert np.max(np.abs(ctx.hphi(b) - want)) < 1e-12 * np.abs(want).max()
    # a pair that is not in the list reads as zeros
    Hd, Sd = ctx.dense_HS()
    Hd_o, Sd_o = O.assemble_dense(frags, blocks)
    assert np.max(np.abs(Hd - Hd_o)) < 1e-12 * np.abs(Hd_o).max()
    assert np.max(np.abs(Sd - Sd_o)) < 1e-12 * max(1.0, np.abs(Sd_o).max())


# ---------------------------------------------------------------- FP32 -----

def fp32_states(grid, frags, seed0):
    # the states as FP32 holds them, so both sides start from the same numbers
    return [random_states(grid, f, seed=seed0 + a).astype(np.float32).astype(np.float64)
            for a, f in enumerate(frags)]


def check_fp32_blocks(ctx, wl, Phis, H, pairs, prec, sample=None):
    """Per-entry bound for FP32 sums: |err| <= 2 (n_chunk_terms) u |a|.|b|,
    plus the FP32 H-apply error (<= 8 u |(|c0+V| |phi| + c1 sum|nbrs|)|)."""
    rng = np.random.default_rng(0)
    if sample is not None and len(pairs) > sample:
        idx = rng.choice(len(pairs), size=sample, replace=False)
        pairs = [pairs[i] for i in sorted(idx)]
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
        K = max(1, int(np.prod(fa.ext)))
        cS = 2 * K * U32 * absS + 1e-30
        cH = (2 * K + 8) * U32 * absH + 1e-30
        eS = np.abs(Sg - Sab)
        eH = np.abs(Hg - Hab)
        assert np.all(eS <= cS), (a, b, (eS / cS).max())
        assert np.all(eH <= cH), (a, b, (eH / cH).max())
        # typical errors are far below the worst case: sqrt(K) scaling
        worst = max(worst, (eS / (math.sqrt(K) * U32 * absS + 1e-30)).max(),
                    (eH / (math.sqrt(K) * U32 * absH + 1e-30)).max())
    assert worst < 8.0, worst


@pytest.mark.parametrize("geom", sorted(GEOMS))
def test_random_states_fp32(ofm, geom):
    grid, frags = GEOMS[geom]
    wl = small_workload(grid_n=grid.n, h=grid.h, frags=frags, seed=3)
    Phis = fp32_states(grid, frags, 200)
    H = O.hamiltonian(wl.grid, wl.V)
    ctx = run_gpu(ofm, wl, Phis, "fp32", "fp32")
    check_fp32_blocks(ctx, wl, Phis, H, O.pair_list(grid, frags), "fp32")


def test_fp64_arithmetic_on_fp32_storage(ofm):
    """FP64 contraction of FP32-stored states: products are exact, so the
    blocks differ from the oracle only through the FP32 H apply."""
    grid, frags = GEOMS["chain"]
    wl = small_workload(grid_n=grid.n, h=grid.h, frags=frags, seed=3)
    Phis = fp32_states(grid, frags, 300)
    H, pairs, blocks = oracle_with_states(wl, Phis)
    ctx = run_gpu(ofm, wl, Phis, "fp32", "fp64")
    for (a, b), (Hab, Sab) in blocks.items():
        Hg, Sg = ctx.block(a, b)
        assert np.max(np.abs(Sg - Sab)) < 1e-13 * max(1.0, abs_overlap(wl.grid, frags[a], Phis[a], frags[b], Phis[b]).max())
        Ea = O.zero_extend(wl.grid, frags[a], Phis[a])
        Eb = O.zero_extend(wl.grid, frags[b], Phis[b])
        absH = (abs(Ea).T @ (abs(H) @ abs(Eb))).toarray()
        assert np.all(np.abs(Hg - Hab) <= 8 * U32 * absH + 1e-14), (a, b)


def test_alkane_full_size_fp32_sampled_pairs(ofm):
    """The 256x32x32 alkane-chain workload at full size (31 boxes 16x32x32,
    32 states), random FP32 states, FP32 contraction: a seeded sample of
    pairs of every kind against the oracle, entry by entry."""
    wl = make_workload("alkane")
    Phis = fp32_states(wl.grid, wl.frags, 400)
    H = O.hamiltonian(wl.grid, wl.V)
    ctx = run_gpu(ofm, wl, Phis, "fp32", "fp32")
    pairs = ctx.pairs()
    assert len(pairs) == 91
    chosen = [(0, 0), (0, 1), (0, 2), (0, 30), (14, 15), (15, 17), (29, 30), (30, 30)]
    check_fp32_blocks(ctx, wl, Phis, H, chosen, "fp32")


# ---------------------------------------------------------------- Eq. 2 ----

@pytest.mark.parametrize("n", [1, 7, 33, 100, 257])
def test_window_solver_random_pencils(ofm, n):
    rng = np.random.default_rng(n)
    X = rng.standard_normal((n, n))
    S = X @ X.T / n + 0.3 * np.eye(n)
    Y = rng.standard_normal((n, n))
    Hm = 0.5 * (Y + Y.T)
    E = O.generalized_eigs(Hm, S)
    ctx = ofm.Context()
    ctx.set_dense_HS(Hm, S)
    got = ctx.eigs_by_index(0, n)
    assert np.max(np.abs(got - E)) < 1e-10 * max(1.0, np.abs(E).max())
    lo, hi = E[n // 3] - 1e-7, E[(2 * n) // 3] + 1e-7
    w, cnt = ctx.window_eigs(lo, hi, max_out=n)
    want = E[(E >= lo) & (E <= hi)]
    assert cnt == len(want)
    assert np.max(np.abs(w - want)) < 1e-10 * max(1.0, np.abs(E).max())


def test_window_solver_reports_indefinite_overlap(ofm):
    ctx = ofm.Context()
    S = np.eye(40)
    S[3, 3] = -1.0
    ctx.set_dense_HS(np.eye(40), S)
    with pytest.raises(ofm.OFMError) as e:
        ctx.eigs_by_index(0, 3)
    assert e.value.status == ofm.OFM_ERR_NOT_POSDEF
    assert "pivot 3" in str(e.value)


def test_status_codes_for_bad_calls(ofm):
    ctx = ofm.Context()
    with pytest.raises(ofm.OFMError) as e:
        ctx.assemble("fp32")
    assert e.value.status == ofm.OFM_ERR_STATE
    wl = make_workload("tiny")
    with pytest.raises(ofm.OFMError) as e:
        ctx.build_fragments(wl.grid, wl.V, [Fragment((0, 0, 0), (31, 12, 12), 6)])
    assert e.value.status == ofm.OFM_ERR_INVALID
    ctx.build_fragments(wl.grid, wl.V, wl.frags, storage="fp64")
    with pytest.raises(ofm.OFMError) as e:
        ctx.assemble("fp64")          # states not set yet
    assert e.value.status == ofm.OFM_ERR_STATE
    for a, f in enumerate(wl.frags):
        ctx.set_fragment_states(a, random_states(wl.grid, f, seed=a))
    with pytest.raises(ofm.OFMError) as e:
        ctx.assemble("fp32")          # FP32 arithmetic needs FP32 storage
    assert e.value.status == ofm.OFM_ERR_INVALID
    ctx.assemble("fp64")


def test_set_potential_and_get_blocks(ofm):
    """A new potential in the same basis (ofm_set_potential): with V -> V + c
    the whole-system H gains c I, so every H_ab gains c S_ab while S_ab stays
    (Eq. 1); the blocks equal the oracle's for the shifted potential.  The
    block export (ofm_get_blocks) is the pair list's [H_ab | S_ab] blocks
    concatenated, bit for bit those of ofm_get_block."""
    import torch
    wl = make_workload("tiny")
    r = O.run_ofm(wl)
    ctx = run_gpu(ofm, wl, r["Phis"], "fp64", "fp64")
    all0 = ctx.get_blocks()
    off = 0
    for a, b in ctx.pairs():
        na, nb = wl.frags[a].n_states, wl.frags[b].n_states
        Hg, Sg = ctx.block(a, b)
        assert np.array_equal(all0[off:off + na * nb].reshape(na, nb), Hg)
        assert np.array_equal(all0[off + na * nb:off + 2 * na * nb].reshape(na, nb), Sg)
        off += 2 * na * nb
    assert off == len(all0) == ctx.blocks_count()
    c = 0.37
    ctx.set_potential(wl.V + c)
    with pytest.raises(ofm.OFMError):
        ctx.block(0, 1)            # blocks of the old H are gone
    ctx.assemble("fp64")
    H2 = O.hamiltonian(wl.grid, wl.V + c)
    for (a, b), (Hab, Sab) in r["blocks"].items():
        Hg, Sg = ctx.block(a, b)
        Ho, So = O.pair_block(H2, wl.grid, wl.frags[a], r["Phis"][a], wl.frags[b], r["Phis"][b])
        if a == b:
            Ho = 0.5 * (Ho + Ho.T)
        assert np.max(np.abs(Hg - (Hab + c * Sab))) < 1e-12
        assert np.max(np.abs(Hg - Ho)) < 1e-12 and np.max(np.abs(Sg - Sab)) < 1e-13
    # device output and a pinned host output give the same blocks
    dev = torch.empty(ctx.blocks_count(), dtype=torch.float64, device="cuda")
    pin = torch.empty(ctx.blocks_count(), dtype=torch.float64).pin_memory()
    ctx.get_blocks(dev)
    ctx.get_blocks(pin)
    assert np.array_equal(dev.cpu().numpy(), pin.numpy())
    assert np.array_equal(pin.numpy(), ctx.get_blocks())


def test_blocks_async_read_back(ofm):
    """ofm_get_blocks_async: the blocks reach the caller's buffer (pinned host
    or device) after ofm_sync_blocks, bit for bit those of ofm_get_blocks,
    also when the next assemblies (another potential each) are enqueued while
    the previous blocks travel; the last call's blocks are the ones held."""
    import torch
    wl = make_workload("tiny")
    r = O.run_ofm(wl)
    ctx = run_gpu(ofm, wl, r["Phis"], "fp64", "fp64")
    n = ctx.blocks_count()
    pin = torch.full((n,), -1.0, dtype=torch.float64).pin_memory()
    dev = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
    for k, c in enumerate((0.0, 0.21, -0.13)):
        ctx.set_potential(wl.V + c)
        ctx.assemble("fp64")
        ctx.get_blocks_async(pin if k % 2 == 0 else dev)
    ctx.sync_blocks()
    last = ctx.get_blocks()
    assert np.array_equal(pin.numpy(), last)           # the third assembly (k = 2)
    ctx.set_potential(wl.V + 0.21)
    ctx.assemble("fp64")
    ref = ctx.get_blocks()
    assert np.array_equal(dev.cpu().numpy(), ref)      # the second assembly (k = 1)
    # the count query and the sync without a pending transfer
    assert ctx.lib.ofm_sync_blocks(ctx.h) == ofm.OFM_OK
