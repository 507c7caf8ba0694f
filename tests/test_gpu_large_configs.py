"""The two largest workloads at their full sizes, in the launch configuration
the benchmark times, against the FP64 oracle on sampled outputs.

Large lattice (384x192x192 grid, 1024 boxes 40^3, 96 states): a cluster of
4x2x2 neighbouring boxes carries seeded random states, every other fragment
zero states; the assembly runs in BF16 hi+lo on the region schedule (the
benchmark's).  At least 64 sampled blocks of cluster pairs are compared
entry by entry with the oracle's, within the inner-product error bound
    |err| <= (2 u_in + 2 K u_32) sum_r |phi_a(r)| |phi_b(r)|
(u_in = 2^-16 for the hi+lo split, K the points of box a, u_32 = 2^-24 for
the FP32 accumulation; the H block adds the FP32 H-apply error), and blocks
of pairs with a zero-state fragment must be exactly zero.

Scaled chains (192^3 grid, ~4000 boxes of 24^3..32^3 along 14 chains, 48
states, ~745k pairs): 12 consecutive boxes of one chain carry random states,
the rest zero; BF16 hi+lo on the per-pair schedule (the region plan does
not apply there: its partial sums would not fit)."""
import numpy as np
import pytest

from ofm_inputs import make_workload

from gpu_util import U32, gpu_lib
from oracle_pool import fp32_states, oracle_blocks

pytestmark = pytest.mark.gpu

U_HILO = 2.0 ** -16


@pytest.fixture(scope="module")
def ofm():
    return gpu_lib()


def load_states(ofm, ctx, wl, active, seed0):
    """Seeded FP32-rounded random states for the active fragments, zeros for
    the rest (imported from a device buffer)."""
    import torch
    zero = {}
    for a, f in enumerate(wl.frags):
        if a in active:
            ctx.set_fragment_states(a, fp32_states(wl.grid, f, seed0 + a))
        else:
            P = f.ext[0] * f.ext[1] * f.ext[2]
            key = (f.n_states, P)
            if key not in zero:
                zero[key] = torch.zeros((f.n_states, P), dtype=torch.float64, device="cuda")
            ctx.set_fragment_states(a, zero[key])


def check(ctx, wl, ref, u_in):
    worst = 0.0
    for (a, b), (Hab, Sab, aS, aH) in ref.items():
        Hg, Sg = ctx.block(a, b)
        K = int(np.prod(wl.frags[a].ext))
        cS = (2 * u_in + 2 * K * U32) * aS + 1e-30
        cH = (2 * u_in + (2 * K + 8) * U32) * aH + 1e-30
        eS, eH = np.abs(Sg - Sab), np.abs(Hg - Hab)
        assert np.all(np.isfinite(Sg)) and np.all(np.isfinite(Hg)), (a, b)
        assert np.all(eS <= cS), (a, b, float((eS / cS).max()))
        assert np.all(eH <= cH), (a, b, float((eH / cH).max()))
        worst = max(worst, float((eS / cS).max()), float((eH / cH).max()))
    return worst


def test_large_lattice_sampled_blocks_bf16x3_region(ofm):
    wl = make_workload("large")
    cx, cy = 16, 8
    cluster = {i + cx * (j + cy * k) for i in range(4) for j in range(2) for k in range(2)}
    pairs = [p for p in ofm.plan_pairs(wl.grid, wl.frags)[0] if p[0] in cluster and p[1] in cluster]
    rng = np.random.default_rng(5)
    sample = sorted(map(tuple, np.array(pairs)[rng.choice(len(pairs), size=min(64, len(pairs)),
                                                          replace=False)].tolist()))
    assert len(sample) >= 64
    ctx = ofm.Context()
    ctx.build_fragments(wl.grid, wl.V, wl.frags, storage="fp32")
    load_states(ofm, ctx, wl, cluster, 3000)
    ctx.assemble("bf16x3", schedule="region")
    ref = oracle_blocks(wl.grid, wl.frags, wl.V, sample, 3000)
    check(ctx, wl, ref, U_HILO)
    # pairs with a zero-state fragment: exactly zero blocks
    outside = [p for p in ctx.pairs() if (p[0] in cluster) != (p[1] in cluster)][:8]
    for a, b in outside:
        Hg, Sg = ctx.block(a, b)
        assert not Hg.any() and not Sg.any(), (a, b)
    ctx.close()


def test_scaled_chains_sampled_blocks_bf16x3_pairs(ofm):
    wl = make_workload("scaled")
    active = set(range(12))   # consecutive fragment centres along the first chain
    pairs = [p for p in ofm.plan_pairs(wl.grid, wl.frags)[0] if p[0] in active and p[1] in active]
    assert len(pairs) >= 64
    rng = np.random.default_rng(6)
    sample = sorted(map(tuple, np.array(pairs)[rng.choice(len(pairs), size=64, replace=False)].tolist()))
    ctx = ofm.Context()
    ctx.build_fragments(wl.grid, wl.V, wl.frags, storage="fp32")
    load_states(ofm, ctx, wl, active, 4000)
    ctx.assemble("bf16x3", schedule="pair")
    ref = oracle_blocks(wl.grid, wl.frags, wl.V, sample, 4000)
    check(ctx, wl, ref, U_HILO)
    ctx.close()
