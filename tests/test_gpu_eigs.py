"""GPU fragment eigensolver (Chebyshev-filtered subspace iteration) and the
end-to-end method (GPU states -> GPU assembly -> GPU window solve) against
the FP64 oracle.  States are compared only where they are unique (gaps
between neighbouring levels); energies are gauge-invariant."""
import itertools
import math
import multiprocessing as mp

import numpy as np
import pytest

from ofm_inputs import Fragment, Grid, make_workload, small_workload
from oracle import ofm_oracle as O

from gpu_util import gpu_lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ofm():
    return gpu_lib()


def closed_form(grid, frag):
    out = []
    for d in range(3):
        n, e, h = grid.n[d], frag.ext[d], grid.h
        if e == n:
            out.append([(1 - math.cos(2 * math.pi * k / n)) / h ** 2 for k in range(n)])
        else:
            out.append([(1 - math.cos(k * math.pi / (e + 1))) / h ** 2 for k in range(1, e + 1)])
    return np.sort([sum(t) for t in itertools.product(*out)])


@pytest.mark.parametrize("storage,tol", [("fp64", 1e-9), ("fp32", 2e-6)])
def test_free_particle_fragment_levels(ofm, storage, tol):
    grid = Grid((18, 10, 12), 0.5)
    frags = [Fragment((3, 0, 9), (7, 10, 6), 6), Fragment((12, 2, 0), (9, 5, 12), 5)]
    wl = small_workload(grid_n=grid.n, h=grid.h, frags=frags, zero_potential=True)
    ctx = ofm.Context()
    ctx.build_fragments(grid, wl.V, frags, storage=storage)
    eps, res, _ = ctx.fragment_eigs()
    k = 0
    for f in frags:
        want = closed_form(grid, f)[:f.n_states]
        assert np.max(np.abs(eps[k:k + f.n_states] - want)) < tol * 20
        k += f.n_states
    assert res.max() <= (1e-9 if storage == "fp64" else 1e-5)


def test_tiny_fp64_end_to_end(ofm):
    """Tiny workload in FP64: fragment energies and states (gauge fixed) vs
    the oracle's dense eigh, then the window eigenvalues of the whole
    method from the GPU's own states vs the oracle's (1e-6 Ha)."""
    wl = make_workload("tiny")
    r = O.run_ofm(wl)
    ctx = ofm.Context()
    ctx.build_fragments(wl.grid, wl.V, wl.frags, storage="fp64")
    eps, res, _ = ctx.fragment_eigs()
    assert res.max() <= 1e-9
    allo = np.concatenate(r["eps"])
    assert np.max(np.abs(eps - allo)) < 1e-10
    for a in range(4):
        e = r["eps"][a]
        g = ctx.get_fragment_states(a)
        for i in range(len(e)):
            gap = min([abs(e[i] - e[j]) for j in range(len(e)) if j != i] + [1.0])
            if gap > 1e-4:
                assert np.max(np.abs(g[:, i] - r["Phis"][a][:, i])) < 1e-6, (a, i)
    ctx.assemble("fp64")
    lo, hi = O.window_bounds(r["E"], wl.window)
    want = r["E"][(r["E"] >= lo - 1e-7) & (r["E"] <= hi + 1e-7)]
    got, n = ctx.window_eigs(lo - 1e-7, hi + 1e-7)
    assert n == len(want)
    assert np.max(np.abs(got - want)) < 1e-6


def _oracle_fragment(args):
    name, a = args
    wl = make_workload(name)
    H = O.hamiltonian(wl.grid, wl.V)
    return O.fragment_eigs(H, wl.grid, wl.frags[a])


def test_alkane_fp32_fragment_energies_sampled(ofm):
    """Full-size alkane workload (31 fragments, 16384 points, 32 states) in
    FP32: energies of sampled fragments vs the oracle's shift-invert
    Lanczos (1e-5 Ha), residuals below tolerance."""
    wl = make_workload("alkane")
    ctx = ofm.Context()
    ctx.build_fragments(wl.grid, wl.V, wl.frags, storage="fp32")
    eps, res, _ = ctx.fragment_eigs()
    assert res.max() <= 1e-5
    sample = [0, 15, 30]
    with mp.get_context("spawn").Pool(len(sample)) as pool:
        outs = pool.map(_oracle_fragment, [("alkane", a) for a in sample])
    for a, (e, _) in zip(sample, outs):
        got = eps[32 * a:32 * (a + 1)]
        assert np.max(np.abs(got - e)) < 1e-5, (a, np.max(np.abs(got - e)))
