"""Both forms of the stencil kernels (shared-memory staged with bulk copies,
register z-marching) give the oracle's H phi, pair blocks and fragment
eigenstates.  The form is chosen when the context plans its launches;
OFM_STENCIL=staged asks for the staged form wherever its tile fits."""
import numpy as np
import pytest

from ofm_inputs import Fragment, Grid, make_workload, random_states, small_workload
from oracle import ofm_oracle as O

from gpu_util import gpu_lib
from test_gpu_assembly import (GEOMS, abs_overlap, check_fp32_blocks, fp32_states,
                               oracle_with_states, run_gpu)
from test_gpu_eigs import closed_form

pytestmark = pytest.mark.gpu

FORMS = ["staged", "register"]


@pytest.fixture(scope="module")
def ofm():
    return gpu_lib()


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("geom", sorted(GEOMS))
def test_forms_fp64_blocks_and_hphi(ofm, monkeypatch, form, geom):
    monkeypatch.setenv("OFM_STENCIL", form)
    grid, frags = GEOMS[geom]
    wl = small_workload(grid_n=grid.n, h=grid.h, frags=frags, seed=5)
    Phis = [random_states(grid, f, seed=300 + a) for a, f in enumerate(frags)]
    H, pairs, blocks = oracle_with_states(wl, Phis)
    ctx = run_gpu(ofm, wl, Phis, "fp64", "fp64")
    for b, f in enumerate(frags):
        want = O.apply_h(H, grid, f, Phis[b])
        assert np.max(np.abs(ctx.hphi(b) - want)) < 1e-12 * np.abs(want).max(), b
    for (a, b), (Hab, Sab) in blocks.items():
        Hg, Sg = ctx.block(a, b)
        bound_s = 1e-13 * max(1.0, abs_overlap(grid, frags[a], Phis[a], frags[b], Phis[b]).max())
        assert np.max(np.abs(Sg - Sab)) < bound_s, (a, b)
        assert np.max(np.abs(Hg - Hab)) < 1e-12 * max(1.0, np.abs(Hab).max()), (a, b)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("geom", sorted(GEOMS))
def test_forms_fp32_blocks(ofm, monkeypatch, form, geom):
    monkeypatch.setenv("OFM_STENCIL", form)
    grid, frags = GEOMS[geom]
    wl = small_workload(grid_n=grid.n, h=grid.h, frags=frags, seed=5)
    Phis = fp32_states(grid, frags, 400)
    H = O.hamiltonian(wl.grid, wl.V)
    ctx = run_gpu(ofm, wl, Phis, "fp32", "fp32")
    check_fp32_blocks(ctx, wl, Phis, H, O.pair_list(grid, frags), "fp32")


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("storage,tol", [("fp64", 1e-9), ("fp32", 2e-6)])
def test_forms_free_particle_levels(ofm, monkeypatch, form, storage, tol):
    """The fragment eigensolver's filter steps run on the chosen form."""
    monkeypatch.setenv("OFM_STENCIL", form)
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


def test_staged_tiny_fp64_window(ofm, monkeypatch):
    """Whole method on the staged form: window eigenvalues vs the oracle."""
    monkeypatch.setenv("OFM_STENCIL", "staged")
    wl = make_workload("tiny")
    r = O.run_ofm(wl)
    ctx = ofm.Context()
    ctx.build_fragments(wl.grid, wl.V, wl.frags, storage="fp64")
    eps, res, _ = ctx.fragment_eigs()
    assert np.max(np.abs(eps - np.concatenate(r["eps"]))) < 1e-10
    ctx.assemble("fp64")
    lo, hi = O.window_bounds(r["E"], wl.window)
    want = r["E"][(r["E"] >= lo - 1e-7) & (r["E"] <= hi + 1e-7)]
    got, n = ctx.window_eigs(lo - 1e-7, hi + 1e-7)
    assert n == len(want)
    assert np.max(np.abs(got - want)) < 1e-6
