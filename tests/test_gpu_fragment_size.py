"""Fragment-size study (the paper's monomer / dimer / trimer comparison, Sec.
III "Choice of fragments", as a synthetic analogue): fragments of 1, 2 and 3
consecutive wells of the tiny workload, whole method on the GPU in FP64.
The lowest levels match the oracle's run of the same method, lie above the
full-grid diagonalisation (the pencil is a Rayleigh-Ritz problem in the span
of the fragment states), and approach it as the fragments grow."""
import numpy as np
import pytest

from ofm_inputs import Fragment, tiny_fragments_of
from oracle import ofm_oracle as O

from gpu_util import gpu_lib

pytestmark = pytest.mark.gpu
N_BOUND = 5   # levels below zero: one per well band that stays bound


@pytest.fixture(scope="module")
def ofm():
    return gpu_lib()


def _gpu_levels(ofm, wl, k):
    ctx = ofm.Context()
    ctx.build_fragments(wl.grid, wl.V, wl.frags, storage="fp64")
    ctx.fragment_eigs()
    ctx.assemble("fp64")
    return ctx.eigs_by_index(0, k)


def test_fragment_size_study(ofm):
    base = tiny_fragments_of(1)
    H = O.hamiltonian(base.grid, base.V)
    full, _ = O.fragment_eigs(H, base.grid, Fragment((0, 0, 0), tuple(base.grid.n), 8))
    errs = []
    for s in (1, 2, 3):
        wl = tiny_fragments_of(s)
        got = _gpu_levels(ofm, wl, 8)
        want = O.run_ofm(wl)["E"][:8]
        assert np.max(np.abs(got - want)) < 1e-7, s
        assert np.all(got >= full - 1e-9), s
        errs.append(got[:N_BOUND] - full[:N_BOUND])
    assert np.all(errs[1] < errs[0]) and np.all(errs[2] < errs[1])
    assert np.max(errs[2]) < 1e-3


def test_whole_grid_fragment_is_the_full_diagonalisation(ofm):
    """One fragment spanning the grid: its eigensolve is the full-grid
    diagonalisation the study compares against."""
    base = tiny_fragments_of(1)
    H = O.hamiltonian(base.grid, base.V)
    whole = Fragment((0, 0, 0), tuple(base.grid.n), 8)
    full, _ = O.fragment_eigs(H, base.grid, whole)
    ctx = ofm.Context()
    ctx.build_fragments(base.grid, base.V, [whole], storage="fp64")
    eps, res, _ = ctx.fragment_eigs()
    assert np.max(np.abs(eps - full)) < 1e-9
