"""Distance cutoff on the pair list (Sec. III.C): the GPU keeps exactly the
oracle's pairs, the kept blocks match the oracle's, dropped pairs are zero
in the blocks and in the dense pencil, and the window eigenvalues are those
of the oracle's truncated pencil."""
import ctypes as C

import numpy as np
import pytest

from ofm_inputs import make_workload
from oracle import ofm_oracle as O

from gpu_util import gpu_lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ofm():
    return gpu_lib()


@pytest.fixture(scope="module")
def tiny():
    wl = make_workload("tiny")
    H = O.hamiltonian(wl.grid, wl.V)
    eps, Phis = zip(*[O.fragment_eigs(H, wl.grid, f) for f in wl.frags])
    return wl, H, list(Phis)


def _ctx(ofm, wl, Phis):
    ctx = ofm.Context()
    ctx.build_fragments(wl.grid, wl.V, wl.frags, storage="fp64")
    for a, P in enumerate(Phis):
        ctx.set_fragment_states(a, P)
    return ctx


@pytest.mark.parametrize("d_cut", [1.0, 0.5])
def test_cutoff_pairs_blocks_and_window(ofm, tiny, d_cut):
    wl, H, Phis = tiny
    atoms = wl.fragment_atoms()
    want = O.cutoff_pairs(wl.grid, wl.frags, atoms, d_cut)
    full = O.pair_list(wl.grid, wl.frags)
    assert len(want) < len(full)
    ctx = _ctx(ofm, wl, Phis)
    ctx.set_pair_cutoff(atoms, d_cut)
    assert ctx.pairs() == want
    ctx.assemble("fp64")
    blocks = O.pair_blocks(H, wl.grid, wl.frags, Phis, want)
    for (a, b), (Hab, Sab) in blocks.items():
        Hg, Sg = ctx.block(a, b)
        assert np.max(np.abs(Sg - Sab)) < 1e-12 * max(1.0, np.abs(Sab).max()), (a, b)
        assert np.max(np.abs(Hg - Hab)) < 1e-11 * max(1.0, np.abs(Hab).max()), (a, b)
    for (a, b) in set(full) - set(want):
        Hg, Sg = ctx.block(a, b)
        assert not Hg.any() and not Sg.any(), (a, b)
    Hd, Sd = O.assemble_dense(wl.frags, blocks)
    Hg, Sg = ctx.dense_HS()
    assert np.max(np.abs(Hg - Hd)) < 1e-11 * np.abs(Hd).max()
    assert np.max(np.abs(Sg - Sd)) < 1e-12 * max(1.0, np.abs(Sd).max())
    E = O.generalized_eigs(Hd, Sd)
    lo, hi = E[0] - 1e-7, E[0] + 0.5
    got, n = ctx.window_eigs(lo, hi)
    ref = O.window_eigs(Hd, Sd, lo, hi)
    assert n == len(ref)
    assert np.max(np.abs(got - ref)) < 1e-9


def test_cutoff_cleared_and_self_pairs(ofm, tiny):
    """A cutoff below every atom distance leaves the self pairs (the spectrum
    is then the union of the fragment energies); clearing it restores the
    geometric list."""
    wl, H, Phis = tiny
    ctx = _ctx(ofm, wl, Phis)
    # one atom per fragment, at least 3 bohr apart (minimum image in 16 bohr)
    far = [np.array([[3.0 * a + 0.1, 0.5, 0.5]]) for a in range(len(wl.frags))]
    ctx.set_pair_cutoff(far, 1.0)
    assert ctx.pairs() == [(a, a) for a in range(len(wl.frags))]
    ctx.assemble("fp64")
    eps = np.sort(np.concatenate([O.fragment_eigs(H, wl.grid, f)[0] for f in wl.frags]))
    got = ctx.eigs_by_index(0, len(eps))
    assert np.max(np.abs(got - eps)) < 1e-9
    ctx.set_pair_cutoff(None, 0.0)
    assert ctx.pairs() == O.pair_list(wl.grid, wl.frags)


def test_cutoff_errors(ofm, tiny):
    wl, H, Phis = tiny
    lib = ofm.load_library()
    fresh = ofm.Context()
    xyz = np.zeros(3)
    off = np.zeros(len(wl.frags) + 1, dtype=np.int32)
    dp = xyz.ctypes.data_as(C.POINTER(C.c_double))
    ip = off.ctypes.data_as(C.POINTER(C.c_int))
    assert lib.ofm_set_pair_cutoff(fresh.h, dp, ip, 1.0) == 7          # OFM_ERR_STATE
    ctx = _ctx(ofm, wl, Phis)
    bad = off.copy()
    bad[0] = 1
    assert lib.ofm_set_pair_cutoff(ctx.h, dp, bad.ctypes.data_as(C.POINTER(C.c_int)), 1.0) == 1
    bad = off.copy()
    bad[2] = 3                                                         # 3 then 0: decreasing
    assert lib.ofm_set_pair_cutoff(ctx.h, dp, bad.ctypes.data_as(C.POINTER(C.c_int)), 1.0) == 1
    assert ctx.pairs() == O.pair_list(wl.grid, wl.frags)               # list untouched
