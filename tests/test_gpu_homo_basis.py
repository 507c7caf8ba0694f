"""Basis of selected fragment states (Sec. III, "Choice of the number of basis
states per fragment") and the occupation rule for a HOMO basis: the GPU
pencil of the selected states matches the oracle's, the distance cutoff
survives a selection, the rule finds the oracle's gap, and a later
fragment eigensolve computes the selected number of states."""
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
    return wl, H, list(eps), list(Phis)


def _ctx(ofm, wl, Phis):
    ctx = ofm.Context()
    ctx.build_fragments(wl.grid, wl.V, wl.frags, storage="fp64")
    for a, P in enumerate(Phis):
        ctx.set_fragment_states(a, P)
    return ctx


def _oracle_pencil(wl, H, Phis, pairs):
    blocks = O.pair_blocks(H, wl.grid, wl.frags, Phis, pairs)
    frags = [type(f)(f.off, f.ext, P.shape[1]) for f, P in zip(wl.frags, Phis)]
    return blocks, O.assemble_dense(frags, blocks)


@pytest.mark.parametrize("first,count", [(4, 2), (0, 6), (5, 1)])
def test_selected_states_pencil(ofm, tiny, first, count):
    wl, H, eps, Phis = tiny
    ctx = _ctx(ofm, wl, Phis)
    ctx.select_states(first, count)
    sel = [P[:, first:first + count] for P in Phis]
    for a in range(len(wl.frags)):
        assert np.array_equal(ctx.get_fragment_states(a), sel[a])
    pairs = O.pair_list(wl.grid, wl.frags)
    assert ctx.pairs() == pairs
    ctx.assemble("fp64")
    blocks, (Hd, Sd) = _oracle_pencil(wl, H, sel, pairs)
    for (a, b), (Hab, Sab) in blocks.items():
        Hg, Sg = ctx.block(a, b)
        assert Hg.shape == (count, count)
        assert np.max(np.abs(Sg - Sab)) < 1e-12, (a, b)
        assert np.max(np.abs(Hg - Hab)) < 1e-11 * max(1.0, np.abs(Hab).max()), (a, b)
    E = O.generalized_eigs(Hd, Sd)
    got = ctx.eigs_by_index(0, len(E))
    assert np.max(np.abs(got - E)) < 1e-9


def test_homo_lumo_rule_matches_oracle(ofm, tiny):
    """Basis of the top two states of each fragment; the rule's reference
    energy is the largest fragment HOMO energy and its gap the oracle's."""
    wl, H, eps, Phis = tiny
    ctx = _ctx(ofm, wl, Phis)
    ctx.select_states(4, 2)
    ctx.assemble("fp64")
    sel = [P[:, 4:6] for P in Phis]
    _, (Hd, Sd) = _oracle_pencil(wl, H, sel, O.pair_list(wl.grid, wl.frags))
    E = O.generalized_eigs(Hd, Sd)
    e_ref = max(O.homo_expectations(H, wl.grid, wl.frags, sel))
    assert abs(e_ref - max(w[-1] for w in eps)) < 1e-10
    k0 = max(int(np.sum(E <= e_ref)) - 1, 0)
    gap_min = 0.5 * float(np.max(np.diff(E[k0:])))   # a spacing at or above e_ref
    want = O.first_gap(E, e_ref, gap_min)
    got = ctx.homo_lumo_gap(gap_min)
    assert abs(got[0] - e_ref) < 1e-10
    assert abs(got[1] - want[0]) < 1e-9 and abs(got[2] - want[1]) < 1e-9
    assert got[3] == want[2]
    with pytest.raises(ofm.OFMError):
        ctx.homo_lumo_gap(1e6)


def test_selection_keeps_cutoff_and_errors(ofm, tiny):
    wl, H, eps, Phis = tiny
    ctx = _ctx(ofm, wl, Phis)
    atoms = wl.fragment_atoms()
    ctx.set_pair_cutoff(atoms, 1.0)
    cut = O.cutoff_pairs(wl.grid, wl.frags, atoms, 1.0)
    ctx.select_states(3, 3)
    assert ctx.pairs() == cut
    with pytest.raises(ofm.OFMError):
        ctx.select_states(2, 2)          # [2, 4) is outside the 3 states now held
    fresh = ofm.Context()
    with pytest.raises(ofm.OFMError):
        fresh.select_states([0], [1])


def test_eigensolve_after_selection(ofm, tiny):
    """The eigensolver's workspace follows the new state counts: a later
    ofm_fragment_eigs returns the lowest count states of every fragment."""
    wl, H, eps, Phis = tiny
    ctx = _ctx(ofm, wl, Phis)
    ctx.select_states(0, 3)
    e, res, _ = ctx.fragment_eigs()
    assert len(e) == 3 * len(wl.frags)
    want = np.concatenate([w[:3] for w in eps])
    assert np.max(np.abs(e - want)) < 1e-9
    assert res.max() <= 1e-9
