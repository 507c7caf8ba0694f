"""The oracle's pins catch plausible mistakes: each case below plants one
mistake in the oracle (on the CPU, through a monkeypatch of one oracle
function) and requires at least one pin of tests/test_oracle_pins.py to
fail.  A pin set that stayed green under a planted mistake would not be
pinning that part of the method."""
import inspect
import os

import numpy as np
import pytest

from oracle import ofm_oracle as O

import test_oracle_pins as PINS

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
# the three slowest pins run last: most mistakes trip a fast one first
SLOW = ("test_homo_expectation_is_the_fragment_energy",
        "test_tiny_workload_matches_stored_oracle_output",
        "test_self_pairs_only_give_the_fragment_spectra",
        "test_stored_alkane_spectrum_matches",
        "test_stored_polymer_spectrum_matches")


def _pins():
    fs = [getattr(PINS, n) for n in sorted(dir(PINS)) if n.startswith("test_")]
    return [f for f in fs if f.__name__ not in SLOW] + [getattr(PINS, n) for n in SLOW]


def _first_failing_pin():
    """Name of the first pin that fails (any exception), or None."""
    for f in _pins():
        mp = pytest.MonkeyPatch()
        try:
            args = []
            for p in inspect.signature(f).parameters:
                args.append(mp if p == "monkeypatch" else ROOT)
            f(*args)
        except Exception:          # an assertion, or an error the mistake causes
            return f.__name__
        finally:
            mp.undo()
    return None


# ------------------------------------------------------- planted mistakes --

def kinetic_weight(mp):
    """-1/h^2 Laplacian instead of -1/(2 h^2) (wrong stencil weight)."""
    orig = O.hamiltonian

    def h(grid, V):
        K = orig(grid, np.zeros(grid.npoints))
        return 2.0 * K + orig(grid, V) - K
    mp.setattr(O, "hamiltonian", h)


def potential_sign(mp):
    """H = T - V."""
    orig = O.hamiltonian
    mp.setattr(O, "hamiltonian", lambda grid, V: orig(grid, -np.asarray(V)))


def apply_on_box_only(mp):
    """H phi kept on the box, the one-point halo dropped."""
    orig = O.apply_h

    def a(H, grid, frag, Phi):
        out = orig(H, grid, frag, Phi)
        _, dext = O.dilated_box(grid, frag)
        keep = []
        for d in range(3):
            m = np.ones(dext[d], dtype=bool)
            if dext[d] != frag.ext[d]:
                m[0] = m[-1] = False
            keep.append(m)
        mask = (keep[2][:, None, None] & keep[1][None, :, None] & keep[0][None, None, :]).ravel()
        return out * mask[:, None]
    mp.setattr(O, "apply_h", a)


def no_dilation(mp):
    """The dilated box taken as the box itself."""
    mp.setattr(O, "dilated_box", lambda grid, frag: (tuple(frag.off), tuple(frag.ext)))


def clamp_not_wrap(mp):
    """Box coordinates clamped at the grid edge instead of wrapped."""
    mp.setattr(O, "box_axes", lambda grid, off, ext: [
        np.clip(off[d] + np.arange(ext[d]), 0, grid.n[d] - 1) for d in range(3)])


def transposed_block(mp):
    """(H_ab, S_ab) returned transposed."""
    orig = O.pair_block

    def pb(H, grid, fa, Pa, fb, Pb):
        Hb, S = orig(H, grid, fa, Pa, fb, Pb)
        return Hb.T.copy(), S.T.copy()
    mp.setattr(O, "pair_block", pb)


def wrong_mirror(mp):
    """The block b > a filled with the block a < b itself, not its transpose."""
    def ad(frags, blocks):
        starts = np.concatenate([[0], np.cumsum([f.n_states for f in frags])])
        n = int(starts[-1])
        Hd, Sd = np.zeros((n, n)), np.zeros((n, n))
        for (a, b), (Hab, Sab) in blocks.items():
            ra, rb = slice(starts[a], starts[a + 1]), slice(starts[b], starts[b + 1])
            Hd[ra, rb], Sd[ra, rb] = Hab, Sab
            if a != b:
                Hd[rb, ra], Sd[rb, ra] = Hab, Sab
        return Hd, Sd
    mp.setattr(O, "assemble_dense", ad)


def window_off_by_one(mp):
    """The window above the gap starting one level too low."""
    orig = O.window_bounds

    def wb(E, rule):
        if rule.kind == "above_gap":
            lo = float(E[rule.n_occ - 1])
            return lo, lo + rule.width
        return orig(E, rule)
    mp.setattr(O, "window_bounds", wb)


def gauge_negative(mp):
    """Sign gauge with the largest component negative."""
    orig = O.gauge_fix
    mp.setattr(O, "gauge_fix", lambda Phi: -orig(Phi))


def gap_scan_from_zero(mp):
    """The occupation rule scanning from the bottom of the spectrum instead
    of from the reference energy."""
    def fg(E, e_ref, gap_min):
        E = np.sort(np.asarray(E, dtype=np.float64))
        for i in range(len(E) - 1):
            if E[i + 1] - E[i] > gap_min:
                return float(E[i]), float(E[i + 1]), i + 1
        raise ValueError("no spacing wider than gap_min")
    mp.setattr(O, "first_gap", fg)


def distance_no_minimum_image(mp):
    """Fragment distance without the periodic minimum image."""
    def fd(grid, atoms_a, atoms_b):
        A = np.asarray(atoms_a, dtype=np.float64).reshape(-1, 3)
        B = np.asarray(atoms_b, dtype=np.float64).reshape(-1, 3)
        if len(A) == 0 or len(B) == 0:
            return float("inf")
        return float(np.min(np.linalg.norm(A[:, None, :] - B[None, :, :], axis=2)))
    mp.setattr(O, "fragment_distance", fd)


MISTAKES = [kinetic_weight, potential_sign, apply_on_box_only, no_dilation, clamp_not_wrap,
            transposed_block, wrong_mirror, window_off_by_one, gauge_negative,
            gap_scan_from_zero, distance_no_minimum_image]


def test_pins_pass_on_the_oracle_as_written():
    assert _first_failing_pin() is None


@pytest.mark.parametrize("plant", MISTAKES, ids=[m.__name__ for m in MISTAKES])
def test_planted_mistake_fails_a_pin(plant, monkeypatch):
    plant(monkeypatch)
    assert _first_failing_pin() is not None, plant.__doc__
