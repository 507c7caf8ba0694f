"""Pins that tie the FP64 oracle to what the mathematics fixes, independently
of the oracle's own code: closed forms, identities, invariants and brute
force.  Each test names the part of the oracle it would catch if wrong."""
import itertools
import math

import numpy as np
import pytest

from ofm_inputs import Fragment, Grid, make_workload, small_workload
from oracle import ofm_oracle as O


def periodic_1d(n, h):
    # eigenvalues of -1/2 d^2 (3-point, periodic, n points)
    return np.array([(1.0 - math.cos(2.0 * math.pi * k / n)) / h ** 2 for k in range(n)])


def dirichlet_1d(n, h):
    # eigenvalues of -1/2 d^2 (3-point, zero outside n points)
    return np.array([(1.0 - math.cos(k * math.pi / (n + 1))) / h ** 2 for k in range(1, n + 1)])


def sums(*lists):
    return np.sort(np.array([sum(t) for t in itertools.product(*lists)]))


# --- step 1: the grid operator ----------------------------------------------

def test_free_particle_spectrum_periodic_grid():
    grid = Grid((6, 5, 4), 0.7)
    H = O.hamiltonian(grid, np.zeros(grid.n[::-1])).toarray()
    assert np.allclose(H, H.T)
    got = np.linalg.eigvalsh(H)
    want = sums(periodic_1d(6, 0.7), periodic_1d(5, 0.7), periodic_1d(4, 0.7))
    assert np.max(np.abs(got - want)) < 1e-12


def test_constant_potential_shifts_spectrum():
    grid = Grid((4, 3, 5), 0.5)
    c = -0.731
    H0 = O.hamiltonian(grid, np.zeros(grid.n[::-1])).toarray()
    H1 = O.hamiltonian(grid, np.full(grid.n[::-1], c)).toarray()
    assert np.max(np.abs(np.linalg.eigvalsh(H1) - np.linalg.eigvalsh(H0) - c)) < 1e-12


def test_potential_sits_on_the_right_grid_point():
    # a potential that is non-zero at one point only: the diagonal entry at
    # that point's linear index (x fastest) carries it
    grid = Grid((5, 4, 3), 0.5)
    V = np.zeros(grid.n[::-1])
    V[2, 1, 3] = -2.5
    H = O.hamiltonian(grid, V)
    lin = 2 * 4 * 5 + 1 * 5 + 3
    assert abs(H[lin, lin] - (3.0 / 0.25 - 2.5)) < 1e-14
    assert abs(H[0, 0] - 3.0 / 0.25) < 1e-14


# --- step 2: fragment eigensolve --------------------------------------------

def test_free_particle_fragment_mixed_boundaries():
    # Dirichlet in x and z (z box wraps through the periodic boundary),
    # periodic in y where the box spans the whole grid
    grid = Grid((12, 6, 10), 0.5)
    H = O.hamiltonian(grid, np.zeros(grid.n[::-1]))
    frag = Fragment((3, 0, 7), (5, 6, 6), 9)
    eps, Phi = O.fragment_eigs(H, grid, frag)
    want = sums(dirichlet_1d(5, 0.5), periodic_1d(6, 0.5), dirichlet_1d(6, 0.5))[:9]
    assert np.max(np.abs(eps - want)) < 1e-12
    assert np.max(np.abs(Phi.T @ Phi - np.eye(9))) < 1e-12


def test_fragment_sparse_path_matches_closed_form(monkeypatch):
    monkeypatch.setattr(O, "DENSE_EIGH_MAX", 100)
    grid = Grid((16, 8, 8), 0.5)
    H = O.hamiltonian(grid, np.zeros(grid.n[::-1]))
    frag = Fragment((14, 2, 0), (7, 5, 8), 6)
    eps, Phi = O.fragment_eigs(H, grid, frag)
    want = sums(dirichlet_1d(7, 0.5), dirichlet_1d(5, 0.5), periodic_1d(8, 0.5))[:6]
    # the first levels are degenerate; compare eigenvalues only
    assert np.max(np.abs(eps - want)) < 1e-10


def test_gauge_largest_component_positive():
    wl = small_workload(seed=3)
    H = O.hamiltonian(wl.grid, wl.V)
    _, Phi = O.fragment_eigs(H, wl.grid, wl.frags[0])
    for c in range(Phi.shape[1]):
        i = np.argmax(np.abs(Phi[:, c]))
        assert Phi[i, c] > 0


# --- step 3: H phi ----------------------------------------------------------

def test_apply_plane_wave_full_span():
    grid = Grid((8, 6, 5), 0.5)
    c = -0.4
    H = O.hamiltonian(grid, np.full(grid.n[::-1], c))
    frag = Fragment((0, 0, 0), grid.n, 1)
    k = (2, 1, 3)
    zz, yy, xx = np.meshgrid(np.arange(5), np.arange(6), np.arange(8), indexing="ij")
    ph = 2 * math.pi * (k[0] * xx / 8 + k[1] * yy / 6 + k[2] * zz / 5) + 0.3
    phi = np.cos(ph).ravel()[:, None]
    Ek = sum((1 - math.cos(2 * math.pi * k[d] / grid.n[d])) / 0.25 for d in range(3)) + c
    Hphi = O.apply_h(H, grid, frag, phi)
    assert Hphi.shape == phi.shape
    assert np.max(np.abs(Hphi - Ek * phi)) < 1e-12


def test_apply_is_zero_beyond_the_dilated_box():
    wl = small_workload(grid_n=(14, 9, 7), seed=1)
    H = O.hamiltonian(wl.grid, wl.V)
    f = Fragment((11, 2, 1), (6, 4, 5), 3)       # wraps in x, Dirichlet everywhere
    Phi = np.random.default_rng(0).standard_normal((6 * 4 * 5, 3))
    full = (H @ O.zero_extend(wl.grid, f, Phi)).toarray()
    doff, dext = O.dilated_box(wl.grid, f)
    inside = np.zeros(wl.grid.npoints, bool)
    inside[O.box_indices(wl.grid, doff, dext)] = True
    assert np.all(full[~inside] == 0.0)


# --- step 4: pair blocks ----------------------------------------------------

def edge_form(grid, V, fa, Pa, fb, Pb):
    """<a|H|b> through the edge form of the kinetic energy:
    (1/2h^2) sum over grid edges (r, r+e_d) of the products of differences,
    plus sum_r V a b.  Written with explicit loops over points and edges."""
    nx, ny, nz = grid.n
    A = np.zeros((nz, ny, nx, Pa.shape[1]))
    B = np.zeros((nz, ny, nx, Pb.shape[1]))
    for (f, P, T) in ((fa, Pa, A), (fb, Pb, B)):
        p = 0
        for z in range(f.ext[2]):
            for y in range(f.ext[1]):
                for x in range(f.ext[0]):
                    T[(f.off[2] + z) % nz, (f.off[1] + y) % ny, (f.off[0] + x) % nx] = P[p]
                    p += 1
    out = np.zeros((Pa.shape[1], Pb.shape[1]))
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                a0, b0 = A[z, y, x], B[z, y, x]
                out += V[z, y, x] * np.outer(a0, b0)
                for (dx, dy, dz) in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
                    a1 = A[(z + dz) % nz, (y + dy) % ny, (x + dx) % nx]
                    b1 = B[(z + dz) % nz, (y + dy) % ny, (x + dx) % nx]
                    out += np.outer(a0 - a1, b0 - b1) / (2 * grid.h ** 2)
    return out


def test_pair_block_edge_form_identity():
    wl = small_workload(grid_n=(10, 6, 5), seed=2)
    rng = np.random.default_rng(7)
    fa = Fragment((7, 0, 1), (6, 6, 3), 3)     # wraps in x, full span in y
    fb = Fragment((1, 2, 0), (5, 3, 5), 4)     # full span in z
    Pa = rng.standard_normal((6 * 6 * 3, 3))
    Pb = rng.standard_normal((5 * 3 * 5, 4))
    H = O.hamiltonian(wl.grid, wl.V)
    Hab, Sab = O.pair_block(H, wl.grid, fa, Pa, fb, Pb)
    want = edge_form(wl.grid, wl.V, fa, Pa, fb, Pb)
    assert np.max(np.abs(Hab - want)) < 1e-11 * max(1.0, np.abs(want).max())


def test_apply_on_the_dilated_box_through_the_edge_form():
    """<a|H phi_b> summed over the points of b's box grown by one point
    (positions enumerated here, x fastest) equals the edge form."""
    wl = small_workload(grid_n=(12, 7, 6), seed=5)
    g = wl.grid
    rng = np.random.default_rng(9)
    fb = Fragment((9, 2, 0), (5, 3, 6), 3)      # wraps in x; full span in z
    fa = Fragment((0, 0, 0), g.n, 2)            # whole grid
    Pb = rng.standard_normal((5 * 3 * 6, 3))
    Pa = rng.standard_normal((g.npoints, 2))
    HPb = O.apply_h(O.hamiltonian(g, wl.V), g, fb, Pb)
    nx, ny, nz = g.n
    pts = [((9 - 1 + x) % nx, (2 - 1 + y) % ny, z % nz)
           for z in range(6) for y in range(5) for x in range(7)]
    assert HPb.shape == (len(pts), 3)
    got = np.zeros((2, 3))
    for k, (x, y, z) in enumerate(pts):
        got += np.outer(Pa[z * nx * ny + y * nx + x], HPb[k])
    want = edge_form(g, wl.V, fa, Pa, fb, Pb)
    assert np.max(np.abs(got - want)) < 1e-11 * np.abs(want).max()


def test_pair_block_symmetry_and_halo_only_pairs():
    wl = small_workload(grid_n=(24, 6, 6), seed=4, frags=[
        Fragment((0, 0, 0), (8, 6, 6), 3), Fragment((8, 0, 0), (8, 6, 6), 3),
        Fragment((4, 0, 0), (8, 6, 6), 3)])
    H = O.hamiltonian(wl.grid, wl.V)
    rng = np.random.default_rng(5)
    Ph = [rng.standard_normal((288, 3)) for _ in wl.frags]
    for a, b in itertools.product(range(3), repeat=2):
        Hab, Sab = O.pair_block(H, wl.grid, wl.frags[a], Ph[a], wl.frags[b], Ph[b])
        Hba, Sba = O.pair_block(H, wl.grid, wl.frags[b], Ph[b], wl.frags[a], Ph[a])
        assert np.max(np.abs(Hab - Hba.T)) < 1e-12
        assert np.max(np.abs(Sab - Sba.T)) < 1e-13
    # boxes 0 and 1 only touch: S_01 = 0 but H_01 != 0 through the halo
    H01, S01 = O.pair_block(H, wl.grid, wl.frags[0], Ph[0], wl.frags[1], Ph[1])
    assert np.all(S01 == 0.0)
    assert np.abs(H01).max() > 1e-3
    assert (0, 1) in O.pair_list(wl.grid, wl.frags)


def test_diagonal_blocks_of_eigenstates():
    wl = small_workload(seed=1)
    r = O.run_ofm(wl)
    for a, f in enumerate(wl.frags):
        Haa, Saa = r["blocks"][(a, a)]
        assert np.max(np.abs(Saa - np.eye(f.n_states))) < 1e-12
        assert np.max(np.abs(Haa - np.diag(r["eps"][a]))) < 1e-11


def test_residual_identity_off_diagonal_blocks():
    """For exact fragment eigenstates, H_ab = S_ab diag(eps_b) + halo term,
    the halo term being -1/(2h^2) sum over the points p just outside box b
    of phi_a(p) phi_b(q) for each neighbour q of p inside box b."""
    wl = small_workload(grid_n=(16, 6, 6), seed=6)
    r = O.run_ofm(wl)
    g = wl.grid
    nx, ny, nz = g.n
    for (a, b) in r["pairs"]:
        if a == b:
            continue
        fa, fb = wl.frags[a], wl.frags[b]
        Hab, Sab = r["blocks"][(a, b)]
        ia = {int(i): k for k, i in enumerate(O.box_indices(g, fa.off, fa.ext))}
        ib = {int(i): k for k, i in enumerate(O.box_indices(g, fb.off, fb.ext))}
        halo = np.zeros_like(Hab)
        for p, kp in ia.items():
            if p in ib:
                continue
            x, y, z = p % nx, (p // nx) % ny, p // (nx * ny)
            for dx, dy, dz in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                q = ((z + dz) % nz) * nx * ny + ((y + dy) % ny) * nx + (x + dx) % nx
                if q in ib:
                    halo += np.outer(r["Phis"][a][kp], r["Phis"][b][ib[q]]) * (-0.5 / g.h ** 2)
        want = Sab * r["eps"][b][None, :] + halo
        assert np.max(np.abs(Hab - want)) < 1e-10


# --- step 5: Eq. 2 ----------------------------------------------------------

def test_generalized_two_by_two_closed_form():
    a, b, c, s = -0.7, 0.21, -0.3, 0.35
    Hd = np.array([[a, b], [b, c]])
    Sd = np.array([[1.0, s], [s, 1.0]])
    A, B, C = 1 - s * s, -(a + c - 2 * b * s), a * c - b * b
    disc = math.sqrt(B * B - 4 * A * C)
    want = np.sort([(-B - disc) / (2 * A), (-B + disc) / (2 * A)])
    assert np.max(np.abs(O.generalized_eigs(Hd, Sd) - want)) < 1e-14
    assert np.max(np.abs(O.generalized_eigs_jacobi(Hd, Sd) - want)) < 1e-14


def test_generalized_solver_two_independent_routes():
    rng = np.random.default_rng(11)
    n = 14
    X = rng.standard_normal((n, n))
    Sd = X @ X.T / n + 0.5 * np.eye(n)
    Y = rng.standard_normal((n, n))
    Hd = 0.5 * (Y + Y.T)
    e1 = O.generalized_eigs(Hd, Sd)
    e2 = O.generalized_eigs_jacobi(Hd, Sd)
    assert np.max(np.abs(e1 - e2)) < 1e-11
    assert np.max(np.abs(O.generalized_eigs(Hd, np.eye(n)) - np.linalg.eigvalsh(Hd))) < 1e-12


def test_window_vectors_two_by_two_and_properties():
    """Eq. 2 vectors: for the 2x2 pencil the eigenvector of E solves
    (a - E) c0 + (b - E s) c1 = 0 with c^T S c = 1; for a random pencil the
    vectors satisfy H C = S C diag(E) and C^T S C = I, with the eigenvalues
    of the hand-written Cholesky + Jacobi route."""
    a, b, c, s = -0.7, 0.21, -0.3, 0.35
    Hd = np.array([[a, b], [b, c]])
    Sd = np.array([[1.0, s], [s, 1.0]])
    E, C = O.window_vectors(Hd, Sd, -10.0, 10.0)
    for k in range(2):
        v = np.array([-(b - E[k] * s), a - E[k]])
        v /= math.sqrt(v @ Sd @ v)
        assert min(np.max(np.abs(C[:, k] - v)), np.max(np.abs(C[:, k] + v))) < 1e-13
    rng = np.random.default_rng(12)
    n = 16
    X = rng.standard_normal((n, n))
    Sd = X @ X.T / n + 0.5 * np.eye(n)
    Y = rng.standard_normal((n, n))
    Hd = 0.5 * (Y + Y.T)
    Eall = O.generalized_eigs_jacobi(Hd, Sd)
    lo, hi = Eall[3] - 1e-9, Eall[9] + 1e-9
    E, C = O.window_vectors(Hd, Sd, lo, hi)
    assert len(E) == 7 and np.max(np.abs(E - Eall[3:10])) < 1e-11
    assert np.max(np.abs(Hd @ C - Sd @ C * E)) < 1e-12
    assert np.max(np.abs(C.T @ Sd @ C - np.eye(7))) < 1e-12


def test_jacobi_rejects_indefinite_overlap():
    with pytest.raises(np.linalg.LinAlgError):
        O.generalized_eigs_jacobi(np.eye(2), np.array([[1.0, 2.0], [2.0, 1.0]]))


def test_window_rules():
    from ofm_inputs import WindowRule
    E = np.array([-3.0, -2.0, -1.0, 0.5, 0.6, 2.0])
    assert O.window_bounds(E, WindowRule("from_lowest", 0.5)) == (-3.0, -2.5)
    assert O.window_bounds(E, WindowRule("above_gap", 0.3, n_occ=3)) == (0.5, 0.8)
    lo, hi = O.window_bounds(E, WindowRule("around_gap", 0.2, n_occ=3))
    assert abs(lo + 1.2) < 1e-15 and abs(hi - 0.7) < 1e-15


# --- whole pipeline ---------------------------------------------------------

def test_single_fragment_covering_the_grid_is_exact():
    wl = small_workload(grid_n=(8, 6, 6), seed=2, frags=[Fragment((0, 0, 0), (8, 6, 6), 10)])
    r = O.run_ofm(wl)
    exact = np.linalg.eigvalsh(r["H"].toarray())[:10]
    assert np.max(np.abs(r["E"] - exact)) < 1e-11


def test_variational_bound_and_nested_bases():
    base = small_workload(grid_n=(16, 6, 6), seed=8)
    exact = np.linalg.eigvalsh(O.hamiltonian(base.grid, base.V).toarray())
    prev = None
    for n in (1, 2, 3, 4, 5):
        frags = [Fragment(f.off, f.ext, n) for f in base.frags]
        wl = small_workload(grid_n=(16, 6, 6), seed=8, frags=frags)
        E = O.run_ofm(wl)["E"]
        assert np.all(E >= exact[:len(E)] - 1e-10)
        if prev is not None:
            assert np.all(E[:len(prev)] <= prev + 1e-10)
        prev = E


def test_constant_shift_of_the_whole_method():
    c = 0.37
    w0 = small_workload(grid_n=(16, 6, 6), seed=9)
    w1 = small_workload(grid_n=(16, 6, 6), seed=9, V_shift=c)
    r0, r1 = O.run_ofm(w0), O.run_ofm(w1)
    for a in range(len(w0.frags)):
        assert np.max(np.abs(r1["eps"][a] - r0["eps"][a] - c)) < 1e-11
    for k in r0["blocks"]:
        H0, S0 = r0["blocks"][k]
        H1, S1 = r1["blocks"][k]
        # eigenvectors are unchanged by the shift (gauge fixed), so blocks follow
        assert np.max(np.abs(S1 - S0)) < 1e-9
        assert np.max(np.abs(H1 - H0 - c * S0)) < 1e-9
    assert np.max(np.abs(r1["E"] - r0["E"] - c)) < 1e-10


# --- geometry ---------------------------------------------------------------

def test_pair_list_of_the_tiny_and_alkane_workloads():
    tiny = make_workload("tiny")
    pairs = O.pair_list(tiny.grid, tiny.frags)
    assert len(pairs) == 10            # every pair meets on the 32-point ring
    alk = make_workload("alkane")
    pairs = O.pair_list(alk.grid, alk.frags)
    assert len(pairs) == 91
    kinds = {"self": 0, "overlap": 0, "halo": 0}
    for a, b in pairs:
        fa, fb = alk.frags[a], alk.frags[b]
        if a == b:
            kinds["self"] += 1
        elif O.overlap_points(alk.grid, fa.off, fa.ext, fb.off, fb.ext) > 0:
            kinds["overlap"] += 1
        else:
            kinds["halo"] += 1
    assert kinds == {"self": 31, "overlap": 30, "halo": 30}


def test_overlap_counts_by_brute_force():
    grid = Grid((10, 7, 6), 0.5)
    rng = np.random.default_rng(3)
    for _ in range(40):
        offa = tuple(int(rng.integers(0, n)) for n in grid.n)
        offb = tuple(int(rng.integers(0, n)) for n in grid.n)
        exta = tuple(int(rng.integers(1, n + 1)) for n in grid.n)
        extb = tuple(int(rng.integers(1, n + 1)) for n in grid.n)
        ia = set(O.box_indices(grid, offa, exta).tolist())
        ib = set(O.box_indices(grid, offb, extb).tolist())
        assert O.overlap_points(grid, offa, exta, offb, extb) == len(ia & ib)
        assert O.boxes_meet(grid, offa, exta, offb, extb) == bool(ia & ib)


def test_pair_flops_of_the_alkane_workload():
    alk = make_workload("alkane")
    pairs = O.pair_list(alk.grid, alk.frags)
    # 31 self pairs (16384 + 16384 points), 30 neighbours (8192 + 9216),
    # 30 halo-only pairs (0 + 1024); 2 * 32 * 32 flops per point pair
    want = 2 * 32 * 32 * (31 * 32768 + 30 * 17408 + 30 * 1024)
    assert O.pair_flops(alk.grid, alk.frags, pairs) == want


# --- stored oracle output (tests/golden/tiny_oracle.json) --------------------

def test_tiny_workload_matches_stored_oracle_output(repo_root):
    import json
    import os
    g = json.load(open(os.path.join(repo_root, "tests", "golden", "tiny_oracle.json")))
    wl = make_workload("tiny", seed=0)
    r = O.run_ofm(wl)
    assert [list(p) for p in r["pairs"]] == g["pairs"]
    for a in range(4):
        assert np.max(np.abs(r["eps"][a] - np.array(g["fragment_eps"][a]))) < 1e-10
    assert np.max(np.abs(r["E"] - np.array(g["ofm_spectrum"]))) < 1e-9
    # variational bound on the stored numbers themselves
    assert np.all(np.array(g["ofm_spectrum"]) >= np.array(g["exact_lowest"]) - 1e-10)
    assert g["S_min_eig"] > 0


def _stored_spectrum_matches(repo_root, key):
    """The stored FP64 oracle runs (tests/golden/{alkane,polymer}_oracle.json)
    belong to the workload the generator makes today: one entry per basis
    function, fragment energies in ascending order per fragment, and the
    smallest fragment's energies recomputed by the oracle now."""
    import json
    import os
    g = json.load(open(os.path.join(repo_root, "tests", "golden", f"{key}_oracle.json")))
    wl = make_workload(key, seed=0)
    assert g["workload"] == wl.name
    assert len(g["ofm_spectrum"]) == sum(f.n_states for f in wl.frags)
    assert [len(e) for e in g["fragment_eps"]] == [f.n_states for f in wl.frags]
    assert all(np.all(np.diff(e) >= 0) for e in g["fragment_eps"])
    assert np.all(np.diff(g["ofm_spectrum"]) >= 0) and g["S_min_eig"] > 0
    a = min(range(len(wl.frags)), key=lambda i: (np.prod(wl.frags[i].ext), wl.frags[i].n_states))
    H = O.hamiltonian(wl.grid, wl.V)
    eps, _ = O.fragment_eigs(H, wl.grid, wl.frags[a])
    assert np.max(np.abs(eps - np.array(g["fragment_eps"][a]))) < 1e-9


def test_stored_alkane_spectrum_matches(repo_root):
    _stored_spectrum_matches(repo_root, "alkane")


def test_stored_polymer_spectrum_matches(repo_root):
    _stored_spectrum_matches(repo_root, "polymer")


# ------------------------------------------------ Sec. III.C distance cutoff --

def test_fragment_distance_minimum_image_and_empty():
    """Two atoms 0.3 bohr apart across the periodic edge of a 5 bohr box (not
    4.7 apart), the smallest pair wins, and a fragment without atoms is
    infinitely far from every other."""
    grid = Grid((10, 10, 10), 0.5)
    a = np.array([[0.2, 1.0, 1.0], [2.5, 2.5, 2.5]])
    b = np.array([[4.9, 1.0, 1.0]])
    assert abs(O.fragment_distance(grid, a, b) - 0.3) < 1e-12
    c = np.array([[2.5, 2.5, 4.5]])              # 2.0 from a[1] along z
    assert abs(O.fragment_distance(grid, a, c) - 2.0) < 1e-12
    assert O.fragment_distance(grid, a, np.zeros((0, 3))) == math.inf


def test_cutoff_pairs_limits():
    """A cutoff above every distance keeps the geometric list; one below
    every distance keeps the self pairs only; in between, exactly the pairs
    closer than the cutoff stay (a ring of four boxes, fragment 2's atom
    moved so that its two neighbours sit 3.5 and 2.5 bohr away)."""
    grid = Grid((24, 8, 8), 0.5)
    frags = [Fragment((6 * a, 0, 0), (8, 8, 8), 2) for a in range(4)]
    atoms = [np.array([[(6 * a + 4) * 0.5, 2.0, 2.0]]) for a in range(4)]   # 3 bohr apart
    atoms[2] = atoms[2] + np.array([[0.5, 0.0, 0.0]])
    full = O.pair_list(grid, frags)
    assert full == [(0, 0), (0, 1), (0, 3), (1, 1), (1, 2), (2, 2), (2, 3), (3, 3)]
    assert O.cutoff_pairs(grid, frags, atoms, 1e9) == full
    assert O.cutoff_pairs(grid, frags, atoms, 2.0) == [(a, a) for a in range(4)]
    assert O.cutoff_pairs(grid, frags, atoms, 3.2) == [(0, 0), (0, 1), (0, 3), (1, 1), (2, 2),
                                                       (2, 3), (3, 3)]


def test_self_pairs_only_give_the_fragment_spectra():
    """With exact fragment eigenstates S_aa = I and H_aa = diag(eps_a), so a
    pencil assembled from the self pairs alone has exactly the union of the
    fragment energies as its spectrum."""
    wl = make_workload("tiny")
    H = O.hamiltonian(wl.grid, wl.V)
    eps, Phis = zip(*[O.fragment_eigs(H, wl.grid, f) for f in wl.frags])
    selfs = [(a, a) for a in range(len(wl.frags))]
    Hd, Sd = O.assemble_dense(wl.frags, O.pair_blocks(H, wl.grid, wl.frags, list(Phis), selfs))
    E = O.generalized_eigs(Hd, Sd)
    assert np.max(np.abs(E - np.sort(np.concatenate(eps)))) < 1e-10


# ------------------------------------- Sec. III basis selection and occupation --

def test_first_gap_by_hand():
    """Spectrum 0, .1, .2 | .9, 1.0 | 2.0 with gap_min 0.5: the first wide
    spacing at or above the reference is (0.2, 0.9) whether the reference
    sits below the spectrum, inside the cluster or inside that gap; a
    smaller gap_min finds the first spacing that exceeds it."""
    E = [1.0, 0.0, 2.0, 0.1, 0.9, 0.2]
    for e_ref in (-1.0, 0.15, 0.5):
        assert O.first_gap(E, e_ref, 0.5) == (0.2, 0.9, 3)
    assert O.first_gap(E, 0.95, 0.5) == (1.0, 2.0, 5)
    assert O.first_gap(E, 0.0, 0.09) == (0.0, 0.1, 1)
    with pytest.raises(ValueError):
        O.first_gap(E, 0.0, 5.0)


def test_homo_expectation_is_the_fragment_energy():
    """phi_HOMO vanishes outside its box, so <phi|H|phi> with the
    whole-system H equals the quadratic form of the box's principal
    submatrix: the fragment's HOMO energy, for exact eigenstates."""
    wl = make_workload("tiny")
    H = O.hamiltonian(wl.grid, wl.V)
    eps, Phis = zip(*[O.fragment_eigs(H, wl.grid, f) for f in wl.frags])
    e = O.homo_expectations(H, wl.grid, wl.frags, list(Phis))
    assert np.max(np.abs(np.array(e) - np.array([w[-1] for w in eps]))) < 1e-12
    top2 = [P[:, -2:] for P in Phis]
    e2 = O.homo_expectations(H, wl.grid, wl.frags, top2)
    assert e2 == e
