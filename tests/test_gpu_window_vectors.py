"""GPU window eigenvectors of Eq. 2 (the optional C of ofm_window_eigs):
S-orthonormal, residual-free, and spanning the oracle's eigenspaces."""
import numpy as np
import pytest

from ofm_inputs import make_workload
from oracle import ofm_oracle as O

from gpu_util import gpu_lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ofm():
    return gpu_lib()


def check_pairs(Hd, Sd, E, C, E_o, C_o, tol_res, tol_span):
    """C against the oracle's (E_o, C_o): residual, S-orthonormality, and the
    S-projector onto each eigenspace (degenerate eigenvalues grouped)."""
    m = len(E)
    assert C.shape == (Hd.shape[0], m)
    scale = max(1.0, np.abs(Hd).max())
    assert np.max(np.abs(Hd @ C - Sd @ C * E)) < tol_res * scale
    assert np.max(np.abs(C.T @ Sd @ C - np.eye(m))) < tol_res * 10
    assert np.max(np.abs(E - E_o)) < 1e-9 * scale
    # groups of (numerically) equal eigenvalues
    groups, start = [], 0
    for j in range(1, m + 1):
        if j == m or E_o[j] - E_o[j - 1] > 1e-8 * scale:
            groups.append((start, j))
            start = j
    for a, b in groups:
        P = C[:, a:b] @ C[:, a:b].T @ Sd
        Po = C_o[:, a:b] @ C_o[:, a:b].T @ Sd
        assert np.max(np.abs(P - Po)) < tol_span, (a, b)


def test_tiny_fp64_window_vectors(ofm):
    wl = make_workload("tiny")
    r = O.run_ofm(wl)
    ctx = ofm.Context()
    ctx.build_fragments(wl.grid, wl.V, wl.frags, storage="fp64")
    for a, P in enumerate(r["Phis"]):
        ctx.set_fragment_states(a, P)
    ctx.assemble("fp64")
    lo, hi = O.window_bounds(r["E"], wl.window)
    lo, hi = lo - 1e-7, hi + 1e-7
    E, C, n = ctx.window_eigs(lo, hi, vectors=True)
    assert n == len(E) > 1
    E_o, C_o = O.window_vectors(r["Hd"], r["Sd"], lo, hi)
    check_pairs(r["Hd"], r["Sd"], E, C, E_o, C_o, 1e-10, 1e-8)


def test_degenerate_pencil_takes_the_cluster_path(ofm):
    """Two identical uncoupled blocks: every eigenvalue is double, so each
    pair is one cluster, orthogonalised inside the cluster."""
    rng = np.random.default_rng(4)
    k = 40
    X = rng.standard_normal((k, k))
    S1 = X @ X.T / k + 0.5 * np.eye(k)
    Y = rng.standard_normal((k, k))
    H1 = 0.5 * (Y + Y.T)
    Z = np.zeros((k, k))
    Hd = np.block([[H1, Z], [Z, H1]])
    Sd = np.block([[S1, Z], [Z, S1]])
    ctx = ofm.Context()
    ctx.set_dense_HS(Hd, Sd)
    Eall = O.generalized_eigs(Hd, Sd)
    lo, hi = Eall[10] - 1e-6, Eall[29] + 1e-6
    E, C, n = ctx.window_eigs(lo, hi, max_out=2 * k, vectors=True, n_basis=2 * k)
    assert n == 20
    E_o, C_o = O.window_vectors(Hd, Sd, lo, hi)
    check_pairs(Hd, Sd, E, C, E_o, C_o, 1e-10, 1e-8)


def test_alkane_fp32_window_vectors_residual(ofm):
    """Bench-sized pencil (n = 992) from the whole FP32 pipeline: the vectors
    of the window above the gap solve the device's own dense pencil."""
    wl = make_workload("alkane")
    ctx = ofm.Context()
    ctx.build_fragments(wl.grid, wl.V, wl.frags, storage="fp32")
    ctx.fragment_eigs()
    ctx.assemble("bf16x3")
    Hd, Sd = ctx.dense_HS()
    n = Hd.shape[0]
    n_occ = wl.window.n_occ
    e_gap = ctx.eigs_by_index(n_occ, n_occ + 1)[0]
    lo, hi = e_gap, e_gap + wl.window.width
    E, C, m = ctx.window_eigs(lo, hi, vectors=True, n_basis=n)
    assert m == len(E) > 0
    scale = np.abs(Hd).max()
    assert np.max(np.abs(Hd @ C - Sd @ C * E)) < 1e-9 * scale
    assert np.max(np.abs(C.T @ Sd @ C - np.eye(m))) < 1e-9


def test_window_from_index_matches_two_step_window(ofm):
    """The index-anchored window equals E_i from ofm_eigs_by_index followed by
    ofm_window_eigs on [E_i, E_i + width] (same multisection per index, so
    the same values), for a narrow, a medium and a whole-spectrum width."""
    wl = make_workload("tiny")
    r = O.run_ofm(wl)
    ctx = ofm.Context()
    ctx.build_fragments(wl.grid, wl.V, wl.frags, storage="fp64")
    for a, P in enumerate(r["Phis"]):
        ctx.set_fragment_states(a, P)
    ctx.assemble("fp64")
    n = len(r["E"])
    for i_lo, width in ((3, 0.05), (1, 0.5), (0, 1e3)):
        e0 = ctx.eigs_by_index(i_lo, i_lo + 1)[0]
        want, m = ctx.window_eigs(e0 - 1e-9, e0 + width)
        got, k = ctx.window_from_index(i_lo, width)
        assert k == m and k >= 1
        assert np.array_equal(got, want)
        ref = r["E"][i_lo:][r["E"][i_lo:] <= r["E"][i_lo] + width]
        assert len(ref) == k and np.max(np.abs(got - ref)) < 1e-9
    assert ctx.window_from_index(0, 1e3)[1] == n
    with pytest.raises(ofm.OFMError):
        ctx.window_from_index(n, 0.1)
