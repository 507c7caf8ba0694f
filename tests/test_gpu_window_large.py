"""Eq. 2 at the sizes the workloads reach, against LAPACK through the oracle.

Seeded random pencils (H symmetric, S symmetric positive definite with a
condition number of a few hundred, like the chain pencils where overlapping
fragments give lambda_min(S) ~ 0.01) at n = 992 (the alkane chain's basis;
shared-memory Householder reduction, multisection from shared memory),
n = 2500 (persistent reduction from global memory) and n = 8700 (beyond the
shared-memory multisection: bisection from global memory).  Every
eigenvalue, the count of a window, and an index-anchored window are checked.

Tolerance: the Cholesky-based reduction is backward stable, so each
eigenvalue moves by at most about c n u ||H|| ||S^-1|| (u = 2^-53); the tests
take c = 64."""
import numpy as np
import pytest

from oracle import ofm_oracle as O

from gpu_util import U64, gpu_lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ofm():
    return gpu_lib()


@pytest.mark.parametrize("n", [992, 2500, 8700])
def test_window_solver_large_random_pencils(ofm, n):
    rng = np.random.default_rng(1000 + n)
    X = rng.standard_normal((n, n))
    S = X @ X.T / n + 0.01 * np.eye(n)
    Y = rng.standard_normal((n, n)) / np.sqrt(n)
    Hm = 0.5 * (Y + Y.T)
    E = O.generalized_eigs(Hm, S)
    s_min = np.linalg.eigvalsh(S)[0]
    tol = 64 * n * U64 * np.linalg.norm(Hm, 2) / s_min
    ctx = ofm.Context()
    ctx.set_dense_HS(Hm, S)
    got = ctx.eigs_by_index(0, n)
    assert np.max(np.abs(got - E)) < tol, (n, float(np.max(np.abs(got - E))), tol)
    # a window in the middle of the spectrum: count and values
    lo, hi = E[n // 3] - 1e-7, E[n // 2] + 1e-7
    w, cnt = ctx.window_eigs(lo, hi, max_out=n)
    want = E[(E >= lo) & (E <= hi)]
    assert cnt == len(want)
    assert np.max(np.abs(w - want)) < tol
    # anchored at an index, as the benchmark's window above the gap
    i0 = n // 4
    width = float(E[i0 + 50] - E[i0]) + 1e-9
    w2, k = ctx.window_from_index(i0, width, max_out=n)
    ref = E[i0:][E[i0:] <= E[i0] + width + 1e-12]
    assert abs(k - len(ref)) <= 1 and k >= 50
    m = min(k, len(ref))
    assert np.max(np.abs(w2[:m] - ref[:m])) < tol
    ctx.close()
