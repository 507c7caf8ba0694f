"""Failure detection without any GPU fault or hang.

- The eigensolver's iteration cap: OFM_ERR_NOT_CONVERGED with every output
  filled (the best states found stay usable).
- Bounded device waits made to run out on purpose (ofm_test_hold_wait: the
  producer withholds what the wait is for -- a flag that nothing sets): the
  region contraction's tensor-core wait and the tridiagonal reduction's grid
  barrier; the call reports OFM_ERR_TIMEOUT and the next call of the same
  context gives the right answer.
- Host-side injection (OFM_FAULT, read when a context is created), which
  never touches the device: oom, timeout, nonconv, notposdef.
"""
import numpy as np
import pytest

from ofm_inputs import make_workload, random_states
from oracle import ofm_oracle as O

from gpu_util import gpu_lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ofm():
    return gpu_lib()


def test_iteration_cap_reports_not_converged(ofm):
    wl = make_workload("tiny")
    ctx = ofm.Context()
    ctx.build_fragments(wl.grid, wl.V, wl.frags, storage="fp64")
    eps, res, st = ctx.fragment_eigs(max_iter=1, allow_not_converged=True)
    assert st == ofm.OFM_ERR_NOT_CONVERGED
    assert np.all(np.isfinite(eps)) and np.all(np.isfinite(res)) and res.max() > 1e-9
    with pytest.raises(ofm.OFMError) as e:
        ctx.fragment_eigs(max_iter=1)
    assert e.value.status == ofm.OFM_ERR_NOT_CONVERGED
    # the capped states are a usable basis; a full solve then converges
    ctx.assemble("fp64")
    eps2, res2, st2 = ctx.fragment_eigs()
    assert st2 == ofm.OFM_OK and res2.max() <= 1e-9
    ref = O.run_ofm(wl)
    assert np.max(np.abs(eps2 - np.concatenate(ref["eps"]))) < 1e-9


def _fp32_states(wl):
    return [random_states(wl.grid, f, seed=70 + a).astype(np.float32).astype(np.float64)
            for a, f in enumerate(wl.frags)]


def test_region_contraction_wait_runs_out(ofm):
    wl = make_workload("alkane")
    Phis = _fp32_states(wl)
    ctx = ofm.Context()
    ctx.build_fragments(wl.grid, wl.V, wl.frags, storage="fp32")
    for a, P in enumerate(Phis):
        ctx.set_fragment_states(a, P)
    ctx.assemble("bf16x3", schedule="region")
    want = ctx.block(0, 1)
    ctx.test_hold_wait("contract", bound=1 << 12)
    ctx.assemble("bf16x3", schedule="region")
    with pytest.raises(ofm.OFMError) as e:
        ctx.block(0, 1)
    assert e.value.status == ofm.OFM_ERR_TIMEOUT
    # the context is still usable: the same blocks, bit for bit
    ctx.assemble("bf16x3", schedule="region")
    got = ctx.block(0, 1)
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
    H = O.hamiltonian(wl.grid, wl.V)
    Hab, Sab = O.pair_block(H, wl.grid, wl.frags[0], Phis[0], wl.frags[1], Phis[1])
    assert np.max(np.abs(got[1] - Sab)) < 1e-4 and np.max(np.abs(got[0] - Hab)) < 1e-3


@pytest.mark.parametrize("n", [300, 2000])
def test_tridiagonal_barrier_wait_runs_out(ofm, n):
    """n = 300 takes the shared-memory reduction, n = 2000 the persistent one."""
    rng = np.random.default_rng(n)
    X = rng.standard_normal((n, n))
    S = X @ X.T / n + 0.2 * np.eye(n)
    Y = rng.standard_normal((n, n)) / np.sqrt(n)
    Hm = 0.5 * (Y + Y.T)
    E = O.generalized_eigs(Hm, S)
    ctx = ofm.Context()
    ctx.set_dense_HS(Hm, S)
    ctx.test_hold_wait("tridiag", bound=1 << 14)
    with pytest.raises(ofm.OFMError) as e:
        ctx.eigs_by_index(0, 5)
    assert e.value.status == ofm.OFM_ERR_TIMEOUT
    got = ctx.eigs_by_index(0, n)
    assert np.max(np.abs(got - E)) < 1e-9 * max(1.0, np.abs(E).max())


@pytest.mark.parametrize("kind", ["oom", "timeout", "nonconv", "notposdef"])
def test_host_side_injection(ofm, kind, monkeypatch):
    wl = make_workload("tiny")
    monkeypatch.setenv("OFM_FAULT", kind)
    ctx = ofm.Context()
    monkeypatch.delenv("OFM_FAULT")
    if kind == "oom":
        with pytest.raises(ofm.OFMError) as e:
            ctx.build_fragments(wl.grid, wl.V, wl.frags, storage="fp64")
        assert e.value.status == ofm.OFM_ERR_OOM and "injected" in str(e.value)
        return
    ctx.build_fragments(wl.grid, wl.V, wl.frags, storage="fp64")
    if kind == "nonconv":
        eps, res, st = ctx.fragment_eigs(allow_not_converged=True)
        assert st == ofm.OFM_ERR_NOT_CONVERGED
        assert np.all(np.isfinite(eps)) and res.max() <= 1e-9   # the solve itself converged
        return
    ctx.fragment_eigs()
    ctx.assemble("fp64")
    if kind == "timeout":
        with pytest.raises(ofm.OFMError) as e:
            ctx.block(0, 1)
        assert e.value.status == ofm.OFM_ERR_TIMEOUT and "injected" in str(e.value)
        ctx.block(0, 1)   # reported once per launch
        return
    with pytest.raises(ofm.OFMError) as e:
        ctx.eigs_by_index(0, 3)
    assert e.value.status == ofm.OFM_ERR_NOT_POSDEF and "injected" in str(e.value)
    # a context created without the variable is unaffected
    clean = ofm.Context()
    clean.build_fragments(wl.grid, wl.V, wl.frags, storage="fp64")
    clean.fragment_eigs()
    clean.assemble("fp64")
    assert len(clean.eigs_by_index(0, 3)) == 3
