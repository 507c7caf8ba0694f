"""Block-sparse products with the assembled pencil (ofm_pencil_apply): H X and
S X from the pair blocks must equal the dense Eq. 2 matrices times X, for
one and several column tiles with a ragged last one, FP64 and mixed-precision
assemblies, and a distance-cut pair list (dropped blocks are zero)."""
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
def torch():
    import torch
    return torch


@pytest.fixture(scope="module")
def stream(torch):
    # one stream for the context and the tensors it reads and writes (the
    # legacy default stream would leave the context on a stream of its own)
    return torch.cuda.Stream()


def _check(ctx, torch, stream, Hd, Sd, k, seed):
    n = Hd.shape[0]
    rng = np.random.default_rng(seed)
    Xh = rng.standard_normal((k, n))
    with torch.cuda.stream(stream):
        X = torch.from_numpy(Xh).cuda()
        torch.cuda.synchronize()
        for which, M in (("H", Hd), ("S", Sd)):
            Yt = ctx.pencil_apply(which, X)
            torch.cuda.synchronize()
            Y = Yt.cpu().numpy()
            want = Xh @ M.T                  # row c of Y is M x_c
            scale = np.abs(Xh) @ np.abs(M).T + 1e-300
            assert np.max(np.abs(Y - want) / scale) < 1e-13, (which, k)


def test_tiny_fp64_against_the_oracle_pencil(ofm, torch, stream):
    wl = make_workload("tiny")
    r = O.run_ofm(wl)
    ctx = ofm.Context(stream)
    ctx.build_fragments(wl.grid, wl.V, wl.frags, storage="fp64")
    for a, P in enumerate(r["Phis"]):
        ctx.set_fragment_states(a, P)
    ctx.assemble("fp64")
    for k, seed in ((1, 0), (5, 1), (33, 2), (64, 3)):
        _check(ctx, torch, stream, r["Hd"], r["Sd"], k, seed)


def test_alkane_bf16x3_against_the_dense_export(ofm, torch, stream):
    """The bench's configuration: the products use the same blocks the
    dense export scatters, so they match it to FP64 summation order."""
    wl = make_workload("alkane")
    ctx = ofm.Context(stream)
    ctx.build_fragments(wl.grid, wl.V, wl.frags, storage="fp32")
    ctx.fragment_eigs()
    ctx.assemble("bf16x3")
    Hd, Sd = ctx.dense_HS()
    _check(ctx, torch, stream, Hd, Sd, 37, 4)
    # a distance cutoff drops the halo-only pairs: their blocks are zero in both
    ctx.set_pair_cutoff(wl.fragment_atoms(), 1.0)
    ctx.assemble("bf16x3")
    Hc, Sc = ctx.dense_HS()
    assert np.count_nonzero(Hc) < np.count_nonzero(Hd)
    _check(ctx, torch, stream, Hc, Sc, 8, 5)


def test_errors(ofm, torch, stream):
    wl = make_workload("tiny")
    ctx = ofm.Context(stream)
    ctx.build_fragments(wl.grid, wl.V, wl.frags, storage="fp64")
    n = sum(f.n_states for f in wl.frags)
    with torch.cuda.stream(stream):
        X = torch.zeros((2, n), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        with pytest.raises(ofm.OFMError):
            ctx.pencil_apply("H", X)                 # nothing assembled
        r = O.run_ofm(wl)
        for a, P in enumerate(r["Phis"]):
            ctx.set_fragment_states(a, P)
        ctx.assemble("fp64")
        with pytest.raises(ofm.OFMError):
            ctx.pencil_apply("H", X, out=X)          # Y overlaps X
        Y = ctx.pencil_apply("S", X)
        torch.cuda.synchronize()
        assert float(Y.abs().max()) == 0.0
