"""The allocation-free pair-block entry point against the oracle and the
regular assembly.

ofm_pair_blocks_noalloc serves callers that cannot allocate device memory
when they need a block (device memory owned by another framework's pool,
latency-critical paths where cudaMalloc/cudaFree may block, sandboxed code
handed ready-made buffers).  Its inputs here are the oracle's: seeded states
and H phi from the oracle's H apply.  It must give the oracle's blocks
within the FP32 inner-product bound, and the blocks of ofm_assemble_HS +
ofm_get_block within the same bound.  Two calls in a row exercise the shared
fixed scratch; the file is collected last so that a failure here comes
after every other test has run.
"""
import numpy as np
import pytest

from ofm_inputs import Fragment, Grid, random_states, small_workload
from oracle import ofm_oracle as O

from gpu_util import U32, gpu_lib

pytestmark = pytest.mark.gpu


def dilated(grid, f):
    lo, dext = [], []
    for d in range(3):
        full = f.ext[d] == grid.n[d]
        lo.append(0 if full else 1)
        dext.append(f.ext[d] if full else f.ext[d] + 2)
    return lo, dext


def storage_from_box(grid, f, box):
    """(P, n) box states -> point-major dilated layout (Pd * ld,), halo 0."""
    lo, (ex, ey, ez) = dilated(grid, f)
    n = f.n_states
    ld = (n + 3) // 4 * 4
    out = np.zeros((ez, ey, ex, ld), dtype=np.float32)
    out[lo[2]:lo[2] + f.ext[2], lo[1]:lo[1] + f.ext[1], lo[0]:lo[0] + f.ext[0], :n] = \
        box.reshape(f.ext[2], f.ext[1], f.ext[0], n)
    return out.ravel()


def storage_from_dilated(grid, f, dil):
    """(Pd, n) values on the dilated box -> point-major layout (Pd * ld,)."""
    _, (ex, ey, ez) = dilated(grid, f)
    n = f.n_states
    ld = (n + 3) // 4 * 4
    out = np.zeros((ex * ey * ez, ld), dtype=np.float32)
    out[:, :n] = dil
    return out.ravel()


def test_noalloc_pair_blocks_match_the_assembly():
    ofm = gpu_lib()
    import torch

    grid = Grid((48, 10, 10), 0.5)
    frags = [Fragment((6 * a, 0, 0), (12, 10, 10), 6 + a % 3) for a in range(4)]
    wl = small_workload(grid_n=grid.n, h=grid.h, frags=frags, seed=5)
    Phis = [random_states(grid, f, seed=700 + a).astype(np.float32).astype(np.float64)
            for a, f in enumerate(frags)]
    H = O.hamiltonian(grid, wl.V)
    ctx = ofm.Context()
    ctx.build_fragments(grid, wl.V, frags, storage="fp32")
    for a, P in enumerate(Phis):
        ctx.set_fragment_states(a, P)
    ctx.assemble("fp32")
    dev = [torch.tensor(storage_from_box(grid, f, Phis[a]), device="cuda")
           for a, f in enumerate(frags)]
    hdev = [torch.tensor(storage_from_dilated(grid, f, O.apply_h(H, grid, f, Phis[a])), device="cuda")
            for a, f in enumerate(frags)]
    stream = torch.cuda.current_stream().cuda_stream
    # two calls in a row on the shared scratch: an off-diagonal and a diagonal pair
    for (a, b) in [(0, 1), (2, 2), (1, 3)]:
        na, nb = frags[a].n_states, frags[b].n_states
        out = torch.full((2 * na * nb,), float("nan"), dtype=torch.float64, device="cuda")
        ofm.pair_blocks_noalloc(grid, frags[a], frags[b], dev[a], dev[b], hdev[b], out, stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        Hg, Sg = got[:na * nb].reshape(na, nb), got[na * nb:].reshape(na, nb)
        Hr, Sr = ctx.block(a, b)
        Ho, So = O.pair_block(H, grid, frags[a], Phis[a], frags[b], Phis[b])
        if a == b:
            Ho, So = 0.5 * (Ho + Ho.T), 0.5 * (So + So.T)
        # FP32 sums: per-entry bound 2 K u |a|.|b| (K = points of box a); the
        # H phi input is rounded to FP32 too (u |H| |phi_b|)
        Ea = O.zero_extend(grid, frags[a], Phis[a])
        Eb = O.zero_extend(grid, frags[b], Phis[b])
        K = int(np.prod(frags[a].ext))
        bS = 2 * K * U32 * (abs(Ea).T @ abs(Eb)).toarray() + 1e-30
        bH = (2 * K + 8) * U32 * (abs(Ea).T @ (abs(H) @ abs(Eb))).toarray() + 1e-30
        assert np.all(np.isfinite(Hg)) and np.all(np.isfinite(Sg))
        assert np.all(np.abs(Sg - So) <= bS), (a, b)
        assert np.all(np.abs(Hg - Ho) <= bH), (a, b)
        assert np.all(np.abs(Sg - Sr) <= 2 * bS), (a, b)
        assert np.all(np.abs(Hg - Hr) <= 2 * bH), (a, b)
    # a pair whose boxes never meet gives zeros
    na, nb = frags[0].n_states, frags[3].n_states
    far = Fragment((30, 0, 0), (12, 10, 10), nb)
    out = torch.full((2 * na * nb,), float("nan"), dtype=torch.float64, device="cuda")
    ofm.pair_blocks_noalloc(grid, frags[0], far, dev[0], dev[3], hdev[3], out, stream)
    torch.cuda.synchronize()
    assert torch.all(out == 0)


def test_noalloc_refuses_a_capturing_stream():
    """The work tables are staged from host memory that lives only for the
    call, so a call on a stream under capture is refused (nothing is
    captured)."""
    ofm = gpu_lib()
    import torch

    grid = Grid((48, 10, 10), 0.5)
    fa = Fragment((0, 0, 0), (12, 10, 10), 6)
    fb = Fragment((6, 0, 0), (12, 10, 10), 6)
    dev = torch.zeros(14 * 10 * 10 * 8, dtype=torch.float32, device="cuda")
    out = torch.zeros(2 * 36, dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    ofm.pair_blocks_noalloc(grid, fa, fb, dev, dev, dev, out, s.cuda_stream)   # look-up before capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with pytest.raises(ofm.OFMError) as e:
        with torch.cuda.graph(g, stream=s):
            ofm.pair_blocks_noalloc(grid, fa, fb, dev, dev, dev, out, s.cuda_stream)
    assert e.value.status == ofm.OFM_ERR_INVALID
