"""Oracle pair blocks of large workloads in parallel worker processes.

Test infrastructure: each worker (started with "spawn", so it shares no
state with a CUDA context in the parent) builds the oracle's sparse H from a
potential saved to disk and computes the blocks of its share of the pairs
from seeded random states, FP32-rounded like the library's storage, together
with the entry-wise magnitudes that the error bounds of the tests need:
    |Phi_a|^T |Phi_b|  and  |Phi_a|^T (|H| |Phi_b|).
"""
import multiprocessing as mp
import os
import tempfile

import numpy as np


def fp32_states(grid, frag, seed):
    from ofm_inputs import random_states
    return random_states(grid, frag, seed=seed).astype(np.float32).astype(np.float64)


def _work(args):
    grid, frags, vpath, pairs, seed0 = args
    from oracle import ofm_oracle as O
    H = O.hamiltonian(grid, np.load(vpath, mmap_mode="r"))
    absH = abs(H)
    states = {}
    out = []
    for a, b in pairs:
        for f in (a, b):
            if f not in states:
                states[f] = fp32_states(grid, frags[f], seed0 + f)
        Hab, Sab = O.pair_block(H, grid, frags[a], states[a], frags[b], states[b])
        if a == b:
            Hab, Sab = 0.5 * (Hab + Hab.T), 0.5 * (Sab + Sab.T)
        Ea = abs(O.zero_extend(grid, frags[a], states[a]))
        Eb = abs(O.zero_extend(grid, frags[b], states[b]))
        out.append(((a, b), Hab, Sab, (Ea.T @ Eb).toarray(), (Ea.T @ (absH @ Eb)).toarray()))
    return out


def oracle_blocks(grid, frags, V, pairs, seed0, workers=8):
    """{(a, b): (H_ab, S_ab, |S| bound base, |H| bound base)} for the pairs,
    states of fragment f drawn with seed seed0 + f."""
    for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    w = max(1, min(workers, len(pairs), os.cpu_count() or 1))
    chunks = [pairs[i::w] for i in range(w)]
    with tempfile.TemporaryDirectory() as tmp:
        vpath = os.path.join(tmp, "V.npy")
        np.save(vpath, np.ascontiguousarray(V))
        with mp.get_context("spawn").Pool(w) as pool:
            res = pool.map(_work, [(grid, frags, vpath, c, seed0) for c in chunks])
    return {ab: rest for part in res for (ab, *rest) in part}
