"""The amorphous polymer end to end from the GPU's own states: 128^3 grid, 56
uneven boxes (16^3 .. 40^3 points, edges multiples of 8), 8-64 states per
box, basis 2033.

FP64 storage and arithmetic throughout: the batched fragment eigensolver,
the assembly (per-pair schedule) and Eq. 2 by the dense FP64 window solver,
against the FP64 oracle's run of the same workload (fragment energies and
the whole spectrum of Eq. 2, tests/golden/polymer_oracle.json, written by
tests/golden/make_golden.py from oracle/ only).  The window is the 0.3 Ha
above E_801 (A9: one occupied level per well, 800 wells); each of its
eigenvalues must match to 1e-6 Ha.

The oracle's S has lambda_min = 2e-9 here, so Eq. 2 is far more sensitive
than for the chains: the GPU's states differ from the oracle's by the
eigensolver's residual (<= 1e-9), and the window still matches, while the
mixed-precision path cannot even factor S (its FP32-accurate entries sit
far above lambda_min); that is reported as OFM_ERR_NOT_POSDEF (A11)."""
import json
import os

import numpy as np
import pytest

from ofm_inputs import make_workload

from gpu_util import gpu_lib

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def ofm():
    return gpu_lib()


def test_polymer_end_to_end_fp64(ofm):
    g = json.load(open(os.path.join(HERE, "golden", "polymer_oracle.json")))
    wl = make_workload("polymer")
    assert wl.name == g["workload"] and len(wl.frags) == 56
    assert {f.n_states for f in wl.frags} <= set(range(8, 65))
    assert len({tuple(f.ext) for f in wl.frags}) > 1
    Eo = np.array(g["ofm_spectrum"])
    n = len(Eo)
    assert n == sum(f.n_states for f in wl.frags)
    ctx = ofm.Context()
    ctx.build_fragments(wl.grid, wl.V, wl.frags, storage="fp64")
    eps, res, st = ctx.fragment_eigs()
    assert st == ofm.OFM_OK and res.max() <= 1e-9
    ef = np.concatenate([np.array(e) for e in g["fragment_eps"]])
    assert np.max(np.abs(eps - ef)) < 1e-9, np.max(np.abs(eps - ef))
    ctx.assemble("fp64")
    assert ctx.last_schedule() == "pair"   # FP64 storage: the per-pair form
    E = ctx.eigs_by_index(0, n)
    i0 = g["window_rule"]["n_occ"]
    width = g["window_rule"]["width"]
    m = int(np.sum((Eo >= Eo[i0]) & (Eo <= Eo[i0] + width)))
    assert m > 300
    err = np.abs(E[i0:i0 + m] - Eo[i0:i0 + m])
    assert err.max() < 1e-6, (float(err.max()), int(np.argmax(err)))
    # the window anchored at the first empty level, as the benchmark takes it
    w, k = ctx.window_from_index(i0, width, max_out=n)
    assert abs(k - m) <= 1
    mm = min(k, m)
    assert np.max(np.abs(w[:mm] - Eo[i0:i0 + mm])) < 1e-6
    ctx.close()
