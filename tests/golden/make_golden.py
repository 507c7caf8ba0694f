"""Writes the FP64 oracle's results used as stored expected values:
  tests/golden/tiny_oracle.json   -- the 32x12x12 tiny workload (4 boxes
                                     16x12x12, 6 states each, seed 0);
  tests/golden/alkane_oracle.json -- the 256x32x32 alkane chain (31 boxes
                                     16x32x32, 32 states each, seed 0): its
                                     fragment energies and the whole spectrum
                                     of Eq. 2 (992 eigenvalues);
  tests/golden/polymer_oracle.json -- the 128^3 amorphous polymer (56 uneven
                                     boxes, 8-64 states, seed 0): the same
                                     (2033 eigenvalues).

Calls only oracle/ and the seeded input generator.  The stored numbers are
the oracle's, not the paper's (the paper prints no worked example: its
figures are not part of the available text).
Run from the repository root:  python tests/golden/make_golden.py [tiny|alkane|polymer]
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from ofm_inputs import make_workload  # noqa: E402
from oracle import ofm_oracle as O  # noqa: E402


def _fragment(args):
    key, a = args
    wl = make_workload(key, seed=0)
    H = O.hamiltonian(wl.grid, wl.V)
    return O.fragment_eigs(H, wl.grid, wl.frags[a])


def alkane(key="alkane"):
    """A workload through the oracle as it stands: fragment eigensolves (one
    process each, spawned), pair blocks, dense Eq. 2."""
    import multiprocessing as mp
    for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    wl = make_workload(key, seed=0)
    with mp.get_context("spawn").Pool(min(len(wl.frags), os.cpu_count() or 1)) as pool:
        res = pool.map(_fragment, [(key, a) for a in range(len(wl.frags))])
    eps = [w for w, _ in res]
    Phis = [U for _, U in res]
    r = O.run_ofm(wl, Phis=Phis)
    out = {
        "workload": wl.name,
        "seed": 0,
        "source": "oracle/ofm_oracle.py fragment_eigs + run_ofm (FP64), tests/golden/make_golden.py",
        "fragment_eps": [list(map(float, e)) for e in eps],
        "n_pairs": len(r["pairs"]),
        "ofm_spectrum": list(map(float, r["E"])),
        "window_rule": {"kind": wl.window.kind, "width": wl.window.width, "n_occ": wl.window.n_occ},
        "S_min_eig": float(np.linalg.eigvalsh(r["Sd"])[0]),
    }
    path = os.path.join(ROOT, "tests", "golden", f"{key}_oracle.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=0)
    print("wrote", path)


def main():
    wl = make_workload("tiny", seed=0)
    r = O.run_ofm(wl)
    lo, hi = O.window_bounds(r["E"], wl.window)
    win = r["E"][(r["E"] >= lo) & (r["E"] <= hi)]
    exact = np.linalg.eigvalsh(r["H"].toarray())
    out = {
        "workload": wl.name,
        "seed": 0,
        "source": "oracle/ofm_oracle.py run_ofm (FP64), tests/golden/make_golden.py",
        "fragment_eps": [list(map(float, e)) for e in r["eps"]],
        "pairs": [list(p) for p in r["pairs"]],
        "ofm_spectrum": list(map(float, r["E"])),
        "window": [lo, hi],
        "window_eigs": list(map(float, win)),
        "exact_lowest": list(map(float, exact[:len(r["E"])])),
        "S_min_eig": float(np.linalg.eigvalsh(r["Sd"])[0]),
        "H_01_corner": [[float(x) for x in row] for row in r["blocks"][(0, 1)][0][:3, :3]],
        "S_01_corner": [[float(x) for x in row] for row in r["blocks"][(0, 1)][1][:3, :3]],
    }
    path = os.path.join(ROOT, "tests", "golden", "tiny_oracle.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    which = sys.argv[1:] or ["tiny"]
    if "tiny" in which:
        main()
    if "alkane" in which:
        alkane()
    if "polymer" in which:
        alkane("polymer")
