"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads, exports
every symbol include/ofm.h declares, and its host-only planner agrees with
the oracle's pair list and overlap counts.  No device compute here."""
import os
import re
import subprocess

import numpy as np
import pytest

from ofm_inputs import Fragment, Grid, make_workload
from oracle import ofm_oracle as O


@pytest.fixture(scope="module")
def lib(repo_root):
    from paper_1011_4764_gb300 import build
    build.build()
    from paper_1011_4764_gb300 import ofm
    return ofm


def header_symbols(repo_root):
    text = open(os.path.join(repo_root, "include", "ofm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ofm_[a-zA-Z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib, repo_root):
    syms = header_symbols(repo_root)
    assert "ofm_assemble_HS" in syms and "ofm_window_eigs" in syms
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    missing = [s for s in syms if s not in exported]
    assert not missing, missing
    assert sorted(lib.EXPORTS) == syms
    L = lib.load_library()
    for s in syms:
        assert hasattr(L, s)


def test_status_strings(lib):
    """Every status the header defines has its name, and the binding's
    constants carry the header's values."""
    import re
    text = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                             "include", "ofm.h")).read()
    codes = dict((n, int(v)) for n, v in re.findall(r"\b(OFM_(?:OK|ERR_[A-Z_]+))\s*=\s*(\d+)", text))
    assert codes["OFM_OK"] == 0 and len(codes) >= 9
    for name, value in codes.items():
        assert lib.status_name(value) == name
        assert getattr(lib, name) == value
    assert lib.status_name(99) == "OFM_ERR_UNKNOWN"


@pytest.mark.parametrize("name", ["tiny", "alkane"])
def test_planner_matches_oracle_pairs_and_counts(lib, name):
    wl = make_workload(name)
    pairs, counts, F = lib.plan_pairs(wl.grid, wl.frags)
    assert pairs == O.pair_list(wl.grid, wl.frags)
    for (a, b), (ks, kh) in zip(pairs, counts):
        fa, fb = wl.frags[a], wl.frags[b]
        doff, dext = O.dilated_box(wl.grid, fb)
        assert ks == O.overlap_points(wl.grid, fa.off, fa.ext, fb.off, fb.ext)
        assert kh == O.overlap_points(wl.grid, fa.off, fa.ext, doff, dext)
    assert F == O.pair_flops(wl.grid, wl.frags, pairs)


def test_planner_on_random_periodic_boxes(lib):
    rng = np.random.default_rng(0)
    grid = Grid((13, 9, 7), 0.5)
    for trial in range(20):
        frags = []
        for _ in range(5):
            ext = []
            for n in grid.n:
                e = int(rng.integers(1, n + 1))
                if e == n - 1:
                    e = n
                ext.append(e)
            off = tuple(int(rng.integers(0, n)) for n in grid.n)
            frags.append(Fragment(off, tuple(ext), 1))
        pairs, counts, F = lib.plan_pairs(grid, frags)
        assert pairs == O.pair_list(grid, frags)
        assert F == O.pair_flops(grid, frags, pairs)


@pytest.mark.parametrize("bad", [
    dict(ext=(12, 4, 4)),          # ext == n - 1 in x (n = 13)
    dict(ext=(14, 4, 4)),          # ext > n
    dict(ext=(0, 4, 4)),           # empty box
    dict(n_states=0),
    dict(n_states=4 * 4 * 4),      # more states than P - 1
])
def test_planner_rejects_invalid_geometry(lib, bad):
    grid = Grid((13, 9, 7), 0.5)
    f = dict(off=(0, 0, 0), ext=(4, 4, 4), n_states=2)
    f.update(bad)
    with pytest.raises(lib.OFMError):
        lib.plan_pairs(grid, [Fragment(**f)])


def test_planner_rejects_bad_spacing(lib):
    with pytest.raises(lib.OFMError):
        lib.plan_pairs(Grid((8, 8, 8), 0.0), [Fragment((0, 0, 0), (4, 4, 4), 1)])


def test_missing_library_raises(lib, monkeypatch, tmp_path):
    """No CPU fallback: without libofm.so the binding refuses to load."""
    monkeypatch.setattr(lib, "_LIB", None)
    with pytest.raises(RuntimeError):
        lib.load_library(str(tmp_path / "libofm.so"))


def test_no_device_is_an_error_not_a_fallback(lib):
    """Without a CUDA device a context cannot be created: the call reports
    the CUDA failure (there is no host path to fall back to)."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(lib.OFMError):
        lib.Context()


@pytest.mark.parametrize("name", ["tiny", "alkane", "polymer"])
def test_region_plan_covers_every_pair_exactly(name):
    """The region plan of the tensor-core assembly (coverage regions: products
    of the segments between dilated-box boundaries) sums each pair over the
    regions that hold both fragments; those regions must contain exactly the
    points of B_a ∩ B_b+ that the oracle counts, for every pair."""
    from paper_1011_4764_gb300 import ofm
    wl = make_workload(name)
    stats, pts = ofm.plan_regions(wl.grid, wl.frags)
    pairs = O.pair_list(wl.grid, wl.frags)
    want = []
    for a, b in pairs:
        doff, dext = O.dilated_box(wl.grid, wl.frags[b])
        want.append(O.overlap_points(wl.grid, wl.frags[a].off, wl.frags[a].ext, doff, dext))
    assert stats["regions"] > 0
    assert list(pts) == want


def test_region_plan_on_wrapping_uneven_boxes():
    """Boxes that wrap the periodic boundary, span whole dimensions, and have
    uneven state counts: the same exact coverage, and the plan applies."""
    from paper_1011_4764_gb300 import ofm
    grid = Grid((20, 9, 8), 0.45)
    frags = [Fragment((15, 0, 0), (9, 9, 5), 5), Fragment((3, 2, 4), (7, 5, 8), 7),
             Fragment((9, 7, 6), (6, 4, 6), 3), Fragment((0, 0, 0), (20, 9, 8), 9),
             Fragment((18, 5, 2), (4, 9, 3), 2)]
    stats, pts = ofm.plan_regions(grid, frags)
    want = []
    for a, b in O.pair_list(grid, frags):
        doff, dext = O.dilated_box(grid, frags[b])
        want.append(O.overlap_points(grid, frags[a].off, frags[a].ext, doff, dext))
    assert stats["ok"] == 1 and list(pts) == want
    # segments merged to at least 4 points: regions coarser, coverage unchanged
    s4, p4 = ofm.plan_regions(grid, frags, w_min=4)
    assert s4["regions"] <= stats["regions"] and list(p4) == want
