"""Checkpoint of the basis (ofm_save_basis / ofm_load_basis): a context built
on the same geometry resumes from the saved states without the eigensolve,
with the same blocks and window bit for bit (FP64 and FP32 storage: the
values are saved in the storage precision, so they round-trip exactly).
Headers of another geometry and files of the wrong length are refused."""
import json

import numpy as np
import pytest

from ofm_inputs import Fragment, make_workload

from gpu_util import gpu_lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ofm():
    return gpu_lib()


@pytest.mark.parametrize("storage,prec", [("fp64", "fp64"), ("fp32", "bf16x3")])
def test_basis_checkpoint_resumes(ofm, tmp_path, storage, prec):
    wl = make_workload("tiny")
    path = tmp_path / "basis"
    a = ofm.Context()
    a.build_fragments(wl.grid, wl.V, wl.frags, storage=storage)
    a.fragment_eigs()
    a.assemble(prec)
    want_blocks, want_E = a.get_blocks(), a.eigs_by_index(0, 10)
    a.save_basis(path)
    hdr = json.load(open(str(path) + ".json"))
    assert hdr["format"] == "ofm-basis-1" and hdr["storage"] == storage
    assert hdr["grid"] == list(wl.grid.n) and len(hdr["fragments"]) == len(wl.frags)
    esz = 8 if storage == "fp64" else 4
    n_vals = sum(int(np.prod(f.ext)) * f.n_states for f in wl.frags)
    assert (tmp_path / "basis.bin").stat().st_size == n_vals * esz
    a.close()
    b = ofm.Context()
    b.build_fragments(wl.grid, wl.V, wl.frags, storage=storage)
    b.load_basis(path)
    b.assemble(prec)
    assert np.array_equal(b.get_blocks(), want_blocks)
    assert np.array_equal(b.eigs_by_index(0, 10), want_E)
    b.close()


def test_basis_checkpoint_refuses_other_geometry(ofm, tmp_path):
    wl = make_workload("tiny")
    path = tmp_path / "basis"
    a = ofm.Context()
    a.build_fragments(wl.grid, wl.V, wl.frags, storage="fp64")
    a.fragment_eigs()
    a.save_basis(path)
    a.close()
    other = [Fragment(f.off, f.ext, f.n_states + (1 if i == 0 else 0)) for i, f in enumerate(wl.frags)]
    c = ofm.Context()
    c.build_fragments(wl.grid, wl.V, other, storage="fp64")
    with pytest.raises(ofm.OFMError) as e:
        c.load_basis(path)
    assert e.value.status == ofm.OFM_ERR_INVALID and "another grid" in str(e.value)
    c.build_fragments(wl.grid, wl.V, wl.frags, storage="fp32")   # storage differs
    with pytest.raises(ofm.OFMError):
        c.load_basis(path)
    c.build_fragments(wl.grid, wl.V, wl.frags, storage="fp64")
    data = (tmp_path / "basis.bin").read_bytes()
    (tmp_path / "basis.bin").write_bytes(data[:-8])
    with pytest.raises(ofm.OFMError) as e:
        c.load_basis(path)
    assert "shorter" in str(e.value)
    (tmp_path / "basis.bin").write_bytes(data + b"\0" * 8)
    with pytest.raises(ofm.OFMError) as e:
        c.load_basis(path)
    assert "longer" in str(e.value)
    c.close()
