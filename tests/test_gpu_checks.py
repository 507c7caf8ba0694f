"""Check mode (ofm_set_checks, or OFM_CHECK=1 when a context is created):
every device buffer carries a guard band that is read after each call, and
the region schedule's pack and tensor-core contraction run forms that test
every gathered index and copied range against their buffers.  The failures
below are made on the host (a byte of a guard band overwritten by a host
call; a copy piece of the host plan pointed past its arena, which the
checking producer refuses before any copy): nothing faults."""
import numpy as np
import pytest

from ofm_inputs import make_workload, small_workload

from gpu_util import gpu_lib
from test_gpu_tensorcore import GEOMS, fp32_states

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ofm():
    return gpu_lib()


def _ctx(ofm, geom, checks):
    grid, frags = GEOMS[geom]
    wl = small_workload(grid_n=grid.n, h=grid.h, frags=frags, seed=3)
    ctx = ofm.Context()
    if checks:
        ctx.set_checks(True)
    ctx.build_fragments(grid, wl.V, frags, storage="fp32")
    for a, P in enumerate(fp32_states(grid, frags, 500)):
        ctx.set_fragment_states(a, P)
    return ctx, wl


@pytest.mark.parametrize("geom", ["wrap", "chain"])
def test_check_mode_gives_the_same_blocks(ofm, geom):
    plain, _ = _ctx(ofm, geom, False)
    checked, _ = _ctx(ofm, geom, True)
    for prec, sched in (("bf16x3", "region"), ("tf32", "region"), ("bf16x3", "pair"),
                        ("fp32", "region"), ("fp64", "region")):
        plain.assemble(prec, schedule=sched)
        checked.assemble(prec, schedule=sched)   # ends with a guard check
        a, b = plain.get_blocks(), checked.get_blocks()
        assert np.array_equal(a, b), (prec, sched)
    checked.check_guards()
    plain.close()
    checked.close()


def test_check_mode_whole_method(ofm):
    """The tiny workload through the eigensolver, the assembly and Eq. 2 with
    checks on: every call's guard check passes, the same results."""
    wl = make_workload("tiny")
    out = []
    for checks in (False, True):
        ctx = ofm.Context()
        ctx.set_checks(checks)
        ctx.build_fragments(wl.grid, wl.V, wl.frags, storage="fp64")
        eps, _, _ = ctx.fragment_eigs()
        ctx.assemble("fp64")
        out.append((eps, ctx.eigs_by_index(0, 10), ctx.get_blocks()))
        ctx.close()
    for x, y in zip(out[0], out[1]):
        assert np.array_equal(x, y)


def test_overwritten_guard_band_is_reported(ofm):
    ctx, _ = _ctx(ofm, "chain", True)
    ctx.assemble("bf16x3")
    ctx.check_guards()
    ctx.test_hold_wait("guard")
    with pytest.raises(ofm.OFMError) as e:
        ctx.check_guards()
    assert e.value.status == ofm.OFM_ERR_CORRUPT and "blocks" in str(e.value)
    with pytest.raises(ofm.OFMError) as e:
        ctx.get_blocks()          # every checked call reports it from now on
    assert e.value.status == ofm.OFM_ERR_CORRUPT
    ctx.close()


def test_refused_copy_piece_is_reported(ofm):
    grid, frags = GEOMS["chain"]
    ctx, wl = _ctx(ofm, "chain", True)
    ctx.assemble("bf16x3", schedule="region")
    want = ctx.get_blocks()
    ctx.test_hold_wait("piece")
    with pytest.raises(ofm.OFMError) as e:
        ctx.assemble("bf16x3", schedule="region")
    assert e.value.status == ofm.OFM_ERR_CORRUPT and "refused" in str(e.value)
    # a new plan: the context works again, the same blocks bit for bit
    ctx.build_fragments(grid, wl.V, frags, storage="fp32")
    for a, P in enumerate(fp32_states(grid, frags, 500)):
        ctx.set_fragment_states(a, P)
    ctx.assemble("bf16x3", schedule="region")
    assert np.array_equal(ctx.get_blocks(), want)
    # the hook is for check mode only
    ctx.set_checks(False)
    with pytest.raises(ofm.OFMError) as e:
        ctx.test_hold_wait("piece")
    assert e.value.status == ofm.OFM_ERR_STATE
    ctx.close()
