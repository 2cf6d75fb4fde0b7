"""Failure detection on the GPU without a fault: a bounded device wait that
runs out ends its kernel normally and reports QTV_COUNT_TIMEOUT, and the
handle (and the CUDA context) stay usable.

The wait exercised is the decoupled look-back of the segment scan, a spin on
a global-memory tile flag.  The injection (qtv_inject_scan_hold) makes one
scan tile withhold its flag, so the next tile's wait has a flag that nothing
sets; a short spin limit (about a millisecond) ends it.  No mbarrier that
guards in-flight bulk copies is involved, no kernel traps, and nothing reads
or writes out of bounds: faces are written only below capacity.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", params=[0, 1], ids=["nibble", "bits"])
def q(request):
    import paper_1911_12070_gb300 as qtv

    qtv.build()
    h = qtv.Qtv(0)
    h.configure_sweep(variant=request.param)
    yield h
    h.inject_scan_hold(-1, 0)
    h.close()


@pytest.fixture(scope="module")
def field():
    # 600 planes of 128 rows: more than one 4096-segment scan tile with
    # either sweep (8 or 19 bands a plane)
    return torch.from_numpy(synth.random_waves_numpy((600, 128, 40),
                                                     synth.wave_spec(31, 256))).cuda()


def test_lookback_wait_runs_out_and_handle_recovers(q, field):
    import paper_1911_12070_gb300 as qtv

    ref_ids, ref_w, _ = q.identify(field)
    n = ref_ids.numel()
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    ids = torch.zeros(n + 64, dtype=torch.int64, device="cuda")
    w = torch.zeros(n + 64, dtype=torch.int8, device="cuda")
    q.inject_scan_hold(0, 1 << 20)  # tile 0 withholds its flag; ~0.5 ms spins
    try:
        q.identify_into(field, ids, w, count)
        torch.cuda.synchronize()  # the kernels ended: no hang, no fault
        assert int(count.item()) == -1  # QTV_COUNT_TIMEOUT read as int64
        with pytest.raises(qtv.QtvError) as e:
            q.identify(field)
        assert e.value.code == qtv.ERR_TIMEOUT
        # identify + localize: the timed-out count bounds nothing beyond capacity
        with pytest.raises(qtv.QtvError):
            q.identify_localize(field, capacity=n + 64)
        torch.cuda.synchronize()
    finally:
        q.inject_scan_hold(-1, 0)
    # the handle and the context are usable: the same results as before
    ids2, w2, _ = q.identify(field)
    assert torch.equal(ids2, ref_ids) and torch.equal(w2, ref_w)
    xyz, _, _ = q.localize(field, ids2, w2)
    assert bool(torch.isfinite(xyz).all())


def test_hold_beyond_the_scan_changes_nothing(q, field):
    # a tile index past the scan's last tile holds nothing back
    ref_ids, _, _ = q.identify(field)
    q.inject_scan_hold(1 << 40, 1 << 20)
    try:
        ids, _, _ = q.identify(field)
    finally:
        q.inject_scan_hold(-1, 0)
    assert torch.equal(ids, ref_ids)


def test_bad_injection_arguments_are_rejected(q):
    import paper_1911_12070_gb300 as qtv

    with pytest.raises(qtv.QtvError) as e:
        q.inject_scan_hold(-2, 0)
    assert e.value.code == qtv.ERR_ARG
    with pytest.raises(qtv.QtvError):
        q.inject_scan_hold(0, -1)
