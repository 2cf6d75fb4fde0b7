"""Stream capture of the identification + localization call (Sec. 2.2.2, Eq. 5;
Sec. 3.3.3, Eq. 6): once the workspace is reserved, the call allocates and
synchronises nothing, so a CUDA graph of it replays the same pipeline.

The graph's outputs must equal the eager call's bit for bit (same kernels,
same inputs), repeat replays too, on a ragged grid and on a field that changes
between replays (the graph reads the field's buffer at replay time).  A traced
launch inside the capture becomes a pair of event-record nodes: after a replay
the trace holds one timed record per captured sweep.  The trace filter accepts
the library's kernel names and rejects others.
"""
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def q():
    import paper_1911_12070_gb300 as qtv

    qtv.build()
    h = qtv.Qtv(0)
    yield h
    h.close()


def _bufs(cap, dev):
    return (torch.empty(cap, dtype=torch.int64, device=dev),
            torch.empty(cap, dtype=torch.int8, device=dev),
            torch.zeros(1, dtype=torch.int64, device=dev),
            torch.empty((cap, 3), dtype=torch.float32, device=dev),
            torch.empty(cap, dtype=torch.float32, device=dev),
            torch.empty(cap, dtype=torch.uint8, device=dev))


def _same(a, b):
    n = int(a[2].item())
    assert n == int(b[2].item())
    for x, y in zip(a[:2] + a[3:], b[:2] + b[3:]):
        assert torch.equal(x[:n], y[:n])
    return n


@pytest.mark.parametrize("shape,seed", [((40, 36, 52), 13), ((33, 70, 62), 4)])
def test_graph_replay_equals_eager(q, shape, seed):
    dev = torch.device("cuda", 0)
    psi = torch.from_numpy(synth.random_waves_numpy(shape, synth.wave_spec(seed, 512))).to(dev)
    cap = 4096 + int(0.03 * psi.numel())
    q.reserve(shape, cap)
    eager = _bufs(cap, dev)
    q.identify_localize_into(psi, *eager)
    torch.cuda.synchronize()
    out = _bufs(cap, dev)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        q.identify_localize_into(psi, *out)  # workspace of this shape exists
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    for t in out:
        t.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        q.identify_localize_into(psi, *out)
    g.replay()
    torch.cuda.synchronize()
    n = _same(eager, out)
    assert n > 100
    for t in out:
        t.zero_()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    _same(eager, out)
    # the graph reads the field at replay time: a new field in the same buffer
    other = torch.from_numpy(synth.random_waves_numpy(shape, synth.wave_spec(seed + 1, 512))).to(dev)
    ref = _bufs(cap, dev)
    q.identify_localize_into(other, *ref)
    psi.copy_(other)
    g.replay()
    torch.cuda.synchronize()
    _same(ref, out)
    del g


def test_traced_capture_times_each_replay(q):
    shape = (48, 48, 48)
    dev = torch.device("cuda", 0)
    psi = torch.from_numpy(synth.random_waves_numpy(shape, synth.wave_spec(21, 512))).to(dev)
    cap = 4096 + int(0.03 * psi.numel())
    q.reserve(shape, cap)
    out = _bufs(cap, dev)
    q.identify_localize_into(psi, *out)
    torch.cuda.synchronize()
    q.trace_read(reset=True)
    g = torch.cuda.CUDAGraph()
    q.trace_enable(True, only="sweep")
    try:
        with torch.cuda.graph(g):
            for _ in range(3):
                q.identify_localize_into(psi, *out)
    finally:
        q.trace_enable(False, only=None)
    g.replay()
    torch.cuda.synchronize()
    tr = q.trace_read(reset=True)
    assert set(tr) == {"sweep"}
    launches, ms = tr["sweep"]
    assert launches == 3 and 0.0 < ms < 1e3
    del g
    # eager tracing is unaffected by the capture
    q.trace_enable(True)
    q.identify_localize_into(psi, *out)
    torch.cuda.synchronize()
    q.trace_enable(False)
    tr = q.trace_read(reset=True)
    assert {"sweep", "localize"} <= set(tr)


def test_trace_filter_names(q):
    import paper_1911_12070_gb300 as qtv

    with pytest.raises(qtv.QtvError):
        q.trace_enable(True, only="no_such_kernel")
    q.trace_enable(False, only=None)
    for name in ("sweep", "localize", "refine", "thin"):
        q.trace_enable(False, only=name)
    q.trace_enable(False, only=None)
