"""qtv_identify_static: identification for callers that cannot allocate device
memory (an engine that owns the whole GPU through its own allocator, or a
latency-critical loop where cudaMalloc / cudaFree would synchronise the
device).  The entry point keeps its scratch in a fixed device array inside
the library; this test calls it through the C ABI and checks that two calls
in a row return exactly what the handle-based qtv_identify returns (windings
are compared bit for bit, as everywhere else).  It sits in its own file,
collected last, and passes alone or after the other tests."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _static_call(lib, psi, capacity):
    import paper_1911_12070_gb300 as qtv

    g = qtv.Grid.of(tuple(psi.shape))
    ids = torch.empty(capacity, dtype=torch.int64, device="cuda")
    w = torch.empty(capacity, dtype=torch.int8, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    rc = lib.qtv_identify_static(ctypes.byref(g), ctypes.c_void_p(psi.data_ptr()),
                                 ctypes.c_void_p(ids.data_ptr()), ctypes.c_void_p(w.data_ptr()),
                                 capacity, ctypes.c_void_p(count.data_ptr()),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, lib.qtv_last_error_string()
    n = int(count.item())
    assert n <= capacity
    return ids[:n].cpu().numpy(), w[:n].cpu().numpy()


def test_static_identify_matches_handle_identify_twice():
    import paper_1911_12070_gb300 as qtv

    qtv.build()
    lib = qtv.lib()
    q = qtv.Qtv(0)
    fields = [synth.random_waves((96, 160, 256), synth.wave_spec(31, 1024), device="cuda"),
              torch.from_numpy(synth.analytic_line_ring()).cuda()]
    for psi in fields:  # two calls in a row, different sizes and contents
        ref_ids, ref_w, _ = q.identify(psi)
        ids, w = _static_call(lib, psi, capacity=max(4096, 2 * ref_ids.numel()))
        assert np.array_equal(ids, ref_ids.cpu().numpy())
        assert np.array_equal(w, ref_w.cpu().numpy())
    # and the same input again: the array keeps the previous contents, which
    # must not leak into the result
    ids2, w2 = _static_call(lib, fields[0], capacity=200000)
    ref_ids, ref_w, _ = q.identify(fields[0])
    assert np.array_equal(ids2, ref_ids.cpu().numpy()) and np.array_equal(w2, ref_w.cpu().numpy())
    q.close()


def test_static_identify_rejects_sizes_beyond_the_limit():
    import paper_1911_12070_gb300 as qtv

    lib = qtv.lib()
    g = qtv.Grid.of((8, 8, 8))
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    psi = torch.zeros((8, 8, 8), dtype=torch.complex64, device="cuda")
    buf = torch.empty(8, dtype=torch.int64, device="cuda")
    rc = lib.qtv_identify_static(ctypes.byref(g), ctypes.c_void_p(psi.data_ptr()),
                                 ctypes.c_void_p(buf.data_ptr()), ctypes.c_void_p(buf.data_ptr()),
                                 (1 << 21) + 1, ctypes.c_void_p(count.data_ptr()), None)
    assert rc == qtv.ERR_ARG
    assert b"QTV_STATIC_MAX_FACES" in lib.qtv_last_error_string()
    g2 = qtv.Grid.of((4096, 7 * 40, 8))
    rc = lib.qtv_identify_static(ctypes.byref(g2), ctypes.c_void_p(psi.data_ptr()), None, None,
                                 0, ctypes.c_void_p(count.data_ptr()), None)
    assert rc == qtv.ERR_ARG
    assert b"QTV_STATIC_MAX_SEGMENTS" in lib.qtv_last_error_string()
