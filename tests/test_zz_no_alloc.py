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


@pytest.mark.parametrize("case", ["odd_nx", "psi_8_byte_aligned"])
def test_static_identify_register_sweep_path(case):
    # odd nx, or psi aligned to 8 but not 16 bytes, takes the register sweep
    # (the staged sweep needs even nx and a 16-byte aligned field); its use of
    # the fixed array must give the handle call's result too
    import paper_1911_12070_gb300 as qtv

    qtv.build()
    lib = qtv.lib()
    q = qtv.Qtv(0)
    if case == "odd_nx":
        psi = torch.from_numpy(synth.random_waves_numpy((63, 64, 95),
                                                        synth.wave_spec(32, 512))).cuda()
    else:
        host = synth.random_waves_numpy((40, 48, 128), synth.wave_spec(33, 512))
        flat = torch.empty(host.size + 1, dtype=torch.complex64, device="cuda")
        psi = flat[1:].view(host.shape)
        psi.copy_(torch.from_numpy(host))
        assert psi.data_ptr() % 16 == 8
    ref_ids, ref_w, _ = q.identify(psi)
    for _ in range(2):
        ids, w = _static_call(lib, psi, capacity=2 * ref_ids.numel() + 64)
        assert np.array_equal(ids, ref_ids.cpu().numpy())
        assert np.array_equal(w, ref_w.cpu().numpy())
    q.close()


def test_static_identify_capacity_below_the_face_count():
    # more pierced faces than capacity: the count is the full total and the
    # first `capacity` faces are the handle call's first faces
    import paper_1911_12070_gb300 as qtv

    qtv.build()
    lib = qtv.lib()
    q = qtv.Qtv(0)
    psi = synth.random_waves((64, 128, 256), synth.wave_spec(34, 1024), device="cuda")
    ref_ids, ref_w, _ = q.identify(psi)
    n = ref_ids.numel()
    cap = n // 3
    g = qtv.Grid.of(tuple(psi.shape))
    ids = torch.empty(cap, dtype=torch.int64, device="cuda")
    w = torch.empty(cap, dtype=torch.int8, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    rc = lib.qtv_identify_static(ctypes.byref(g), ctypes.c_void_p(psi.data_ptr()),
                                 ctypes.c_void_p(ids.data_ptr()), ctypes.c_void_p(w.data_ptr()),
                                 cap, ctypes.c_void_p(count.data_ptr()),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, lib.qtv_last_error_string()
    assert int(count.item()) == n
    assert torch.equal(ids, ref_ids[:cap]) and torch.equal(w, ref_w[:cap])
    q.close()
