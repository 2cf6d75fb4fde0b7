"""GB300 vortex-core identification and sub-grid localization.

Python binding of libqtv (``include/qtv.h``).  It only marshals arguments:
every step of identification, localization and emission runs in the CUDA
kernels of ``csrc/``.  PyTorch supplies device memory and streams.  There is
no CPU fallback: if ``_build/libqtv.so`` cannot be loaded, :func:`lib` raises.

Low-level: :func:`lib` returns the ctypes library whose functions carry the
C names (``qtv_identify``, ``qtv_localize``, ``qtv_emit_samples``, ...).
High-level: :class:`Qtv` wraps a handle and works on torch tensors.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

LOCATOR_PARAMS = 99587

__all__ = ["lib", "Qtv", "Grid", "Stats", "Sample", "QtvError", "PLAIN", "LEARNED",
           "FLAG_ANOMALOUS", "FLAG_FALLBACK", "FLAG_LEARNED", "SAMPLE_DTYPE", "build"]

PLAIN, LEARNED = 0, 1
FLAG_ANOMALOUS, FLAG_FALLBACK, FLAG_LEARNED = 1, 2, 4
OK, WARN_NONFINITE, ERR_ARG, ERR_CAPACITY, ERR_CUDA, ERR_TIMEOUT, ERR_STATE = 0, 1, -1, -2, -3, -4, -5

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libqtv.so")


REFINE_CONVERGED, REFINE_NO_TANGENT, REFINE_MAX_ITER = 1, 2, 4


PIECE_DTYPE = np.dtype([("first", "<u8"), ("count", "<u4"), ("component", "<u4"),
                        ("closed", "u1"), ("comp_type", "u1"), ("reversed", "u1"),
                        ("reserved", "u1", 5)])


def pieces_numpy(pieces):
    """qtv_piece records (uint8 tensor [np, 24]) as a numpy structured array."""
    return pieces.cpu().numpy().reshape(-1).view(PIECE_DTYPE)


class QtvError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"qtv error {code}: {msg}")
        self.code = code


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("h", ctypes.c_float), ("origin", ctypes.c_float * 3), ("periodic", ctypes.c_uint32)]

    @classmethod
    def of(cls, shape, h=1.0, origin=(0.0, 0.0, 0.0)):
        nz, ny, nx = shape
        g = cls()
        g.nx, g.ny, g.nz, g.h = nx, ny, nz, h
        for i in range(3):
            g.origin[i] = origin[i]
        g.periodic = 0
        return g


class Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("faces_scanned", "pierced", "ambiguous",
                                              "zero_node_faces", "nonfinite_faces", "anomalous",
                                              "fallbacks", "reserved")]


class Sample(ctypes.Structure):
    _fields_ = [("x", ctypes.c_float), ("y", ctypes.c_float), ("z", ctypes.c_float),
                ("resid", ctypes.c_float), ("face_id", ctypes.c_uint64), ("winding", ctypes.c_int8),
                ("flags", ctypes.c_uint8), ("reserved0", ctypes.c_uint16),
                ("reserved1", ctypes.c_uint32)]


class TraceEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_uint32),
                ("total_ms", ctypes.c_float)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("nodes", ctypes.c_uint64), ("faces", ctypes.c_uint64),
                ("warps_per_tile", ctypes.c_int32), ("tile_columns", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("zscale", ctypes.c_float),
                ("concurrent", ctypes.c_int32), ("variant", ctypes.c_int32),
                ("stages", ctypes.c_int32), ("sweeps", ctypes.c_int32),
                ("grid", ctypes.c_int32), ("source", ctypes.c_int32),
                ("candidates", ctypes.c_int32), ("tuned_ms", ctypes.c_float)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


SAMPLE_DTYPE = np.dtype([("x", "<f4"), ("y", "<f4"), ("z", "<f4"), ("resid", "<f4"),
                         ("face_id", "<u8"), ("winding", "i1"), ("flags", "u1"),
                         ("reserved0", "<u2"), ("reserved1", "<u4")])
assert SAMPLE_DTYPE.itemsize == ctypes.sizeof(Sample) == 32

_lib = None


def build(force: bool = False) -> str:
    from . import nvcc_build

    return nvcc_build.build(force=force)


def lib() -> ctypes.CDLL:
    """Load libqtv.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_1911_12070_gb300.build() first")
        L = ctypes.CDLL(LIB_PATH)
        P, u64, i32, f32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_float
        L.qtv_version.restype = i32
        L.qtv_last_error_string.restype = ctypes.c_char_p
        L.qtv_create.argtypes = [ctypes.POINTER(P), i32]
        L.qtv_destroy.argtypes = [P]
        L.qtv_reserve.argtypes = [P, ctypes.POINTER(Grid), u64]
        L.qtv_identify.argtypes = [P, ctypes.POINTER(Grid), P, P, P, u64, P, P, P]
        L.qtv_localize.argtypes = [P, ctypes.POINTER(Grid), P, P, P, u64, P, i32, f32, P, P, P, P]
        L.qtv_emit_samples.argtypes = [P, u64, P, P, P, P, P, P, P]
        L.qtv_identify_localize.argtypes = [P, ctypes.POINTER(Grid), P, P, P, u64, P, P, P, P, P,
                                             P]
        L.qtv_identify_localize.restype = i32
        L.qtv_identify_static.argtypes = [ctypes.POINTER(Grid), P, P, P, u64, P, P]
        L.qtv_identify_static.restype = i32
        L.qtv_locator_init.argtypes = [P, u64]
        L.qtv_locator_get.argtypes = [P, P, P, ctypes.POINTER(u64)]
        L.qtv_locator_set.argtypes = [P, P, P, u64]
        L.qtv_locator_encode.argtypes = [P, ctypes.POINTER(Grid), P, P, P, u64, P, P, P, P, P]
        L.qtv_locator_forward.argtypes = [P, P, u64, P, P]
        L.qtv_locator_gradients.argtypes = [P, P, P, u64, P, P, P]
        L.qtv_locator_train_step.argtypes = [P, P, P, u64, f32, P, P]
        L.qtv_locator_save.argtypes = [P, ctypes.c_char_p]
        L.qtv_locator_load.argtypes = [P, ctypes.c_char_p]
        L.qtv_locator_set_tensor_path.argtypes = [P, i32]
        L.qtv_locator_set_tensor_path.restype = i32
        for name in ("qtv_locator_init", "qtv_locator_get", "qtv_locator_set", "qtv_locator_encode",
                     "qtv_locator_forward", "qtv_locator_gradients", "qtv_locator_train_step",
                     "qtv_locator_save", "qtv_locator_load"):
            getattr(L, name).restype = i32
        L.qtv_configure_sweep.argtypes = [P, i32, i32, i32, i32]
        L.qtv_configure_sweep.restype = i32
        L.qtv_inject_scan_hold.argtypes = [P, ctypes.c_int64, ctypes.c_int64]
        L.qtv_inject_scan_hold.restype = i32
        L.qtv_batch_plan.argtypes = [P, i32, ctypes.POINTER(Grid), ctypes.POINTER(P),
                                     ctypes.c_char_p, P]
        L.qtv_batch_info_get.argtypes = [P, ctypes.POINTER(BatchInfo)]
        L.qtv_batch_run.argtypes = [P, P, P, u64, P, P, P, P, i32, f32, P]
        for name in ("qtv_batch_plan", "qtv_batch_info_get", "qtv_batch_run"):
            getattr(L, name).restype = i32
        L.qtv_node_circulation.argtypes = [P, ctypes.POINTER(Grid), P, P, P, u64, P, P, P]
        L.qtv_density_error.argtypes = [P, ctypes.POINTER(Grid), P, P, u64, P, P, P, P]
        L.qtv_refine_samples.argtypes = [P, ctypes.POINTER(Grid), P, P, P, u64, P, i32, f32, P, P,
                                         P, P, P, P, P]
        L.qtv_face_graph.argtypes = [P, ctypes.POINTER(Grid), P, u64, P, P, P, P, P, P]
        L.qtv_line_pieces.argtypes = [P, u64, P, P, P, P, P, P, P, P, u64, P, u64, P, P]
        L.qtv_piece_curves.argtypes = [P, P, P, P, u64, P, i32, P, u64, P, P, P, P]
        L.qtv_identify_localize_host.argtypes = [P, ctypes.POINTER(Grid), P, u64, P, P, P]
        L.qtv_thin_pieces.argtypes = [P, P, P, P, u64, u64, f32, P, u64, P, P, P]
        L.qtv_node_graph.argtypes = [P, ctypes.POINTER(Grid), P, u64, P, P, P, P, P, P]
        L.qtv_box_reduce.argtypes = [P, u64, P, P, P, i32, P, f32, i32, P, P, P, P]
        L.qtv_box_reduce.restype = i32
        L.qtv_node_circulation_faces.argtypes = [P, ctypes.POINTER(Grid), P, P, u64, P, P, P, u64,
                                                 P, P, P]
        L.qtv_node_circulation_faces.restype = i32
        for name in ("qtv_node_circulation", "qtv_density_error", "qtv_refine_samples",
                     "qtv_face_graph", "qtv_line_pieces", "qtv_piece_curves",
                     "qtv_identify_localize_host", "qtv_thin_pieces", "qtv_node_graph"):
            getattr(L, name).restype = i32
        L.qtv_trace_enable.argtypes = [P, i32]
        L.qtv_trace_filter.argtypes = [P, ctypes.c_char_p]
        L.qtv_trace_read.argtypes = [P, ctypes.POINTER(TraceEntry), i32, ctypes.POINTER(i32), i32]
        for name in ("qtv_create", "qtv_destroy", "qtv_reserve", "qtv_identify", "qtv_localize",
                     "qtv_emit_samples", "qtv_trace_enable", "qtv_trace_filter", "qtv_trace_read"):
            getattr(L, name).restype = i32
        _lib = L
    return _lib


def _check(rc):
    if rc < 0:
        raise QtvError(rc, lib().qtv_last_error_string().decode())
    return rc


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    import torch

    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


class Qtv:
    """A libqtv handle bound to one CUDA device."""

    def __init__(self, device: int = 0):
        self.device = device
        h = ctypes.c_void_p()
        _check(lib().qtv_create(ctypes.byref(h), device))
        self.h = h

    def close(self):
        if self.h:
            lib().qtv_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def trace_enable(self, on: bool = True, only: str | None = None):
        """Kernel timing trace on or off; `only` restricts it to one kernel name."""
        _check(lib().qtv_trace_filter(self.h, (only or "").encode()))
        _check(lib().qtv_trace_enable(self.h, 1 if on else 0))

    def trace_read(self, reset: bool = True):
        """{kernel name: (launches, total device ms)} recorded since the last reset."""
        cap = 64
        buf = (TraceEntry * cap)()
        n = ctypes.c_int(0)
        _check(lib().qtv_trace_read(self.h, buf, cap, ctypes.byref(n), 1 if reset else 0))
        return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms))
                for i in range(min(n.value, cap))}

    def configure_sweep(self, variant: int = -1, warps_per_tile: int = 0, stages: int = 0,
                        ctas_per_sm: int = 0):
        """Sweep shape of this handle's single-snapshot calls (qtv_configure_sweep)."""
        _check(lib().qtv_configure_sweep(self.h, int(variant), int(warps_per_tile), int(stages),
                                         int(ctas_per_sm)))

    def inject_scan_hold(self, hold_tile: int = -1, spin_cycles: int = 0):
        """Failure injection (qtv_inject_scan_hold): look-back tile hold_tile of
        the segment scan never publishes, and look-back waits give up after
        spin_cycles SM cycles (0 = default); (-1, 0) restores normal calls."""
        _check(lib().qtv_inject_scan_hold(self.h, int(hold_tile), int(spin_cycles)))

    def reserve(self, shape, max_faces: int):
        g = Grid.of(shape)
        _check(lib().qtv_reserve(self.h, ctypes.byref(g), int(max_faces)))

    # -- identification -------------------------------------------------------------
    def identify_into(self, psi, face_ids, winding, count, stats=None, grid=None, stream=None):
        """Raw call: all tensors preallocated on the device (count: uint64[1])."""
        g = grid or Grid.of(tuple(psi.shape))
        cap = 0 if face_ids is None else face_ids.numel()
        _check(lib().qtv_identify(self.h, ctypes.byref(g), _ptr(psi), _ptr(face_ids),
                                  _ptr(winding), cap, _ptr(count), _ptr(stats),
                                  _stream_ptr(stream)))

    def identify(self, psi, capacity: int | None = None, stats: bool = False, stream=None):
        """Pierced faces of psi (complex64 [nz, ny, nx] on the device).

        Returns (face_ids uint64-as-int64 tensor [n], winding int8 [n], stats dict or None).
        Grows the output and retries when the capacity is too small."""
        import torch

        dev = psi.device
        nz, ny, nx = psi.shape
        if capacity is None:
            capacity = max(1024, int(0.02 * nx * ny * nz))
        count = torch.zeros(1, dtype=torch.int64, device=dev)
        st = torch.zeros(8, dtype=torch.int64, device=dev) if stats else None
        for _ in range(2):
            ids = torch.empty(capacity, dtype=torch.int64, device=dev)
            w = torch.empty(capacity, dtype=torch.int8, device=dev)
            self.identify_into(psi, ids, w, count, st, stream=stream)
            n = int(count.item())
            if n < 0:  # QTV_COUNT_TIMEOUT read as int64
                raise QtvError(ERR_TIMEOUT, "a bounded device wait gave up")
            if n <= capacity:
                break
            capacity = n
        sd = None
        if stats:
            vals = st.cpu().numpy().astype(np.uint64)
            sd = {f[0]: int(v) for f, v in zip(Stats._fields_, vals)}
        return ids[:n], w[:n], sd

    def identify_localize_into(self, psi, face_ids, winding, count, xyz, resid, flags,
                               stats=None, grid=None, stream=None):
        """Raw fused call: identification + plain localization, preallocated outputs."""
        g = grid or Grid.of(tuple(psi.shape))
        cap = 0 if face_ids is None else face_ids.numel()
        _check(lib().qtv_identify_localize(self.h, ctypes.byref(g), _ptr(psi), _ptr(face_ids),
                                           _ptr(winding), cap, _ptr(count), _ptr(xyz),
                                           _ptr(resid), _ptr(flags), _ptr(stats),
                                           _stream_ptr(stream)))

    def identify_localize(self, psi, capacity: int | None = None, stream=None):
        """(face_ids, winding, xyz, resid, flags) of psi in one fused call."""
        import torch

        dev = psi.device
        nz, ny, nx = psi.shape
        if capacity is None:
            capacity = max(1024, int(0.02 * nx * ny * nz))
        count = torch.zeros(1, dtype=torch.int64, device=dev)
        for _ in range(2):
            ids = torch.empty(capacity, dtype=torch.int64, device=dev)
            w = torch.empty(capacity, dtype=torch.int8, device=dev)
            xyz = torch.empty((capacity, 3), dtype=torch.float32, device=dev)
            resid = torch.empty(capacity, dtype=torch.float32, device=dev)
            flags = torch.empty(capacity, dtype=torch.uint8, device=dev)
            self.identify_localize_into(psi, ids, w, count, xyz, resid, flags, stream=stream)
            n = int(count.item())
            if n < 0:  # QTV_COUNT_TIMEOUT read as int64
                raise QtvError(ERR_TIMEOUT, "a bounded device wait gave up")
            if n <= capacity:
                break
            capacity = n
        return ids[:n], w[:n], xyz[:n], resid[:n], flags[:n]

    def identify_localize_host_into(self, psi_host, capacity, out, count, grid=None,
                                    stream=None):
        """End-to-end call from host memory (qtv_identify_localize_host): psi_host a
        pinned complex64 [nz, ny, nx] host tensor, out a pinned uint8 host tensor of
        at least capacity * 32 bytes, count a pinned int64 host tensor of one element.
        Asynchronous: synchronise the stream before reading out and count."""
        g = grid or Grid.of(tuple(psi_host.shape))
        _check(lib().qtv_identify_localize_host(self.h, ctypes.byref(g), _ptr(psi_host),
                                                int(capacity), _ptr(out), _ptr(count),
                                                _stream_ptr(stream)))

    def identify_localize_host(self, psi_host, capacity: int | None = None, stream=None):
        """Samples (numpy SAMPLE_DTYPE records) of a pinned host field, end to end."""
        import torch

        nz, ny, nx = psi_host.shape
        if capacity is None:
            capacity = max(1024, int(0.02 * nx * ny * nz))
        count = torch.zeros(1, dtype=torch.int64, pin_memory=True)
        for _ in range(2):
            out = torch.empty(capacity * 32, dtype=torch.uint8, pin_memory=True)
            self.identify_localize_host_into(psi_host, capacity, out, count, stream=stream)
            (torch.cuda.current_stream() if stream is None else stream).synchronize()
            n = int(count[0])
            if n <= capacity:
                break
            capacity = n
        return out.numpy()[: n * 32].view(SAMPLE_DTYPE)

    # -- localization ---------------------------------------------------------------
    def localize_into(self, psi, face_ids, winding, xyz, resid, flags, n=None, n_dev=None,
                      mode=PLAIN, fallback_resid=1e-3, grid=None, stream=None):
        g = grid or Grid.of(tuple(psi.shape))
        nn = face_ids.numel() if n is None else int(n)
        _check(lib().qtv_localize(self.h, ctypes.byref(g), _ptr(psi), _ptr(face_ids),
                                  _ptr(winding), nn, _ptr(n_dev), int(mode),
                                  float(fallback_resid), _ptr(xyz), _ptr(resid), _ptr(flags),
                                  _stream_ptr(stream)))

    def localize(self, psi, face_ids, winding, mode=PLAIN, fallback_resid=1e-3, grid=None,
                 stream=None):
        import torch

        n = face_ids.numel()
        dev = psi.device
        xyz = torch.empty((n, 3), dtype=torch.float32, device=dev)
        resid = torch.empty(n, dtype=torch.float32, device=dev)
        flags = torch.empty(n, dtype=torch.uint8, device=dev)
        self.localize_into(psi, face_ids, winding, xyz, resid, flags, mode=mode,
                           fallback_resid=fallback_resid, grid=grid, stream=stream)
        return xyz, resid, flags

    # -- batches of snapshots ---------------------------------------------------------
    def batch_plan(self, psis, tune_cache=None, grids=None, stream=None):
        """Plans one pass over the snapshots psis (list of complex64 [nz, ny, nx]
        device tensors, kept alive by the handle); returns the plan's info."""
        n = len(psis)
        gs = (Grid * n)(*[grids[i] if grids else Grid.of(tuple(p.shape)) for i, p in enumerate(psis)])
        ps = (ctypes.c_void_p * n)(*[p.data_ptr() for p in psis])
        path = None if tune_cache is None else str(tune_cache).encode()
        self._batch_psis = list(psis)
        _check(lib().qtv_batch_plan(self.h, n, gs, ps, path, _stream_ptr(stream)))
        return self.batch_info()

    def batch_info(self):
        info = BatchInfo()
        _check(lib().qtv_batch_info_get(self.h, ctypes.byref(info)))
        return info.as_dict()

    def batch_run_into(self, face_ids, winding, offsets, xyz=None, resid=None, flags=None,
                       mode=PLAIN, fallback_resid=1e-3, stream=None):
        """Raw call: preallocated device outputs; offsets int64 [n + 1]."""
        cap = 0 if face_ids is None else face_ids.numel()
        _check(lib().qtv_batch_run(self.h, _ptr(face_ids), _ptr(winding), cap, _ptr(offsets),
                                   _ptr(xyz), _ptr(resid), _ptr(flags), int(mode),
                                   float(fallback_resid), _stream_ptr(stream)))

    def batch_run(self, capacity=None, localize=True, mode=PLAIN, fallback_resid=1e-3,
                  stream=None):
        """Runs the planned batch; returns one dict per snapshot with ids, w and
        (localize) xyz, resid, flags, views into shared output tensors."""
        import torch

        psis = self._batch_psis
        dev = psis[0].device
        if capacity is None:
            capacity = int(self.batch_info()["faces"] * 1.02) + 1024
        n = len(psis)
        while True:
            ids = torch.empty(capacity, dtype=torch.int64, device=dev)
            w = torch.empty(capacity, dtype=torch.int8, device=dev)
            off = torch.zeros(n + 1, dtype=torch.int64, device=dev)
            xyz = resid = fl = None
            if localize:
                xyz = torch.empty((capacity, 3), dtype=torch.float32, device=dev)
                resid = torch.empty(capacity, dtype=torch.float32, device=dev)
                fl = torch.empty(capacity, dtype=torch.uint8, device=dev)
            self.batch_run_into(ids, w, off, xyz, resid, fl, mode, fallback_resid, stream)
            o = off.cpu().numpy().view(np.uint64)
            if o[n] == 0xFFFFFFFFFFFFFFFF:
                raise QtvError(-4, "batch: a bounded device wait gave up")
            if int(o[n]) <= capacity:
                break
            capacity = int(o[n]) + 1024
        out = []
        for i in range(n):
            a, b = int(o[i]), int(o[i + 1])
            d = {"ids": ids[a:b], "w": w[a:b]}
            if localize:
                d.update(xyz=xyz[a:b], resid=resid[a:b], flags=fl[a:b])
            out.append(d)
        return out

    # -- learned locator ------------------------------------------------------------
    def locator_init(self, seed: int = 0):
        _check(lib().qtv_locator_init(self.h, int(seed)))

    def locator_set_tensor_path(self, path: int):
        """Dense layers of forward passes on mma.sync (0) or tcgen05 (1)."""
        _check(lib().qtv_locator_set_tensor_path(self.h, int(path)))

    def locator_get(self):
        """(params float32 [P], adam float32 [2P], step) copied to the host."""
        p = np.zeros(LOCATOR_PARAMS, np.float32)
        a = np.zeros(2 * LOCATOR_PARAMS, np.float32)
        st = ctypes.c_uint64(0)
        _check(lib().qtv_locator_get(self.h, p.ctypes.data, a.ctypes.data, ctypes.byref(st)))
        return p, a, int(st.value)

    def locator_set(self, params, adam=None, step: int = 0):
        p = np.ascontiguousarray(params, dtype=np.float32)
        a = None if adam is None else np.ascontiguousarray(adam, dtype=np.float32)
        _check(lib().qtv_locator_set(self.h, p.ctypes.data, None if a is None else a.ctypes.data,
                                     int(step)))

    def locator_encode(self, psi, face_ids, winding, grid=None, stream=None):
        """(x uint16-as-int16 [n,128] BF16 bits, ok uint8 [n], rms float32 [n])."""
        import torch

        n = face_ids.numel()
        dev = psi.device
        x = torch.empty((n, 128), dtype=torch.int16, device=dev)
        ok = torch.empty(n, dtype=torch.uint8, device=dev)
        rms = torch.empty(n, dtype=torch.float32, device=dev)
        g = grid or Grid.of(tuple(psi.shape))
        _check(lib().qtv_locator_encode(self.h, ctypes.byref(g), _ptr(psi), _ptr(face_ids),
                                        _ptr(winding), n, None, _ptr(x), _ptr(ok), _ptr(rms),
                                        _stream_ptr(stream)))
        return x, ok, rms

    def locator_forward(self, x, stream=None):
        import torch

        n = x.shape[0]
        y = torch.empty((n, 3), dtype=torch.float32, device=x.device)
        _check(lib().qtv_locator_forward(self.h, _ptr(x), n, _ptr(y), _stream_ptr(stream)))
        return y

    def locator_gradients(self, x, targets, stream=None):
        """(grads float32 [P], loss) for one batch (rows a multiple of 64)."""
        import torch

        n = x.shape[0]
        g = torch.empty(LOCATOR_PARAMS, dtype=torch.float32, device=x.device)
        loss = torch.zeros(1, dtype=torch.float32, device=x.device)
        _check(lib().qtv_locator_gradients(self.h, _ptr(x), _ptr(targets), n, _ptr(g), _ptr(loss),
                                           _stream_ptr(stream)))
        return g, loss

    def locator_train_step(self, x, targets, lr: float, loss=None, stream=None):
        """One Adam step on a batch; loss (device float[1]) receives the batch loss."""
        import torch

        if loss is None:
            loss = torch.zeros(1, dtype=torch.float32, device=x.device)
        _check(lib().qtv_locator_train_step(self.h, _ptr(x), _ptr(targets), x.shape[0], float(lr),
                                            _ptr(loss), _stream_ptr(stream)))
        return loss

    def locator_save(self, path: str):
        _check(lib().qtv_locator_save(self.h, path.encode()))

    def locator_load(self, path: str):
        _check(lib().qtv_locator_load(self.h, path.encode()))

    # -- node form of the circulation and the density error ---------------------------
    def node_circulation_into(self, psi, node_ids, circ, count, dense=None, grid=None,
                              stream=None):
        """Raw call: preallocated device outputs (count: uint64[1])."""
        g = grid or Grid.of(tuple(psi.shape))
        cap = 0 if node_ids is None else node_ids.numel()
        _check(lib().qtv_node_circulation(self.h, ctypes.byref(g), _ptr(psi), _ptr(node_ids),
                                          _ptr(circ), cap, _ptr(count), _ptr(dense),
                                          _stream_ptr(stream)))

    def node_circulation(self, psi, capacity: int | None = None, dense: bool = False,
                         stream=None):
        """Vortex nodes of psi by the ring circulation of every node and plane.

        Returns (node_ids int64 [n] ascending, circ int8 [n, 3] = C / (2 pi) of the
        planes xy, yz, zx, dense int8 [3, nz, ny, nx] or None).  Grows the output
        and retries when the capacity is too small."""
        import torch

        dev = psi.device
        nz, ny, nx = psi.shape
        if capacity is None:
            capacity = max(1024, int(0.06 * nx * ny * nz))
        count = torch.zeros(1, dtype=torch.int64, device=dev)
        d = torch.empty((3, nz, ny, nx), dtype=torch.int8, device=dev) if dense else None
        for _ in range(2):
            ids = torch.empty(capacity, dtype=torch.int64, device=dev)
            circ = torch.empty((capacity, 3), dtype=torch.int8, device=dev)
            self.node_circulation_into(psi, ids, circ, count, d, stream=stream)
            n = int(count.item())
            if n <= capacity:
                break
            capacity = n
        return ids[:n], circ[:n], d

    def node_circulation_faces_into(self, shape, face_ids, winding, node_ids, circ, count, tie,
                                    n_dev=None, grid=None, stream=None):
        """Raw call: preallocated device outputs (count: uint64[1], tie: int32[1])."""
        g = grid or Grid.of(tuple(shape))
        cap = 0 if node_ids is None else node_ids.numel()
        _check(lib().qtv_node_circulation_faces(
            self.h, ctypes.byref(g), _ptr(face_ids), _ptr(winding), face_ids.numel(), _ptr(n_dev),
            _ptr(node_ids), _ptr(circ), cap, _ptr(count), _ptr(tie), _stream_ptr(stream)))

    def node_circulation_faces(self, shape, face_ids, winding, capacity: int | None = None,
                               n_dev=None, stream=None):
        """The node form from the face list of identify (same grid shape
        (nz, ny, nx)): (node_ids int64 [n] ascending, circ int8 [n, 3], tie);
        tie true means a face of winding 2 was met and the lists are not
        valid (use node_circulation)."""
        import torch

        dev = face_ids.device
        if capacity is None:
            capacity = max(1024, 3 * face_ids.numel())
        count = torch.zeros(1, dtype=torch.int64, device=dev)
        tie = torch.zeros(1, dtype=torch.int32, device=dev)
        for _ in range(2):
            ids = torch.empty(capacity, dtype=torch.int64, device=dev)
            circ = torch.empty((capacity, 3), dtype=torch.int8, device=dev)
            self.node_circulation_faces_into(shape, face_ids, winding, ids, circ, count, tie,
                                             n_dev=n_dev, stream=stream)
            n = int(count.item())
            if n <= capacity:
                break
            capacity = n
        return ids[:n], circ[:n], bool(int(tie.item()))

    def density_error(self, psi, xyz, n_dev=None, want_rho: bool = False, grid=None,
                      stream=None):
        """Eq. 7 at the points xyz (float32 [n, 3] on the device).

        Returns (e, mean |rho| over the points, rho_bar) as floats, plus rho
        (float32 [n]) when want_rho."""
        import torch

        g = grid or Grid.of(tuple(psi.shape))
        n = xyz.shape[0]
        out = torch.zeros(3, dtype=torch.float64, device=psi.device)
        rho = torch.empty(max(n, 1), dtype=torch.float32, device=psi.device) if want_rho else None
        _check(lib().qtv_density_error(self.h, ctypes.byref(g), _ptr(psi),
                                       _ptr(xyz) if n else None, n, _ptr(n_dev), _ptr(rho),
                                       _ptr(out), _stream_ptr(stream)))
        e, m, rb = (float(v) for v in out.cpu().tolist())
        return (e, m, rb, rho[:n]) if want_rho else (e, m, rb)

    def refine_samples(self, psi, xyz0=None, face_ids=None, n_dev=None, max_iter: int = 200,
                       tol: float = 1e-7, grid=None, stream=None):
        """Sample refinement of Sec. 3.3.3 from points xyz0 (float32 [n, 3], world
        coordinates) or from the centres of faces face_ids.

        Returns dict of device tensors: xyz [n, 3], rho [n], t [n, 3], detj [n],
        iters int32 [n], flags uint8 [n] (REFINE_* bits)."""
        import torch

        g = grid or Grid.of(tuple(psi.shape))
        src = xyz0 if xyz0 is not None else face_ids
        n = src.shape[0]
        dev = psi.device
        out = {"xyz": torch.empty((n, 3), dtype=torch.float32, device=dev),
               "rho": torch.empty(n, dtype=torch.float32, device=dev),
               "t": torch.empty((n, 3), dtype=torch.float32, device=dev),
               "detj": torch.empty(n, dtype=torch.float32, device=dev),
               "iters": torch.empty(n, dtype=torch.int32, device=dev),
               "flags": torch.empty(n, dtype=torch.uint8, device=dev)}
        _check(lib().qtv_refine_samples(self.h, ctypes.byref(g), _ptr(psi), _ptr(xyz0),
                                        _ptr(face_ids), n, _ptr(n_dev), int(max_iter),
                                        float(tol), _ptr(out["xyz"]), _ptr(out["rho"]),
                                        _ptr(out["t"]), _ptr(out["detj"]), _ptr(out["iters"]),
                                        _ptr(out["flags"]), _stream_ptr(stream)))
        return out

    def face_graph(self, shape, face_ids, n_dev=None, grid=None, stream=None):
        """Adjacency (faces sharing a unit cell) and connected components of a
        pierced-face list (ascending ids) on a grid of the given [nz, ny, nx] shape.

        Returns (nbr int32 [n, 10] with -1 for none, deg uint8 [n], comp int32 [n]
        = lowest face index of the component, number of components)."""
        import torch

        g = grid or Grid.of(tuple(shape))
        n = face_ids.numel()
        dev = face_ids.device
        nbr = torch.empty((max(n, 1), 10), dtype=torch.int32, device=dev)
        deg = torch.empty(max(n, 1), dtype=torch.uint8, device=dev)
        comp = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        nc = torch.zeros(1, dtype=torch.int64, device=dev)
        _check(lib().qtv_face_graph(self.h, ctypes.byref(g), _ptr(face_ids), n, _ptr(n_dev),
                                    _ptr(nbr), _ptr(deg), _ptr(comp), _ptr(nc),
                                    _stream_ptr(stream)))
        k = int(nc.item())
        if k < 0:
            raise QtvError(ERR_TIMEOUT, "a bounded union-find retry loop gave up")
        return nbr[:n], deg[:n], comp[:n], k

    def box_reduce(self, nbr, deg, xyz, box: float = 4.0, max_passes: int = 10, n_dev=None,
                   stream=None):
        """Box-mean reduction of a sample graph (qtv_box_reduce): nbr / deg as
        from face_graph or node_graph, xyz float32 [n, 3] non-negative positions.

        Returns (label int32 [n] = lowest node index of each node's cluster,
        reps int64 [c] = the cluster labels in ascending order, xyz float64
        [c, 3] = their mean positions, passes)."""
        import torch

        n = xyz.shape[0]
        dev = xyz.device
        label = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        out = torch.empty((max(n, 1), 3), dtype=torch.float64, device=dev)
        counts = torch.zeros(2, dtype=torch.int64, device=dev)
        _check(lib().qtv_box_reduce(self.h, n, _ptr(n_dev), _ptr(nbr), _ptr(deg),
                                    int(nbr.shape[1]) if n else 10, _ptr(xyz), float(box),
                                    int(max_passes), _ptr(label), _ptr(out), _ptr(counts),
                                    _stream_ptr(stream)))
        c = counts.cpu()
        if int(c[0]) < 0:
            raise QtvError(ERR_TIMEOUT, "a bounded union-find retry loop gave up")
        label = label[:n]
        reps = torch.nonzero(label == torch.arange(n, device=dev, dtype=torch.int32))[:, 0]
        assert reps.numel() == int(c[0])
        return label, reps, out[reps], int(c[1])

    def node_graph(self, shape, node_ids, n_dev=None, grid=None, stream=None):
        """Graph of vortex nodes (6-connectivity) and its components: (nbr int32
        [n, 6] with -1 for none, deg uint8 [n], comp int32 [n], number of components)."""
        import torch

        g = grid or Grid.of(tuple(shape))
        n = node_ids.numel()
        dev = node_ids.device
        nbr = torch.empty((max(n, 1), 6), dtype=torch.int32, device=dev)
        deg = torch.empty(max(n, 1), dtype=torch.uint8, device=dev)
        comp = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        nc = torch.zeros(1, dtype=torch.int64, device=dev)
        _check(lib().qtv_node_graph(self.h, ctypes.byref(g), _ptr(node_ids), n, _ptr(n_dev),
                                    _ptr(nbr), _ptr(deg), _ptr(comp), _ptr(nc),
                                    _stream_ptr(stream)))
        k = int(nc.item())
        if k < 0:
            raise QtvError(ERR_TIMEOUT, "a bounded union-find retry loop gave up")
        return nbr[:n], deg[:n], comp[:n], k

    def line_pieces(self, nbr, deg, comp, xyz, face_ids=None, winding=None, stream=None):
        """Pieces of the vortex-core lines of a face graph (qtv_line_pieces).

        Returns (pieces: uint8 device tensor [np, 24] of qtv_piece records, use
        pieces_numpy() to read them; nodes: int32 device tensor of sample indices)."""
        import torch

        n = deg.numel()
        dev = deg.device
        counts = torch.zeros(2, dtype=torch.int64, device=dev)
        args = (_ptr(nbr), _ptr(deg), _ptr(comp), _ptr(xyz), _ptr(face_ids), _ptr(winding))
        _check(lib().qtv_line_pieces(self.h, n, None, *args, None, 0, None, 0, _ptr(counts),
                                     _stream_ptr(stream)))
        npc, nnd = (int(v) for v in counts.cpu().tolist())
        pieces = torch.empty((max(npc, 1), 24), dtype=torch.uint8, device=dev)
        nodes = torch.empty(max(nnd, 1), dtype=torch.int32, device=dev)
        _check(lib().qtv_line_pieces(self.h, n, None, *args, _ptr(pieces), npc, _ptr(nodes), nnd,
                                     _ptr(counts), _stream_ptr(stream)))
        return pieces[:npc], nodes[:nnd]

    def piece_curves(self, xyz, nodes, pieces, per_segment: int = 8, stream=None):
        """Catmull-Rom curves of line pieces (qtv_piece_curves): (curve float32 [m, 3],
        first point of each piece int64 [np], length float32 [np])."""
        import torch

        npc = pieces.shape[0]
        dev = xyz.device
        first = torch.empty(max(npc, 1), dtype=torch.int64, device=dev)
        length = torch.empty(max(npc, 1), dtype=torch.float32, device=dev)
        total = torch.zeros(1, dtype=torch.int64, device=dev)
        args = (_ptr(xyz), _ptr(nodes), _ptr(pieces), npc, None, int(per_segment))
        _check(lib().qtv_piece_curves(self.h, *args, None, 0, _ptr(first), _ptr(length),
                                      _ptr(total), _stream_ptr(stream)))
        m = int(total.item())
        curve = torch.empty((max(m, 1), 3), dtype=torch.float32, device=dev)
        _check(lib().qtv_piece_curves(self.h, *args, _ptr(curve), m, _ptr(first), _ptr(length),
                                      _ptr(total), _stream_ptr(stream)))
        return curve[:m], first[:npc], length[:npc]

    def thin_pieces(self, xyz, nodes, pieces, box: float, stream=None):
        """Arc-length thinning of line pieces (qtv_thin_pieces): (means float32 [m, 3],
        pieces over the means as a uint8 tensor [np, 24] of qtv_piece records)."""
        import torch

        npc = pieces.shape[0]
        nn = nodes.numel()
        dev = xyz.device
        out = torch.empty((max(nn, 1), 3), dtype=torch.float32, device=dev)
        outp = torch.empty((max(npc, 1), 24), dtype=torch.uint8, device=dev)
        total = torch.zeros(1, dtype=torch.int64, device=dev)
        _check(lib().qtv_thin_pieces(self.h, _ptr(xyz), _ptr(nodes), _ptr(pieces), npc, nn,
                                     float(box), _ptr(out), nn, _ptr(outp), _ptr(total),
                                     _stream_ptr(stream)))
        m = int(total.item())
        return out[:m], outp[:npc]

    # -- emission -------------------------------------------------------------------
    def emit_samples(self, face_ids, winding, xyz, resid, flags, out=None, stream=None):
        """Samples packed into host memory (numpy structured array, SAMPLE_DTYPE)."""
        import torch

        n = face_ids.numel()
        if out is None:
            out = torch.empty(n * 32, dtype=torch.uint8, pin_memory=True)
        _check(lib().qtv_emit_samples(self.h, n, _ptr(face_ids), _ptr(winding), _ptr(xyz),
                                      _ptr(resid), _ptr(flags), _ptr(out), _stream_ptr(stream)))
        (torch.cuda.current_stream() if stream is None else stream).synchronize()
        return out.numpy()[: n * 32].view(SAMPLE_DTYPE)
