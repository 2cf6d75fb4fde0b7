"""Plain FP64 CPU oracle for vortex-core identification and localization.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  It shares no code with
the CUDA path.  ``qtv_oracle.c`` holds identification (Sec. 2.2.2, Eq. 5) and
plaquette localization (Sec. 3.3.3, Eq. 6), the node form of the circulation,
the density of the interpolated field and the refinement of sample points in
the plane normal to the pseudo-vorticity (Sec. 3.3.3); ``graph.py`` holds the graph
pipeline of Sec. 3.1-3.4; ``mlp.py`` holds the learned-locator network in FP64.

Flag bits returned by :func:`identify` (per face):
  AMBIGUOUS  an edge phase difference within 1e-4 rad of +-pi
  ZERO_NODE  a corner with psi == 0 exactly (given phase 0, see qtv_oracle.c)
  NONFINITE  a corner with a NaN/Inf component (W forced to 0)
  ABSENT     the face does not exist (a corner lies outside the grid)
  RESIDUAL   the FP64 circulation sum is not within 1e-9 of 2*pi*W
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

AMBIGUOUS, ZERO_NODE, NONFINITE, ABSENT, RESIDUAL = 1, 2, 4, 8, 16
L_ANOMALOUS, L_ILLCOND = 1, 2
R_CONVERGED, R_NO_TANGENT, R_MAX_ITER = 1, 2, 4

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qtv_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile qtv_oracle.c with gcc (-ffp-contract=off, OpenMP if available)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
            "-Wall", "-o", _LIB + ".tmp", _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i32, i64, f64 = ctypes.c_int, ctypes.c_long, ctypes.c_double
        L.oracle_identify.argtypes = [i32, i32, i32, i32, i32, P, P, P, P]
        L.oracle_identify.restype = i64
        L.oracle_node_circulation.argtypes = [i32, i32, i32, P, P, P]
        L.oracle_node_circulation.restype = None
        L.oracle_localize.argtypes = [i32, i32, i32, P, i64, P, P, f64, P, P, P, P, P, P]
        L.oracle_localize.restype = i64
        L.oracle_density.argtypes = [i32, i32, i32, P, i64, P, P]
        L.oracle_density.restype = None
        L.oracle_refine.argtypes = [i32, i32, i32, P, i64, P, i32, ctypes.c_double, P, P, P, P,
                                    P, P]
        L.oracle_refine.restype = None
        L.oracle_set_threads.argtypes = [i32]
        L.oracle_max_threads.restype = i32
        _lib = L
    return _lib


def _psi_f32(psi: np.ndarray) -> np.ndarray:
    assert psi.ndim == 3 and psi.dtype == np.complex64, "psi must be complex64 [nz][ny][nx]"
    return np.ascontiguousarray(psi)


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))


def max_threads() -> int:
    return int(lib().oracle_max_threads())


def identify(psi: np.ndarray, k0: int = 0, k1: int | None = None, want_circ: bool = False):
    """Winding W and flags of every face with minimum corner in planes [k0, k1).

    Returns (w int8 [3][k1-k0][ny][nx], flags uint8 same shape[, circ f64]).
    """
    psi = _psi_f32(psi)
    nz, ny, nx = psi.shape
    k1 = nz if k1 is None else k1
    nk = k1 - k0
    w = np.zeros((3, nk, ny, nx), np.int8)
    fl = np.zeros((3, nk, ny, nx), np.uint8)
    circ = np.zeros((3, nk, ny, nx), np.float64) if want_circ else None
    bad = lib().oracle_identify(nx, ny, nz, k0, k1, psi.ctypes.data, w.ctypes.data,
                                fl.ctypes.data, circ.ctypes.data if want_circ else None)
    assert bad == 0, f"{bad} faces with a circulation residual above 1e-9"
    return (w, fl, circ) if want_circ else (w, fl)


def node_circulation(psi: np.ndarray):
    """Ring-path circulation per node and plane, and the vortex-node flag."""
    psi = _psi_f32(psi)
    nz, ny, nx = psi.shape
    c = np.zeros((3, nz, ny, nx), np.float64)
    v = np.zeros((nz, ny, nx), np.uint8)
    lib().oracle_node_circulation(nx, ny, nz, psi.ctypes.data, c.ctypes.data, v.ctypes.data)
    return c, v


def face_list(w: np.ndarray, k0: int = 0):
    """Face ids (ascending) and windings of the nonzero entries of a dense field."""
    _, nk, ny, nx = w.shape
    o, kk, j, i = np.nonzero(w)
    lin = ((kk.astype(np.int64) + k0) * ny + j) * nx + i
    ids = (lin.astype(np.uint64) << np.uint64(2)) | o.astype(np.uint64)
    order = np.argsort(ids, kind="stable")
    return ids[order], w[o, kk, j, i][order].astype(np.int8)


def localize(psi: np.ndarray, face_ids: np.ndarray, winding: np.ndarray, h: float = 1.0,
             origin=(0.0, 0.0, 0.0)):
    """Zero of the bilinear interpolant in each listed face.

    Returns dict with uv [n,2], xyz [n,3], resid [n] (|F|^2), detn [n]
    (|det J|/max|corner|^2), flags [n] (L_ANOMALOUS | L_ILLCOND).
    """
    psi = _psi_f32(psi)
    nz, ny, nx = psi.shape
    ids = np.ascontiguousarray(face_ids, dtype=np.uint64)
    w = np.ascontiguousarray(winding, dtype=np.int8)
    n = ids.shape[0]
    uv = np.zeros((n, 2)); xyz = np.zeros((n, 3)); r = np.zeros(n); dn = np.zeros(n)
    fl = np.zeros(n, np.uint8)
    org = np.ascontiguousarray(origin, dtype=np.float64)
    lib().oracle_localize(nx, ny, nz, psi.ctypes.data, n, ids.ctypes.data, w.ctypes.data,
                          float(h), org.ctypes.data, uv.ctypes.data, xyz.ctypes.data,
                          r.ctypes.data, dn.ctypes.data, fl.ctypes.data)
    return {"uv": uv, "xyz": xyz, "resid": r, "detn": dn, "flags": fl}


def density(psi: np.ndarray, points: np.ndarray) -> np.ndarray:
    """Trilinearly interpolated |psi|^2 at points given in grid coordinates."""
    psi = _psi_f32(psi)
    nz, ny, nx = psi.shape
    p = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
    rho = np.zeros(p.shape[0])
    lib().oracle_density(nx, ny, nz, psi.ctypes.data, p.shape[0], p.ctypes.data, rho.ctypes.data)
    return rho


def refine(psi: np.ndarray, x0: np.ndarray, max_iter: int = 200, tol: float = 1e-7):
    """Sample refinement of Sec. 3.3.3: gradient descent of rho in the plane
    through each x0 (grid coordinates, [n, 3]) normal to the pseudo-vorticity.

    Returns dict: xyz [n, 3], rho [n], t [n, 3] (unit tangent), detj [n] (2x2
    in-plane Jacobian determinant of psi at the result), iters [n], flags [n]
    (R_CONVERGED, R_NO_TANGENT, R_MAX_ITER)."""
    psi = _psi_f32(psi)
    nz, ny, nx = psi.shape
    p = np.ascontiguousarray(x0, dtype=np.float64).reshape(-1, 3)
    n = p.shape[0]
    xyz = np.zeros((n, 3))
    rho = np.zeros(n)
    t = np.zeros((n, 3))
    dj = np.zeros(n)
    it = np.zeros(n, np.int32)
    fl = np.zeros(n, np.uint8)
    lib().oracle_refine(nx, ny, nz, psi.ctypes.data, n, p.ctypes.data, int(max_iter), float(tol),
                        xyz.ctypes.data, rho.ctypes.data, t.ctypes.data, dj.ctypes.data,
                        it.ctypes.data, fl.ctypes.data)
    return {"xyz": xyz, "rho": rho, "t": t, "detj": dj, "iters": it, "flags": fl}
