"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
(via the thin binding) and compare it with the oracle on the same input."""
from __future__ import annotations

import numpy as np

import oracle


def split_ids(ids, shape):
    nz, ny, nx = shape
    ids = np.asarray(ids, dtype=np.uint64)
    o = (ids & np.uint64(3)).astype(np.int64)
    lin = (ids >> np.uint64(2)).astype(np.int64)
    i = lin % nx
    j = (lin // nx) % ny
    k = lin // (nx * ny)
    return o, i, j, k


def dense_from_list(ids, w, shape, k0=0, k1=None):
    """Dense [3][k1-k0][ny][nx] winding field from a face list (faces outside
    the plane range are dropped)."""
    nz, ny, nx = shape
    k1 = nz if k1 is None else k1
    out = np.zeros((3, k1 - k0, ny, nx), np.int8)
    o, i, j, k = split_ids(ids, shape)
    sel = (k >= k0) & (k < k1)
    out[o[sel], k[sel] - k0, j[sel], i[sel]] = np.asarray(w)[sel]
    return out


def compare_windings(gpu_dense, ora_w, ora_fl):
    """Bit-exact comparison on every face the oracle does not flag ambiguous.
    Returns (n_mismatch_unambiguous, n_ambiguous, n_ambiguous_differing)."""
    amb = (ora_fl & oracle.AMBIGUOUS) != 0
    diff = gpu_dense != ora_w
    return int(np.count_nonzero(diff & ~amb)), int(amb.sum()), int(np.count_nonzero(diff & amb))


def gpu_identify(q, psi_dev, stats=False, capacity=None):
    ids, w, st = q.identify(psi_dev, capacity=capacity, stats=stats)
    return ids.cpu().numpy().view(np.uint64), w.cpu().numpy(), st


def position_tolerance(xyz):
    """1e-4 h plus half an FP32 ulp of the absolute coordinate (the output is
    FP32 in grid units)."""
    return 1e-4 + np.abs(xyz) * 2.0 ** -24 * 2


def compare_positions(gpu_xyz, ora, ora_ok):
    tol = position_tolerance(ora["xyz"])
    err = np.abs(gpu_xyz.astype(np.float64) - ora["xyz"])
    bad = np.any(err > tol, axis=1) & ora_ok
    return int(bad.sum()), float(np.max(err[ora_ok])) if ora_ok.any() else 0.0
