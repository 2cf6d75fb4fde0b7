"""The oracle against its stored expected values (tests/golden/, written by
tests/golden/make_golden.py from the oracle alone): the pierced faces of the
64^3 analytic line and ring field (Eq. 5, Sec. 2.2.2) and their samples (the
zero of the bilinear interpolant, Eq. 6, Sec. 3.3.3).

A change to the oracle's arithmetic that moves any of these values has to be
justified by the passage it follows and the fixture rewritten by the script.
The file also carries facts fixed independently of the oracle, checked here:
the line along z pierces one xy face per plane with winding +1 at the analytic
axis, every sample lies on its own face, and every residual is an FP64 zero.
"""
import os

import numpy as np

import synth

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "analytic_line_ring_64.txt")


def _load():
    rows = np.loadtxt(GOLDEN, comments="#", dtype=object)
    ids = np.array([int(v) for v in rows[:, 0]], dtype=np.uint64)
    w = rows[:, 1].astype(np.int64)
    xyz = rows[:, 2:5].astype(np.float64)
    resid = rows[:, 5].astype(np.float64)
    flags = rows[:, 6].astype(np.int64)
    return ids, w, xyz, resid, flags


def test_oracle_reproduces_the_stored_faces_and_samples():
    import importlib.util

    spec = importlib.util.spec_from_file_location(
        "make_golden", os.path.join(HERE, "golden", "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    shape, ids, wn, loc = mg.analytic_rows()
    gids, gw, gxyz, gres, gfl = _load()
    assert shape == (64, 64, 64)
    assert np.array_equal(ids, gids)
    assert np.array_equal(wn.astype(np.int64), gw)
    assert np.max(np.abs(loc["xyz"] - gxyz)) < 1e-12
    assert np.array_equal(loc["flags"].astype(np.int64), gfl)
    assert np.all(loc["resid"] <= 1e-20)


def test_stored_values_agree_with_the_analytic_field():
    ids, w, xyz, resid, flags = _load()
    n = 64
    o = (ids & np.uint64(3)).astype(np.int64)
    lin = (ids >> np.uint64(2)).astype(np.int64)
    i, j, k = lin % n, (lin // n) % n, lin // (n * n)
    # the straight line along z through (31.37, 30.81): one xy face per plane,
    # the face containing the axis, winding +1, sample within 0.02 h of the axis
    # (the field is zero on the axis; its bilinear interpolant, of a factor
    # r / sqrt(r^2 + xi^2) times the ring factor, is zero nearby)
    line = (o == 0) & (i == 31) & (j == 30)
    assert sorted(k[line].tolist()) == list(range(n))
    assert np.all(w[line] == 1)
    assert np.max(np.abs(xyz[line, 0] - 31.37)) < 2e-2
    assert np.max(np.abs(xyz[line, 1] - 30.81)) < 2e-2
    # every sample lies on its own face (the face's two in-plane axes within
    # [0, 1] of its minimum corner, the normal coordinate on the corner's plane)
    base = np.stack([i, j, k], 1).astype(np.float64)
    d = xyz - base
    normal = np.where(o == 0, 2, np.where(o == 1, 0, 1))
    for a in range(3):
        on = normal == a
        assert np.all(np.abs(d[on, a]) < 1e-12)
        assert np.all((d[~on, a] > -1e-9) & (d[~on, a] < 1 + 1e-9))
    assert np.all(resid <= 1e-20) and np.all(flags == 0)
    # the field is what the script read
    psi = synth.analytic_line_ring()
    assert psi.shape == (n, n, n) and psi.dtype == np.complex64
