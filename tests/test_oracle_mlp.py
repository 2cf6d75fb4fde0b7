"""Pins of the learned-locator oracle (oracle/mlp.py) against the mathematics:

* gradients of the loss equal central finite differences (relative 1e-6);
* one Adam step equals the closed form for the first step (m/(sqrt(v)+eps)
  with bias correction gives lr * sign(g) for |g| >> eps);
* the encoding has unit mean |psi|^2, places the face at block nodes
  a, b in {1, 2}, c = 1, turns a W = -1 face into the W = +1 encoding of the
  conjugate field, and is the same for the three orientations when the field
  is rotated so that the face frame becomes (x, y, z).
"""
import numpy as np
import pytest

import oracle
from oracle import mlp


@pytest.fixture(scope="module")
def small_problem():
    rng = np.random.default_rng(3)
    p = mlp.init_params(5)
    x = rng.standard_normal((7, 128))
    t = rng.standard_normal((7, 3))
    return p, x, t


def test_gradients_match_central_differences(small_problem):
    p, x, t = small_problem
    loss, g = mlp.loss_and_grads(p, x, t)
    rng = np.random.default_rng(9)
    for key in ("W1", "b1", "W2", "b2", "W3", "b3"):
        flat = p[key].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            h = 1e-6 * max(1.0, abs(flat[idx]))
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = mlp.loss_and_grads(p, x, t)
            flat[idx] = old - h
            lm, _ = mlp.loss_and_grads(p, x, t)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[key].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)) + 1e-9, (key, idx, fd, an)


def test_first_adam_step_is_lr_times_sign(small_problem):
    p, x, t = small_problem
    q = {k: v.copy() for k, v in p.items()}
    _, g = mlp.loss_and_grads(q, x, t)
    m = {k: np.zeros_like(v) for k, v in q.items()}
    v = {k: np.zeros_like(v) for k, v in q.items()}
    mlp.adam_step(q, g, m, v, t=1, lr=1e-3, eps=1e-12)
    for key in q:
        big = np.abs(g[key]) > 1e-6
        assert np.allclose((p[key] - q[key])[big], 1e-3 * np.sign(g[key][big]), rtol=1e-6)


def _field(seed, shape=(10, 11, 12)):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)


def test_encoding_normalisation_and_face_position():
    psi = _field(1)
    nz, ny, nx = psi.shape
    i, j, k = 4, 5, 3
    fid = np.array([(((k * ny + j) * nx + i) << 2) | 0], np.uint64)
    x, ok, rms = mlp.encode(psi, fid, np.array([1], np.int8))
    assert ok[0]
    assert abs(np.sum(x[0] ** 2) / 64 - 1.0) < 1e-12
    z = (x[0, 0::2] + 1j * x[0, 1::2]).reshape(4, 4, 4) * rms[0]  # [c][b][a]
    # the minimum corner is rotated onto the positive real axis
    ph = np.conj(psi[k, j, i]) / abs(psi[k, j, i])
    assert abs(z[1, 1, 1].imag) < 1e-12 and z[1, 1, 1].real > 0
    # face corners of an xy face at block (a, b) in {1,2}, c = 1
    assert np.allclose(z[1, 1, 1], psi[k, j, i] * ph) and np.allclose(z[1, 1, 2], psi[k, j, i + 1] * ph)
    assert np.allclose(z[1, 2, 2], psi[k, j + 1, i + 1] * ph)
    assert np.allclose(z[1, 2, 1], psi[k, j + 1, i] * ph)
    assert np.allclose(z[0, 0, 0], psi[k - 1, j - 1, i - 1] * ph)


def test_encoding_is_phase_invariant():
    psi = _field(6)
    nz, ny, nx = psi.shape
    fid = np.array([(((4 * ny + 5) * nx + 6) << 2) | 2], np.uint64)
    w = np.array([1], np.int8)
    x0, _, _ = mlp.encode(psi, fid, w)
    x1, _, _ = mlp.encode((psi * np.complex64(np.exp(1j * 2.1))).astype(np.complex64), fid, w)
    assert np.allclose(x0, x1, atol=1e-6)


def test_encoding_of_negative_winding_is_conjugate():
    psi = _field(2)
    nz, ny, nx = psi.shape
    fid = np.array([(((4 * ny + 4) * nx + 4) << 2) | 1], np.uint64)
    xm, _, _ = mlp.encode(psi, fid, np.array([-1], np.int8))
    xp, _, _ = mlp.encode(np.conj(psi), fid, np.array([1], np.int8))
    assert np.allclose(xm, xp)


def test_encoding_is_frame_covariant():
    psi = _field(3, shape=(9, 9, 9))  # [z][y][x]
    n = 9
    i, j, k = 3, 4, 5

    def fid(i, j, k, o):
        return np.array([(((k * n + j) * n + i) << 2) | o], np.uint64)

    w = np.array([1], np.int8)
    x0, _, _ = mlp.encode(psi, fid(i, j, k, 0), w)
    # yz face: frame (u, v, n) = (y, z, x).  Rotate so that y -> x', z -> y',
    # x -> z': psi'[z'][y'][x'] = psi[y'][x'][z'] ... psi'(x', y', z') = psi(z', x', y')
    rot = np.transpose(psi, (2, 0, 1))  # rot[x][z][y] -> index [z'=x][y'=z][x'=y]
    x1, _, _ = mlp.encode(rot, fid(j, k, i, 0), w)
    y1, _, _ = mlp.encode(psi, fid(i, j, k, 1), w)
    assert np.allclose(x1, y1)
    # zx face: frame (z, x, y): psi''(x'', y'', z'') = psi(y'', z'', x'')
    rot2 = np.transpose(psi, (1, 2, 0))  # index [z''=y][y''=x][x''=z]
    x2, _, _ = mlp.encode(rot2, fid(k, i, j, 0), w)
    y2, _, _ = mlp.encode(psi, fid(i, j, k, 2), w)
    assert np.allclose(x2, y2)
    assert not np.allclose(x0, y1)


def test_encoding_rejects_boundary_faces():
    psi = _field(4)
    nz, ny, nx = psi.shape
    fid = np.array([(((0 * ny + 5) * nx + 5) << 2) | 0, (((5 * ny + 5) * nx + 5) << 2) | 0],
                   np.uint64)
    _, ok, _ = mlp.encode(psi, fid, np.array([1, 1], np.int8))
    assert list(ok) == [False, True]
