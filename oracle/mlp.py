"""FP64 oracle of the learned locator (no counterpart in the paper; the paper's
localization is the density-guided optimisation of Sec. 3.3.3, Eq. 6, which
this network is trained to imitate).

TEST INFRASTRUCTURE ONLY (tests, smoke, bench CPU baseline).  Plain numpy,
written from the definitions:

* encoding -- the 4 x 4 x 4 neighbourhood of a pierced face in the face frame
  (u, v, n) = (x, y, z) for xy faces, (y, z, x) for yz faces, (z, x, y) for zx
  faces; node (a, b, c) of the block is grid node
  min_corner + (a - 1) e_u + (b - 1) e_v + (c - 1) e_n, so the face spans
  a, b in {1, 2} at c = 1.  psi is conjugated when W = -1 (the zero of the
  interpolant does not move and the winding becomes +1), multiplied by
  conj(P0)/|P0| with P0 the value at the face's minimum corner (block node
  (1, 1, 1); a constant phase does not move the zero either) and divided by
  the RMS of |psi| over the block.  Input vector index ((c * 4 + b) * 4 + a) * 2 +
  {0: Re, 1: Im}.  Faces whose block leaves the grid are not encoded.
* network -- y = W3 relu(W2 relu(W1 x + b1) + b2) + b3, sizes 128-256-256-3;
  W_l has shape (out, in).
* loss -- mean over the batch of the squared error summed over the 3 outputs.
* Adam -- standard bias-corrected moments (Kingma & Ba 2015).
"""
from __future__ import annotations

import numpy as np

SIZES = (128, 256, 256, 3)


def init_params(seed: int = 0):
    """He-normal weights, zero biases (FP64)."""
    rng = np.random.default_rng(seed)
    p = {}
    for l, (fi, fo) in enumerate(zip(SIZES[:-1], SIZES[1:]), start=1):
        p[f"W{l}"] = rng.standard_normal((fo, fi)) * np.sqrt(2.0 / fi)
        p[f"b{l}"] = np.zeros(fo)
    return p


def forward(p, x):
    """Returns (y, cache) for inputs x [B, 128]."""
    z1 = x @ p["W1"].T + p["b1"]
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ p["W2"].T + p["b2"]
    a2 = np.maximum(z2, 0.0)
    y = a2 @ p["W3"].T + p["b3"]
    return y, (x, z1, a1, z2, a2)


def loss_and_grads(p, x, t):
    """Mean squared error (summed over outputs, averaged over the batch) and its
    gradients by the chain rule."""
    y, (x, z1, a1, z2, a2) = forward(p, x)
    B = x.shape[0]
    diff = y - t
    loss = float(np.sum(diff * diff) / B)
    dy = 2.0 * diff / B
    g = {"W3": dy.T @ a2, "b3": dy.sum(0)}
    da2 = dy @ p["W3"]
    dz2 = da2 * (z2 > 0)
    g["W2"] = dz2.T @ a1
    g["b2"] = dz2.sum(0)
    da1 = dz2 @ p["W2"]
    dz1 = da1 * (z1 > 0)
    g["W1"] = dz1.T @ x
    g["b1"] = dz1.sum(0)
    return loss, g


def adam_step(p, g, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update of every parameter in place; t is the 1-based step."""
    for key in p:
        m[key] = beta1 * m[key] + (1 - beta1) * g[key]
        v[key] = beta2 * v[key] + (1 - beta2) * g[key] * g[key]
        mh = m[key] / (1 - beta1 ** t)
        vh = v[key] / (1 - beta2 ** t)
        p[key] = p[key] - lr * mh / (np.sqrt(vh) + eps)


# face frame axes: (u, v, n) as grid axes (0 = x, 1 = y, 2 = z)
_FRAME = {0: (0, 1, 2), 1: (1, 2, 0), 2: (2, 0, 1)}


def encode(psi: np.ndarray, face_ids: np.ndarray, winding: np.ndarray):
    """Neighbourhood encodings of faces; returns (x [n, 128] float64, ok [n]
    bool, rms [n]).  Rows of faces whose block leaves the grid are zero."""
    nz, ny, nx = psi.shape
    ids = np.asarray(face_ids, dtype=np.uint64)
    n = ids.shape[0]
    out = np.zeros((n, 128))
    ok = np.zeros(n, bool)
    rms = np.zeros(n)
    dims = (nx, ny, nz)
    for f in range(n):
        fid = int(ids[f])
        o = fid & 3
        lin = fid >> 2
        corner = (lin % nx, (lin // nx) % ny, lin // (nx * ny))
        au, av, an = _FRAME[o]
        vals = np.zeros((4, 4, 4), np.complex128)
        inside = True
        for c in range(4):
            for b in range(4):
                for a in range(4):
                    pos = list(corner)
                    pos[au] += a - 1
                    pos[av] += b - 1
                    pos[an] += c - 1
                    if not all(0 <= pos[d] < dims[d] for d in range(3)):
                        inside = False
                        break
                    vals[c, b, a] = complex(psi[pos[2], pos[1], pos[0]])
                if not inside:
                    break
            if not inside:
                break
        if not inside:
            continue
        if int(winding[f]) == -1:
            vals = np.conj(vals)
        p0 = vals[1, 1, 1]
        if abs(p0) > 0:
            vals = vals * (np.conj(p0) / abs(p0))
        r = np.sqrt(np.mean(np.abs(vals) ** 2))
        if not r > 0:
            continue
        vals = vals / r
        out[f, 0::2] = vals.real.reshape(-1)
        out[f, 1::2] = vals.imag.reshape(-1)
        ok[f] = True
        rms[f] = r
    return out, ok, rms
