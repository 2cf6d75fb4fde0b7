"""Training and evaluation driver of the learned locator.

Only orchestration lives here: fields come from ``synth``, faces and plain
positions from qtv_identify_localize, encodings, forward and backward passes
and Adam steps from the library's kernels (qtv_locator_*).  Labels are the
face coordinates (u, v, 0) of the plain localization (Sec. 3.3.3, Eq. 6) of a
clean field; inputs are the encodings of the same faces in a field with 5%
multiplicative amplitude noise (phases and windings unchanged), so the network
is trained to recover the clean cores from noisy data.
"""
from __future__ import annotations

import numpy as np

import synth

from . import FLAG_ANOMALOUS, Qtv


def face_uv(face_ids, xyz, shape, h=1.0, origin=(0.0, 0.0, 0.0)):
    """Face coordinates (u, v) of positions xyz on their faces (torch)."""
    import torch

    nz, ny, nx = shape
    ids = face_ids
    o = (ids & 3).long()
    lin = ids >> 2
    i = (lin % nx).float()
    j = ((lin // nx) % ny).float()
    k = (lin // (nx * ny)).float()
    g = (xyz - torch.tensor(origin, device=xyz.device)) / h
    gx, gy, gz = g[:, 0], g[:, 1], g[:, 2]
    u = torch.where(o == 0, gx - i, torch.where(o == 1, gy - j, gz - k))
    v = torch.where(o == 0, gy - j, torch.where(o == 1, gz - k, gx - i))
    return torch.stack([u, v], 1)


def field_pair(seed: int, n: int, waves: int, noise: float, device):
    """(clean, noisy) random-wave fields of one seed."""
    clean = synth.random_waves((n, n, n), synth.wave_spec(seed, waves), device=device)
    noisy = synth.multiplicative_noise(clean, seed + 100000, noise) if noise > 0 else clean
    return clean, noisy


def make_examples(q: Qtv, clean, noisy):
    """Encodings of noisy-field neighbourhoods and clean plain labels.

    Returns dict with x (BF16 bits [m,128]), t (float32 [m,3]: u, v, 0),
    ids, winding, and the clean plain positions; only faces whose block lies in
    the grid and whose plain solve found a zero are kept."""
    import torch

    ids, w, xyz, resid, flags = q.identify_localize(clean)
    x, ok, rms = q.locator_encode(noisy, ids, w)
    keep = (ok != 0) & ((flags & FLAG_ANOMALOUS) == 0)
    uv = face_uv(ids, xyz, tuple(clean.shape))
    t = torch.cat([uv, torch.zeros_like(uv[:, :1])], 1)
    return {"x": x[keep].contiguous(), "t": t[keep].contiguous(), "ids": ids[keep].contiguous(),
            "w": w[keep].contiguous(), "xyz": xyz[keep].contiguous()}


def train(q: Qtv, x, t, steps: int, batch: int = 4096, lr: float = 2e-3, seed: int = 0,
          lr_final: float = 1e-4, log_every: int = 0):
    """Adam on shuffled minibatches with a cosine learning-rate decay; returns
    the per-step losses (host floats)."""
    import torch

    m = x.shape[0]
    nb = m // batch
    if nb < 1:
        raise ValueError("fewer examples than one batch")
    gen = torch.Generator(device="cpu").manual_seed(seed)
    losses = []
    loss_buf = torch.zeros(steps, dtype=torch.float32, device=x.device)
    perm = torch.randperm(m, generator=gen).to(x.device)
    for s in range(steps):
        b = s % nb
        if b == 0 and s > 0:
            perm = torch.randperm(m, generator=gen).to(x.device)
        idx = perm[b * batch:(b + 1) * batch]
        xb = x[idx].contiguous()
        tb = t[idx].contiguous()
        c = 0.5 * (1 + np.cos(np.pi * s / max(1, steps - 1)))
        rate = lr_final + (lr - lr_final) * c
        q.locator_train_step(xb, tb, rate, loss=loss_buf[s:s + 1])
        if log_every and s % log_every == 0:
            print(f"step {s} loss {float(loss_buf[s]):.3e}")
    return loss_buf.cpu().numpy()


TRAIN_SEEDS = tuple(range(101, 113))


def fit(q: Qtv, seeds=TRAIN_SEEDS, n: int = 256, waves: int = 4096, noise: float = 0.05,
        steps: int = 20000, batch: int = 4096, lr: float = 2e-3, init_seed: int = 1):
    """Trains the handle's locator from scratch on the random-wave fields of the
    given seeds (12 seeds of 256^3 give about 2.0e6 faces); returns the losses."""
    import torch

    ex = [make_examples(q, *field_pair(s, n, waves, noise, "cuda")) for s in seeds]
    x = torch.cat([e["x"] for e in ex])
    t = torch.cat([e["t"] for e in ex])
    del ex
    q.locator_init(init_seed)
    return train(q, x, t, steps=steps, batch=batch, lr=lr)


def rms_h(a, b):
    """Root mean square distance (rows of a, b) as a float."""
    import torch

    return float(torch.sqrt(torch.mean(torch.sum((a - b) ** 2, 1))))
