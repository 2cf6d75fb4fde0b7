"""Seeded synthetic wave-function fields (test and benchmark inputs).

This module only makes inputs.  It holds none of the arithmetic of the
identification or localization methods, and both the CUDA path and the oracle
consume what it makes.  The paper's 2048^3 NLKG snapshots (Sec. 2.1.3) are not
available, so these fields stand in for them: complex64 grids whose vortex
cores are resolved by a few cells, as in the paper's data (healing length of
at least two grid cells, Sec. 5 "Vectorization uncertainty").

Fields are complex64 arrays indexed [z][y][x] (x fastest), grid spacing h = 1,
node (i, j, k) at physical position (i, j, k).

* :func:`analytic_line_ring` -- product of one straight vortex line along z
  and one vortex ring in a z-plane, each factor r e^{i phi} / sqrt(r^2 + xi^2).
* :func:`random_waves` -- psi = sum_n A_n exp(i k_n . x) with |k_n| uniform in a
  shell, directions uniform on the sphere, A_n ~ CN(0, 1/W), so <|psi|^2> = 1.
  Random-wave fields carry a dense tangle of vortex lines (phase
  singularities), the synthetic stand-in for quantum turbulence.
* :func:`multiplicative_noise` -- psi * (1 + level * g), g ~ N(0, 1) real.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

__all__ = ["analytic_line_ring", "WaveSpec", "wave_spec", "random_waves", "random_waves_numpy",
           "multiplicative_noise", "config_field"]


def _coords(shape):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    return x, y, z


def line_factor(x, y, x0, y0, xi):
    """Straight vortex line parallel to z through (x0, y0), winding +1 about +z."""
    re, im = x - x0, y - y0
    s = np.sqrt(re * re + im * im + xi * xi)
    return (re + 1j * im) / s


def ring_factor(x, y, z, center, radius, xi):
    """Vortex ring of the given radius in the plane z = center[2], normal z."""
    rho = np.sqrt((x - center[0]) ** 2 + (y - center[1]) ** 2) - radius
    zc = z - center[2]
    s = np.sqrt(rho * rho + zc * zc + xi * xi)
    return (rho + 1j * zc) / s


def analytic_line_ring(n: int = 64, xi: float = 2.0, line_xy=(31.37, 30.81),
                       ring_center=(32.0, 32.0, 40.0), ring_radius: float = 12.0,
                       with_line: bool = True, with_ring: bool = True) -> np.ndarray:
    """Product of analytic vortex factors on an n^3 grid, evaluated in FP64 and
    rounded once to complex64."""
    x, y, z = _coords((n, n, n))
    psi = np.ones((n, n, n), np.complex128)
    if with_line:
        psi = psi * line_factor(x, y, line_xy[0], line_xy[1], xi)
    if with_ring:
        psi = psi * ring_factor(x, y, z, ring_center, ring_radius, xi)
    return psi.astype(np.complex64)


@dataclass
class WaveSpec:
    k: np.ndarray      # [W, 3] float64 wave vectors (rad / h)
    amp: np.ndarray    # [W] complex128 amplitudes


def wave_spec(seed: int, n_waves: int, kmin: float = 0.15, kmax: float = 0.35) -> WaveSpec:
    """W plane waves: |k| ~ U[kmin, kmax] (uniform in magnitude), direction
    uniform on S^2, amplitude complex Gaussian with E|A|^2 = 1/W."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d = rng.standard_normal((n_waves, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    kmag = rng.uniform(kmin, kmax, n_waves)
    amp = (rng.standard_normal(n_waves) + 1j * rng.standard_normal(n_waves)) * np.sqrt(
        0.5 / n_waves)
    return WaveSpec(k=d * kmag[:, None], amp=amp)


def random_waves_numpy(shape, spec: WaveSpec) -> np.ndarray:
    """FP64 evaluation on the host (small grids): psi[z] = (A * ez[:, z]) ey^T ex."""
    nz, ny, nx = shape
    ex = np.exp(1j * np.outer(spec.k[:, 0], np.arange(nx)))
    ey = np.exp(1j * np.outer(spec.k[:, 1], np.arange(ny)))
    ez = np.exp(1j * np.outer(spec.k[:, 2], np.arange(nz)))
    out = np.empty(shape, np.complex64)
    for z in range(nz):
        m = (spec.amp * ez[:, z])[None, :] * ey.T  # [ny, W]
        out[z] = (m @ ex).astype(np.complex64)
    return out


def random_waves(shape, spec: WaveSpec, device="cpu", chunk: int | None = None):
    """Random-wave field as a torch complex64 tensor on `device`.

    Phase tables are built in FP64 and rounded to complex64; each z-plane is a
    complex GEMM (ny x W) @ (W x nx) accumulated in FP32.  Used for the large
    grids, where the host evaluation would take hours.
    """
    import torch

    nz, ny, nx = shape
    dev = torch.device(device)
    k = torch.as_tensor(spec.k, dtype=torch.float64, device=dev)
    amp = torch.as_tensor(spec.amp, dtype=torch.complex128, device=dev)

    def table(col, n):
        ph = torch.outer(k[:, col], torch.arange(n, dtype=torch.float64, device=dev))
        return torch.polar(torch.ones_like(ph), ph)

    ex = table(0, nx).to(torch.complex64)                  # [W, nx]
    eyt = table(1, ny).transpose(0, 1).contiguous()        # [ny, W] complex128
    ez = table(2, nz)                                      # [W, nz] complex128
    out = torch.empty((nz, ny, nx), dtype=torch.complex64, device=dev)
    W = spec.k.shape[0]
    if chunk is None:
        chunk = max(1, min(nz, int(2 ** 28 // max(1, ny * W))))
    for z0 in range(0, nz, chunk):
        z1 = min(nz, z0 + chunk)
        m = (amp[None, :] * ez[:, z0:z1].transpose(0, 1))[:, None, :] * eyt[None, :, :]
        out[z0:z1] = torch.matmul(m.to(torch.complex64), ex)
    return out


def multiplicative_noise(psi, seed: int, level: float = 0.05):
    """psi * (1 + level * g) with one real standard normal g per node.

    A positive real factor does not change any phase, so the winding field is
    unchanged wherever 1 + level * g > 0 (always, in practice, at 5%)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    g = rng.standard_normal(tuple(psi.shape)).astype(np.float32)
    fac = (1.0 + level * g).astype(np.float32)
    if isinstance(psi, np.ndarray):
        return (psi * fac).astype(np.complex64)
    import torch

    return psi * torch.as_tensor(fac, device=psi.device)


# the 16 snapshots of the uneven batch workload: (edge, waves), seeds 201..216
BATCH16 = [(256, 4096)] * 8 + [(384, 4096)] * 4 + [(512, 16384)] * 3 + [(768, 16384)]


def batch_fields(device="cuda", sizes=None, seed0: int = 201):
    """Random-wave tangles of an uneven batch: one snapshot per (edge, waves)
    entry of sizes (default BATCH16: 8 x 256^3, 4 x 384^3, 3 x 512^3,
    1 x 768^3), seeds seed0, seed0 + 1, ... (torch)."""
    sizes = BATCH16 if sizes is None else sizes
    return [random_waves((n, n, n), wave_spec(seed0 + i, w), device=device)
            for i, (n, w) in enumerate(sizes)]


def config_field(name: str, device="cpu", seed: int | None = None):
    """Fields of the named workloads.

    '64_analytic'        64^3 line x ring product, xi = 2h (numpy complex64)
    '256_waves'          256^3, 4096 waves, seed 1 by default (torch)
    '512_waves_noise'    512^3, 16384 waves seed 7, 5% noise seed 8 (torch)
    """
    if name == "64_analytic":
        return analytic_line_ring()
    if name == "256_waves":
        return random_waves((256, 256, 256), wave_spec(1 if seed is None else seed, 4096),
                            device=device)
    if name == "512_waves_noise":
        psi = random_waves((512, 512, 512), wave_spec(7 if seed is None else seed, 16384),
                           device=device)
        return multiplicative_noise(psi, 8)
    raise KeyError(name)
