"""Z-slab sharding validated with virtual slabs on one GPU: each virtual rank
identifies and localizes its planes plus a one-plane halo (a pointer offset
into the field) and keeps the faces whose minimum corner lies in its planes;
the lists concatenated in rank order must equal the single-grid call: the
same ascending face ids and windings bit for bit, the same flags, and the same
positions up to the FP32 rounding of the shifted origin.  The slabs run one
after another; no kernel waits on another."""
import numpy as np
import pytest

import synth
from paper_1911_12070_gb300 import slabs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def q():
    import paper_1911_12070_gb300 as qtv

    qtv.build()
    h = qtv.Qtv(0)
    yield h
    h.close()


def _check(q, psi, parts):
    full = q.identify_localize(psi)
    got = [slabs.identify_localize_slab(q, psi, z0, z1)
           for z0, z1 in slabs.slab_bounds(psi.shape[0], parts)]
    cat = [torch.cat([g[i] for g in got]) for i in range(5)]
    assert torch.equal(cat[0], full[0]) and torch.equal(cat[1], full[1])
    assert torch.equal(cat[4], full[4])
    dx = (cat[2] - full[2]).abs().max().item() if full[2].numel() else 0.0
    assert dx <= 1e-4 + float(full[2].abs().max().item()) * 2.0 ** -23 if full[2].numel() else True
    assert torch.allclose(cat[3], full[3], rtol=1e-5, atol=1e-9)
    return full[0].numel()


@pytest.mark.parametrize("parts", [1, 2, 3, 5, 7, 40])
def test_virtual_slabs_equal_single_grid(q, parts):
    host = synth.random_waves_numpy((40, 36, 52), synth.wave_spec(13, 512))
    n = _check(q, torch.from_numpy(host).cuda(), parts)
    assert n > 300


def test_virtual_slabs_512(q):
    psi = synth.config_field("512_waves_noise", device="cuda")
    for parts in (4, 8):
        _check(q, psi, parts)


def test_slab_bounds():
    assert slabs.slab_bounds(10, 3) == [(0, 4), (4, 8), (8, 10)]
    assert slabs.slab_bounds(5, 7)[-1] == (5, 5)
    assert sum(z1 - z0 for z0, z1 in slabs.slab_bounds(513, 8)) == 513
