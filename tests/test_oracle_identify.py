"""Pins of the oracle's identification (Sec. 2.2.2, Eq. 5) against what the
paper and the mathematics fix, not against the oracle itself.

* A straight vortex line along z pierces exactly one xy plaquette per z-plane,
  with winding +1 (|C| = 2 pi at a core, Sec. 2.2.2; sign = direction).
* Conjugating psi reverses every circulation (sign = direction).
* The net winding out of every closed unit cell is zero (a vortex line that
  enters a cell leaves it; discrete Stokes theorem).
* A positive real rescaling per node leaves every phase, hence every winding,
  unchanged.
* A generic vortex ring crosses exactly the lattice faces that integer
  enumeration of the analytic circle predicts, with the right-hand-rule sign.
* Random-wave tangles pierce about <k^2>/(2 pi) faces per node (isotropic line
  density <k^2>/(3 pi), times 3/2 lattice-plane crossings per unit length);
  a +-10% sanity check from the random-wave literature.
* The paper's node form (ring path around a node, max over three planes,
  threshold pi) equals 2 pi times the sum of the four incident plaquette
  windings.
"""
import numpy as np
import pytest

import oracle
import synth

TWO_PI = 2 * np.pi


def _field(n, waves, seed):
    return synth.random_waves_numpy((n, n, n), synth.wave_spec(seed, waves))


@pytest.fixture(scope="module")
def rw48():
    return _field(48, 512, 11)


def test_straight_line_one_face_per_plane():
    psi = synth.analytic_line_ring(with_ring=False)
    w, fl = oracle.identify(psi)
    o, k, j, i = np.nonzero(w)
    assert len(o) == 64
    assert set(o.tolist()) == {0}
    assert set(zip(i.tolist(), j.tolist())) == {(31, 30)}
    assert sorted(k.tolist()) == list(range(64))
    assert set(w[w != 0].tolist()) == {1}
    assert np.count_nonzero(fl & oracle.AMBIGUOUS) == 0


def test_straight_line_reversed_direction():
    # (x - x0) - i (y - y0) winds the other way about +z
    psi = np.conj(synth.analytic_line_ring(with_ring=False))
    w, _ = oracle.identify(psi)
    assert set(w[w != 0].tolist()) == {-1}
    assert np.count_nonzero(w) == 64


@pytest.mark.parametrize("which", ["config0", "waves"])
def test_conjugation_flips_every_sign(which, rw48):
    psi = synth.analytic_line_ring() if which == "config0" else rw48
    w, fl = oracle.identify(psi)
    wc, flc = oracle.identify(np.conj(psi))
    ok = ((fl | flc) & (oracle.AMBIGUOUS | oracle.ABSENT)) == 0
    assert np.array_equal(wc[ok], -w[ok])
    assert np.count_nonzero(w[ok]) > 0


def _cell_flux(w):
    """Outward net winding of every unit cell: faces whose normal points out of
    the cell count +W, faces whose normal points in count -W."""
    wxy, wyz, wzx = (w[o].astype(np.int32) for o in range(3))
    return ((wxy[1:, :-1, :-1] - wxy[:-1, :-1, :-1])
            + (wyz[:-1, :-1, 1:] - wyz[:-1, :-1, :-1])
            + (wzx[:-1, 1:, :-1] - wzx[:-1, :-1, :-1]))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_closed_cells_have_zero_net_flux(seed):
    psi = _field(40, 256, seed)
    w, fl = oracle.identify(psi)
    flux = _cell_flux(w)
    assert np.count_nonzero(w) > 100
    assert np.count_nonzero(flux) == 0


def test_closed_cells_zero_flux_config0():
    w, _ = oracle.identify(synth.analytic_line_ring())
    assert np.count_nonzero(_cell_flux(w)) == 0


def test_cell_flux_detects_a_planted_error(rw48):
    # the flux check is sharp enough to see one wrong face
    w, _ = oracle.identify(rw48)
    o, k, j, i = [a[0] for a in np.nonzero(w)]
    w2 = w.copy()
    w2[o, k, j, i] = -w2[o, k, j, i]
    assert np.count_nonzero(_cell_flux(w2)) > 0


def test_positive_real_rescaling_keeps_windings(rw48):
    w, fl = oracle.identify(rw48)
    noisy = synth.multiplicative_noise(rw48, seed=8, level=0.05)
    wn, fln = oracle.identify(noisy)
    ok = ((fl | fln) & oracle.AMBIGUOUS) == 0
    assert np.array_equal(w[ok], wn[ok])
    assert np.count_nonzero(~ok) <= 8


def _ring_crossings(center, radius, n):
    """Faces crossed by the circle |(x,y) - c| = R in the plane z = cz, by
    integer enumeration of the lattice planes x = i and y = j it meets.
    Returns {(o, i, j, k): expected winding}.  The ring factor's phase winds
    counter-clockwise in the (rho, z) half plane, so its direction is -theta
    (right-hand rule), i.e. tangent (sin t, -cos t, 0) at angle t."""
    cx, cy, cz = center
    k = int(np.floor(cz))
    out = {}
    for i in range(n):
        dx = i - cx
        if abs(dx) < radius:
            for s in (+1, -1):
                y = cy + s * np.sqrt(radius ** 2 - dx ** 2)
                # yz face at x = i, normal +x: winding = sign(tangent_x) = sign(y - cy)
                out[(1, i, int(np.floor(y)), k)] = s
    for j in range(n):
        dy = j - cy
        if abs(dy) < radius:
            for s in (+1, -1):
                x = cx + s * np.sqrt(radius ** 2 - dy ** 2)
                # zx face at y = j, normal +y: winding = sign(tangent_y) = -sign(x - cx)
                out[(2, int(np.floor(x)), j, k)] = -s
    return out


@pytest.mark.parametrize("center", [(32.29, 31.63, 40.47), (30.71, 33.18, 20.33)])
def test_generic_ring_crossing_count_and_signs(center):
    R = 12.0
    psi = synth.analytic_line_ring(with_line=False, ring_center=center, ring_radius=R)
    w, fl = oracle.identify(psi)
    expect = _ring_crossings(center, R, 64)
    assert len(expect) == 8 * int(R)  # 96 lattice-plane crossings for R = 12
    got = {(o, i, j, k): int(w[o, k, j, i]) for o, k, j, i in zip(*np.nonzero(w))}
    assert len(got) == len(expect)
    # every analytic crossing face is pierced with the right-hand-rule sign,
    # allowing a crossing within 0.1 h of a face edge to land in the neighbour
    for (o, i, j, k), s in expect.items():
        if (o, i, j, k) in got:
            assert got[(o, i, j, k)] == s
        else:
            near = [key for key in got if key[0] == o and abs(key[1] - i) + abs(key[2] - j)
                    + abs(key[3] - k) == 1]
            assert near, (o, i, j, k)
            assert all(got[key] == s for key in near)


def test_random_wave_face_density():
    kmin, kmax = 0.15, 0.35
    k2 = (kmax ** 3 - kmin ** 3) / (3 * (kmax - kmin))
    expect = k2 / (2 * np.pi)
    dens = []
    for seed in (3, 4):
        w, _ = oracle.identify(_field(96, 1024, seed))
        dens.append(np.count_nonzero(w) / 96 ** 3)
    assert abs(np.mean(dens) / expect - 1) < 0.10, (dens, expect)


def test_node_form_equals_incident_plaquette_sum(rw48):
    w, fl = oracle.identify(rw48)
    c, vortex = oracle.node_circulation(rw48)
    nz, ny, nx = rw48.shape
    wi = w.astype(np.int64)
    # for node (i,j,k) and plane o, the four plaquettes of that plane with the
    # node as a corner: min corners (u-1,v-1), (u,v-1), (u,v), (u-1,v)
    s = np.zeros_like(c)
    # o = 0: (u,v) = (x,y)
    s[0, :, 1:-1, 1:-1] = (wi[0, :, :-2, :-2] + wi[0, :, :-2, 1:-1] + wi[0, :, 1:-1, 1:-1]
                           + wi[0, :, 1:-1, :-2])[:, :, :]
    # o = 1: (u,v) = (y,z)
    s[1, 1:-1, 1:-1, :] = (wi[1, :-2, :-2, :] + wi[1, :-2, 1:-1, :] + wi[1, 1:-1, 1:-1, :]
                           + wi[1, 1:-1, :-2, :])
    # o = 2: (u,v) = (z,x)
    s[2, 1:-1, :, 1:-1] = (wi[2, :-2, :, :-2] + wi[2, 1:-1, :, :-2] + wi[2, 1:-1, :, 1:-1]
                           + wi[2, :-2, :, 1:-1])
    inner = np.zeros_like(c, dtype=bool)
    inner[0, :, 1:-1, 1:-1] = True
    inner[1, 1:-1, 1:-1, :] = True
    inner[2, 1:-1, :, 1:-1] = True
    assert np.max(np.abs(c[inner] - TWO_PI * s[inner])) < 1e-9
    # vortex node <=> max over planes |C| > pi (threshold of Sec. 2.2.2)
    interior = np.zeros(rw48.shape, bool)
    interior[1:-1, 1:-1, 1:-1] = True
    vn = (np.abs(s).max(axis=0) >= 1) & interior
    assert np.array_equal(vortex.astype(bool) & interior, vn)
    assert vn.sum() > 0


def test_nonfinite_faces_forced_to_zero(rw48):
    psi = rw48.copy()
    psi[10, 20, 30] = np.complex64(complex(np.nan, 0.0))
    psi[30, 5, 7] = np.complex64(complex(0.0, np.inf))
    w, fl = oracle.identify(psi)
    bad = (fl & oracle.NONFINITE) != 0
    # each non-finite node touches 12 faces (4 per orientation) away from the boundary
    assert bad.sum() == 24
    assert np.count_nonzero(w[bad]) == 0


def test_zero_nodes_flagged_config0():
    # the ring of config 0 is tangent to x = 20, 44 and y = 20, 44 at nodes,
    # where psi vanishes exactly
    psi = synth.analytic_line_ring()
    zero = np.argwhere(psi == 0)
    assert sorted(map(tuple, zero.tolist())) == sorted([(40, 32, 20), (40, 32, 44), (40, 20, 32),
                                                        (40, 44, 32)])
    _, fl = oracle.identify(psi)
    assert np.count_nonzero(fl & oracle.ZERO_NODE) == 4 * 12


def test_absent_faces_on_the_upper_boundary():
    psi = _field(9, 64, 1)[:, :7, :5].copy()  # nz=9, ny=7, nx=5
    w, fl = oracle.identify(psi)
    absent = (fl & oracle.ABSENT) != 0
    nz, ny, nx = psi.shape
    assert absent[0].sum() == nz * ny * nx - nz * (ny - 1) * (nx - 1)
    assert absent[1].sum() == nz * ny * nx - (nz - 1) * (ny - 1) * nx
    assert absent[2].sum() == nz * ny * nx - (nz - 1) * ny * (nx - 1)
    assert np.count_nonzero(w[absent]) == 0


def test_plane_range_matches_full_grid(rw48):
    w, fl = oracle.identify(rw48)
    w2, fl2 = oracle.identify(rw48, k0=17, k1=23)
    assert np.array_equal(w2, w[:, 17:23])
    assert np.array_equal(fl2, fl[:, 17:23])
