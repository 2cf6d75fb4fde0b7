"""GPU parity of the node form of the circulation (Sec. 2.2.2) and of the
density error of Eq. 7 (Sec. 5), through the C ABI.

Node form: for every node and plane, the ring circulation C = 2 pi S of the
CUDA path must equal the FP64 oracle's ring sum bit for bit (as the integer S)
on every ring whose edges lie at least 1e-4 rad from +-pi and avoid exact zero
nodes (the rings whose four incident plaquettes the oracle does not flag);
the vortex-node list must be the ascending list of nodes with some S != 0.
Cases: ragged x / y / z tails across warp column segments and row bands,
wide rows, degenerate grids, NaN/Inf and zero nodes, the analytic line and
ring, capacity overflow, repeat calls, and the 512^3 workload the benchmark
times, checked on sub-blocks the oracle evaluates exactly.

Density error: rho at every point within the FP32 interpolation bound, e and
rho_bar within 1e-5 / 1e-6 relative of the oracle.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import graph as ograph
from qtv_testutil import dense_from_list, gpu_identify

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TWO_PI = 2.0 * np.pi


@pytest.fixture(scope="module")
def q():
    import paper_1911_12070_gb300 as qtv

    qtv.build()
    h = qtv.Qtv(0)
    yield h
    h.close()


def _waves(shape, seed, waves=512):
    return synth.random_waves_numpy(shape, synth.wave_spec(seed, waves))


def _oracle_rings(psi):
    """Oracle ring sums as integers S [3][nz][ny][nx], the vortex flag, and the
    rings to exclude (an incident plaquette flagged ambiguous or zero-node)."""
    c, v = oracle.node_circulation(psi)
    s = np.rint(c / TWO_PI)
    assert np.max(np.abs(c - TWO_PI * s)) < 1e-6
    _, fl = oracle.identify(psi)
    f = (fl & (oracle.AMBIGUOUS | oracle.ZERO_NODE)) != 0
    ex = np.zeros(c.shape, bool)
    # plane o, node (u, v): plaquettes with minimum corners (u-1..u, v-1..v)
    ex[0, :, 1:-1, 1:-1] = (f[0, :, :-2, :-2] | f[0, :, :-2, 1:-1] | f[0, :, 1:-1, :-2]
                            | f[0, :, 1:-1, 1:-1])
    ex[1, 1:-1, 1:-1, :] = (f[1, :-2, :-2, :] | f[1, :-2, 1:-1, :] | f[1, 1:-1, :-2, :]
                            | f[1, 1:-1, 1:-1, :])
    ex[2, 1:-1, :, 1:-1] = (f[2, :-2, :, :-2] | f[2, :-2, :, 1:-1] | f[2, 1:-1, :, :-2]
                            | f[2, 1:-1, :, 1:-1])
    return s.astype(np.int8), v.astype(bool), ex


def _gpu_rings(q, psi_dev, capacity=None):
    ids, circ, dense = q.node_circulation(psi_dev, capacity=capacity, dense=True)
    return ids.cpu().numpy(), circ.cpu().numpy(), dense.cpu().numpy()


def _check(q, psi, max_excluded_frac=0.01):
    s_or, vortex_or, ex = _oracle_rings(psi)
    ids, circ, dense = _gpu_rings(q, torch.from_numpy(psi).cuda())
    assert dense.shape == s_or.shape
    bad = (dense != s_or) & ~ex
    assert not bad.any(), f"{bad.sum()} rings differ, first at {np.argwhere(bad)[:5]}"
    assert ex.mean() <= max_excluded_frac
    # the list: ascending nodes with some S != 0, carrying their three S
    want = np.flatnonzero((dense != 0).any(axis=0).ravel())
    assert np.array_equal(ids, want)
    assert np.array_equal(circ, dense.reshape(3, -1)[:, ids].T)
    # vortex-node flag (max |C| > pi) wherever no plane is excluded
    clean = ~ex.any(axis=0)
    gv = (dense != 0).any(axis=0)
    assert np.array_equal(gv[clean], vortex_or[clean])
    return len(ids), int(ex.sum())


@pytest.mark.parametrize("shape", [(20, 33, 61), (9, 17, 128), (40, 40, 40), (13, 8, 30),
                                   (7, 70, 300), (5, 9, 31), (24, 16, 1000)])
def test_random_waves_match_oracle(q, shape):
    n, nex = _check(q, _waves(shape, seed=sum(shape)))
    if np.prod(shape) >= 16000:  # smaller grids may hold no core at all
        assert n > 0


def test_analytic_line_and_ring(q):
    # exact zero nodes and exact pi ties of the ring in a node plane
    psi = synth.analytic_line_ring()
    n, nex = _check(q, psi, max_excluded_frac=0.02)
    assert n > 200


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 5, 7), (3, 3, 3), (2, 2, 2), (5, 1, 9),
                                   (4, 6, 1), (3, 40, 3)])
def test_degenerate_grids(q, shape):
    psi = (np.random.default_rng(11).standard_normal(shape + (2,)).astype(np.float32)
           .view(np.complex64)[..., 0])
    _check(q, np.ascontiguousarray(psi), max_excluded_frac=1.0)


def test_empty_grid_counts_zero(q):
    psi = torch.zeros((0, 4, 4), dtype=torch.complex64, device="cuda")
    ids, circ, _ = q.node_circulation(psi)
    assert ids.numel() == 0 and circ.shape == (0, 3)


def test_nonfinite_and_zero_nodes(q):
    psi = _waves((14, 26, 95), seed=12)
    psi[5, 10, 29] = np.complex64(complex(np.nan, 1.0))   # last column of warp segment 0
    psi[6, 7, 30] = np.complex64(complex(np.inf, 0.0))    # first column of segment 1
    psi[6, 8, 60] = np.complex64(complex(0.0, -np.inf))   # band halo row (j = 8)
    psi[3, 15, 44] = np.complex64(complex(np.nan, np.nan))
    psi[9, 20, 50] = 0                                    # exact zero node
    psi[9, 21, 50] = 0
    _check(q, psi, max_excluded_frac=0.05)
    ids, circ, dense = _gpu_rings(q, torch.from_numpy(psi).cuda())
    # rings through a non-finite node are 0; the node's own rings are not affected
    assert dense[0, 5, 10, 28] == 0 and dense[0, 5, 11, 29] == 0 and dense[1, 4, 10, 29] == 0


def test_ring_equals_incident_plaquette_windings_on_gpu(q):
    # on a finite field the ring sum equals the sum of the four plaquette
    # windings of qtv_identify (interior edges cancel exactly)
    psi = synth.random_waves((96, 160, 256), synth.wave_spec(31, 1024), device="cuda")
    ids, w, _ = gpu_identify(q, psi)
    wd = dense_from_list(ids, w, tuple(psi.shape)).astype(np.int32)
    _, _, dense = _gpu_rings(q, psi)
    s = np.zeros(dense.shape, np.int32)
    s[0, :, 1:-1, 1:-1] = wd[0, :, :-2, :-2] + wd[0, :, :-2, 1:-1] + wd[0, :, 1:-1, :-2] + \
        wd[0, :, 1:-1, 1:-1]
    s[1, 1:-1, 1:-1, :] = wd[1, :-2, :-2, :] + wd[1, :-2, 1:-1, :] + wd[1, 1:-1, :-2, :] + \
        wd[1, 1:-1, 1:-1, :]
    s[2, 1:-1, :, 1:-1] = wd[2, :-2, :, :-2] + wd[2, :-2, :, 1:-1] + wd[2, 1:-1, :, :-2] + \
        wd[2, 1:-1, :, 1:-1]
    assert np.array_equal(dense.astype(np.int32), s)
    assert (dense != 0).any(axis=0).sum() > 0.02 * dense[0].size


def test_capacity_overflow_reports_required_count(q):
    psi = torch.from_numpy(_waves((24, 48, 90), seed=8)).cuda()
    full_ids, full_circ, _ = _gpu_rings(q, psi)
    n = len(full_ids)
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    small = torch.empty(n // 3, dtype=torch.int64, device="cuda")
    sc = torch.empty((n // 3, 3), dtype=torch.int8, device="cuda")
    q.node_circulation_into(psi, small, sc, count)
    assert int(count.item()) == n
    q.node_circulation_into(psi, None, None, count)   # count only
    assert int(count.item()) == n
    ids, circ, _ = _gpu_rings(q, psi, capacity=16)    # binding retries
    assert np.array_equal(ids, full_ids) and np.array_equal(circ, full_circ)


def test_repeat_calls_are_deterministic(q):
    psi = synth.random_waves((64, 128, 200), synth.wave_spec(5, 1024), device="cuda")
    a = _gpu_rings(q, psi)
    b = _gpu_rings(q, psi)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.fixture(scope="module")
def field512():
    return synth.config_field("512_waves_noise", device="cuda")


def test_512_workload_sub_blocks(q, field512):
    """The bench workload in the bench's launch shape; the oracle evaluates
    48^3 sub-blocks (plus a one-node rim), whose interior rings are exact."""
    ids, circ, dense = q.node_circulation(field512, dense=True)
    host = field512.cpu().numpy()
    d = dense.cpu().numpy()
    n = 512
    w = 48
    for a in [(0, 0, 0), (232, 240, 250), (464, 464, 464), (100, 0, 300), (0, 471, 17)]:
        lo = [max(c - 1, 0) for c in a]
        hi = [min(c + w + 1, n) for c in a]
        sub = np.ascontiguousarray(host[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]])
        s_or, _, ex = _oracle_rings(sub)
        sl = tuple(slice(c - l, c - l + w) for c, l in zip(a, lo))
        got = d[:, a[0]:a[0] + w, a[1]:a[1] + w, a[2]:a[2] + w]
        want = s_or[(slice(None),) + sl]
        exs = ex[(slice(None),) + sl]
        assert not ((got != want) & ~exs).any()
    nv = len(ids)
    assert 0.01 < nv / n ** 3 < 0.08
    idn = ids.cpu().numpy()
    assert np.all(np.diff(idn) > 0)
    assert np.array_equal(idn, np.flatnonzero((d != 0).any(axis=0).ravel()))


# ---------------------------------------------------------------------------
# density error (Eq. 7)
# ---------------------------------------------------------------------------
def _rho_tol(psi, rho_ref):
    # FP32 trilinear interpolation: |d psi| <= ~8e-7 max|psi| (weights and
    # eight FMAs), so |d rho| <= 2 max|psi| |d psi| + rounding of rho
    m2 = float(np.max(np.abs(psi.astype(np.complex128)) ** 2))
    return 2e-6 * m2 + 1e-6 * np.abs(rho_ref)


def test_density_error_random_points_match_oracle(q):
    psi = _waves((40, 36, 52), seed=3)
    rng = np.random.default_rng(4)
    nz, ny, nx = psi.shape
    pts = rng.uniform(0, 1, (5000, 3)) * np.array([nx - 1, ny - 1, nz - 1])
    pts[:7] = [[0, 0, 0], [nx - 1, ny - 1, nz - 1], [nx - 1, 0, 3.5], [2.25, ny - 1, 0],
               [10, 11, 12], [0.5, 0.5, nz - 1], [nx - 1.5, ny - 1, nz - 1]]
    pts = pts.astype(np.float32)
    dev = torch.from_numpy(psi).cuda()
    e, m, rho_bar, rho = q.density_error(dev, torch.from_numpy(pts).cuda(), want_rho=True)
    ref = oracle.density(psi, pts.astype(np.float64))
    got = rho.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - ref) <= _rho_tol(psi, ref))
    e_or = ograph.density_error(psi, pts.astype(np.float64))
    assert abs(e - e_or) <= 1e-5 * e_or
    rb = float(np.mean(np.abs(psi.astype(np.complex128)) ** 2))
    assert abs(rho_bar - rb) <= 1e-6 * rb
    assert abs(m - np.mean(np.abs(ref))) <= 1e-5 * np.mean(np.abs(ref))


def test_density_error_of_plain_samples_is_rounding_level(q):
    # a plain sample is the zero of the face's bilinear interpolant, which is
    # the trilinear interpolant restricted to the face: rho there is zero up
    # to the FP32 rounding of the position
    psi = _waves((32, 40, 48), seed=6)
    dev = torch.from_numpy(psi).cuda()
    ids, w, xyz, resid, flags = q.identify_localize(dev)
    assert len(ids) > 100
    e, m, rho_bar = q.density_error(dev, xyz)
    e_or = ograph.density_error(psi, xyz.cpu().numpy().astype(np.float64))
    assert e < 1e-6 and e_or < 1e-6
    # the same samples moved off their faces (inside the grid) are far from cores
    off = xyz * 0.97 + 0.3
    e2, _, _ = q.density_error(dev, off)
    e2_or = ograph.density_error(psi, off.cpu().numpy().astype(np.float64))
    assert e2 > 1e-3 and abs(e2 - e2_or) <= 1e-5 * e2_or


def test_density_error_edge_cases(q):
    psi = _waves((10, 12, 14), seed=2)
    dev = torch.from_numpy(psi).cuda()
    none = torch.empty((0, 3), dtype=torch.float32, device="cuda")
    e, m, rb = q.density_error(dev, none)
    assert e == 0.0 and m == 0.0 and rb > 0
    pts = torch.tensor([[1.0, 2.0, 3.0], [13.5, 1.0, 1.0], [-0.1, 0.0, 0.0]], device="cuda")
    e, m, rb, rho = q.density_error(dev, pts, want_rho=True)
    r = rho.cpu().numpy()
    assert np.isfinite(r[0]) and np.isnan(r[1]) and np.isnan(r[2]) and np.isnan(e)
    # n_dev limits the points without a host synchronisation
    nd = torch.tensor([1], dtype=torch.int64, device="cuda")
    e1, _, _ = q.density_error(dev, pts, n_dev=nd)
    e_or = ograph.density_error(psi, pts[:1].cpu().numpy().astype(np.float64))
    assert abs(e1 - e_or) <= 1e-5 * e_or


def test_density_error_512_workload(q, field512):
    ids, w, xyz, resid, flags = q.identify_localize(field512)
    e, m, rho_bar = q.density_error(field512, xyz)
    rb = float((field512.real.double() ** 2 + field512.imag.double() ** 2).mean())
    assert abs(rho_bar - rb) <= 1e-6 * rb
    assert e < 1e-6
    # repeat calls agree bit for bit
    assert q.density_error(field512, xyz) == (e, m, rho_bar)
