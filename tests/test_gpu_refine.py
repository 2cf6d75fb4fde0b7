"""GPU parity of sample refinement (Sec. 3.3.3, "Locating more accurate sample
points") through the C ABI: descent of rho = |psi|^2 in the plane through x0
normal to the pseudo-vorticity, FP32 on the GPU against the FP64 oracle.

Compared on the same initial points (face centres of pierced faces, and the
box means of the oracle's graph reduction of the GPU samples, which is the
paper's own input): the no-tangent flags exactly, tangents within 1e-3, and
positions within 1e-4 h wherever the oracle converged away from the grid and
box boundaries at a well-conditioned zero (|det J| >= 1e-3 max|psi|^2; the
other cases are counted).  Closed forms on the GPU: a tilted anisotropic line
refines to its nearest point.  Edge cases: points outside the grid, a field
with no tangent, a step limit of 0, the device count limit, world coordinates
(h, origin), repeat calls, and the 512^3 workload on a sample of its faces.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import graph

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def q():
    import paper_1911_12070_gb300 as qtv

    qtv.build()
    h = qtv.Qtv(0)
    yield h
    h.close()


# density agreement off the strict subset: relative to the oracle's density
# there, plus an absolute floor relative to max |psi|^2 (FP32 evaluation of rho)
RHO_REL, RHO_ABS = 1e-3, 1e-7


def _face_centres(ids, shape):
    nz, ny, nx = shape
    o = (ids & np.uint64(3)).astype(np.int64)
    lin = (ids >> np.uint64(2)).astype(np.int64)
    c = np.column_stack([lin % nx, (lin // nx) % ny, lin // (nx * ny)]).astype(np.float64)
    half = np.array([[0.5, 0.5, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5]])
    return c + half[o]


def _host(out):
    return {k: v.cpu().numpy() for k, v in out.items()}


def _compare(host, x0, g, r, min_sel=0.6):
    """Every sample is checked.  Flags: no-tangent exactly; converged / step
    limit equal except where both searches ended at a zero of rho (a search
    that reaches a zero stops within a step or two of the step limit in FP32
    and FP64 alike, so the limit may be hit on one side only).  Positions within
    1e-4 h on the strict subset (both converged, away from the grid and box
    boundaries, well-conditioned zero); on every other sample the two searches
    must end at the same density, since rho is what the descent minimizes and
    flat directions of rho leave the position itself loosely fixed."""
    m2 = float(np.max(np.abs(host.astype(np.complex128)) ** 2))
    nt_g = (g["flags"] & 2) != 0
    nt_o = (r["flags"] & oracle.R_NO_TANGENT) != 0
    assert np.array_equal(nt_g, nt_o)
    both = ~nt_o
    assert np.max(np.abs(g["t"][both] - r["t"][both]), initial=0.0) < 1e-3
    at_zero = (g["rho"] < 1e-9 * m2) & (r["rho"] < 1e-9 * m2)
    differ = both & (g["flags"] != r["flags"])
    assert not np.any(differ & ~at_zero), np.nonzero(differ & ~at_zero)[0][:10]
    assert differ.sum() <= max(2, 0.002 * both.sum()), int(differ.sum())
    hi = np.array(host.shape[::-1]) - 1
    dx = r["xyz"] - x0
    sel = both & (r["flags"] == oracle.R_CONVERGED) & (g["flags"] == oracle.R_CONVERGED) & \
        np.all((r["xyz"] > 1e-6) & (r["xyz"] < hi - 1e-6), axis=1) & \
        (np.max(np.abs(dx), axis=1) < 1 - 1e-6) & (np.abs(r["detj"]) >= 1e-3 * m2)
    assert sel.mean() >= min_sel, sel.mean()
    err = np.max(np.abs(g["xyz"].astype(np.float64) - r["xyz"]), axis=1)
    tol = 1e-4 + np.max(np.abs(r["xyz"]), axis=1) * 2.0 ** -23
    bad = sel & (err > tol)
    assert not bad.any(), (int(bad.sum()), float(err[sel].max()))
    assert np.max(g["rho"][sel]) < 1e-9 * m2
    # off the strict subset, start points inside the grid: both searches end
    # at the same density; start points on the grid boundary: a direction that
    # leaves the grid is rejected, so an FP32 and an FP64 direction that differ
    # by rounding may decide whether the search moves at all; there both only
    # never increase rho
    inner = np.all((x0 > 1e-6) & (x0 < hi - 1e-6), axis=1)
    rest = both & ~sel & inner
    edge = both & ~sel & ~inner
    drho = np.abs(g["rho"].astype(np.float64) - r["rho"])
    rho_tol = RHO_REL * r["rho"] + RHO_ABS * m2
    print(f"strict {int(sel.sum())}, rest {int(rest.sum())}, boundary {int(edge.sum())}, "
          f"flags differ {int(differ.sum())}, "
          f"max |drho|/m2 on rest {np.max(drho[rest] / m2, initial=0.0):.2e}")
    assert not np.any(rest & (drho > rho_tol)), (
        int(np.sum(rest & (drho > rho_tol))), float(np.max((drho / rho_tol)[rest])))
    rho0 = oracle.density(host, x0)
    assert np.all(r["rho"][both] <= rho0[both] * (1 + 1e-12) + 1e-15 * m2)
    assert np.all(g["rho"][both] <= rho0[both] * (1 + 1e-5) + 1e-9 * m2)
    # the position never leaves the search box around x0 on either side
    assert np.all(np.max(np.abs(g["xyz"][both] - x0[both]), axis=1) <= 1 + 1e-5)
    return int(sel.sum()), float(err[sel].max())


def test_face_centres_match_oracle(q):
    host = synth.random_waves_numpy((40, 36, 52), synth.wave_spec(13, 512))
    dev = torch.from_numpy(host).cuda()
    ids, w, _ = q.identify(dev)
    g = _host(q.refine_samples(dev, face_ids=ids))
    x0 = _face_centres(ids.cpu().numpy().view(np.uint64), host.shape)
    r = oracle.refine(host, x0)
    n, e = _compare(host, x0, g, r)
    assert n > 300


def test_box_means_of_the_graph_reduction_match_oracle(q):
    # the paper's input: box means of the reduced sample graph (Sec. 3.3.2)
    host = synth.random_waves_numpy((40, 40, 40), synth.wave_spec(23, 512))
    dev = torch.from_numpy(host).cuda()
    ids, w, xyz, _, _ = q.identify_localize(dev)
    fg = graph.face_graph(ids.cpu().numpy().view(np.uint64), w.cpu().numpy(),
                          xyz.cpu().numpy().astype(np.float64), host.shape)
    red, _ = graph.reduce(fg, d=4.0)
    x0 = np.ascontiguousarray(red.pos, dtype=np.float64)
    g = _host(q.refine_samples(dev, xyz0=torch.from_numpy(x0.astype(np.float32)).cuda()))
    r = oracle.refine(host, x0.astype(np.float32).astype(np.float64))
    n, e = _compare(host, x0.astype(np.float32).astype(np.float64), g, r, min_sel=0.5)
    assert n > 30
    # the refined samples sit on cores: Eq. 7 error far below the box means'
    e0 = graph.density_error(host, x0)
    e1 = graph.density_error(host, g["xyz"].astype(np.float64))
    assert e1 < 0.1 * e0


@pytest.mark.parametrize("aniso", [(1.0, 1.0), (2.0, 0.5)])
def test_tilted_line_nearest_point_on_gpu(q, aniso):
    rng = np.random.default_rng(17)
    qq, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    u, v = qq[:, 0], qq[:, 1]
    d = np.cross(u, v)
    p = np.array([7.3, 6.1, 5.7])
    shape = (12, 13, 15)
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    r3 = np.stack([x, y, z], axis=-1) - p
    host = (aniso[0] * (r3 @ u) + 1j * aniso[1] * (r3 @ v)).astype(np.complex64)
    x0 = (p + rng.uniform(-0.45, 0.45, (40, 3))).astype(np.float32)
    g = _host(q.refine_samples(torch.from_numpy(host).cuda(), xyz0=torch.from_numpy(x0).cuda()))
    want = p + ((x0 - p) @ d)[:, None] * d
    assert np.all(g["flags"] == 1)
    assert np.max(np.abs(g["xyz"] - want)) < 1e-4
    assert np.max(np.abs(g["t"] - d)) < 1e-4


def test_edge_cases(q):
    host = synth.random_waves_numpy((10, 12, 14), synth.wave_spec(3, 128))
    dev = torch.from_numpy(host).cuda()
    pts = torch.tensor([[5.2, 5.1, 4.3], [-0.5, 2.0, 2.0], [13.5, 1.0, 1.0],
                        [float("nan"), 1.0, 1.0], [0.0, 0.0, 0.0], [13.0, 11.0, 9.0]],
                       device="cuda")
    g = _host(q.refine_samples(dev, xyz0=pts))
    assert list(g["flags"][1:4] & 2) == [2, 2, 2]
    assert np.array_equal(g["xyz"][1:3], pts.cpu().numpy()[1:3])
    r = oracle.refine(host, pts.cpu().numpy().astype(np.float64))
    assert np.array_equal((g["flags"] & 2) != 0, (r["flags"] & 2) != 0)
    # a step limit of 0 leaves x0 and flags the limit
    g0 = _host(q.refine_samples(dev, xyz0=pts[:1], max_iter=0))
    assert g0["flags"][0] == 4 and np.array_equal(g0["xyz"][0], pts[0].cpu().numpy())
    # constant field: no tangent anywhere
    ones = torch.ones((6, 7, 8), dtype=torch.complex64, device="cuda")
    g1 = _host(q.refine_samples(ones, xyz0=torch.tensor([[3.0, 3.0, 3.0]], device="cuda")))
    assert g1["flags"][0] == 2 and g1["iters"][0] == 0
    # the device count limits the samples processed
    out = q.refine_samples(dev, xyz0=pts, n_dev=torch.tensor([1], dtype=torch.int64,
                                                                 device="cuda"))
    assert out["flags"].shape[0] == 6
    g2 = _host(q.refine_samples(dev, xyz0=pts[:1]))
    assert np.array_equal(out["xyz"][:1].cpu().numpy(), g2["xyz"])


def test_world_coordinates(q):
    import paper_1911_12070_gb300 as qtv

    host = synth.random_waves_numpy((24, 26, 28), synth.wave_spec(8, 256))
    dev = torch.from_numpy(host).cuda()
    ids, _, _ = q.identify(dev)
    x0 = _face_centres(ids.cpu().numpy().view(np.uint64), host.shape)
    a = _host(q.refine_samples(dev, xyz0=torch.from_numpy(x0.astype(np.float32)).cuda()))
    grid = qtv.Grid.of(host.shape, h=0.5, origin=(1.0, -2.0, 3.0))
    xw = (np.array([1.0, -2.0, 3.0]) + 0.5 * x0).astype(np.float32)
    b = _host(q.refine_samples(dev, xyz0=torch.from_numpy(xw).cuda(), grid=grid))
    assert np.array_equal(a["flags"], b["flags"])
    back = (b["xyz"].astype(np.float64) - np.array([1.0, -2.0, 3.0])) / 0.5
    assert np.max(np.abs(back - a["xyz"])) < 1e-4


def test_repeat_calls_identical(q):
    host = synth.random_waves_numpy((32, 32, 32), synth.wave_spec(9, 256))
    dev = torch.from_numpy(host).cuda()
    ids, _, _ = q.identify(dev)
    a = _host(q.refine_samples(dev, face_ids=ids))
    b = _host(q.refine_samples(dev, face_ids=ids))
    for k in a:
        assert np.array_equal(a[k], b[k], equal_nan=True)


def test_512_workload_sampled(q):
    psi = synth.config_field("512_waves_noise", device="cuda")
    ids, w, _ = q.identify(psi)
    g = q.refine_samples(psi, face_ids=ids)
    rng = np.random.default_rng(5)
    n = ids.numel()
    sel = np.unique(np.concatenate([np.arange(2000), rng.choice(n, 4000, replace=False),
                                    np.arange(n - 1000, n)]))
    gi = {k: v.cpu().numpy()[sel] for k, v in g.items()}
    host = psi.cpu().numpy()
    x0 = _face_centres(ids.cpu().numpy().view(np.uint64)[sel], host.shape)
    r = oracle.refine(host, x0)
    nsel, e = _compare(host, x0, gi, r)
    conv = (g["flags"] == 1).float().mean().item()
    assert conv > 0.9
