"""GPU parity at the paper's own resolution: a 2048^3 complex64 field (64 GiB,
more than 2^32 nodes, the size of the paper's NLKG snapshots) identified and
localized in one call on one GPU (Sec. 2.2.2, Eq. 5; Sec. 3.3.3, Eq. 6).

Face by face on sampled planes, planes past node index 2^32 and the first and
last planes among them: every unambiguous face's winding equals the FP64
oracle's (run on the two planes the faces need), no face is listed where the
grid has none, and every well-conditioned position is within 1e-4 h (plus
half an FP32 ulp of the absolute coordinate, about 1.2e-4 h at z = 2047).
The list is strictly ascending over the whole field.  Both the bit-sliced
sweep (the default) and, with the nibble setting, the register sweep (rows
wider than the nibble sweep's 1024 columns) are checked.  The node form from
psi and from the face list give the same vortex nodes and circulations there.
"""
import numpy as np
import pytest

import oracle
import synth
from qtv_testutil import compare_windings, dense_from_list, position_tolerance

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N = 2048
PLANES = [0, 1, 777, 1023, 1024, 1500, 2046, 2047]


@pytest.fixture(scope="module")
def field():
    if torch.cuda.get_device_properties(0).total_memory < 120 * 2 ** 30:
        pytest.skip("needs about 100 GB of device memory")
    # 1024 waves of the random-wave spectrum (the 512^3 field's shell)
    psi = synth.random_waves((N, N, N), synth.wave_spec(2048, 1024), device="cuda")
    torch.cuda.synchronize()
    torch.cuda.empty_cache()  # the generator's temporaries
    yield psi
    del psi
    torch.cuda.empty_cache()


@pytest.fixture(scope="module", params=[1, 0], ids=["bits", "nibble"])
def q(request):
    import paper_1911_12070_gb300 as qtv

    qtv.build()
    h = qtv.Qtv(0)
    h.configure_sweep(variant=request.param)
    yield h
    h.close()
    torch.cuda.empty_cache()


def test_paper_resolution_face_by_face(q, field):
    ids_d, w_d, xyz_d, _, flags_d = q.identify_localize(field)
    n = ids_d.numel()
    assert n > 10_000_000
    assert bool(torch.all(ids_d[1:] > ids_d[:-1]))
    assert int(ids_d[-1]) >> 2 < N ** 3
    ids = ids_d.cpu().numpy().view(np.uint64)
    w = w_d.cpu().numpy()
    xyz = xyz_d.cpu().numpy()
    flags = flags_d.cpu().numpy()
    del ids_d, w_d, xyz_d, flags_d
    o = (ids & np.uint64(3)).astype(np.int64)
    lin = (ids >> np.uint64(2)).astype(np.int64)
    k = lin // (N * N)
    checked = 0
    for kk in PLANES:
        sel = np.nonzero(k == kk)[0]
        slab = field[kk:kk + 2].cpu().numpy()
        local = (((lin[sel] - kk * N * N) << 2) | o[sel]).astype(np.uint64)
        ow, ofl = oracle.identify(slab, k0=0, k1=1)
        g = dense_from_list(local, w[sel], (1, N, N))
        bad, _, _ = compare_windings(g, ow, ofl)
        assert bad == 0, f"plane {kk}: {bad} unambiguous faces differ"
        assert not np.any(g[(ofl & oracle.ABSENT) != 0]), f"plane {kk}: a non-face listed"
        ora = oracle.localize(slab, local, w[sel])
        f = ofl.reshape(3, -1)[o[sel], lin[sel] - kk * N * N]
        ok = ((ora["flags"] & (oracle.L_ANOMALOUS | oracle.L_ILLCOND)) == 0) & \
            ((f & (oracle.AMBIGUOUS | oracle.ZERO_NODE)) == 0)
        ref = ora["xyz"] + np.array([0.0, 0.0, float(kk)])
        err = np.abs(xyz[sel].astype(np.float64) - ref)
        badp = np.any(err > position_tolerance(ref), axis=1) & ok
        assert not badp.any(), f"plane {kk}: {int(badp.sum())} positions off (max {err[ok].max()})"
        assert not np.any((flags[sel] & 1)[ok])
        checked += int(ok.sum())
    print(f"2048^3: {n} pierced faces; {checked} positions checked on {len(PLANES)} planes")
    assert checked > 50_000


def test_paper_resolution_node_form(q, field):
    """The node form (Sec. 2.2.2) at 2048^3, from psi and from the face list:
    the same vortex nodes and ring circulations, node for node."""
    ids, w, _ = q.identify(field)
    a_ids, a_circ, _ = q.node_circulation(field)
    b_ids, b_circ, tie = q.node_circulation_faces(tuple(field.shape), ids, w)
    del ids, w
    assert not tie
    assert a_ids.numel() > 10_000_000
    assert bool(torch.all(a_ids[1:] > a_ids[:-1]))
    assert torch.equal(a_ids, b_ids) and torch.equal(a_circ, b_circ)
