"""GPU parity of identification (Sec. 2.2.2, Eq. 5) through the C ABI.

The CUDA winding field must equal the FP64 oracle bit for bit on every face
whose edge phase differences lie at least 1e-4 rad from +-pi; the remaining
faces are counted and reported.  Sizes span several CTA bands and warps,
ragged tails in x, y and z, odd nx (scalar-load path), nx above 512 (wider
CTAs) and up to 2048 (more than 32 tile warps per band row), a field with
every face pierced, degenerate grids, non-finite input, capacity overflow, and the full
512^3 workload that the benchmark times (checked on sampled planes), each
with the nibble sweep and with the bit-sliced sweep.
"""
import numpy as np
import pytest

import oracle
import synth
from qtv_testutil import compare_windings, dense_from_list, gpu_identify, split_ids

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", params=[0, 1], ids=["nibble", "bits"])
def q(request):
    """A handle whose single-snapshot calls use the nibble sweep or the
    bit-sliced sweep (rows wider than 1024 columns take the register sweep
    with the nibble setting); every test runs with both."""
    import paper_1911_12070_gb300 as qtv

    qtv.build()
    h = qtv.Qtv(0)
    h.configure_sweep(variant=request.param)
    yield h
    h.close()


def _waves(shape, seed, waves=512):
    return synth.random_waves_numpy(shape, synth.wave_spec(seed, waves))


def _check_full(q, psi, max_amb_diff=None):
    dev = torch.from_numpy(psi).cuda()
    ids, w, _ = gpu_identify(q, dev)
    assert np.all(np.diff(ids.astype(np.int64)) > 0), "face ids must be strictly ascending"
    ow, ofl = oracle.identify(psi)
    g = dense_from_list(ids, w, psi.shape)
    bad, namb, damb = compare_windings(g, ow, ofl)
    assert bad == 0, f"{bad} unambiguous faces differ"
    assert not np.any(g[(ofl & oracle.ABSENT) != 0]), "a non-existing face was listed"
    return len(ids), namb, damb


def test_config0_analytic_bit_exact(q):
    psi = synth.analytic_line_ring()
    n, namb, damb = _check_full(q, psi)
    assert n > 150
    # the straight line alone: exactly one xy face per plane at (31, 30)
    ids, w, _ = gpu_identify(q, torch.from_numpy(synth.analytic_line_ring(with_ring=False)).cuda())
    assert len(ids) == 64 and set(w.tolist()) == {1}
    o, i, j, k = split_ids(ids, (64, 64, 64))
    assert set(o.tolist()) == {0} and set(i.tolist()) == {31} and set(j.tolist()) == {30}
    assert sorted(k.tolist()) == list(range(64))


@pytest.mark.parametrize("shape", [(33, 45, 67), (40, 50, 130), (20, 29, 200), (9, 15, 1024),
                                   (6, 8, 1999), (7, 14, 64), (17, 7, 128), (12, 13, 2),
                                   (11, 33, 248), (5, 16, 126), (8, 17, 992), (6, 31, 124),
                                   (4, 48, 250), (13, 3, 62), (4, 20, 1026), (5, 33, 1538),
                                   (3, 18, 1986), (4, 17, 1996), (3, 40, 2048)])
def test_ragged_random_waves_bit_exact(q, shape):
    psi = _waves(shape, seed=sum(shape))
    n, namb, damb = _check_full(q, psi)
    assert n > 0


@pytest.mark.parametrize("shape,kmin,kmax", [((10, 40, 992), 0.9, 1.5), ((9, 35, 500), 0.5, 0.9),
                                             ((7, 20, 300), 1.2, 2.0)])
def test_dense_tangles_bit_exact(q, shape, kmin, kmax):
    # short wavelengths: a plane band holds hundreds of lanes with faces, so the
    # expand pass takes both its register-held and its reloading path
    psi = synth.random_waves_numpy(shape, synth.wave_spec(sum(shape), 512, kmin=kmin, kmax=kmax))
    n, namb, damb = _check_full(q, psi)
    assert n > 0.03 * psi.size


def _all_pierced(shape):
    """A field whose every plaquette of all three orientations is pierced:
    phases 2 pi f / 5 with f a fixed pattern of period 2 in x, y and z (edge
    differences 0, +-2 pi / 5, +-4 pi / 5, none near +-pi), unit modulus."""
    f = np.array([0, 0, 1, 3, 3, 2, 1, 4])  # f[x % 2 + 2 (y % 2) + 4 (z % 2)]
    z, y, x = np.indices(shape)
    th = 2 * np.pi * f[x % 2 + 2 * (y % 2) + 4 * (z % 2)] / 5
    return np.exp(1j * th).astype(np.complex64)


@pytest.mark.parametrize("shape", [(3, 17, 2048), (3, 35, 1000), (4, 20, 66)])
def test_every_face_pierced(q, shape):
    # a 16-row band of a 2048-column plane then holds 3 x 16 x 2047 faces,
    # above 2^16: the expand pass's row offsets must not wrap
    psi = _all_pierced(shape)
    nz, ny, nx = shape
    full = (nx - 1) * (ny - 1) * nz + nx * (ny - 1) * (nz - 1) + (nx - 1) * ny * (nz - 1)
    n, namb, damb = _check_full(q, psi)
    assert n == full and namb == 0


@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 2, 2), (1, 5, 6), (3, 1, 7), (4, 6, 1),
                                   (2, 9, 3)])
def test_degenerate_grids(q, shape):
    psi = (np.random.default_rng(5).standard_normal(shape + (2,)).astype(np.float32)
           .view(np.complex64)[..., 0])
    _check_full(q, np.ascontiguousarray(psi))


def test_empty_grid(q):
    import paper_1911_12070_gb300 as qtv

    psi = torch.zeros((0, 4, 4), dtype=torch.complex64, device="cuda")
    count = torch.full((1,), 7, dtype=torch.int64, device="cuda")
    q.identify_into(psi, None, None, count)
    assert int(count.item()) == 0


def test_conjugation_flips_every_sign_256(q):
    psi = synth.random_waves((96, 160, 256), synth.wave_spec(21, 1024), device="cuda")
    ids, w, _ = gpu_identify(q, psi)
    idc, wc, _ = gpu_identify(q, torch.conj(psi).resolve_conj())
    # windings are exactly antisymmetric away from exact +-pi ties
    common = np.intersect1d(ids, idc)
    assert len(common) >= 0.999 * len(ids)
    wd = dict(zip(ids.tolist(), w.tolist()))
    wcd = dict(zip(idc.tolist(), wc.tolist()))
    assert all(wd[i] == -wcd[i] for i in common.tolist())


def test_closed_cells_zero_flux_on_gpu_output(q):
    psi = synth.random_waves((64, 96, 128), synth.wave_spec(3, 1024), device="cuda")
    ids, w, _ = gpu_identify(q, psi)
    d = dense_from_list(ids, w, tuple(psi.shape)).astype(np.int32)
    flux = ((d[0, 1:, :-1, :-1] - d[0, :-1, :-1, :-1]) + (d[1, :-1, :-1, 1:] - d[1, :-1, :-1, :-1])
            + (d[2, :-1, 1:, :-1] - d[2, :-1, :-1, :-1]))
    assert np.count_nonzero(flux) == 0


def test_nonfinite_nodes_zero_their_faces(q):
    psi = _waves((24, 40, 130), seed=9)
    psi[5, 10, 63] = np.complex64(complex(np.nan, 1.0))      # lane-31 / warp boundary column
    psi[6, 20, 64] = np.complex64(complex(np.inf, 0.0))      # first column of warp 1
    psi[12, 6, 7] = np.complex64(complex(0.0, -np.inf))      # band halo row (j = 7k - 1)
    psi[23, 39, 129] = np.complex64(complex(np.nan, np.nan))  # far corner
    n, namb, damb = _check_full(q, psi)
    st = gpu_identify(q, torch.from_numpy(psi).cuda(), stats=True)[2]
    ow, ofl = oracle.identify(psi)
    assert st["nonfinite_faces"] == int(np.count_nonzero(ofl & oracle.NONFINITE))


def test_zero_field_and_zero_nodes(q):
    psi = np.zeros((8, 9, 10), np.complex64)
    ids, w, st = gpu_identify(q, torch.from_numpy(psi).cuda(), stats=True)
    assert len(ids) == 0
    assert st["zero_node_faces"] == st["faces_scanned"] > 0
    # config 0 has four exact zeros of psi on the ring (oracle reading: phase 0)
    psi = synth.analytic_line_ring()
    _, _, st = gpu_identify(q, torch.from_numpy(psi).cuda(), stats=True)
    _, ofl = oracle.identify(psi)
    assert st["zero_node_faces"] == int(np.count_nonzero(ofl & oracle.ZERO_NODE)) == 48


def test_stats_counts(q):
    psi = _waves((40, 50, 130), seed=4)
    ids, w, st = gpu_identify(q, torch.from_numpy(psi).cuda(), stats=True)
    ow, ofl = oracle.identify(psi)
    assert st["pierced"] == len(ids) == int(np.count_nonzero(ow))
    assert st["faces_scanned"] == int(np.count_nonzero((ofl & oracle.ABSENT) == 0))
    amb = int(np.count_nonzero(ofl & oracle.AMBIGUOUS))
    assert abs(st["ambiguous"] - amb) <= max(2, amb // 10)


def test_capacity_overflow_reports_required_count(q):
    psi = torch.from_numpy(_waves((32, 64, 128), seed=8)).cuda()
    full_ids, full_w, _ = gpu_identify(q, psi)
    n = len(full_ids)
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    ids = torch.empty(n // 3, dtype=torch.int64, device="cuda")
    w = torch.empty(n // 3, dtype=torch.int8, device="cuda")
    q.identify_into(psi, ids, w, count)
    assert int(count.item()) == n
    # count-only call
    count.zero_()
    q.identify_into(psi, None, None, count)
    assert int(count.item()) == n
    # the binding retries with a larger capacity and gets the full list
    ids2, w2, _ = gpu_identify(q, psi, capacity=16)
    assert np.array_equal(ids2, full_ids) and np.array_equal(w2, full_w)


def test_repeat_calls_are_deterministic(q):
    psi = synth.random_waves((64, 128, 256), synth.wave_spec(5, 1024), device="cuda")
    a = gpu_identify(q, psi)
    b = gpu_identify(q, psi)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_config1_256_full_parity(q):
    psi = synth.config_field("256_waves", device="cuda", seed=1)
    host = psi.cpu().numpy()
    n, namb, damb = _check_full(q, host)
    dens = n / 256 ** 3
    assert 0.009 < dens < 0.012
    print(f"256^3 seed 1: {n} pierced faces, {namb} ambiguous ({damb} differing)")


@pytest.fixture(scope="module")
def field512():
    return synth.config_field("512_waves_noise", device="cuda")


def test_config2_512_sampled_planes(q, field512):
    psi = field512
    ids, w, st = gpu_identify(q, psi, stats=True)
    host = psi.cpu().numpy()
    shape = tuple(psi.shape)
    total_bad = 0
    for k0 in (0, 1, 6, 7, 137, 255, 256, 383, 510, 511):
        ow, ofl = oracle.identify(host, k0=k0, k1=k0 + 1)
        g = dense_from_list(ids, w, shape, k0=k0, k1=k0 + 1)
        bad, namb, damb = compare_windings(g, ow, ofl)
        total_bad += bad
    assert total_bad == 0
    assert st["pierced"] == len(ids)
    assert 0.009 < len(ids) / 512 ** 3 < 0.012


def test_config2_noise_does_not_change_windings(q, field512):
    clean = synth.random_waves((512, 512, 512), synth.wave_spec(7, 16384), device="cuda")
    a = gpu_identify(q, clean)
    b = gpu_identify(q, field512)
    common = np.intersect1d(a[0], b[0])
    # a positive real factor never moves a phase; only exact +-pi ties may differ
    assert len(common) >= len(a[0]) - 5 and len(common) >= len(b[0]) - 5
