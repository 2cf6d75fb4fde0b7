"""GPU parity and behaviour of the learned locator (no counterpart in the
paper; trained on the plain localization of Sec. 3.3.3, Eq. 6).

* the encoding kernel equals the FP64 oracle encoding to BF16 rounding (plus
  the FP32 rounding of the phase rotation);
* the forward pass, the gradients of all six parameter tensors and the Adam
  update equal the FP64 oracle within BF16 tolerances (cosine > 0.999 and
  relative error < 2e-2 for the gradients);
* a checkpoint resumes training bit for bit;
* trained on noisy neighbourhoods (12 seeds of 256^3, about 2e6 faces) with
  labels from the plain solve of the clean field, the network's positions are
  within 0.05 h RMS of those labels on a held-out field; what it gains is
  measured against the plain method on the same noisy field and reported;
* learned localization falls back to the plain result exactly where it must.
"""
import os
import tempfile

import numpy as np
import pytest

import oracle
import synth
from oracle import mlp

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def q():
    import paper_1911_12070_gb300 as qtv

    qtv.build()
    h = qtv.Qtv(0)
    yield h
    h.close()


def bf16_to_f64(t):
    b = t.cpu().numpy().view(np.uint16).astype(np.uint32) << 16
    return b.view(np.float32).astype(np.float64)


def round_bf16(a):
    a32 = np.asarray(a, np.float32)
    bits = a32.view(np.uint32).astype(np.uint64)
    bits = (bits + 0x7FFF + ((bits >> 16) & 1)) >> 16
    return (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def params_to_dict(p):
    p = np.asarray(p, np.float64)
    o = 0
    d = {}
    for l, (fi, fo) in enumerate(zip(mlp.SIZES[:-1], mlp.SIZES[1:]), start=1):
        d[f"W{l}"] = p[o:o + fi * fo].reshape(fo, fi)
        o += fi * fo
        d[f"b{l}"] = p[o:o + fo].copy()
        o += fo
    assert o == p.size
    return d


def dict_to_params(d):
    return np.concatenate([np.concatenate([d[f"W{l}"].reshape(-1), d[f"b{l}"]]) for l in (1, 2, 3)])


@pytest.fixture(scope="module")
def small_faces(q):
    host = synth.random_waves_numpy((24, 40, 130), synth.wave_spec(12, 512))
    psi = torch.from_numpy(host).cuda()
    ids, w, _ = q.identify(psi)
    return host, psi, ids, w


def test_encoding_matches_oracle(q, small_faces):
    host, psi, ids, w = small_faces
    x, ok, rms = q.locator_encode(psi, ids, w)
    xo, oko, rmso = mlp.encode(host, ids.cpu().numpy().view(np.uint64), w.cpu().numpy())
    okg = ok.cpu().numpy().astype(bool)
    assert np.array_equal(okg, oko)
    assert okg.sum() > 100 and (~okg).sum() > 0
    xg = bf16_to_f64(x)[okg]
    ref = xo[okg]
    # BF16 rounding (half an ulp, 2^-8 relative) plus the FP32 rounding of the
    # phase rotation and normalisation, a few ulp of the unit-RMS block values
    assert np.all(np.abs(xg - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-5)
    assert np.allclose(rms.cpu().numpy()[okg], rmso[okg], rtol=1e-5)


def _batch(q, small_faces, n=128):
    host, psi, ids, w = small_faces
    x, ok, _ = q.locator_encode(psi, ids, w)
    xb = x[ok.bool()][:n].contiguous()
    assert xb.shape[0] == n
    rng = np.random.default_rng(1)
    t = torch.from_numpy(rng.uniform(0, 1, (n, 3)).astype(np.float32)).cuda()
    return xb, t


def _oracle_with_bf16_weights(q):
    p, _, _ = q.locator_get()
    d = params_to_dict(p)
    # the tensor cores see BF16 copies of W1 and W2
    d["W1"] = round_bf16(d["W1"])
    d["W2"] = round_bf16(d["W2"])
    return p, d


def test_forward_matches_oracle(q, small_faces):
    """The mma.sync layer kernels (the path training uses) against the FP64
    oracle."""
    q.locator_init(7)
    xb, _ = _batch(q, small_faces)
    q.locator_set_tensor_path(0)
    try:
        y = q.locator_forward(xb).cpu().numpy().astype(np.float64)
    finally:
        q.locator_set_tensor_path(1)
    _, d = _oracle_with_bf16_weights(q)
    yo, _ = mlp.forward(d, bf16_to_f64(xb))
    scale = np.sqrt(np.mean(yo ** 2))
    assert np.max(np.abs(y - yo)) < 2e-2 * scale


def test_tcgen05_forward_matches_oracle(q, small_faces):
    """The fused tcgen05 network (the default inference path: accumulators and
    hidden activations in tensor memory) against the FP64 oracle."""
    q.locator_init(7)
    xb, _ = _batch(q, small_faces)
    y = q.locator_forward(xb).cpu().numpy().astype(np.float64)
    _, d = _oracle_with_bf16_weights(q)
    yo, _ = mlp.forward(d, bf16_to_f64(xb))
    scale = np.sqrt(np.mean(yo ** 2))
    assert np.max(np.abs(y - yo)) < 2e-2 * scale


@pytest.mark.parametrize("n", [1, 64, 129, 128 * 151 + 1])
def test_tcgen05_forward_small_and_ragged(q, n):
    """Row counts below one tile, one row past a tile, and one row past one
    tile per SM (the grid smaller than, or one tile past, the SM count): the
    tensor copies read the rows past the end as zeros and the first and last
    rows match the oracle."""
    q.locator_init(11)
    g = torch.Generator(device="cpu").manual_seed(n)
    xf = torch.randn((n, 128), generator=g) * 0.7
    x = xf.to(torch.bfloat16).view(torch.int16).cuda()
    y = q.locator_forward(x)
    _, d = _oracle_with_bf16_weights(q)
    rows = np.unique(np.r_[0:min(n, 3), max(0, n - 3):n])
    yo, _ = mlp.forward(d, bf16_to_f64(x[torch.from_numpy(rows).cuda()]))
    # the output scale of this network on 256 rows of the same distribution
    xs = (torch.randn((256, 128), generator=g) * 0.7).to(torch.bfloat16).view(torch.int16)
    ys, _ = mlp.forward(d, bf16_to_f64(xs))
    scale = float(np.sqrt(np.mean(ys ** 2)))
    assert y.shape == (n, 3) and bool(torch.isfinite(y).all())
    assert np.max(np.abs(y[torch.from_numpy(rows).cuda()].cpu().numpy() - yo)) < 2e-2 * scale


def test_tcgen05_matches_mma_path_on_many_tiles(q):
    """Ragged row count over many 128-row tiles (more tiles than SMs, so every
    persistent CTA loops and prefetches): the two tensor paths agree to
    accumulation order."""
    q.locator_init(3)
    n = 128 * 152 * 3 + 77
    g = torch.Generator(device="cpu").manual_seed(5)
    xf = torch.randn((n, 128), generator=g) * 0.7
    x = xf.to(torch.bfloat16).view(torch.int16).cuda()
    q.locator_set_tensor_path(0)
    try:
        y0 = q.locator_forward(x)
    finally:
        q.locator_set_tensor_path(1)
    y1 = q.locator_forward(x)
    scale = float(torch.sqrt(torch.mean(y0 ** 2)))
    assert torch.isfinite(y1).all()
    assert float(torch.max(torch.abs(y1 - y0))) < 2e-2 * scale
    # rows on both sides of tile and CTA boundaries against the FP64 oracle
    _, d = _oracle_with_bf16_weights(q)
    rows = np.r_[0:3, 125:131, 127 * 152 - 2:127 * 152 + 3, n - 80:n]
    yo, _ = mlp.forward(d, bf16_to_f64(x[torch.from_numpy(rows).cuda()]))
    assert np.max(np.abs(y1[torch.from_numpy(rows).cuda()].cpu().numpy() - yo)) < 2e-2 * scale


def test_gradients_match_oracle(q, small_faces):
    q.locator_init(11)
    xb, t = _batch(q, small_faces)
    g, loss = q.locator_gradients(xb, t)
    gg = params_to_dict(g.cpu().numpy())
    _, d = _oracle_with_bf16_weights(q)
    lo, go = mlp.loss_and_grads(d, bf16_to_f64(xb), t.cpu().numpy().astype(np.float64))
    assert abs(float(loss.item()) - lo) < 1e-2 * lo
    for key in ("W1", "b1", "W2", "b2", "W3", "b3"):
        a, b = gg[key].reshape(-1), go[key].reshape(-1)
        cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b))
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        assert cos > 0.999 and rel < 2e-2, (key, cos, rel)


@pytest.fixture(scope="module")
def more_faces(q):
    host = synth.random_waves_numpy((64, 96, 128), synth.wave_spec(14, 512))
    psi = torch.from_numpy(host).cuda()
    ids, w, _ = q.identify(psi)
    return host, psi, ids, w


@pytest.mark.parametrize("n", [64, 192, 4096])
def test_tcgen05_training_gradients_match_oracle(q, more_faces, n):
    """Training on tcgen05 (the default path): forward, data-gradient and
    weight-gradient GEMMs with accumulators in tensor memory, batches of 1, 3
    and 64 K chunks of 64 rows (the weight gradients split along the batch
    into 1, 3 and 16 parts summed in a fixed order), against the FP64 oracle;
    and against the mma.sync layer kernels (the same BF16 operands, another
    accumulation order)."""
    q.locator_init(21)
    xb, t = _batch(q, more_faces, n=n)
    q.locator_set_tensor_path(1)
    g1, loss1 = q.locator_gradients(xb, t)
    q.locator_set_tensor_path(0)
    try:
        g0, loss0 = q.locator_gradients(xb, t)
    finally:
        q.locator_set_tensor_path(1)
    _, d = _oracle_with_bf16_weights(q)
    lo, go = mlp.loss_and_grads(d, bf16_to_f64(xb), t.cpu().numpy().astype(np.float64))
    assert abs(float(loss1.item()) - lo) < 1e-2 * lo
    gg1 = params_to_dict(g1.cpu().numpy())
    gg0 = params_to_dict(g0.cpu().numpy())
    for key in ("W1", "b1", "W2", "b2", "W3", "b3"):
        a, b = gg1[key].reshape(-1), go[key].reshape(-1)
        cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b))
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        assert cos > 0.999 and rel < 2e-2, (key, cos, rel)
        c = gg0[key].reshape(-1)
        assert np.linalg.norm(a - c) / np.linalg.norm(c) < 1e-2, key
    # deterministic: the same gradients bit for bit on a second call
    g2, _ = q.locator_gradients(xb, t)
    assert torch.equal(g1, g2)


def test_adam_step_matches_oracle(q, small_faces):
    q.locator_init(13)
    xb, t = _batch(q, small_faces)
    p0, _, s0 = q.locator_get()
    g, _ = q.locator_gradients(xb, t)
    q.locator_train_step(xb, t, lr=1e-3)
    torch.cuda.synchronize()
    p1, adam, s1 = q.locator_get()
    assert s1 == s0 + 1
    d = params_to_dict(p0)
    gd = params_to_dict(g.cpu().numpy())
    m = {k: np.zeros_like(v) for k, v in d.items()}
    v = {k: np.zeros_like(v) for k, v in d.items()}
    mlp.adam_step(d, gd, m, v, t=1, lr=1e-3)
    ref = dict_to_params(d)
    assert np.max(np.abs(p1 - ref)) < 1e-6
    assert np.allclose(adam[:len(p1)], dict_to_params(m), rtol=1e-5, atol=1e-12)


def test_checkpoint_resumes_bit_exactly(q, small_faces):
    import paper_1911_12070_gb300 as qtv

    xb, t = _batch(q, small_faces)
    q.locator_init(17)
    for _ in range(5):
        q.locator_train_step(xb, t, lr=1e-3)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "loc.qtv")
        q.locator_save(path)
        for _ in range(3):
            q.locator_train_step(xb, t, lr=1e-3)
        pa, aa, sa = q.locator_get()
        q2 = qtv.Qtv(0)
        q2.locator_load(path)
        for _ in range(3):
            q2.locator_train_step(xb, t, lr=1e-3)
        pb, ab, sb = q2.locator_get()
        q2.close()
        # a corrupted file is rejected
        raw = bytearray(open(path, "rb").read())
        raw[100] ^= 0xFF
        open(path, "wb").write(bytes(raw))
        with pytest.raises(qtv.QtvError):
            q.locator_load(path)
    assert sa == sb == 8
    assert np.array_equal(pa, pb) and np.array_equal(aa, ab)


@pytest.fixture(scope="module")
def trained(q):
    from paper_1911_12070_gb300 import learned

    losses = learned.fit(q)
    clean, noisy = learned.field_pair(120, 256, 4096, 0.05, "cuda")
    test = learned.make_examples(q, clean, noisy)
    return losses, test, clean, noisy


def test_training_reduces_loss_and_meets_accuracy(q, trained):
    from paper_1911_12070_gb300 import learned

    losses, test, clean, noisy = trained
    assert losses[-50:].mean() < 0.1 * losses[:10].mean()
    y = q.locator_forward(test["x"])
    rms_learned = learned.rms_h(y[:, :2], test["t"][:, :2])
    print(f"held-out: {len(test['t'])} faces, learned RMS {rms_learned:.4f} h")
    assert rms_learned <= 0.05


def _gain(q, noise):
    """(plain RMS, network RMS, worst-decile plain RMS, network RMS there) in h
    against the clean plain cores of the held-out field (seed 120) with the
    given multiplicative noise: plain solves the noisy field, the network
    sees the noisy 4 x 4 x 4 neighbourhoods."""
    from paper_1911_12070_gb300 import learned

    clean, noisy = learned.field_pair(120, 256, 4096, noise, "cuda")
    test = learned.make_examples(q, clean, noisy)
    y = q.locator_forward(test["x"])
    xyz_n, _, _ = q.localize(noisy, test["ids"], test["w"])
    uvp = learned.face_uv(test["ids"], xyz_n, tuple(noisy.shape))
    ep = torch.sqrt(torch.sum((uvp - test["t"][:, :2]) ** 2, 1))
    el = torch.sqrt(torch.sum((y[:, :2] - test["t"][:, :2]) ** 2, 1))
    hard = ep > torch.quantile(ep, 0.9)
    rms = lambda e: float(torch.sqrt(torch.mean(e ** 2)))  # noqa: E731
    return rms(ep), rms(el), rms(ep[hard]), rms(el[hard])


def test_gain_over_plain_on_noisy_field(q, trained):
    """What the network adds, measured against the clean plain cores.  At 5%
    noise the plain zero of the noisy field is 0.015 h away and the network
    0.019 h: no gain on average, but on the tenth of the faces where the plain
    solve is worst (a noisy corner moves the zero most) the network, which
    sees 64 nodes, is closer (about 0.021 against 0.030 h)."""
    p, n, ph, nh = _gain(q, 0.05)
    print(f"5% noise vs clean cores: plain {p:.4f} h, network {n:.4f} h; "
          f"worst-decile plain faces: plain {ph:.4f} h, network {nh:.4f} h")
    assert p <= 0.05 and n <= 0.05
    assert nh < 0.85 * ph


def test_gain_at_higher_noise():
    """A locator trained and tested at 15% noise: the network's 64-node
    receptive field averages the noise the 4-corner solve cannot (measured
    about 0.026 h against 0.046 h for plain), so it gains over the method
    without it on all faces."""
    import paper_1911_12070_gb300 as qtv
    from paper_1911_12070_gb300 import learned

    q2 = qtv.Qtv(0)
    try:
        learned.fit(q2, noise=0.15)
        p, n, ph, nh = _gain(q2, 0.15)
    finally:
        q2.close()
    print(f"15% noise vs clean cores: plain {p:.4f} h, network {n:.4f} h; "
          f"worst-decile plain faces: plain {ph:.4f} h, network {nh:.4f} h")
    assert n <= 0.05 and n < 0.75 * p and nh < 0.5 * ph


def test_learned_localize_tcgen05_path(q, trained):
    """Learned localization on the tcgen05 network: the same faces accepted (up
    to a handful at the acceptance threshold) and positions close to the
    mma.sync layer kernels: RMS difference below 1e-3 h, every face within
    1e-2 h (the accumulation orders differ, which can flip the BF16 rounding of
    a hidden activation)."""
    import paper_1911_12070_gb300 as qtv

    _, test, clean, noisy = trained
    ids, w = test["ids"], test["w"]
    q.locator_set_tensor_path(0)
    try:
        xyz0, _, fl0 = q.localize(clean, ids, w, mode=qtv.LEARNED, fallback_resid=1e-3)
    finally:
        q.locator_set_tensor_path(1)
    xyz1, _, fl1 = q.localize(clean, ids, w, mode=qtv.LEARNED, fallback_resid=1e-3)
    same = fl0 == fl1
    assert float(same.float().mean()) > 0.999
    d = torch.linalg.norm(xyz1 - xyz0, dim=1)[same]
    print(f"tcgen05 vs mma.sync: RMS {float(torch.sqrt(torch.mean(d ** 2))):.2e} h, "
          f"max {float(d.max()):.2e} h")
    assert float(torch.sqrt(torch.mean(d ** 2))) < 1e-3
    assert float(d.max()) < 1e-2


def test_learned_localize_fallback_is_plain(q, trained):
    import paper_1911_12070_gb300 as qtv

    _, test, clean, noisy = trained
    ids, w = test["ids"], test["w"]
    xyz_l, resid_l, flags_l = q.localize(clean, ids, w, mode=qtv.LEARNED, fallback_resid=1e-3)
    xyz_p, resid_p, flags_p = q.localize(clean, ids, w)
    fl = flags_l.cpu().numpy()
    learned_mask = (fl & qtv.FLAG_LEARNED) != 0
    fb = (fl & qtv.FLAG_FALLBACK) != 0
    assert np.all(learned_mask ^ fb)
    assert torch.equal(xyz_l[torch.from_numpy(fb).cuda()], xyz_p[torch.from_numpy(fb).cuda()])
    d = torch.linalg.norm(xyz_l - xyz_p, dim=1).cpu().numpy()
    print(f"learned accepted {learned_mask.mean():.3f}, RMS vs plain {np.sqrt(np.mean(d**2)):.4f} h")
    assert np.sqrt(np.mean(d ** 2)) <= 0.05


def test_learned_batch_against_oracle(q, trained):
    """The uneven batch with the trained locator on (the batched workload runs
    it): every face is accepted (LEARNED) or falls back (FALLBACK), never both;
    fallback samples are the oracle's plain zeros within 1e-4 h (Sec. 3.3.3,
    Eq. 6) on unambiguous, well-conditioned faces; an accepted sample lies in
    its face, its reported residual is the oracle's interpolated density there
    (linear interpolation, Sec. 5), that density meets the acceptance rule
    against the oracle's neighbourhood RMS, and accepted samples are within
    0.05 h RMS of the oracle's plain zeros."""
    import paper_1911_12070_gb300 as qtv
    from oracle import mlp
    from qtv_testutil import compare_positions

    shapes = [(40, 48, 130), (24, 64, 96), (33, 45, 66)]
    hosts = [synth.multiplicative_noise(
        synth.random_waves_numpy(s, synth.wave_spec(400 + i, 512)), 500 + i)
        for i, s in enumerate(shapes)]
    devs = [torch.from_numpy(h).cuda() for h in hosts]
    q.batch_plan(devs)
    out = q.batch_run(mode=qtv.LEARNED, fallback_resid=1e-3)
    n_acc = n_all = 0
    for host, d in zip(hosts, out):
        ids = d["ids"].cpu().numpy().view(np.uint64)
        w = d["w"].cpu().numpy()
        xyz = d["xyz"].cpu().numpy()
        resid = d["resid"].cpu().numpy()
        fl = d["flags"].cpu().numpy()
        acc = (fl & qtv.FLAG_LEARNED) != 0
        fb = (fl & qtv.FLAG_FALLBACK) != 0
        assert np.all(acc ^ fb)
        ora = oracle.localize(host, ids, w)
        _, ofl = oracle.identify(host)
        o = (ids & np.uint64(3)).astype(np.int64)
        lin = (ids >> np.uint64(2)).astype(np.int64)
        f = ofl.reshape(3, -1)[o, lin]
        ok = ((ora["flags"] & (oracle.L_ANOMALOUS | oracle.L_ILLCOND)) == 0) & \
            ((f & (oracle.AMBIGUOUS | oracle.ZERO_NODE)) == 0)
        bad, emax = compare_positions(xyz[fb], {"xyz": ora["xyz"][fb]}, ok[fb])
        assert bad == 0, (bad, emax)
        m2 = float(np.max(np.abs(host.astype(np.complex128)) ** 2))
        _, okenc, rms = mlp.encode(host, ids[acc], w[acc])
        assert okenc.all()
        corner = np.column_stack([lin % host.shape[2], (lin // host.shape[2]) % host.shape[1],
                                  lin // (host.shape[2] * host.shape[1])])[acc]
        normal = np.array([2, 0, 1])[o[acc]]  # the axis the face does not span
        rel = xyz[acc] - corner
        assert np.all(np.abs(rel[np.arange(len(rel)), normal]) == 0)
        assert np.all((rel > -0.01 - 1e-5) & (rel < 1.01 + 1e-5))
        # inside the face the trilinear interpolant the oracle evaluates is the
        # face's bilinear one (a sample up to 0.01 beyond an edge is in the
        # neighbouring face's territory, where the two differ)
        inside = np.all((rel >= 0) & (rel <= 1), axis=1)
        rho = oracle.density(host, xyz[acc][inside].astype(np.float64))
        # |F| at the FP32 sample against |F| at its FP32 grid coordinates: the
        # coordinates round by |x| 2^-24, and |grad F| <= 4 max|psi| on a face
        slack = (4 * np.sqrt(m2) * np.max(np.abs(xyz[acc][inside]), axis=1) * 2.0 ** -23 +
                 1e-6 * np.sqrt(m2))
        assert np.all(np.abs(np.sqrt(resid[acc][inside]) - np.sqrt(rho)) <= slack)
        assert np.all(np.sqrt(rho) <= np.sqrt(1e-3) * rms[inside] + slack)
        assert inside.mean() > 0.9
        dd = np.linalg.norm(xyz[acc] - ora["xyz"][acc], axis=1)
        assert np.sqrt(np.mean(dd ** 2)) <= 0.05
        n_acc += int(acc.sum())
        n_all += len(ids)
    print(f"learned batch: {n_acc} of {n_all} faces accepted")
    assert n_acc > 0.8 * n_all
