"""GPU parity of batched identification (Sec. 2.2.2, Eq. 5) and localization
(Sec. 3.3.3, Eq. 6): many snapshots of uneven sizes in one persistent sweep
launch, one finalize pass and one localization pass, replayed as a CUDA graph.

* every snapshot's slice of the batch output equals the FP64 oracle bit for
  bit on unambiguous faces (windings) and within 1e-4 h (positions), for each
  sweep shape (nibble sweep: one tile width of 64 to 1024 columns for all
  snapshots, or one sweep per row-width group, serial or concurrent;
  bit-sliced sweep: tiles of 62, 124 or 248 columns, 2 or 3 ring stages,
  rows up to 2048 columns;
  various CTAs per SM and z-block heights), shapes pinned through a
  tune-cache line with the key "*";
* the slices equal the single-snapshot calls bit for bit (ids, windings, plain
  and learned positions and flags);
* capacity overflow reports the total, replays are deterministic, and new data
  written into the planned buffers is picked up by the replay;
* the autotuner stores its choice in the cache and a second plan reads it;
* the full 16-snapshot workload (8 x 256^3, 4 x 384^3, 3 x 512^3, 1 x 768^3)
  matches the oracle on sampled planes of every snapshot.
"""
import os
import tempfile

import numpy as np
import pytest

import oracle
import synth
from qtv_testutil import compare_positions, compare_windings, dense_from_list

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SMALL = [(20, 40, 130), (13, 29, 64), (9, 15, 1024), (7, 33, 200), (16, 16, 2), (1, 5, 6),
         (25, 31, 384), (3, 8, 66)]
# the bit-sliced sweep also takes rows wider than the nibble sweep's 1024
# columns (up to 96 tile warps of 31 columns per band row)
SMALL_BITS = [(20, 40, 130), (13, 33, 64), (9, 15, 992), (7, 34, 200), (16, 16, 2), (1, 5, 6),
              (25, 31, 384), (3, 8, 66), (6, 17, 124), (5, 18, 126), (4, 20, 2048),
              (3, 18, 1986)]


@pytest.fixture(scope="module")
def q():
    import paper_1911_12070_gb300 as qtv

    qtv.build()
    h = qtv.Qtv(0)
    yield h
    h.close()


def _fields(shapes, seed0):
    hosts = [synth.random_waves_numpy(s, synth.wave_spec(seed0 + i, 512)) for i, s in enumerate(shapes)]
    return hosts, [torch.from_numpy(h).cuda() for h in hosts]


@pytest.fixture(scope="module")
def small_batch():
    return _fields(SMALL, 300)


@pytest.fixture(scope="module")
def small_batch_bits():
    return _fields(SMALL_BITS, 350)


def _pin(path, nwt, ctas, zscale, concurrent=0, variant=0, stages=3):
    with open(path, "w") as f:
        f.write(f"qtv-tune-v3 * {variant} {nwt} {ctas} {zscale} {concurrent} {stages} 0.0\n")


def _check_slices(hosts, out):
    for host, d in zip(hosts, out):
        ids = d["ids"].cpu().numpy().view(np.uint64)
        w = d["w"].cpu().numpy()
        assert np.all(np.diff(ids.astype(np.int64)) > 0)
        ow, ofl = oracle.identify(host)
        g = dense_from_list(ids, w, host.shape)
        bad, _, _ = compare_windings(g, ow, ofl)
        assert bad == 0, f"{bad} unambiguous faces differ in a {host.shape} snapshot"
        assert not np.any(g[(ofl & oracle.ABSENT) != 0])
        if len(ids) == 0:
            continue
        ora = oracle.localize(host, ids, w)
        o = (ids & np.uint64(3)).astype(np.int64)
        lin = (ids >> np.uint64(2)).astype(np.int64)
        f = ofl.reshape(3, -1)[o, lin]
        ok = ((ora["flags"] & (oracle.L_ANOMALOUS | oracle.L_ILLCOND)) == 0) & \
             ((f & (oracle.AMBIGUOUS | oracle.ZERO_NODE)) == 0)
        nbad, emax = compare_positions(d["xyz"].cpu().numpy(), ora, ok)
        assert nbad == 0, f"{nbad} positions off in a {host.shape} snapshot (max {emax})"


@pytest.mark.parametrize("shape", [(1, 0, 1.0, 0), (2, 0, 0.5, 0), (4, 2, 1.0, 0), (8, 1, 2.0, 0),
                                   (16, 0, 1.0, 0), (4, 0, 3.0, 0), (0, 0, 1.0, 0),
                                   (0, 0, 1.0, 1), (0, 1, 0.5, 1)])
def test_small_batch_matches_oracle_for_each_tile_shape(q, small_batch, shape):
    hosts, devs = small_batch
    nwt, ctas, zs, conc = shape
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "tune.txt")
        _pin(path, nwt, ctas, zs, conc)
        info = q.batch_plan(devs, tune_cache=path)
    assert info["source"] == 1 and info["warps_per_tile"] == nwt
    assert info["concurrent"] == conc and info["variant"] == 0
    # per-snapshot widths: one sweep per distinct row width in warps
    assert info["sweeps"] == (1 if nwt else len({(s[2] + 63) // 64 for s in SMALL}))
    out = q.batch_run()
    _check_slices(hosts, out)


@pytest.mark.parametrize("shape", [(2, 0, 1.0, 2), (4, 0, 1.0, 3), (8, 0, 2.0, 2), (4, 1, 0.5, 3),
                                   (8, 1, 1.0, 3)])
def test_small_batch_bit_sliced_sweep_matches_oracle(q, small_batch_bits, shape):
    hosts, devs = small_batch_bits
    nwt, ctas, zs, stages = shape
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "tune.txt")
        _pin(path, nwt, ctas, zs, 0, variant=1, stages=stages)
        info = q.batch_plan(devs, tune_cache=path)
    assert info["source"] == 1 and info["variant"] == 1 and info["warps_per_tile"] == nwt
    out = q.batch_run()
    _check_slices(hosts, out)


def test_wide_snapshots_autotuned(q):
    # snapshots wider than the nibble sweep's 1024 columns: the counting pass
    # and every candidate the autotuner keeps use the bit-sliced sweep
    hosts, devs = _fields([(4, 20, 2048), (6, 24, 130), (3, 17, 1538)], 370)
    with tempfile.TemporaryDirectory() as d:
        info = q.batch_plan(devs, tune_cache=os.path.join(d, "tune.txt"))
    assert info["source"] == 2 and info["variant"] == 1
    out = q.batch_run()
    _check_slices(hosts, out)
    for dev, d in zip(devs, out):
        ids, w, _ = q.identify(dev)
        assert torch.equal(ids, d["ids"]) and torch.equal(w, d["w"])


def test_batch_equals_single_calls(q, small_batch):
    import paper_1911_12070_gb300 as qtv

    hosts, devs = small_batch
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "tune.txt")
        _pin(path, 0, 0, 1.0, 1)
        q.batch_plan(devs, tune_cache=path)
    out = q.batch_run()
    q.locator_init(5)
    outl = q.batch_run(mode=qtv.LEARNED, fallback_resid=1e-3)
    for dev, d, dl in zip(devs, out, outl):
        ids, w, _ = q.identify(dev)
        assert torch.equal(ids, d["ids"]) and torch.equal(w, d["w"])
        assert torch.equal(ids, dl["ids"])
        if ids.numel() == 0:
            continue
        xyz, resid, fl = q.localize(dev, ids, w)
        assert torch.equal(xyz, d["xyz"]) and torch.equal(resid, d["resid"])
        assert torch.equal(fl, d["flags"])
        xyzl, residl, fll = q.localize(dev, ids, w, mode=qtv.LEARNED, fallback_resid=1e-3)
        assert torch.equal(fll, dl["flags"])
        assert torch.equal(xyzl, dl["xyz"]) and torch.equal(residl, dl["resid"])


def test_capacity_overflow_and_replay(q, small_batch):
    hosts, devs = small_batch
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "tune.txt")
        _pin(path, 4, 0, 1.0)
        info = q.batch_plan(devs, tune_cache=path)
    total = info["faces"]
    n = len(devs)
    dev = devs[0].device
    cap = total // 2
    ids = torch.empty(cap, dtype=torch.int64, device=dev)
    w = torch.empty(cap, dtype=torch.int8, device=dev)
    off = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    q.batch_run_into(ids, w, off)
    torch.cuda.synchronize()
    assert int(off[n]) == total
    full = q.batch_run()
    got = torch.cat([x["ids"] for x in full])
    assert torch.equal(ids, got[:cap])
    # replays of the captured graph are deterministic
    a = q.batch_run(capacity=total + 7)
    b = q.batch_run(capacity=total + 7)
    for x, y in zip(a, b):
        assert torch.equal(x["ids"], y["ids"]) and torch.equal(x["xyz"], y["xyz"])


def test_replay_sees_new_data_in_planned_buffers(q):
    shapes = [(12, 20, 96), (10, 24, 160)]
    devs = [torch.from_numpy(synth.random_waves_numpy(s, synth.wave_spec(400 + i, 512))).cuda()
            for i, s in enumerate(shapes)]
    q.batch_plan(devs)
    cap = 20000
    ids = torch.empty(cap, dtype=torch.int64, device="cuda")
    w = torch.empty(cap, dtype=torch.int8, device="cuda")
    off = torch.zeros(3, dtype=torch.int64, device="cuda")
    xyz = torch.empty((cap, 3), dtype=torch.float32, device="cuda")
    resid = torch.empty(cap, dtype=torch.float32, device="cuda")
    fl = torch.empty(cap, dtype=torch.uint8, device="cuda")
    q.batch_run_into(ids, w, off, xyz, resid, fl)
    hosts = [synth.random_waves_numpy(s, synth.wave_spec(500 + i, 512)) for i, s in enumerate(shapes)]
    for dv, hst in zip(devs, hosts):
        dv.copy_(torch.from_numpy(hst))
    q.batch_run_into(ids, w, off, xyz, resid, fl)  # same outputs: graph replay
    o = off.cpu().numpy()
    assert int(o[2]) <= cap
    out = [{"ids": ids[o[i]:o[i + 1]], "w": w[o[i]:o[i + 1]], "xyz": xyz[o[i]:o[i + 1]]}
           for i in range(2)]
    _check_slices(hosts, out)


def test_autotuner_stores_and_reuses_choice(q, small_batch):
    _, devs = small_batch
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "tune.txt")
        info = q.batch_plan(devs, tune_cache=path)
        assert info["source"] == 2 and info["candidates"] >= 6 and info["tuned_ms"] > 0
        lines = open(path).read().splitlines()
        assert len(lines) == 1 and lines[0].startswith("qtv-tune-v3 ")
        info2 = q.batch_plan(devs, tune_cache=path)
        assert info2["source"] == 1
        for k in ("variant", "warps_per_tile", "ctas_per_sm", "zscale", "concurrent", "stages"):
            assert info2[k] == info[k]


def test_full_batch16_sampled_planes(q):
    """The 16-snapshot workload that the benchmark times, in the launch
    configuration the autotuner picks: every snapshot checked on sampled
    planes against the oracle."""
    devs = synth.batch_fields("cuda")
    info = q.batch_plan(devs)
    out = q.batch_run()
    assert sum(d["ids"].numel() for d in out) == info["faces"]
    total_bad = 0
    for psi, d in zip(devs, out):
        n = psi.shape[0]
        ids = d["ids"].cpu().numpy().view(np.uint64)
        w = d["w"].cpu().numpy()
        assert np.all(np.diff(ids.astype(np.int64)) > 0)
        assert 0.009 < len(ids) / psi.numel() < 0.012
        for k0 in (0, n // 2 - 1, n - 1):
            slab = psi[k0:k0 + 2].cpu().numpy()
            ow, ofl = oracle.identify(slab, k0=0, k1=1)
            sel = ((ids >> np.uint64(2)) // np.uint64(psi.shape[1] * psi.shape[2])) == k0
            sid = ids[sel] - np.uint64(k0 * psi.shape[1] * psi.shape[2] * 4)
            g = dense_from_list(sid, w[sel], slab.shape, k0=0, k1=1)
            bad, _, _ = compare_windings(g, ow, ofl)
            total_bad += bad
            # positions of the plane's faces
            xyz = d["xyz"].cpu().numpy()[sel]
            ora = oracle.localize(slab, sid, w[sel])
            ok = (ora["flags"] & (oracle.L_ANOMALOUS | oracle.L_ILLCOND)) == 0
            ora["xyz"] = ora["xyz"] + np.array([0.0, 0.0, float(k0)])
            nbad, emax = compare_positions(xyz, ora, ok)
            assert nbad == 0, f"{nbad} positions off (max {emax})"
    assert total_bad == 0
