"""GPU parity of the node form derived from the pierced-face list
(qtv_node_circulation_faces; Sec. 2.2.2: a ring's circulation is the sum of
the windings of the four plaquettes it encloses) against the node form from
psi (qtv_node_circulation, itself pinned to the FP64 oracle) and, on small
fields, against the oracle's ring sums directly.

Both lists must be equal element for element (ids ascending, the three S of
each node) on finite fields without winding-2 faces: ragged shapes, dense
tangles with branches, zero nodes, one-cell-thick grids, the 512^3 benchmark
field; plus the tie flag, a device count limit, capacity overflow and an
empty list.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def q():
    import paper_1911_12070_gb300 as qtv

    qtv.build()
    h = qtv.Qtv(0)
    yield h
    h.close()


def _both(q, psi):
    ids, w, _ = q.identify(psi)
    a_ids, a_circ, _ = q.node_circulation(psi)
    b_ids, b_circ, tie = q.node_circulation_faces(tuple(psi.shape), ids, w)
    return (a_ids, a_circ), (b_ids, b_circ, tie), (ids, w)


def _assert_equal(a, b):
    assert not b[2]
    assert torch.equal(a[0], b[0])
    assert torch.equal(a[1], b[1])


@pytest.mark.parametrize("shape,seed,waves", [((40, 48, 64), 81, 512), ((33, 45, 67), 82, 512),
                                              ((24, 64, 130), 83, 512), ((64, 64, 64), 84, 1024),
                                              ((3, 3, 3), 85, 64), ((2, 50, 70), 86, 256),
                                              ((17, 2, 90), 87, 256), ((20, 30, 1), 88, 256)])
def test_matches_psi_form(q, shape, seed, waves):
    psi = torch.from_numpy(synth.random_waves_numpy(shape, synth.wave_spec(seed, waves))).cuda()
    a, b, _ = _both(q, psi)
    _assert_equal(a, b)


def test_dense_tangle_with_noise(q):
    host = synth.random_waves_numpy((48, 56, 72), synth.wave_spec(89, 512, kmin=0.4, kmax=0.7))
    host = (host * (1.0 + 0.05 * np.random.default_rng(90).standard_normal(host.shape))
            ).astype(np.complex64)
    a, b, _ = _both(q, torch.from_numpy(host).cuda())
    assert a[0].numel() > 1000
    _assert_equal(a, b)


def test_zero_nodes(q):
    host = synth.random_waves_numpy((32, 40, 48), synth.wave_spec(91, 512))
    rng = np.random.default_rng(92)
    z = rng.integers(0, host.size, 200)
    host.reshape(-1)[z] = 0
    a, b, _ = _both(q, torch.from_numpy(host).cuda())
    _assert_equal(a, b)


def test_against_oracle_rings(q):
    """S of every ring whose four plaquettes the oracle does not flag
    (ambiguous edge or zero node) equals the oracle's FP64 ring sum."""
    host = synth.random_waves_numpy((20, 24, 28), synth.wave_spec(93, 512))
    ids, w, _ = q.identify(torch.from_numpy(host).cuda())
    b_ids, b_circ, tie = q.node_circulation_faces(host.shape, ids, w)
    assert not tie
    c, _ = oracle.node_circulation(host)
    s = np.rint(c / (2 * np.pi)).astype(np.int64)  # [3][nz][ny][nx]
    _, fl = oracle.identify(host)
    f = (fl & (oracle.AMBIGUOUS | oracle.ZERO_NODE)) != 0
    ex = np.zeros(c.shape, bool)
    ex[0, :, 1:-1, 1:-1] = (f[0, :, :-2, :-2] | f[0, :, :-2, 1:-1] | f[0, :, 1:-1, :-2]
                            | f[0, :, 1:-1, 1:-1])
    ex[1, 1:-1, 1:-1, :] = (f[1, :-2, :-2, :] | f[1, :-2, 1:-1, :] | f[1, 1:-1, :-2, :]
                            | f[1, 1:-1, 1:-1, :])
    ex[2, 1:-1, :, 1:-1] = (f[2, :-2, :, :-2] | f[2, :-2, :, 1:-1] | f[2, 1:-1, :, :-2]
                            | f[2, 1:-1, :, 1:-1])
    got = np.zeros((3, host.size), np.int64)
    got[:, b_ids.cpu().numpy()] = b_circ.cpu().numpy().astype(np.int64).T
    got = got.reshape(s.shape)
    assert (~ex).sum() > 0.9 * ex.size
    assert np.array_equal(got[~ex], s[~ex])


def test_512_workload(q):
    psi = synth.config_field("512_waves_noise", device="cuda")
    a, b, _ = _both(q, psi)
    assert a[0].numel() > 3_000_000
    _assert_equal(a, b)


def test_tie_count_limit_capacity_and_empty(q):
    shape = (32, 40, 48)
    psi = torch.from_numpy(synth.random_waves_numpy(shape, synth.wave_spec(94, 512))).cuda()
    ids, w, _ = q.identify(psi)
    ref_ids, ref_circ, tie = q.node_circulation_faces(shape, ids, w)
    assert not tie and ref_ids.numel() > 100
    # a face of winding 2 (W mod 4 = 2): flagged
    w2 = w.clone()
    w2[w2.numel() // 2] = 2
    _, _, tie2 = q.node_circulation_faces(shape, ids, w2)
    assert tie2
    # a device count limit: the same as the truncated list
    m = ids.numel() // 3
    ndev = torch.tensor([m], dtype=torch.int64, device="cuda")
    l_ids, l_circ, _ = q.node_circulation_faces(shape, ids, w, n_dev=ndev)
    t_ids, t_circ, _ = q.node_circulation_faces(shape, ids[:m].contiguous(), w[:m].contiguous())
    assert torch.equal(l_ids, t_ids) and torch.equal(l_circ, t_circ)
    # capacity below the count: the count is the total, the prefix is exact
    cap = ref_ids.numel() // 2
    out_ids = torch.zeros(cap, dtype=torch.int64, device="cuda")
    out_circ = torch.zeros((cap, 3), dtype=torch.int8, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    tie_d = torch.zeros(1, dtype=torch.int32, device="cuda")
    q.node_circulation_faces_into(shape, ids, w, out_ids, out_circ, count, tie_d)
    assert int(count.item()) == ref_ids.numel()
    assert torch.equal(out_ids, ref_ids[:cap]) and torch.equal(out_circ, ref_circ[:cap])
    # no faces: no vortex nodes
    e_ids, e_circ, e_tie = q.node_circulation_faces(
        shape, torch.empty(0, dtype=torch.int64, device="cuda"),
        torch.empty(0, dtype=torch.int8, device="cuda"))
    assert e_ids.numel() == 0 and not e_tie
