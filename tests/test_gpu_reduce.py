"""GPU parity of the box-mean reduction (Sec. 3.3.1-3.3.2, lattice reading:
qtv_box_reduce) through the C ABI against the oracle's graph.box_reduce:
cluster labels and fixed-point mean positions bit for bit, and the number of
passes, on the face graphs of random-wave tangles (branches included), on
the paper's node graph, on hand graphs with closed forms, with a device
count limit, one pass, empty input, and on the 512^3 workload (every face
through the GPU; the oracle on the first 64 planes, clusters that lie well
inside them compared)."""
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


def _table(adj, stride):
    n = len(adj)
    nbr = np.full((max(n, 1), stride), -1, np.int32)
    deg = np.zeros(max(n, 1), np.uint8)
    for a, s in enumerate(adj):
        v = sorted(s)
        nbr[a, :len(v)] = v
        deg[a] = len(v)
    return torch.from_numpy(nbr[:n]).cuda(), torch.from_numpy(deg[:n]).cuda()


def _gpu(q, g, box, stride=10, max_passes=10):
    nbr, deg = _table(g.adj, stride)
    xyz = torch.from_numpy(g.pos.astype(np.float32)).cuda()
    label, reps, pos, passes = q.box_reduce(nbr, deg, xyz, box=box, max_passes=max_passes)
    return label.cpu().numpy(), reps.cpu().numpy(), pos.cpu().numpy(), passes


def _check(q, g, box, stride=10, max_passes=10):
    g = graph.Graph(g.pos.astype(np.float32).astype(np.float64), g.dirs, g.adj)
    red, lab, qfix, passes = graph.box_reduce(g, box, max_passes=max_passes)
    glab, greps, gpos, gpasses = _gpu(q, g, box, stride, max_passes)
    assert gpasses == passes
    assert np.array_equal(glab, lab)
    assert np.array_equal(greps, np.unique(lab))
    assert np.array_equal(gpos, red.pos)  # exact: both are fixed-point means
    return red, passes


def _face_graph_of(q, host):
    dev = torch.from_numpy(host).cuda()
    ids, w, xyz, _, _ = q.identify_localize(dev)
    return graph.face_graph(ids.cpu().numpy().view(np.uint64), w.cpu().numpy(),
                            xyz.cpu().numpy().astype(np.float64), host.shape)


@pytest.mark.parametrize("shape,seed,box", [((40, 48, 64), 71, 4.0), ((33, 45, 67), 72, 3.0),
                                            ((24, 64, 130), 73, 6.0), ((64, 64, 64), 74, 4.0)])
def test_face_graph_reduction_matches_oracle(q, shape, seed, box):
    g = _face_graph_of(q, synth.random_waves_numpy(shape, synth.wave_spec(seed, 512)))
    red, passes = _check(q, g, box)
    deg = red.degrees()
    print(f"{shape}: {g.n} samples -> {red.n} means in {passes} passes, "
          f"{int(np.sum(deg > 2))} branch means")
    assert red.n < g.n / 2


def test_dense_tangle_with_branches(q):
    host = synth.random_waves_numpy((48, 48, 48), synth.wave_spec(75, 512, kmin=0.4, kmax=0.7))
    g = _face_graph_of(q, host)
    assert np.any(g.degrees() > 2)
    _check(q, g, 4.0)


def test_node_graph_reduction_matches_oracle(q):
    psi = synth.random_waves_numpy((40, 40, 40), synth.wave_spec(76, 512))
    c, v = oracle.node_circulation(psi)
    g = graph.node_graph(v.astype(bool), c)
    _check(q, g, 4.0, stride=6)


def test_uneven_chain_by_hand(q):
    xs = np.arange(0.0, 20.0, 0.75)
    pos = np.stack([xs, np.full_like(xs, 3.0), np.full_like(xs, 5.0)], 1)
    adj = [set(x for x in (a - 1, a + 1) if 0 <= x < len(xs)) for a in range(len(xs))]
    g = graph.Graph(pos, np.zeros_like(pos), adj)
    red, passes = _check(q, g, 4.0)
    assert passes == 4 and list(red.pos[:, 0]) == [1.875, 7.875, 13.875, 18.0]


def test_one_pass_device_limit_and_empty(q):
    import paper_1911_12070_gb300 as qtv

    g = _face_graph_of(q, synth.random_waves_numpy((32, 40, 48), synth.wave_spec(77, 512)))
    _check(q, g, 4.0, max_passes=1)
    # a device count limit: the graph of the first m nodes
    m = g.n // 2
    nbr, deg = _table(g.adj, 10)
    xyz = torch.from_numpy(g.pos.astype(np.float32)).cuda()
    ndev = torch.tensor([m], dtype=torch.int64, device="cuda")
    label, reps, pos, passes = q.box_reduce(nbr, deg, xyz, box=4.0, n_dev=ndev)
    sub = graph.Graph(g.pos[:m].astype(np.float32).astype(np.float64), g.dirs[:m],
                      [set(v for v in g.adj[u] if v < m) for u in range(m)])
    red, lab, _, p2 = graph.box_reduce(sub, 4.0)
    assert passes == p2 and np.array_equal(label.cpu().numpy()[:m], lab)
    keep = reps.cpu().numpy() < m
    assert np.array_equal(pos.cpu().numpy()[keep], red.pos)
    # empty input and argument checks
    e = torch.empty((0, 3), dtype=torch.float32, device="cuda")
    label, reps, pos, passes = q.box_reduce(torch.empty((0, 10), dtype=torch.int32, device="cuda"),
                                            torch.empty(0, dtype=torch.uint8, device="cuda"), e)
    assert label.numel() == 0 and reps.numel() == 0 and passes == 0
    with pytest.raises(qtv.QtvError):
        q.box_reduce(nbr, deg, xyz, box=0.0)
    with pytest.raises(qtv.QtvError):
        q.box_reduce(nbr, deg, xyz, box=4.0, max_passes=0)


def test_repeat_calls_identical(q):
    g = _face_graph_of(q, synth.random_waves_numpy((32, 32, 32), synth.wave_spec(78, 512)))
    a = _gpu(q, g, 4.0)
    b = _gpu(q, g, 4.0)
    assert all(np.array_equal(x, y) for x, y in zip(a[:3], b[:3])) and a[3] == b[3]


def test_512_workload(q):
    """Every face of the benchmark field through the GPU reduction; the oracle
    reduces the face graph of the first 64 planes, whose clusters with every
    member below plane 24 (ten boxes from the cut, more than a pass can
    reach per box) must be the GPU's clusters, at the same means."""
    psi = synth.config_field("512_waves_noise", device="cuda")
    ids, w, xyz, _, _ = q.identify_localize(psi)
    nbr, deg, _, _ = q.face_graph(tuple(psi.shape), ids)
    label, reps, pos, passes = q.box_reduce(nbr, deg, xyz, box=4.0)
    n = ids.numel()
    lab = label.cpu().numpy()
    assert 2 <= passes <= 10 and np.all(lab <= np.arange(n)) and np.all(lab[lab] == lab)
    host_ids = ids.cpu().numpy().view(np.uint64)
    z = (host_ids >> np.uint64(2)) // np.uint64(512 * 512)
    m = int(np.searchsorted(z, 64))
    g = graph.face_graph(host_ids[:m], w.cpu().numpy()[:m],
                         xyz.cpu().numpy()[:m].astype(np.float64), tuple(psi.shape))
    red, olab, _, _ = graph.box_reduce(g, 4.0)
    zmax = np.zeros(n, np.int64)
    np.maximum.at(zmax, lab, z.astype(np.int64))
    inner = np.unique(lab[:m][zmax[lab[:m]] < 24])
    assert len(inner) > 1000
    sel = np.isin(lab[:m], inner)
    assert np.array_equal(olab[sel], lab[:m][sel])
    opos = {int(r): red.pos[a] for a, r in enumerate(np.unique(olab))}
    gp = pos.cpu().numpy()
    gr = reps.cpu().numpy()
    for a in np.flatnonzero(np.isin(gr, inner)):
        assert np.array_equal(gp[a], opos[int(gr[a])])
    print(f"512^3: {n} samples -> {reps.numel()} means in {passes} passes; "
          f"{len(inner)} clusters compared with the oracle")
