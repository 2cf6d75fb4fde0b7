"""GPU parity of the sample graph over pierced faces (Sec. 3.1: faces that
bound the same unit cell are adjacent) and of its connected components (the
independent lines of Sec. 3.2), through the C ABI.

Index work, so bit-exact: the neighbour table must equal the oracle's
adjacency sets (`oracle.graph.face_graph`) and the component labels must name
the oracle's depth-first components (`oracle.graph.components`) by their
lowest face index.  Cases: random tangles with ragged shapes, the analytic
line and ring, a face list chained from qtv_identify without a host
synchronisation (device count), an empty list and a single face, repeat
calls, and the 512^3 workload (sampled neighbours against a host search of
the face list, and the union-find invariants on every face).
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


def _check(q, host):
    dev = torch.from_numpy(host).cuda()
    ids, w, _ = q.identify(dev)
    nbr, deg, comp, ncomp = q.face_graph(host.shape, ids)
    idn = ids.cpu().numpy().view(np.uint64)
    og = graph.face_graph(idn, w.cpu().numpy(), np.zeros((len(idn), 3)), host.shape)
    nb = nbr.cpu().numpy().astype(np.int64)
    dg = deg.cpu().numpy()
    for a in range(len(idn)):
        assert list(nb[a, :dg[a]]) == sorted(og.adj[a]), a
        assert np.all(nb[a, dg[a]:] == -1)
    comps = graph.components(og)
    want = np.empty(len(idn), np.int64)
    for c in comps:
        want[c] = min(c)
    assert np.array_equal(comp.cpu().numpy().astype(np.int64), want)
    assert ncomp == len(comps)
    return len(idn), ncomp


@pytest.mark.parametrize("shape,seed", [((40, 36, 52), 13), ((17, 48, 33), 5), ((48, 48, 48), 21),
                                        ((9, 130, 70), 2)])
def test_random_tangles_match_oracle(q, shape, seed):
    n, nc = _check(q, synth.random_waves_numpy(shape, synth.wave_spec(seed, 512)))
    assert n > 100 and nc >= 1


def test_analytic_line_and_ring(q):
    n, nc = _check(q, synth.analytic_line_ring())
    assert nc >= 2


def test_chained_with_device_count_and_edge_cases(q):
    host = synth.random_waves_numpy((32, 30, 34), synth.wave_spec(7, 256))
    dev = torch.from_numpy(host).cuda()
    ids, w, _ = q.identify(dev)
    n = ids.numel()
    # identify into a larger buffer; the graph reads the count on the device
    cap = n + 500
    big = torch.empty(cap, dtype=torch.int64, device="cuda")
    wb = torch.empty(cap, dtype=torch.int8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    q.identify_into(dev, big, wb, cnt)
    a = q.face_graph(host.shape, big, n_dev=cnt)
    b = q.face_graph(host.shape, ids)
    assert a[3] == b[3]
    assert torch.equal(a[0][:n], b[0]) and torch.equal(a[1][:n], b[1]) and \
        torch.equal(a[2][:n], b[2])
    # empty list and a single face
    e = q.face_graph(host.shape, ids[:0])
    assert e[3] == 0
    s = q.face_graph(host.shape, ids[:1])
    assert s[3] == 1 and int(s[1][0]) == 0 and int(s[2][0]) == 0
    # repeat calls are identical
    c = q.face_graph(host.shape, ids)
    for x, y in zip(b[:3], c[:3]):
        assert torch.equal(x, y)


def test_512_workload(q):
    psi = synth.config_field("512_waves_noise", device="cuda")
    ids, w, _ = q.identify(psi)
    nbr, deg, comp, ncomp = q.face_graph(tuple(psi.shape), ids)
    idn = ids.cpu().numpy().view(np.uint64)
    nb = nbr.cpu().numpy().astype(np.int64)
    dg = deg.cpu().numpy().astype(np.int64)
    cp = comp.cpu().numpy().astype(np.int64)
    n = len(idn)
    nx = ny = nz = 512
    # sampled neighbours against a host search of the sorted list
    rng = np.random.default_rng(3)
    for a in np.unique(np.concatenate([np.arange(300), rng.choice(n, 3000, replace=False)])):
        f = int(idn[a])
        want = []
        for c in graph.face_cells(f, (nz, ny, nx)):
            i, j, k = c
            base = (k * ny + j) * nx + i
            for g in ((base << 2) | 0, ((base + nx * ny) << 2) | 0, (base << 2) | 1,
                      ((base + 1) << 2) | 1, (base << 2) | 2, ((base + nx) << 2) | 2):
                if g == f:
                    continue
                p = int(np.searchsorted(idn, np.uint64(g)))
                if p < n and int(idn[p]) == g:
                    want.append(p)
        assert list(nb[a, :dg[a]]) == sorted(want)
    # symmetric adjacency, labels constant on edges, roots are the minima
    src = np.repeat(np.arange(n), dg)
    dst = nb[nb >= 0]
    assert len(src) == len(dst)
    key = np.sort(src * n + dst)
    rev = np.sort(dst * n + src)
    assert np.array_equal(key, rev)
    assert np.all(cp[src] == cp[dst])
    assert np.all(cp <= np.arange(n)) and np.all(cp[cp] == cp)
    assert ncomp == int(np.count_nonzero(cp == np.arange(n)))
    # the partition equals the connected components of the same adjacency
    # (a library routine), each named by its lowest member
    sparse = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    mat = sparse.coo_matrix((np.ones(len(src), np.int8), (src, dst)), shape=(n, n))
    nlab, lab = csgraph.connected_components(mat, directed=False)
    assert nlab == ncomp
    low = np.full(nlab, n)
    np.minimum.at(low, lab, np.arange(n))
    assert np.array_equal(low[lab], cp)


@pytest.mark.parametrize("shape,seed", [((40, 36, 52), 13), ((30, 33, 70), 4)])
def test_vortex_node_graph_matches_oracle(q, shape, seed):
    # the paper's graph: vortex nodes of the node form, 6-connected
    host = synth.random_waves_numpy(shape, synth.wave_spec(seed, 512))
    dev = torch.from_numpy(host).cuda()
    nid, circ, _ = q.node_circulation(dev)
    nbr, deg, comp, ncomp = q.node_graph(shape, nid)
    ids = nid.cpu().numpy()
    mask = np.zeros(int(np.prod(shape)), bool)
    mask[ids] = True
    og = graph.node_graph(mask.reshape(shape))
    nb = nbr.cpu().numpy().astype(np.int64)
    dg = deg.cpu().numpy()
    for a in range(len(ids)):
        assert list(nb[a, :dg[a]]) == sorted(og.adj[a])
    comps = graph.components(og)
    want = np.empty(len(ids), np.int64)
    for c in comps:
        want[c] = min(c)
    assert np.array_equal(comp.cpu().numpy().astype(np.int64), want)
    assert ncomp == len(comps) and len(ids) > 500
