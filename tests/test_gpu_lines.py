"""GPU parity of line extraction over the pierced-face graph (Sec. 3.4):
classification of components (Type I / II / III), their simple pieces in
walk order, orientation along the circulation direction (right-hand rule),
and uniform Catmull-Rom curves with their lengths, through the C ABI.

The oracle runs `graph.classify`, `graph.ordered_lines`, `graph.orient`,
`graph.catmull_rom` and `graph.curve_length` on the same face graph (the GPU
samples as positions).  Index work is bit-exact: the set of oriented pieces
(sample sequences and closed flags) and the component types must be equal
(the GPU lists pieces by their start; the oracle by component).  Curve points
agree within FP32 rounding (1e-4 absolute on coordinates below 512); each
length is the polyline length of the GPU's points (1e-6) and differs from the
oracle's by at most twice the summed point deviations.  Cases: random tangles (Type I, II and III), the
analytic line and ring (one Type I and one Type II line), a single face,
repeat calls, and the 512^3 workload (every piece checked for structure, and
the oracle on a sample of components).
"""
import numpy as np
import pytest

import synth
from oracle import graph

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TYPES = {"I": 1, "II": 2, "III": 3}


@pytest.fixture(scope="module")
def q():
    import paper_1911_12070_gb300 as qtv

    qtv.build()
    h = qtv.Qtv(0)
    yield h
    h.close()


def _gpu(q, dev, shape):
    import paper_1911_12070_gb300 as qtv

    ids, w, xyz, _, _ = q.identify_localize(dev)
    nbr, deg, comp, ncomp = q.face_graph(shape, ids)
    pieces, nodes = q.line_pieces(nbr, deg, comp, xyz, ids, w)
    curve, first, length = q.piece_curves(xyz, nodes, pieces, 8)
    return {"ids": ids.cpu().numpy().view(np.uint64), "w": w.cpu().numpy(),
            "xyz": xyz.cpu().numpy().astype(np.float64), "comp": comp.cpu().numpy(),
            "pieces": qtv.pieces_numpy(pieces), "nodes": nodes.cpu().numpy(),
            "curve": curve.cpu().numpy().astype(np.float64), "first": first.cpu().numpy(),
            "length": length.cpu().numpy(), "ncomp": ncomp}


def _gpu_pieces(r):
    out = {}
    for k, p in enumerate(r["pieces"]):
        seq = tuple(int(v) for v in r["nodes"][p["first"]:p["first"] + p["count"]])
        out[(seq, bool(p["closed"]))] = k
    return out


def _check(r, shape, comps_subset=None):
    g = graph.face_graph(r["ids"], r["w"], r["xyz"], shape)
    comps = graph.components(g)
    if comps_subset is not None:
        comps = [comps[i] for i in comps_subset]
    gp = _gpu_pieces(r)
    seen = 0
    for c in comps:
        kind = graph.classify(g, c)
        lo = min(c)
        for piece, path, closed in graph.ordered_lines(g, c):
            path = graph.orient(g, path, closed)
            key = (tuple(int(v) for v in path), bool(closed))
            assert key in gp, (kind, key[:1])
            k = gp[key]
            p = r["pieces"][k]
            assert p["comp_type"] == TYPES[kind] and p["component"] == lo
            want = graph.catmull_rom(r["xyz"][path], closed)
            f = r["first"][k]
            got = r["curve"][f:f + len(want)]
            assert got.shape == want.shape
            assert np.max(np.abs(got - want)) < 1e-4
            # the reported length is the polyline length of the GPU's own points;
            # that differs from the oracle's by at most the triangle-inequality
            # bound of the point deviations (FP32 rounding of the points)
            Lg = graph.curve_length(got, closed)
            assert abs(float(r["length"][k]) - Lg) <= 1e-6 * max(Lg, 1.0)
            L = graph.curve_length(want, closed)
            dev = np.linalg.norm(got - want, axis=1)
            bound = 2.0 * dev.sum() + 1e-9
            assert abs(Lg - L) <= bound
            seen += 1
    if comps_subset is None:
        assert seen == len(r["pieces"])
    return seen


@pytest.mark.parametrize("shape,seed", [((40, 36, 52), 13), ((48, 48, 48), 21),
                                        ((17, 48, 33), 5), ((9, 130, 70), 2)])
def test_random_tangles_match_oracle(q, shape, seed):
    host = synth.random_waves_numpy(shape, synth.wave_spec(seed, 512))
    r = _gpu(q, torch.from_numpy(host).cuda(), shape)
    n = _check(r, shape)
    assert n > 5


def test_analytic_line_and_ring(q):
    host = synth.analytic_line_ring()
    r = _gpu(q, torch.from_numpy(host).cuda(), host.shape)
    _check(r, host.shape)
    closed = r["pieces"]["closed"].astype(bool)
    assert closed.any() and (~closed).any()


def test_single_face_and_repeat(q):
    import paper_1911_12070_gb300 as qtv

    host = synth.random_waves_numpy((24, 26, 28), synth.wave_spec(8, 256))
    dev = torch.from_numpy(host).cuda()
    ids, w, xyz, _, _ = q.identify_localize(dev)
    nbr, deg, comp, _ = q.face_graph(host.shape, ids[:1])
    pieces, nodes = q.line_pieces(nbr, deg, comp, xyz[:1], ids[:1], w[:1])
    pn = qtv.pieces_numpy(pieces)
    assert len(pn) == 1 and pn[0]["count"] == 1 and int(nodes[0]) == 0
    curve, first, length = q.piece_curves(xyz[:1], nodes, pieces)
    assert curve.shape[0] == 1 and torch.equal(curve[0], xyz[0]) and float(length[0]) == 0.0
    a = _gpu(q, dev, host.shape)
    b = _gpu(q, dev, host.shape)
    for k in ("nodes", "curve", "first", "length"):
        assert np.array_equal(a[k], b[k])
    assert np.array_equal(a["pieces"], b["pieces"])


def test_512_workload(q):
    psi = synth.config_field("512_waves_noise", device="cuda")
    r = _gpu(q, psi, tuple(psi.shape))
    P = r["pieces"]
    n = len(r["ids"])
    # every sample appears; pieces are contiguous and consecutive samples adjacent
    assert np.all(P["first"][1:] == P["first"][:-1] + P["count"][:-1])
    assert int(P["first"][-1] + P["count"][-1]) == len(r["nodes"])
    assert np.array_equal(np.unique(r["nodes"]), np.arange(n))
    # the oracle on a sample of components (the largest and small ones)
    sizes = np.bincount(r["comp"], minlength=n)
    roots = np.flatnonzero(sizes)
    order = np.argsort(-sizes[roots], kind="stable")
    big = roots[order[:3]]
    rng = np.random.default_rng(4)
    small = rng.choice(roots, 200, replace=False)
    g = graph.face_graph(r["ids"], r["w"], r["xyz"], tuple(psi.shape))
    comps = graph.components(g)
    index = {min(c): i for i, c in enumerate(comps)}
    subset = sorted({index[int(x)] for x in np.concatenate([big, small])})
    seen = _check(r, tuple(psi.shape), subset)
    assert seen >= 200
    # all three types occur in a tangle of this size
    assert set(int(t) for t in P["comp_type"]) == {1, 2, 3}


@pytest.mark.parametrize("box", [1.5, 4.0])
def test_thinning_matches_oracle_bit_for_bit(q, box):
    import paper_1911_12070_gb300 as qtv

    host = synth.random_waves_numpy((48, 48, 48), synth.wave_spec(21, 512))
    dev = torch.from_numpy(host).cuda()
    ids, w, xyz, _, _ = q.identify_localize(dev)
    nbr, deg, comp, _ = q.face_graph(host.shape, ids)
    pieces, nodes = q.line_pieces(nbr, deg, comp, xyz, ids, w)
    means, tp = q.thin_pieces(xyz, nodes, pieces, box)
    P = qtv.pieces_numpy(pieces)
    T = qtv.pieces_numpy(tp)
    nd = nodes.cpu().numpy()
    x64 = xyz.cpu().numpy().astype(np.float64)
    m = means.cpu().numpy()
    assert T["first"][0] == 0 and np.all(T["first"][1:] == T["first"][:-1] + T["count"][:-1])
    assert int(T["first"][-1] + T["count"][-1]) == len(m)
    for k in range(len(P)):
        pts = x64[nd[P["first"][k]:P["first"][k] + P["count"][k]]]
        want, _ = graph.thin_piece(pts, bool(P["closed"][k]), box)
        got = m[T["first"][k]:T["first"][k] + T["count"][k]]
        assert np.array_equal(got, want.astype(np.float32)), k
        assert T["closed"][k] == P["closed"][k] and T["component"][k] == P["component"][k]
    assert len(m) < 0.6 * len(nd)


def test_thin_refine_curves_pipeline(q):
    # identification -> samples -> lines -> box means -> refinement (Sec. 3.3.3)
    # -> Catmull-Rom: refined means lie on cores (Eq. 7 error far below the means')
    import paper_1911_12070_gb300 as qtv

    host = synth.random_waves_numpy((48, 48, 48), synth.wave_spec(21, 512))
    dev = torch.from_numpy(host).cuda()
    ids, w, xyz, _, _ = q.identify_localize(dev)
    nbr, deg, comp, _ = q.face_graph(host.shape, ids)
    pieces, nodes = q.line_pieces(nbr, deg, comp, xyz, ids, w)
    means, tp = q.thin_pieces(xyz, nodes, pieces, 4.0)
    ref = q.refine_samples(dev, xyz0=means)
    idn = torch.arange(means.shape[0], dtype=torch.int32, device="cuda")
    curve, first, length = q.piece_curves(ref["xyz"], idn, tp, 8)
    e_means, _, _ = q.density_error(dev, means)
    e_ref, _, _ = q.density_error(dev, ref["xyz"])
    assert e_ref < 0.2 * e_means
    assert curve.shape[0] > means.shape[0] and float(length.sum()) > 0
