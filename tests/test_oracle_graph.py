"""Pins of the oracle's graph pipeline (oracle/graph.py: Sec. 3.1-3.4 and
Eq. 7) against closed forms, hand-built graphs and the analytic cores:

* Catmull-Rom: passes through its control points, reproduces straight lines
  with uniform spacing (linear precision), has the closed-form midpoint
  (-P0 + 9 P1 + 9 P2 - P3) / 16, wraps around for loops, and on a regular
  24-gon inscribed in a circle has a length between the polygon's perimeter
  and 2 pi R;
* Eq. 7 is 0 at exact nodal zeros, 1 for a constant unit field, and has a
  closed form for a linear field;
* components, the box-mean reduction of a unit chain (worked out by hand),
  an idempotent pass, and classification / splitting of a path, a cycle, a
  Y and a loop through one branch point;
* a straight analytic line gives one Type-I line within one cell of its axis
  and oriented along its circulation (right-hand rule); the conjugate field
  reverses it; a ring gives one Type-II loop within one cell of the circle,
  whose length approaches 2 pi R as the box shrinks; line + ring give one of
  each; two perpendicular lines joined by a bridge give a Type-III line with
  two branch points, split into five Type-I pieces.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import graph


def _path_graph(pos, edges):
    pos = np.asarray(pos, np.float64)
    adj = [set() for _ in range(len(pos))]
    for a, b in edges:
        adj[a].add(b)
        adj[b].add(a)
    return graph.Graph(pos, np.zeros_like(pos), adj)


# ---------------------------------------------------------------- Catmull-Rom
def test_catmull_rom_interpolates_and_closed_form_midpoint():
    rng = np.random.default_rng(1)
    P = rng.standard_normal((6, 3))
    c = graph.catmull_rom(P, closed=False)
    assert c.shape == (8 * 5 + 1, 3)
    assert np.allclose(c[::8], P, atol=1e-14)
    # midpoint of segment 2 (between P2 and P3) from the closed form
    mid = (-P[1] + 9 * P[2] + 9 * P[3] - P[4]) / 16
    assert np.allclose(c[2 * 8 + 4], mid, atol=1e-14)
    # open ends repeat the end point as the outer control point
    mid0 = (-P[0] + 9 * P[0] + 9 * P[1] - P[2]) / 16
    assert np.allclose(c[4], mid0, atol=1e-14)


def test_catmull_rom_linear_precision():
    P = np.outer(np.arange(5.0), [1.0, 2.0, -0.5]) + [3.0, 1.0, 2.0]
    c = graph.catmull_rom(P, closed=False)
    # interior segments: uniform points on the line
    inner = c[8:8 * 3 + 1]
    d = np.diff(inner, axis=0)
    assert np.allclose(d, d[0], atol=1e-13)
    assert np.allclose(np.cross(c - P[0], [1.0, 2.0, -0.5]), 0.0, atol=1e-12)


def test_catmull_rom_closed_circle():
    R, m = 5.0, 24
    th = 2 * np.pi * np.arange(m) / m
    P = np.stack([R * np.cos(th), R * np.sin(th), np.zeros(m)], 1)
    c = graph.catmull_rom(P, closed=True)
    assert c.shape == (8 * m, 3)
    assert np.allclose(c[::8], P, atol=1e-14)
    L = graph.curve_length(c, closed=True)
    poly = m * 2 * R * np.sin(np.pi / m)
    assert poly < L < 2 * np.pi * R
    assert abs(L - 2 * np.pi * R) < 2e-3 * 2 * np.pi * R


# ---------------------------------------------------------------- Eq. 7
def test_density_error_zero_at_nodal_zeros():
    n = 12
    z, y, x = np.meshgrid(*(np.arange(n, dtype=float),) * 3, indexing="ij")
    psi = ((x - 5) + 1j * (y - 7)).astype(np.complex64)
    pts = np.stack([np.full(n, 5.0), np.full(n, 7.0), np.arange(n, dtype=float)], 1)
    assert graph.density_error(psi, pts) == 0.0


def test_density_error_constant_and_linear_fields():
    """rho is |trilinear psi|^2: 1 everywhere for a constant unit field, and
    for a linear field psi = (x - x0) + i (y - y0), which trilinear
    interpolation reproduces exactly, (x - x0)^2 + (y - y0)^2 at every point."""
    n = 10
    pts = np.random.default_rng(2).uniform(0, n - 1, (50, 3))
    psi = np.full((n, n, n), 0.6 + 0.8j, np.complex64)
    assert abs(graph.density_error(psi, pts) - 1.0) < 1e-6
    z, y, x = np.meshgrid(*(np.arange(n, dtype=float),) * 3, indexing="ij")
    x0, y0 = 5.5, 7.25  # node values exact in FP32
    psi = ((x - x0) + 1j * (y - y0)).astype(np.complex64)
    rho = (pts[:, 0] - x0) ** 2 + (pts[:, 1] - y0) ** 2
    rho_bar = np.mean((x - x0) ** 2 + (y - y0) ** 2)
    assert abs(graph.density_error(psi, pts) - rho.sum() / (rho_bar * len(pts))) < 1e-12


# ---------------------------------------------------------------- graphs
def test_components_lowest_index_first():
    g = _path_graph(np.zeros((7, 3)), [(0, 3), (3, 5), (1, 2), (2, 6)])
    comps = graph.components(g)
    assert [sorted(c) for c in comps] == [[0, 3, 5], [1, 2, 6], [4]]
    assert comps[0][0] == 0 and comps[1][0] == 1


def test_reduction_of_unit_chain_by_hand():
    n = 20
    pos = np.stack([np.arange(n, dtype=float), np.zeros(n), np.zeros(n)], 1)
    g = _path_graph(pos, [(i, i + 1) for i in range(n - 1)])
    r, passes = graph.reduce(g, d=4.0)
    # box |dx| <= 2 around node 0 takes 0..2 (mean 1); the next box starts at
    # node 3 and takes 3..5 (1 and 2 are processed), and so on; 18, 19 -> 18.5.
    # The second pass moves nothing (samples 3 apart exceed the half box).
    assert np.allclose(r.pos[:, 0], [1, 4, 7, 10, 13, 16, 18.5])
    assert passes == 2
    assert r.degrees().tolist() == [1, 2, 2, 2, 2, 2, 1]


def test_pass_with_small_box_is_identity():
    rng = np.random.default_rng(3)
    pos = np.cumsum(rng.uniform(3, 4, (10, 3)), axis=0)
    g = _path_graph(pos, [(i, i + 1) for i in range(9)] + [(0, 9)])
    r, move = graph.reduce_pass(g, d=2.0)
    assert move == 0.0 and np.array_equal(r.pos, g.pos)
    assert [sorted(a) for a in r.adj] == [sorted(a) for a in g.adj]


def test_classification_and_splitting():
    z = np.zeros((8, 3))
    path = _path_graph(z, [(0, 1), (1, 2), (2, 3)])
    assert graph.classify(path, [0, 1, 2, 3]) == "I"
    (kind, nodes, closed), = graph.ordered_lines(path, [0, 1, 2, 3])
    assert kind == "I" and nodes == [0, 1, 2, 3] and not closed
    cyc = _path_graph(z, [(0, 1), (1, 2), (2, 3), (3, 0)])
    assert graph.classify(cyc, [0, 1, 2, 3]) == "II"
    (kind, nodes, closed), = graph.ordered_lines(cyc, [0, 1, 2, 3])
    assert kind == "II" and closed and nodes == [0, 1, 2, 3]
    y = _path_graph(z, [(0, 1), (1, 2), (1, 3), (3, 4), (1, 5)])
    assert graph.classify(y, [0, 1, 2, 3, 4, 5]) == "III"
    pieces = graph.ordered_lines(y, [0, 1, 2, 3, 4, 5])
    assert sorted(p[1] for p in pieces) == [[1, 0], [1, 2], [1, 3, 4], [1, 5]]
    assert all(p[0] == "I" for p in pieces)
    # a loop through one branch point plus a tail
    lp = _path_graph(z, [(0, 1), (1, 2), (2, 0), (0, 3)])
    pieces = graph.ordered_lines(lp, [0, 1, 2, 3])
    kinds = sorted((p[0], len(p[1]), p[2]) for p in pieces)
    assert kinds == [("I", 2, False), ("II", 3, True)]


def test_face_graph_links_faces_of_one_cell():
    psi = synth.analytic_line_ring(with_ring=False)
    w, _ = oracle.identify(psi)
    ids, wind = oracle.face_list(w)
    loc = oracle.localize(psi, ids, wind)
    g = graph.face_graph(ids, wind, loc["xyz"], psi.shape)
    assert g.n == 64
    deg = g.degrees()
    assert sorted(deg.tolist()) == [1, 1] + [2] * 62
    assert len(graph.components(g)) == 1


# ---------------------------------------------------------------- analytic cores
def _faces(psi):
    w, _ = oracle.identify(psi)
    ids, wind = oracle.face_list(w)
    loc = oracle.localize(psi, ids, wind)
    return graph.face_graph(ids, wind, loc["xyz"], psi.shape)


def _nodes(psi):
    c, v = oracle.node_circulation(psi)
    return graph.node_graph(v.astype(bool), c)


@pytest.mark.parametrize("form", ["faces", "nodes"])
def test_straight_line_is_one_type_I_line_on_its_axis(form):
    psi = synth.analytic_line_ring(with_ring=False)
    g = _faces(psi) if form == "faces" else _nodes(psi)
    out = graph.vectorize(g, d=4.0)
    assert len(out["lines"]) == 1 and out["reconnections"] == 0
    line = out["lines"][0]
    assert line["type"] == "I" and not line["closed"]
    c = line["curve"]
    r = np.hypot(c[:, 0] - 31.37, c[:, 1] - 30.81)
    assert np.max(r) < 1.0
    # W = +1 about +z: the ordered line runs towards +z
    assert line["samples"][-1, 2] > line["samples"][0, 2] + 50


def test_conjugate_reverses_line_direction():
    psi = np.conj(synth.analytic_line_ring(with_ring=False))
    line = graph.vectorize(_faces(psi), d=4.0)["lines"][0]
    assert line["samples"][-1, 2] < line["samples"][0, 2] - 50


@pytest.mark.parametrize("form", ["faces", "nodes"])
def test_ring_is_one_type_II_loop_near_the_circle(form):
    psi = synth.analytic_line_ring(with_line=False)
    g = _faces(psi) if form == "faces" else _nodes(psi)
    out = graph.vectorize(g, d=4.0)
    assert len(out["lines"]) == 1
    loop = out["lines"][0]
    assert loop["type"] == "II" and loop["closed"]
    c = loop["curve"]
    dist = np.hypot(np.hypot(c[:, 0] - 32, c[:, 1] - 32) - 12.0, c[:, 2] - 40.0)
    assert np.max(dist) < 1.0
    assert abs(loop["length"] - 2 * np.pi * 12) < 0.03 * 2 * np.pi * 12


def test_ring_length_approaches_2_pi_r_as_box_shrinks():
    g = _faces(synth.analytic_line_ring(with_line=False))
    target = 2 * np.pi * 12
    err = [abs(graph.vectorize(g, d=d)["lines"][0]["length"] - target) for d in (8.0, 6.0, 4.0, 3.0)]
    assert all(a > b for a, b in zip(err[:-1], err[1:])), err
    assert err[-1] < 2e-3 * target


def test_config0_line_and_ring():
    out = graph.vectorize(_faces(synth.analytic_line_ring()), d=4.0)
    kinds = sorted(l["type"] for l in out["lines"])
    assert kinds == ["I", "II"] and out["reconnections"] == 0
    pts = np.vstack([l["curve"] for l in out["lines"]])
    assert graph.density_error(synth.analytic_line_ring(), pts) < 0.02


def test_bridged_perpendicular_lines_are_type_III():
    v = np.zeros((32, 32, 32), bool)   # [z][y][x]
    v[8, 8, 2:30] = True               # line along x at y = 8, z = 8
    v[8:17, 8, 20] = True              # bridge along z at x = 20, y = 8
    v[16, 2:30, 20] = True             # line along y at x = 20, z = 16
    out = graph.vectorize(graph.node_graph(v), d=3.0)
    assert out["reconnections"] == 2
    assert {l["type"] for l in out["lines"]} == {"III"}
    assert len(out["lines"]) == 5 and all(l["piece"] == "I" for l in out["lines"])
    # the pieces cover the three segments: total length ~ 27 + 27 + 8
    assert 55 < sum(l["length"] for l in out["lines"]) < 66


# ------------------------------------------- lattice box reduction (Sec. 3.3.2)
def _f32(g):
    """The graph with FP32 positions (as the GPU sample stream has them)."""
    return graph.Graph(g.pos.astype(np.float32).astype(np.float64), g.dirs, g.adj)


def _chain(xs, y=3.0, z=5.0):
    xs = np.asarray(xs, np.float64)
    pos = np.stack([xs, np.full_like(xs, y), np.full_like(xs, z)], 1)
    return _path_graph(pos, [(a, a + 1) for a in range(len(xs) - 1)])


@pytest.mark.parametrize("step", [1.0, 0.5, 0.25])
def test_box_reduce_chain_closed_form(step):
    # a straight chain with a spacing that divides the box: the first lattice
    # groups the nodes x in [4 m, 4 m + 4) and each group becomes its mean,
    # 4 m + 2 - step / 2, so the means are 4 apart; the shifted lattice then
    # finds each mean alone in its box, and so does the first again: three
    # passes
    xs = np.arange(0.0, 20.0, step)
    red, lab, q, passes = graph.box_reduce(_chain(xs), 4.0)
    groups = [xs[(xs >= 4 * m) & (xs < 4 * m + 4)] for m in range(5)]
    assert passes == 3
    assert np.allclose(red.pos[:, 0], [g.mean() for g in groups], atol=1e-9)
    assert np.all(red.pos[:, 1:] == [3.0, 5.0])
    assert list(lab) == [int(np.flatnonzero(xs >= 4 * np.floor(x / 4))[0]) for x in xs]
    assert [len(a) for a in red.adj] == [1, 2, 2, 2, 1]


def test_box_reduce_merges_across_the_first_lattice():
    # nodes at x = 3.5 and 4.5 sit in different boxes of the first lattice and
    # in one box of the shifted lattice (side 4, shifted by 2)
    red, lab, _, passes = graph.box_reduce(_chain([3.5, 4.5]), 4.0)
    assert len(red.adj) == 1 and red.pos[0, 0] == 4.0 and list(lab) == [0, 0]
    assert passes == 4  # merge on pass 2, then one quiet pass of each lattice


def test_box_reduce_never_merges_unconnected_nodes():
    pos = np.array([[1.0, 1.0, 1.0], [1.5, 1.0, 1.0], [2.0, 1.0, 1.0]])
    red, lab, _, _ = graph.box_reduce(_path_graph(pos, [(0, 1)]), 4.0)
    assert list(lab) == [0, 0, 2] and len(red.adj) == 2


def test_box_reduce_rounds_means_in_fixed_point():
    # mean of 0, 2^-32 and 2^-32 (in h) is 2/3 of a unit: rounded to 1 unit
    u = 2.0 ** -32
    red, _, q, _ = graph.box_reduce(_chain([0.0, u, u]), 4.0)
    assert q[0][0] == 1 and red.pos[0, 0] == u


def test_box_reduce_keeps_a_branch_point():
    # three arms from a centre: the reduced graph is still a tree with one
    # node of degree three (a reconnection point, Sec. 3.4)
    c = np.array([10.0, 10.0, 10.0])
    pos, edges = [c], []
    for d in ((1, 0, 0), (0, 1, 0), (-1, 0, 0)):
        prev = 0
        for s in range(1, 9):
            pos.append(c + s * np.array(d, np.float64))
            edges.append((prev, len(pos) - 1))
            prev = len(pos) - 1
    red, _, _, _ = graph.box_reduce(_path_graph(pos, edges), 4.0)
    deg = sorted(len(a) for a in red.adj)
    assert deg.count(3) == 1 and deg.count(1) == 3 and set(deg) <= {1, 2, 3}
    assert sum(deg) == 2 * (len(deg) - 1)  # a tree


def test_box_reduce_does_not_depend_on_the_numbering():
    g = _f32(_faces(synth.random_waves_numpy((24, 28, 32), synth.wave_spec(61, 256))))
    red, lab, q, passes = graph.box_reduce(g, 4.0)
    perm = np.random.default_rng(3).permutation(g.n)
    inv = np.argsort(perm)
    gp = graph.Graph(g.pos[perm], g.dirs[perm], [set(int(inv[v]) for v in g.adj[u]) for u in perm])
    red2, lab2, q2, passes2 = graph.box_reduce(gp, 4.0)
    assert passes2 == passes and sorted(q2) == sorted(q)
    # the same partition of the original nodes
    part = {frozenset(np.flatnonzero(lab == r)) for r in np.unique(lab)}
    part2 = {frozenset(perm[np.flatnonzero(lab2 == r)]) for r in np.unique(lab2)}
    assert part == part2


def test_box_reduce_is_a_fixed_point():
    g = _f32(_faces(synth.random_waves_numpy((24, 28, 32), synth.wave_spec(62, 256))))
    red, _, q, passes = graph.box_reduce(g, 4.0)
    assert 3 <= passes <= 10
    again, lab, q2, p2 = graph.box_reduce(red, 4.0)
    assert p2 == 2 and q2 == q and list(lab) == list(range(red.n))


def test_box_reduce_of_the_straight_line_and_the_ring():
    # config 0 line: one xy face per plane, z = k exactly: means at 4 m + 1.5
    red, _, _, _ = graph.box_reduce(_f32(_faces(synth.analytic_line_ring(with_ring=False))), 4.0)
    assert np.array_equal(red.pos[:, 2], 4.0 * np.arange(16) + 1.5)
    assert np.all(np.abs(red.pos[:, 0] - 31.37) < 1) and np.all(np.abs(red.pos[:, 1] - 30.81) < 1)
    # the ring stays one loop; its polygon length approaches 2 pi R
    g = _f32(_faces(synth.analytic_line_ring(with_line=False)))
    target = 2 * np.pi * 12
    errs = []
    for d in (6.0, 4.0, 3.0):
        red, _, _, _ = graph.box_reduce(g, d)
        assert all(len(a) == 2 for a in red.adj)
        (nodes,) = graph.components(red)
        _, path, closed = graph.ordered_lines(red, nodes)[0]
        assert closed
        errs.append(abs(graph.curve_length(red.pos[path], True) - target))
    assert errs[-1] < 0.03 * target and errs[-1] < errs[0]


def test_box_reduce_uneven_chain_by_hand():
    # x = 0, 0.75, ..., 19.5: the first lattice gives means 1.875, 6, 9.75,
    # 13.875, 18; on the shifted lattice (boxes [4 m + 2, 4 m + 6)) 6 and 9.75
    # share box m = 1 and merge into 7.875; then neither lattice merges
    # anything (keys 0, 1, 3, 4 and -1, 1, 2, 4): four passes
    red, lab, _, passes = graph.box_reduce(_chain(np.arange(0.0, 20.0, 0.75)), 4.0)
    assert passes == 4
    assert list(red.pos[:, 0]) == [1.875, 7.875, 13.875, 18.0]
    assert list(lab) == [0] * 6 + [6] * 10 + [16] * 6 + [22] * 5
