"""Graph pipeline of the vectorization (Sec. 3.1 global graph construction,
Sec. 3.2 node extraction, Sec. 3.3.1-3.3.2 box-mean sample estimation and
iterative graph reduction, Sec. 3.4 classification, re-ordering and
Catmull-Rom vectorization) and the density error metric (Eq. 7).

TEST INFRASTRUCTURE ONLY (tests, smoke, bench CPU baseline).  Plain Python
and numpy in FP64, written step by step from the text of those sections; it
shares no code with the CUDA path.  Input is either a set of vortex nodes
(grid nodes whose ring circulation exceeds pi, Sec. 2.2.2) or a list of
pierced plaquettes with their localized samples (the GPU sample stream).

Readings where the text leaves details open:

* node graph: nodes are the vortex nodes, numbered in scan order with x
  fastest, then y, then z; two nodes are adjacent when they are neighbours
  along a grid line (6-connectivity);
* face graph: nodes are the pierced faces in ascending face-id order, at their
  sample positions; two faces are adjacent when they bound the same unit cell
  (a cell with 4 or 6 pierced faces links all of them, as at a reconnection);
* traversals (components, box sub-graphs) visit neighbours in ascending index
  order and start at the lowest unvisited index; the sets they find do not
  depend on the order;
* box: axis-aligned cube of side d = k h centred on the current node,
  membership |p - c|_inf <= d / 2 inclusive; the sub-graph is what a
  traversal from the current node reaches through unprocessed nodes inside
  the box; its mean replaces it, carrying the union of the edges that leave
  it; the next node is the lowest-index unprocessed neighbour of the new node,
  else the lowest-index unprocessed node;
* passes repeat with the same d until no sample moves by 1e-3 h or more
  (a sample's move: its distance from the node its box was centred on),
  at most 10 passes;
* classification by degree: Type I (all degrees <= 2, two ends of degree 1,
  or a single node), Type II (all degrees 2), Type III (a degree above 2);
  Type III is split at its branch points into Type I pieces (or Type II
  pieces for loops through one branch point);
* ordering: Type I from its lower-index end, Type II from its lowest-index
  node towards its lower-index neighbour, pieces from their branch point;
  each ordered line is then turned so that it runs along the circulation
  direction (right-hand rule, Sec. 3.4) of its samples;
* vectorization: uniform Catmull-Rom through the ordered samples, 8 points
  per segment; open lines repeat their end points, loops wrap around;
* Eq. 7: e = sum |rho(x_i)| / (mean rho over the field * N) over the spline
  points x_i, rho trilinearly interpolated;
* lattice box reduction (`box_reduce`, an order-independent parallel reading
  of Sec. 3.3.1-3.3.2): positions are held in fixed point, integers in units
  of 2^-32 h (a position times 2^32, rounded to the nearest integer, ties to
  even; a sample may lie slightly outside the grid, so positions may be
  negative); pass p lays a
  lattice of boxes of side D = round(d 2^32) over space, shifted by
  floor(D / 2) in every axis on odd passes; the nodes of one box that are
  connected through edges inside that box form one cluster, which collapses
  to one node at the rounded mean floor((sum + floor(c / 2)) / c) of its members'
  positions (each current node counted once), named by the lowest original
  index it contains and carrying the union of its members' external edges;
  passes repeat until two consecutive passes (one of each lattice) merge
  nothing, at most 10 passes.  Unlike the sequential traversal of `reduce`,
  its result does not depend on the numbering of the nodes;
* arc-length thinning (`thin_piece`, a parallel reading of the box means of
  Sec. 3.3.2 on ordered pieces): consecutive samples of a piece are grouped by
  the box index floor(s / d) of their arc length s along the piece, each group
  collapsing to its mean; s is a sum of per-segment lengths rounded to units
  of 2^-32 h, so it is exact in any summation order.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

PER_SEGMENT = 8


@dataclass
class Graph:
    """Nodes with positions (grid units), circulation directions (summed over
    the nodes a node stands for) and adjacency sets."""
    pos: np.ndarray                      # [n, 3] float64 (x, y, z)
    dirs: np.ndarray                     # [n, 3] float64
    adj: list = field(default_factory=list)  # list of sets of node indices

    @property
    def n(self):
        return len(self.adj)

    def degrees(self):
        return np.array([len(a) for a in self.adj], np.int64)


# ---------------------------------------------------------------------------
# Sec. 3.1: global graph construction
# ---------------------------------------------------------------------------
def node_graph(vortex: np.ndarray, circulation: np.ndarray | None = None) -> Graph:
    """Graph of vortex nodes (vortex: [nz, ny, nx] bool); circulation
    [3, nz, ny, nx] (ring circulation in the xy, yz and zx planes, i.e. about
    the z, x and y axes), if given, sets each node's direction
    (C_yz, C_zx, C_xy)."""
    vortex = np.asarray(vortex, bool)
    nz, ny, nx = vortex.shape
    lin = np.flatnonzero(vortex.reshape(-1))  # ascending: x fastest, then y, then z
    index = {int(v): a for a, v in enumerate(lin)}
    k, rem = np.divmod(lin, nx * ny)
    j, i = np.divmod(rem, nx)
    pos = np.stack([i, j, k], 1).astype(np.float64)
    dirs = np.zeros_like(pos)
    if circulation is not None:
        c = np.asarray(circulation, np.float64).reshape(3, -1)
        dirs = np.stack([c[1, lin], c[2, lin], c[0, lin]], 1)
    adj = [set() for _ in range(len(lin))]
    for a, v in enumerate(lin):
        x, y, z = int(i[a]), int(j[a]), int(k[a])
        for dx, dy, dz in ((-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)):
            X, Y, Z = x + dx, y + dy, z + dz
            if 0 <= X < nx and 0 <= Y < ny and 0 <= Z < nz:
                b = index.get((Z * ny + Y) * nx + X)
                if b is not None:
                    adj[a].add(b)
    return Graph(pos, dirs, adj)


_NORMAL = {0: (0.0, 0.0, 1.0), 1: (1.0, 0.0, 0.0), 2: (0.0, 1.0, 0.0)}


def face_cells(face_id: int, shape):
    """The (up to two) unit cells, as (i, j, k) min corners, that a face bounds."""
    nz, ny, nx = shape
    o = face_id & 3
    lin = face_id >> 2
    i, j, k = lin % nx, (lin // nx) % ny, lin // (nx * ny)
    if o == 0:    # xy face at height k: cells k - 1 and k
        cand = [(i, j, k - 1), (i, j, k)]
    elif o == 1:  # yz face at x = i
        cand = [(i - 1, j, k), (i, j, k)]
    else:         # zx face at y = j
        cand = [(i, j - 1, k), (i, j, k)]
    return [c for c in cand if 0 <= c[0] < nx - 1 and 0 <= c[1] < ny - 1 and 0 <= c[2] < nz - 1]


def face_graph(face_ids, winding, xyz, shape) -> Graph:
    """Graph of pierced faces at their sample positions xyz (grid units);
    each face's direction is W times its normal."""
    ids = [int(v) for v in np.asarray(face_ids, np.uint64)]
    w = np.asarray(winding, np.int64)
    pos = np.asarray(xyz, np.float64).reshape(-1, 3).copy()
    dirs = np.array([np.multiply(_NORMAL[f & 3], float(w[a])) for a, f in enumerate(ids)],
                    np.float64).reshape(-1, 3)
    cells = {}
    for a, f in enumerate(ids):
        for c in face_cells(f, shape):
            cells.setdefault(c, []).append(a)
    adj = [set() for _ in ids]
    for members in cells.values():
        for a in members:
            for b in members:
                if a != b:
                    adj[a].add(b)
    return Graph(pos, dirs, adj)


# ---------------------------------------------------------------------------
# Sec. 3.2: node extraction (independent lines by depth-first traversal)
# ---------------------------------------------------------------------------
def components(g: Graph):
    """Node sets of the connected sub-graphs, each in traversal order, in the
    order of their lowest index."""
    seen = np.zeros(g.n, bool)
    out = []
    for s in range(g.n):
        if seen[s]:
            continue
        seen[s] = True
        order, stack = [], [s]
        while stack:
            u = stack.pop()
            order.append(u)
            for v in sorted(g.adj[u], reverse=True):  # pops visit ascending
                if not seen[v]:
                    seen[v] = True
                    stack.append(v)
        out.append(order)
    return out


# ---------------------------------------------------------------------------
# Sec. 3.3.1-3.3.2: box-mean candidates and iterative graph reduction
# ---------------------------------------------------------------------------
def reduce_pass(g: Graph, d: float):
    """One pass of box-mean estimation and collapse; returns (reduced graph,
    largest move of a sample from the node its box was centred on)."""
    n = g.n
    processed = np.zeros(n, bool)
    owner = np.full(n, -1, np.int64)
    new_pos, new_dirs, seeds = [], [], []
    half = 0.5 * d
    nxt = 0
    remaining = n
    lowest = 0
    while remaining:
        c = nxt
        centre = g.pos[c]
        members = [c]
        inset = {c}
        stack = [c]
        while stack:
            u = stack.pop()
            for v in sorted(g.adj[u]):
                if processed[v] or v in inset:
                    continue
                if np.max(np.abs(g.pos[v] - centre)) <= half:
                    inset.add(v)
                    members.append(v)
                    stack.append(v)
        knew = len(new_pos)
        new_pos.append(g.pos[members].mean(axis=0))
        new_dirs.append(g.dirs[members].sum(axis=0))
        seeds.append(c)
        for m in members:
            processed[m] = True
            owner[m] = knew
        remaining -= len(members)
        if not remaining:
            break
        ext = [v for m in members for v in g.adj[m] if not processed[v]]
        if ext:
            nxt = min(ext)
        else:
            while processed[lowest]:
                lowest += 1
            nxt = lowest
    adj = [set() for _ in new_pos]
    for u in range(n):
        for v in g.adj[u]:
            a, b = owner[u], owner[v]
            if a != b:
                adj[a].add(int(b))
                adj[b].add(int(a))
    new_pos = np.array(new_pos, np.float64).reshape(-1, 3)
    move = float(np.max(np.linalg.norm(new_pos - g.pos[seeds], axis=1))) if seeds else 0.0
    return Graph(new_pos, np.array(new_dirs, np.float64).reshape(-1, 3), adj), move


def reduce(g: Graph, d: float = 4.0, tol: float = 1e-3, max_passes: int = 10):
    """Passes of reduce_pass with the same box until no sample moves by tol or
    more (at most max_passes); returns (graph, number of passes)."""
    passes = 0
    while passes < max_passes:
        g, move = reduce_pass(g, d)
        passes += 1
        if move < tol:
            break
    return g, passes


FIX = 2 ** 32  # fixed-point units per grid spacing of box_reduce


def _fixed(pos):
    """Fixed-point integers (units of 2^-32 h) of positions below 2^31 in
    magnitude: x 2^32 (exact in FP64 for an FP32 x) rounded to the nearest
    integer, ties to even."""
    out = []
    for p in np.asarray(pos, np.float64).reshape(-1, 3):
        row = []
        for x in p:
            assert abs(x) < 2.0 ** 31, "positions must be below 2^31 in magnitude"
            row.append(round(float(x) * FIX))
        out.append(tuple(row))
    return out


def box_reduce(g: Graph, d: float = 4.0, max_passes: int = 10):
    """Lattice box reduction of a graph (the order-independent reading of Sec.
    3.3.1-3.3.2 in the module header).  Returns (reduced graph, label of every
    node of g = the lowest node index of its final cluster, fixed-point
    positions of the reduced nodes, number of passes).  Reduced nodes are in
    ascending order of their labels."""
    D = int(round(d * FIX))
    assert D > 0
    # current graph: nodes named by their lowest original index
    names = list(range(g.n))
    qpos = dict(zip(names, _fixed(g.pos)))
    dirs = {u: np.array(g.dirs[u], np.float64) for u in names}
    adj = {u: set(g.adj[u]) for u in names}
    label = list(range(g.n))
    quiet = 0
    passes = 0
    while passes < max_passes and quiet < 2:
        off = 0 if passes % 2 == 0 else D // 2
        key = {u: tuple((c - off) // D for c in qpos[u]) for u in names}
        seen, clusters = set(), []
        for s in sorted(names):
            if s in seen:
                continue
            seen.add(s)
            members, stack = [s], [s]
            while stack:
                u = stack.pop()
                for v in adj[u]:
                    if v not in seen and key[v] == key[u]:
                        seen.add(v)
                        members.append(v)
                        stack.append(v)
            clusters.append(sorted(members))
        new_of = {}
        nq, nd, nadj = {}, {}, {}
        for m in clusters:
            rep = m[0]
            c = len(m)
            nq[rep] = tuple((sum(qpos[u][a] for u in m) + c // 2) // c for a in range(3))
            nd[rep] = sum((dirs[u] for u in m), np.zeros(3))
            for u in m:
                new_of[u] = rep
        for u in names:
            a = new_of[u]
            nadj.setdefault(a, set())
            for v in adj[u]:
                b = new_of[v]
                if a != b:
                    nadj[a].add(b)
        merged = len(clusters) < len(names)
        names = sorted(nq)
        qpos, dirs, adj = nq, nd, nadj
        label = [new_of[x] for x in label]
        passes += 1
        quiet = 0 if merged else quiet + 1
    index = {u: a for a, u in enumerate(names)}
    red = Graph(np.array([[c / FIX for c in qpos[u]] for u in names], np.float64).reshape(-1, 3),
                np.array([dirs[u] for u in names], np.float64).reshape(-1, 3),
                [set(index[v] for v in adj[u]) for u in names])
    return red, np.array(label, np.int64), [qpos[u] for u in names], passes


# ---------------------------------------------------------------------------
# Sec. 3.4: classification, splitting and re-ordering
# ---------------------------------------------------------------------------
def classify(g: Graph, nodes) -> str:
    """'I', 'II' or 'III' for the connected node set `nodes`."""
    deg = [len(g.adj[u]) for u in nodes]
    if max(deg) > 2:
        return "III"
    if len(nodes) > 1 and min(deg) == 2:
        return "II"
    return "I"


def _walk(g: Graph, start: int, first: int, stop):
    """Nodes from start through first until a node in stop (included) or a
    dead end; returns (path, closed) where closed means it came back to start."""
    path = [start, first]
    prev, cur = start, first
    while cur not in stop:
        nb = [v for v in sorted(g.adj[cur]) if v != prev]
        if not nb:
            break
        prev, cur = cur, nb[0]
        if cur == start:
            return path, True
        path.append(cur)
    return path, False


def ordered_lines(g: Graph, nodes):
    """Ordered node lists of the simple lines of one connected set, as
    (type, nodes, closed) with type 'I' or 'II'."""
    kind = classify(g, nodes)
    nodes = sorted(nodes)
    if len(nodes) == 1:
        return [("I", nodes, False)]
    if kind == "I":
        start = min(u for u in nodes if len(g.adj[u]) == 1)
        path, _ = _walk(g, start, min(g.adj[start]), set())
        return [("I", path, False)]
    if kind == "II":
        start = nodes[0]
        path, _ = _walk(g, start, min(g.adj[start]), set())
        return [("II", path, True)]
    branch = {u for u in nodes if len(g.adj[u]) > 2}
    used = set()
    out = []
    for b in sorted(branch):
        for v in sorted(g.adj[b]):
            if (b, v) in used:
                continue
            path, closed = _walk(g, b, v, branch)
            for a, c in zip(path[:-1], path[1:]):
                used.add((a, c))
                used.add((c, a))
            if closed:
                used.add((path[-1], b))
                used.add((b, path[-1]))
            out.append(("II" if closed else "I", path, closed))
    return out


def orient(g: Graph, path, closed):
    """Turns an ordered line to run along its samples' circulation direction
    (right-hand rule); lines without direction information stay as they are."""
    p = g.pos[path]
    if len(path) < 2:
        return path
    seg = np.diff(np.vstack([p, p[:1]]) if closed else p, axis=0)
    dots = np.einsum("ij,ij->", seg, g.dirs[path][: len(seg)])
    if dots < 0:
        if closed:
            return [path[0]] + path[1:][::-1]
        return path[::-1]
    return path


# ---------------------------------------------------------------------------
# Sec. 3.4: Catmull-Rom vectorization and Eq. 7
# ---------------------------------------------------------------------------
def catmull_rom(points, closed: bool, per_segment: int = PER_SEGMENT) -> np.ndarray:
    """Uniform Catmull-Rom curve through the ordered points."""
    P = np.asarray(points, np.float64).reshape(-1, 3)
    m = len(P)
    if m < 2:
        return P.copy()
    if closed:
        ext = np.vstack([P[-1:], P, P[:2]])
        nseg = m
    else:
        ext = np.vstack([P[:1], P, P[-1:]])
        nseg = m - 1
    t = np.arange(per_segment, dtype=np.float64) / per_segment
    t2, t3 = t * t, t * t * t
    out = []
    for s in range(nseg):
        p0, p1, p2, p3 = ext[s], ext[s + 1], ext[s + 2], ext[s + 3]
        c = (2.0 * p1[None, :] + np.outer(t, p2 - p0)
             + np.outer(t2, 2.0 * p0 - 5.0 * p1 + 4.0 * p2 - p3)
             + np.outer(t3, -p0 + 3.0 * p1 - 3.0 * p2 + p3)) * 0.5
        out.append(c)
    if not closed:
        out.append(P[-1:])
    return np.vstack(out)


def curve_length(points, closed: bool) -> float:
    p = np.asarray(points, np.float64).reshape(-1, 3)
    if len(p) < 2:
        return 0.0
    if closed:
        p = np.vstack([p, p[:1]])
    return float(np.sum(np.linalg.norm(np.diff(p, axis=0), axis=1)))


THIN_UNIT = 2.0 ** 32  # arc-length units per h


def thin_piece(points, closed: bool, d: float):
    """Arc-length thinning of one ordered piece: (group means [g, 3] float64,
    group index of every sample).  Segment i runs from sample i to i + 1 (the
    last one of a closed piece back to sample 0, which does not move any
    sample's arc length); s_i = sum of the rounded lengths of segments < i."""
    P = np.asarray(points, np.float64).reshape(-1, 3)
    m = len(P)
    if m == 0:
        return np.zeros((0, 3)), np.zeros(0, np.int64)
    s = np.zeros(m, np.int64)
    acc = 0
    for i in range(1, m):
        dx, dy, dz = P[i] - P[i - 1]
        seg = np.sqrt((dx * dx + dy * dy) + dz * dz)
        acc += int(np.rint(seg * THIN_UNIT))
        s[i] = acc
    D = int(np.rint(d * THIN_UNIT))
    box = s // D
    group = np.zeros(m, np.int64)
    for i in range(1, m):
        group[i] = group[i - 1] + (1 if box[i] != box[i - 1] else 0)
    means = np.zeros((group[-1] + 1, 3))
    for gi in range(group[-1] + 1):
        members = np.flatnonzero(group == gi)
        acc3 = np.zeros(3)
        for a in members:
            acc3 = acc3 + P[a]
        means[gi] = acc3 / len(members)
    return means, group


def density_error(psi: np.ndarray, points) -> float:
    """Eq. 7: mean |rho| at the points over the mean density of the field."""
    from . import density

    pts = np.asarray(points, np.float64).reshape(-1, 3)
    if len(pts) == 0:
        return 0.0
    rho = density(psi, pts)
    a = np.asarray(psi).astype(np.complex128)
    rho_bar = float(np.mean(a.real ** 2 + a.imag ** 2))
    return float(np.sum(np.abs(rho)) / (rho_bar * len(pts)))


# ---------------------------------------------------------------------------
# the whole pipeline
# ---------------------------------------------------------------------------
def vectorize(g: Graph, d: float = 4.0, tol: float = 1e-3, max_passes: int = 10):
    """Components, reduction, classification, ordering and splines.

    Returns dict: reduced graph, passes, and lines: list of dicts with
    component (index), type ('I' / 'II' / 'III' of the component), piece
    ('I' / 'II'), closed, nodes (reduced-graph indices in order), samples
    [m, 3], curve [p, 3], length."""
    comps = components(g)
    lines = []
    passes = 0
    reduced = []
    for ci, nodes in enumerate(comps):
        sub, remap = _subgraph(g, nodes)
        r, p = reduce(sub, d, tol, max_passes)
        passes = max(passes, p)
        reduced.append(r)
        for rc in components(r):
            kind = classify(r, rc)
            for piece, path, closed in ordered_lines(r, rc):
                path = orient(r, path, closed)
                samples = r.pos[path]
                curve = catmull_rom(samples, closed)
                lines.append({"component": ci, "type": kind, "piece": piece, "closed": closed,
                              "nodes": path, "samples": samples, "curve": curve,
                              "length": curve_length(curve, closed),
                              "branch_points": int(np.sum(r.degrees()[rc] > 2))})
    return {"lines": lines, "passes": passes, "reduced": reduced,
            "reconnections": int(sum(int(np.sum(r.degrees() > 2)) for r in reduced))}


def _subgraph(g: Graph, nodes):
    nodes = sorted(nodes)
    remap = {u: a for a, u in enumerate(nodes)}
    adj = [{remap[v] for v in g.adj[u]} for u in nodes]
    return Graph(g.pos[nodes].copy(), g.dirs[nodes].copy(), adj), remap
