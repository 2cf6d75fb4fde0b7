"""Z-slab sharding of one snapshot over ranks (host logic; the compute is the
library's identification and localization on each rank's slab).

Faces are independent given a one-plane halo: rank r owns the planes
[z0, z1) of a ceil(nz / P)-plane partition and runs on psi[z0 : z1 + 1] (its
planes plus the first plane of the next rank), keeping the faces whose
minimum corner lies in its own planes.  Global face ids are the local ones
shifted by z0 * nx * ny nodes, and positions use a grid origin shifted by z0
planes, so the concatenation of the ranks' lists in rank order is the
single-grid result: ascending face ids, the same windings, the same samples.
Gathering to one rank is an all-gather of the counts, an exclusive scan, and
an all-gather of the (padded) lists.
"""
from __future__ import annotations


def slab_bounds(nz: int, parts: int):
    """[(z0, z1)] of a partition of nz planes into `parts` slabs of
    ceil(nz / parts) planes (trailing slabs may be short or empty)."""
    step = -(-nz // parts) if parts > 0 else nz
    out = []
    for r in range(parts):
        z0 = min(nz, r * step)
        z1 = min(nz, z0 + step)
        out.append((z0, z1))
    return out


def owned_mask(face_ids, z0: int, z1: int, nx: int, ny: int):
    """Faces (local ids of the slab psi[z0 : z1 + 1]) whose minimum corner lies in
    the rank's own planes (local plane < z1 - z0)."""
    lin = face_ids >> 2
    k = lin // (nx * ny)
    return k < (z1 - z0)


def to_global(face_ids, z0: int, nx: int, ny: int):
    """Local face ids of a slab starting at plane z0 -> ids of the full grid."""
    return face_ids + ((z0 * nx * ny) << 2)


def identify_localize_slab(q, psi, z0: int, z1: int, h: float = 1.0, origin=(0.0, 0.0, 0.0)):
    """Faces and plain samples owned by the slab [z0, z1) of psi ([nz, ny, nx] on
    the device): (face_ids, winding, xyz, resid, flags) with global ids and
    positions."""
    import paper_1911_12070_gb300 as qtv

    import torch

    nz, ny, nx = psi.shape
    if z1 <= z0:
        dev = psi.device
        return (torch.empty(0, dtype=torch.int64, device=dev),
                torch.empty(0, dtype=torch.int8, device=dev),
                torch.empty((0, 3), dtype=torch.float32, device=dev),
                torch.empty(0, dtype=torch.float32, device=dev),
                torch.empty(0, dtype=torch.uint8, device=dev))
    view = psi[z0:min(nz, z1 + 1)]
    grid = qtv.Grid.of(tuple(view.shape), h=h,
                       origin=(origin[0], origin[1], origin[2] + h * z0))
    ids, w, xyz, resid, flags = _identify_localize(q, view, grid)
    keep = owned_mask(ids, z0, z1, nx, ny)
    return (to_global(ids[keep], z0, nx, ny), w[keep], xyz[keep], resid[keep], flags[keep])


def _identify_localize(q, view, grid):
    import torch

    dev = view.device
    nz, ny, nx = view.shape
    cap = max(1024, int(0.02 * nx * ny * nz))
    count = torch.zeros(1, dtype=torch.int64, device=dev)
    for _ in range(2):
        ids = torch.empty(cap, dtype=torch.int64, device=dev)
        w = torch.empty(cap, dtype=torch.int8, device=dev)
        xyz = torch.empty((cap, 3), dtype=torch.float32, device=dev)
        resid = torch.empty(cap, dtype=torch.float32, device=dev)
        flags = torch.empty(cap, dtype=torch.uint8, device=dev)
        q.identify_localize_into(view, ids, w, count, xyz, resid, flags, grid=grid)
        n = int(count.item())
        if n <= cap:
            break
        cap = n
    return ids[:n], w[:n], xyz[:n], resid[:n], flags[:n]


def gather_to_all(t, group=None):
    """All-gather of a 1-D or 2-D tensor of any length per rank, concatenated in
    rank order (counts all-gathered, lists padded to the largest)."""
    import torch
    import torch.distributed as dist

    ws = dist.get_world_size(group)
    n = torch.tensor([t.shape[0]], dtype=torch.int64, device=t.device)
    counts = [torch.zeros_like(n) for _ in range(ws)]
    dist.all_gather(counts, n, group=group)
    counts = [int(c.item()) for c in counts]
    m = max(counts) if counts else 0
    pad = t.new_zeros((m,) + tuple(t.shape[1:]))
    pad[: t.shape[0]] = t
    parts = [torch.zeros_like(pad) for _ in range(ws)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([p[:c] for p, c in zip(parts, counts)])
