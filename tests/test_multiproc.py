"""The multi-GPU paths on CPU ranks (gloo, world size 2).  The benchmark runs
replicas, so its only cross-rank steps are the barrier and the maximum of the
ranks' times; the whole-job value counts every rank's grid points over the
slowest rank's time; the reference arm runs on rank 0 alone.  The z-slab
sharding of one snapshot: each rank identifies its planes plus a one-plane
halo (here with the FP64 oracle on the host) and the face lists gathered in
rank order equal the single-grid list."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_env()
    mine = 10.0 + 5.0 * rank  # rank 1 is the slowest
    dist.barrier()
    ms = bench.slowest_ms(mine, "cpu")
    value = bench.job_value(ws, 512 ** 3, 7, ms)
    out.put((rank, ws, r, local, ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ws, r, local, ms, value in res:
        assert (ws, r, local) == (2, rank, rank)
        assert ms == 15.0
        assert value == 2 * 512 ** 3 * 7 / 15e-3


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:  # the reference arm must return before touching its arguments
        def __getattr__(self, name):
            raise AssertionError(f"rank 1 read args.{name}")

    assert bench.run_reference(A()) == 0


def _slab_rank(rank, world, port, out):
    import numpy as np
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import oracle
    import synth
    from paper_1911_12070_gb300 import slabs

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    host = synth.random_waves_numpy((23, 30, 34), synth.wave_spec(9, 256))
    nz, ny, nx = host.shape
    z0, z1 = slabs.slab_bounds(nz, world)[rank]
    w, _ = oracle.identify(np.ascontiguousarray(host[z0:min(nz, z1 + 1)]))
    ids, wv = oracle.face_list(w)
    ids = torch.from_numpy(ids.astype(np.int64))
    keep = slabs.owned_mask(ids, z0, z1, nx, ny)
    gids = slabs.to_global(ids[keep], z0, nx, ny)
    allids = slabs.gather_to_all(gids)
    allw = slabs.gather_to_all(torch.from_numpy(wv.astype(np.int8))[keep])
    if rank == 0:
        fw, _ = oracle.identify(host)
        fids, fwv = oracle.face_list(fw)
        out.put((bool(np.array_equal(allids.numpy(), fids.astype(np.int64))),
                 bool(np.array_equal(allw.numpy(), fwv)), int(len(fids))))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_one_snapshot_by_z_slabs():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_slab_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    same_ids, same_w, n = out.get(timeout=180)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert same_ids and same_w and n > 50
