"""The N > 1 path is replicas only (each rank runs its own network, no data-path
collective); bench.aggregate combines the ranks: units summed, time = slowest
rank. Checked with world_size 2 over gloo on CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_env()
    assert (ws, r, local) == (world, rank, rank)
    units, secs = bench.aggregate(1000.0 * (rank + 1), 0.5 + rank, ws)
    out.put((rank, units, secs))
    dist.destroy_process_group()


def test_aggregate_two_ranks_gloo():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    for rank, units, secs in res:
        assert units == pytest.approx(3000.0)   # 1000 + 2000: whole-job searches
        assert secs == pytest.approx(1.5)       # slowest rank


def test_single_rank_passthrough():
    import bench
    assert bench.aggregate(123.0, 0.25, 1) == (123.0, 0.25)


def test_profile_counters_are_tied_to_the_kernel_sources(monkeypatch):
    """roofline.traffic (and the issue-active share) come from the committed ncu
    summary only while the search sources hash to the value recorded there; any
    other sources give no counters."""
    import builtins
    import hashlib
    import io

    import bench
    assert isinstance(bench.profile_counters(), dict)
    files = {f: f"// {f}\n".encode() for f in ("search.cu", "device.cuh", "octree.cu")}
    h = hashlib.sha256()
    for f in ("search.cu", "device.cuh", "octree.cu"):
        h.update(files[f])
    summary = (f"x\nsources-sha256: {h.hexdigest()}\ntraffic-bytes-per-launch: 1234\n"
               f"issue-active-first-update: 71.5\n")
    real_open = builtins.open

    def fake_open(path, mode="r", *args, **kwargs):
        name = os.path.basename(str(path))
        if name in files:
            return io.BytesIO(files[name])
        if name == "bh_search_traffic_gaussian_clusters_2p20.md":
            return io.StringIO(summary)
        return real_open(path, mode, *args, **kwargs)

    monkeypatch.setattr(builtins, "open", fake_open)
    monkeypatch.setattr(bench.os.path, "exists", lambda path: True)
    assert bench.profile_counters() == {"traffic": 1234.0, "issue_active": 71.5}
    files["search.cu"] = b"// changed\n"
    assert bench.profile_counters() == {}
