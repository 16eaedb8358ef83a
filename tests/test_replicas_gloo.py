"""Multi-process paths on the CPU (gloo, world size 2, 127.0.0.1).

* Sharding by packet range is exact: two ranks run halves of one request's
  packet range (the oracle, counter-based random numbers keyed by the global
  packet index) and an integer sum-reduce of their histograms and counters
  equals the single-process run bit for bit. This is the one exchange a
  sharded spectrum would need.
* The replica benchmark's bookkeeping: each rank's workload has its own seed,
  and the job's times are the maximum over ranks (bench.reduce_max)."""
import importlib.util
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _shard_worker(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    from oracle import oracle as O
    from paper_2012_00963_gb300 import workloads as W
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl = W.cfg1(n_packets=6000, r_ap=3e-3, cone_alpha=0.5, t_snap=(1e-6, 2e-6))
        per = wl.n_packets // world
        r = O.simulate(wl, n_packets=per, packet_begin=rank * per, n_threads=2)
        h = torch.from_numpy(r["hist"].astype(np.int64))
        c = torch.from_numpy(r["counters"].astype(np.int64))
        dist.all_reduce(h, op=dist.ReduceOp.SUM)
        dist.all_reduce(c, op=dist.ReduceOp.SUM)
        if rank == 0:
            np.save(os.path.join(out_dir, "hist.npy"), h.numpy())
            np.save(os.path.join(out_dir, "cnt.npy"), c.numpy())
    finally:
        dist.destroy_process_group()


def _timing_worker(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _bench()

        class A:
            packets = 1000
            snapshots = 5
        wl = b.workload(A, rank)
        seeds = [None] * world
        dist.all_gather_object(seeds, wl.seed)
        t = torch.tensor([1.0 + rank, 10.0 - rank], dtype=torch.float64)
        t = b.reduce_max(t, world)
        if rank == 0:
            np.save(os.path.join(out_dir, "t.npy"), t.numpy())
            np.save(os.path.join(out_dir, "seeds.npy"), np.array(seeds))
    finally:
        dist.destroy_process_group()


def test_packet_range_sharding_is_exact(tmp_path):
    from oracle import oracle as O
    from paper_2012_00963_gb300 import workloads as W
    mp.start_processes(_shard_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2,
                       start_method="spawn")
    wl = W.cfg1(n_packets=6000, r_ap=3e-3, cone_alpha=0.5, t_snap=(1e-6, 2e-6))
    full = O.simulate(wl, n_threads=2)
    assert np.array_equal(np.load(tmp_path / "hist.npy"), full["hist"].astype(np.int64))
    assert np.array_equal(np.load(tmp_path / "cnt.npy"), full["counters"].astype(np.int64))


def test_replica_seeds_and_max_timing(tmp_path):
    mp.start_processes(_timing_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2,
                       start_method="spawn")
    assert np.array_equal(np.load(tmp_path / "t.npy"), [2.0, 10.0])
    seeds = np.load(tmp_path / "seeds.npy")
    assert len(set(seeds.tolist())) == 2
