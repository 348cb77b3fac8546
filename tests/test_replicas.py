"""Replicas over ranks (CPU, gloo, world size 2): the trajectory-id ranges of
the ranks' handles are disjoint, and the job time and update count combine as
the bench reports them (max over ranks, sum of updates)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sizes = {24: 700, 48: 680, 64: 668}
        per_rank = 2048
        offs = bench.trajectory_offsets(rank, per_rank, sizes)
        ranges = [(offs[n], offs[n] + sizes[n]) for n in sizes]
        gathered = [None] * world
        dist.all_gather_object(gathered, ranges)
        ms, upd = bench.combine_over_ranks(torch, dist, 10.0 + 2.0 * rank, 100 + 20 * rank, "cpu")
        dist.barrier()
        out.put((rank, gathered, ms, upd))
    finally:
        dist.destroy_process_group()


def test_replica_ranges_and_reduction():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, gathered, ms, upd in results:
        assert ms == 12.0 and upd == 220.0
        spans = sorted(span for ranks in gathered for span in ranks)
        for (a0, a1), (b0, b1) in zip(spans, spans[1:]):
            assert a1 <= b0, spans


def _merge_worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import numpy as np
    from paper_2508_05745_gb300 import replicas as RP
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rng = np.random.default_rng(17)
        data = rng.standard_normal((20, 6)) * np.logspace(-8, 2, 6)   # per-trajectory observables
        split = [0, 7, 20]                                            # uneven: 7 and 13 trajectories
        mine = data[split[rank]:split[rank + 1]]
        # the rank's trajectories sit in two handles (sizes of a batch)
        mean, se = RP.merged_observables(dist, [mine[:3], mine[3:]])
        out.put((rank, mean, se))
    finally:
        dist.destroy_process_group()


def test_observable_merge_is_exact_over_ranks():
    """Two gloo ranks hold 7 and 13 trajectories of synthetic per-trajectory
    observables (spread over two handles each); the merged mean and standard
    error equal the single-process merge bit for bit, and a plain numpy
    estimate to rounding."""
    import numpy as np
    from paper_2508_05745_gb300 import replicas as RP
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_merge_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    rng = np.random.default_rng(17)
    data = rng.standard_normal((20, 6)) * np.logspace(-8, 2, 6)
    ref_mean, ref_se = RP.finalize(RP.exact_sums(data))
    for rank, mean, se in results:
        assert np.array_equal(mean, ref_mean) and np.array_equal(se, ref_se), rank
    assert np.allclose(ref_mean, data.mean(axis=0), rtol=1e-14, atol=0)
    assert np.allclose(ref_se, data.std(axis=0, ddof=1) / np.sqrt(20), rtol=1e-12, atol=0)
