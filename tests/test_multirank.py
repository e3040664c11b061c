"""The N > 1 path of bench.py on CPU: two gloo ranks.  The CTM does not shard
(every move needs all enlarged corners and a global SVD per cut), so N GPUs
run N independent replicas: each rank contracts its own synthetic state, no
collective touches the data, and only the timing is reduced (max over ranks)
into the whole-job throughput."""
import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    import synth
    dist = bench.init_dist(world)
    local_seconds = 0.5 + rank  # rank 1 is the slower replica
    t_max = bench.max_over_ranks(local_seconds, dist)
    value = bench.job_value(8, world, t_max)
    seed = bench.rank_seed(rank)
    w = synth.workload("product_noise", seed=seed, D=2, chi=8)
    scan = synth.scan(seed=seed, n=4, Ds=(2, 3), chis=(9, 12))
    q.put((rank, dist.get_backend(), t_max, value, seed, float(np.abs(w["tensors"][0]).sum()),
           [(i["D"], i["chi"]) for i in scan]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_replicas_and_max_timing():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, b0, t0, v0, s0, n0, sc0), (r1, b1, t1, v1, s1, n1, sc1) = out
    assert b0 == b1 == "gloo"
    assert t0 == t1 == 1.5  # the slowest rank's time on every rank
    assert v0 == v1 == 2 * 8 / 1.5  # all ranks' units over the slowest time
    assert s0 != s1 and n0 != n1  # independent replicas: different states per rank
    assert sc0 != sc1  # and different scan instance mixes (r = seed mod 12)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.init_dist(1) is None
    assert bench.max_over_ranks(0.25, None) == 0.25
    assert bench.job_value(4, 1, 0.5) == 8.0
