"""The multi-rank path on CPU (gloo, world size 2).  Vectors are independent
(Eq. (3)), so ranks run replicas with their own seeds and exchange nothing on
the data path; the benchmark only reduces its figures over ranks: the max of
the times and the sum of the walker-steps.  The reference arm runs on rank 0
alone."""
import argparse
import os
import socket

import torch.multiprocessing as mp


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out = bench.reduce_over_ranks(dist, (10.0 + rank, 100.0 * (rank + 1), 2.0 * rank, 7.0), "cpu")
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def test_replica_figures_reduce_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # times: max over ranks; walker-steps: sum over ranks
    for r in range(2):
        assert res[r] == (11.0, 300.0, 2.0, 14.0)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    import bench
    args = argparse.Namespace(workload="ghz4", steps=1, warmup=3)
    bench.run_reference(args, 1, 2)
    assert capsys.readouterr().out == ""
