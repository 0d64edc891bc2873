"""The multi-rank host logic of bench.py on CPU: two gloo ranks.

Each rank of a multi-GPU run solves its own batch (weak scaling, no
collective on the data path); the only collectives are the barriers and the
maximum of the per-rank step times.  These tests run that logic with the
gloo backend on the host, without a GPU.
"""
import os
import socket
import sys

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


def _rank_main(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    # step times of this rank: rank 1 is the slower one
    ms = [10.0 + 5.0 * rank, 12.0 + 5.0 * rank, 14.0 + 5.0 * rank]
    agg = bench._agg_ms(ms, ws, torch.device("cpu"))
    W = dict(bench.WORKLOADS["darcy100"])
    K, _ = bench._inputs(W, 3, bench._rank_seed(W, rank))
    mine = torch.tensor([float(np.sum(K)), float(K.shape[1])], dtype=torch.float64)
    allv = [torch.zeros(2, dtype=torch.float64) for _ in range(ws)]
    dist.all_gather(allv, mine)
    dist.barrier()
    q.put((rank, agg, [v.tolist() for v in allv], bench._dist()))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank_and_solve_distinct_batches():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for rank, agg, allv, d in out:
        assert agg == pytest.approx(17.0)          # max over ranks of the per-rank means (12, 17)
        assert d == (2, rank, rank)                 # WORLD_SIZE, RANK, LOCAL_RANK read from the env
        assert allv[0][1] == allv[1][1]             # same workload shape on every rank
        assert allv[0][0] != allv[1][0]             # but each rank its own batch
    assert out[0][2] == out[1][2]


def test_single_rank_mean_without_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench._agg_ms([3.0, 5.0], 1, None) == 4.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        workload, precond, pc_blocks, warm_start = "darcy100", None, 72, False
        steps, warmup, ref_seconds = 1, 0, 1.0

    assert bench.run_reference(Args()) is None
    assert capsys.readouterr().out == ""
