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


def test_reference_arm_prints_one_contract_line():
    # the oracle arm of bench.py needs no GPU: one short sample on Darcy 100^2
    import json
    import subprocess
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "darcy100", "--steps", "1", "--warmup", "0", "--ref-seconds", "2"],
                         capture_output=True, text=True, timeout=600, env=env, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["unit"] == "systems/s" and d["steps"] == 1 and d["warmup"] == 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"] and cb["cpu"]
    assert d["e2e"] == {"value": d["value"], "unit": "systems/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "darcy2d 100x100" in d["config"]["workload"]
