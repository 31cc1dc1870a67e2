"""Host logic of the multi-rank benchmark on CPU: two gloo ranks.

Instances shard across ranks with no data-path collective; the process group
carries the barrier and the max-over-ranks of the timings, and the job value
is the units all ranks processed over the slowest rank's time.
"""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    ctx = bench.Ctx(device="cpu")
    ctx.barrier()
    ms_local = 10.0 + 5.0 * rank           # rank 1 is the slowest
    ms_max = ctx.max_over_ranks(ms_local)
    value = ctx.job_rate(100, ms_max)
    ctx.barrier()
    ctx.dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"world": ctx.world, "ms_max": ms_max, "value": value}, f)


@pytest.mark.timeout(120)
def test_two_gloo_ranks_max_and_job_rate(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r in res:
        assert r["world"] == world
        assert r["ms_max"] == 15.0                          # the slowest rank's time on every rank
        assert abs(r["value"] - 200 / 15e-3) < 1e-6         # 2 ranks x 100 units / 15 ms


def test_rank_seeds_distinct():
    sys.path.insert(0, ROOT)
    import bench
    seeds = {bench.rank_seed(r, b, a) for r in range(8) for b in range(6) for a in range(3)}
    assert len(seeds) == 8 * 6 * 3


def test_reference_arm_only_rank0_prints(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    args = type("A", (), dict(steps=1, warmup=3, gpus=2, workload="batch1d", ragged_n=10000))()
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args)
    assert buf.getvalue() == ""


@pytest.mark.parametrize("workload", ["single64", "ns2d"])
def test_reference_arm_json_line(monkeypatch, capsys, workload):
    """The reference arm (the FP64 oracle on the host cores) prints one JSON
    line with the contract's keys, its own cpu_baseline and a zero-copy e2e."""
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "0")
    args = type("A", (), dict(steps=1, warmup=3, gpus=1, workload=workload, ragged_n=10000))()
    bench.run_reference(args)
    line = capsys.readouterr().out.strip().splitlines()
    assert len(line) == 1
    d = json.loads(line[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"] == bench.WORKLOAD_NAMES[workload]


def test_explicit_fft_cpu_rate():
    """The second CPU timing of the 1D batch (the paper's explicit method in
    FP64 on the host): a positive rate over the sub-configurations."""
    sys.path.insert(0, ROOT)
    import bench
    rate, sample = bench.oracle_rate_explicit_1d(0.2, bench.L1D, bench.SUBS)
    assert rate > 0 and "explicit" in sample
