"""Host logic of the multi-rank benchmark on CPU: two gloo ranks (127.0.0.1)
agree on the slowest rank's time, the whole-job throughput counts every rank's
signals, and the oracle arm runs on rank 0 only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(1.5 + rank, tdist, device="cpu")   # rank r "took" 1.5 + r seconds
    v = bench.job_throughput(world, 1000, t)
    out.put((rank, t, v))
    tdist.barrier()
    tdist.destroy_process_group()


def test_max_over_ranks_and_whole_job_throughput_with_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    # both ranks need the same port: pick it once
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in res:
        assert t == 2.5                       # the slowest rank's time on every rank
        assert v == pytest.approx(2 * 1000 / 2.5)


def test_max_over_ranks_without_group_is_identity():
    import bench
    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.job_throughput(1, 500, 2.0) == 250.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")

    class A:
        workload = "tiny"
        cpu_sample = 100
        steps = 1
        warmup = 0
        gpus = 2
    bench.run_reference(A())
    assert capsys.readouterr().out == ""


def test_reference_arm_json_line_carries_the_contract_keys(monkeypatch, capsys):
    """Rank 0 of the oracle arm prints one JSON line with the keys the bench
    contract names, its e2e moving no bytes and its cpu_baseline describing the
    same run."""
    import json

    import bench
    monkeypatch.setenv("RANK", "0")

    class A:
        workload = "tiny"
        cpu_sample = 200
        steps = 1
        warmup = 0
        gpus = 1
    bench.run_reference(A())
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "impl",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["config"]["workload"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
