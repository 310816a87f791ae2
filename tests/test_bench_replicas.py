"""The multi-rank path of bench.py (N independent replicas, one per rank), checked on CPU with
two gloo ranks: the job's step time is the maximum over ranks, the whole-job rate counts every
rank's units at that time, and only rank 0 reports. No GPU is involved."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, ws: int, port: int, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        local_ms = 10.0 + 5.0 * rank            # rank 1 is the slow replica
        ms = bench.job_time_ms(local_ms, ws, "cpu")
        rate = bench.job_rate(64, ms, ws)
        env = bench.dist_env()
        out.put((rank, ms, rate, env))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_report_max_time_and_job_rate():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rate, env in res:
        assert ms == pytest.approx(15.0)                 # max over ranks, seen by every rank
        assert rate == pytest.approx(2 * 64 * 1000.0 / 15.0)
        assert env == (ws, rank, rank)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_time_ms(12.5, 1, "cpu") == 12.5
    assert bench.job_rate(1.0, 4.0, 1) == pytest.approx(250.0)


def _run_bench(args, env_extra):
    import json
    import subprocess
    env = dict(os.environ)
    env.update(env_extra)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    return r.returncode, [json.loads(l) for l in lines]


def test_reference_arm_line():
    """`bench.py --impl reference` times the CPU oracle (no GPU) and prints one JSON line with the
    contract's keys, its own sample sizes and a zero-copy e2e entry (here on the channel, whose
    oracle step takes seconds; the cylinder's takes minutes)."""
    code, lines = _run_bench(["--impl", "reference", "--workload", "bfs33", "--steps", "1", "--warmup", "1"],
                             {"RANK": "0", "WORLD_SIZE": "1", "LOCAL_RANK": "0"})
    assert code == 0 and len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["unit"] == "steps/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["ms_per_step"] == pytest.approx(1000.0 / d["value"])
    assert d["steps"] == 1 and d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("bfs33: backward-facing step, coarse 65,308 / fine 259,117 nodes")


def test_reference_arm_other_ranks_exit_quietly():
    code, lines = _run_bench(["--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "1"],
                             {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert code == 0 and lines == []


def test_bench_accounting_helpers():
    """The byte and launch counts behind the bench line's roofline and gpu_launches keys: the
    momentum solve's algorithmic bytes (two products of (v + 4) nnz + 4 n + 4 v n bytes and 90 v / 8
    bytes of vector passes per row per iteration, 12 nnz + 52 n per FP64 refinement pass) and the
    batched step's one launch per stage for all instances."""
    import types
    sys.path.insert(0, ROOT)
    import bench
    nnz, n = 7, 1
    # one FP32 iteration (v = 4) and one refinement pass (outer 0 -> one residual)
    assert bench.momentum_alg_bytes(nnz, n, 4, 1.0, 0.0) == 2 * (8 * 7 + 4 + 16) + 45 + (12 * 7 + 52)
    # FP64 iterations: ~330 bytes per row at 7 entries per row
    per_iter = bench.momentum_alg_bytes(nnz, n, 8, 1.0, -1.0)
    assert 320 <= per_iter <= 340
    flow = lambda lv, fo, ws: types.SimpleNamespace(info=types.SimpleNamespace(levels=lv, fine_order=fo),
                                                    params=types.SimpleNamespace(warm_start=ws))
    # permute, assembly, 2 predictor launches, momentum, restriction, coarse CG, 1 prolongation,
    # gradient, mass, correction
    assert bench.batch_launches_per_step([flow(1, 0, 3)] * 3) == 11
    assert bench.batch_launches_per_step([flow(1, 1, 0)]) == 8


def test_clock_record_from_sampled_lines():
    """The `clocks` key: median SM clock under load, the maximum clock and every throttle reason
    that was active in any sample (nvidia-smi's csv,noheader,nounits lines); lines that do not
    parse are skipped."""
    sys.path.insert(0, ROOT)
    import bench
    c = bench.ClockSampler(0)
    c.lines = [
        "0, 2070, 2070, 900.50, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1965, 2070, 1399.12, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1100.00, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070, 1100.00, 0x0, Not Active, Not Active, Not Active, Not Active",
        "not a sample",
    ]
    assert c.summary() == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    c.lines.append("0, 1500, 2070, 1200.00, 0x0000000000000008, Active, Not Active, Not Active, Not Active")
    s = c.summary()
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"] and s["samples"] == 4 and s["sm_mhz"] == 2017.5
    c.lines = []
    assert c.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
