"""The multi-GPU path of the benchmark is replicas only (one factorization
does not shard without a panel exchange per step): every rank runs the same
evaluations, the timed region's time is the maximum over ranks and the
throughput counts the evaluations of all ranks.  Checked here with two gloo
ranks on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [120.0, 180.0][rank]
    ms = bench.max_over_ranks(local_ms, world, "cpu")
    evals, tflops = bench.replica_throughput(ms, world, 5, 2.0e13)
    q.put((rank, ms, evals, tflops))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank_and_sum_the_work():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    for rank, ms, evals, tflops in out:
        assert ms == 180.0                                  # the slowest rank
        assert abs(evals - 2 * 5 / 0.18) < 1e-9             # evaluations of both ranks
        assert abs(tflops - 2 * 5 * 2.0e13 / 0.18 / 1e12) < 1e-6


def test_single_rank_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(42.0, 1, "cpu") == 42.0
    evals, tflops = bench.replica_throughput(500.0, 1, 5, 2.0e13)
    assert abs(evals - 10.0) < 1e-12 and abs(tflops - 200.0) < 1e-9


def test_tile_mix_roofline_sums_the_unit_terms():
    # T* = sum of F_unit / P_unit over the kernel's units + 2 x stored bytes / BW
    import types
    import bench
    rows = [{"kernel": "dag_kernel (test)", "unit_lower_bounds_ms": {"a": 3.0, "b": 5.0, "c": 90.0}},
            {"kernel": "other", "unit_lower_bounds_ms": {"z": 1000.0}}]
    ts = types.SimpleNamespace(lay=types.SimpleNamespace(bytes_dp=1_000_000_000, bytes_sp=2_000_000_000))
    r = bench.tile_mix_roofline(rows, ts, 200.0)
    bw = bench.measured_hbm_gbs()[0]
    hbm_ms = 2 * 3e9 / (bw * 1e9) * 1e3
    assert abs(r["t_star_ms"] - (98.0 + hbm_ms)) < 1e-9
    assert abs(r["frac"] - r["t_star_ms"] / 200.0) < 1e-12
    assert r["largest_term_ms"] == 90.0
    assert bench.tile_mix_roofline([{"kernel": "other", "unit_lower_bounds_ms": {}}], ts, 1.0) is None


def test_dag_traffic_is_keyed_by_the_kernel_sources():
    import bench
    h = bench.dag_source_hash()
    assert len(h) == 16 and int(h, 16) >= 0
    assert h == bench.dag_source_hash()          # stable
    for key, val in bench.DAG_TRAFFIC.items():
        assert len(key) == 16 and val > 0


def _shard_rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    costs = [float(n) ** 3 for n in (500, 8000, 3000, 3000, 700, 6000, 1200)]
    mine = bench.shard_problems(costs, rank, world)
    local = {"ms": 100.0 + 10 * rank, "completion_ms": [float(b) for b in mine], "problems": len(mine)}
    q.put((rank, mine, bench.gather_shards(local, world)))
    dist.barrier()
    dist.destroy_process_group()


def test_batch_shards_are_disjoint_balanced_and_gathered():
    """Batched problems are independent units: each rank takes a disjoint,
    cost-balanced share, and every rank gathers the slowest rank's time and
    every problem's completion."""
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_rank, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    shares = [o[1] for o in out]
    assert sorted(shares[0] + shares[1]) == list(range(7)) and not set(shares[0]) & set(shares[1])
    costs = [float(n) ** 3 for n in (500, 8000, 3000, 3000, 700, 6000, 1200)]
    work = [sum(costs[b] for b in sh) for sh in shares]
    assert max(work) <= sum(costs) / world + max(costs)          # the greedy's bound
    assert shares[0] == [1]                                      # the largest problem alone on one rank
    for _, _, (ms, comp, nprob) in out:
        assert ms == 110.0 and nprob == 7 and sorted(comp) == [float(b) for b in range(7)]


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` (the CPU oracle on its bounded sample) prints
    one JSON line with the main arm's metric and the keys the driver reads."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, check=True, timeout=600).stdout
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    import bench
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "TFLOP/s"
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["n"] == bench.CPU_SAMPLE_M ** 2


def test_batch_tensor_work_closed_form_matches_the_task_counts():
    """The batch roofline's closed-form tensor work of a band-1 factorization
    equals the task-by-task count the single-problem roofline uses."""
    import bench
    for p in (1, 2, 3, 5, 9, 20):
        nb = 128
        f64, f64u, f32, lp = bench.algorithmic_flops(p, nb, 1)
        want = lp * bench.TC_PAIRS + f64u * bench.EX_PAIRS
        assert abs(bench.tensor_work_band1(p * nb - 3, nb) - want) <= 1e-9 * max(1.0, want)
