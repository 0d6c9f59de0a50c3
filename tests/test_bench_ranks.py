"""The multi-GPU path of bench.py (one replica per rank, no data-path
collective): rank bookkeeping, the max over ranks of the timed region and the
whole-job value, run as two gloo ranks on the CPU."""
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, w, local = bench.rank_env()
    ms = bench.max_over_ranks(10.0 + 3.0 * rank, dist, "cpu")   # rank 1 is the slow one
    q.put((r, w, local, ms, bench.replica_seed(r), bench.job_value(1000, 5, ms, w)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time_and_the_job_value():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [x[0] for x in res] == [0, 1] and all(x[1] == 2 for x in res)
    assert all(x[3] == 13.0 for x in res)                # max over ranks
    assert res[0][4] != res[1][4]                        # independent replicas
    assert res[0][5] == res[1][5] == pytest.approx(1000 * 5 * 2 / (13.0 * 1e6))


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_report_line_carries_the_contract_keys():
    """The JSON line of bench.py (built from timings, here synthetic) holds the
    contract's keys and the roofline objects, including the ALU rooflines and
    the smoothing leg, without a GPU."""
    import contextlib
    import io
    import json
    import types
    sys.path.insert(0, ROOT)
    import bench
    args = types.SimpleNamespace(steps=20, warmup=3, no_cpu_baseline=True, smooth=1, gpus=1, no_ensemble=True)
    w = dict(bench.WORKLOADS["thermal3d_128"], smooth=1)
    common = dict(ms_direct=160.0, field_ms=7.0, smooth_ms=1.3, ncell=128 ** 3, clocks={"sm_mhz": 2070.0},
                  diag={"gauss_max": 1e-6, "rho_max": 1.5, "step": 140})
    mixed = dict(common, ms=160.0, steps=20, push_ms=120.0, push_n=20, sort_ms=30.0,
                 counters={"bytes_per_particle_step": 56.0, "launches_per_step": 9.0},
                 tuning={"tile": [8, 8, 8], "sort_interval": 3, "halo": 3})
    fp64 = dict(common, ms=1300.0, steps=5, push_ms=1290.0, push_n=5, sort_ms=0.0,
                counters={"bytes_per_particle_step": 96.0, "launches_per_step": 5.0}, tuning=None)
    alu = {"fp32_fma_tflops": 78.3, "fp64_fma_tflops": 1.25}
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench._report(args, w, {"mixed": mixed, "fp64": fp64}, 134217728, 1, 0, 3.0, 6.5e9, 6.5e9, None, 1, alu)
    d = json.loads(buf.getvalue())
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks"):
        assert k in d, k
    r = d["roofline"]
    assert r["bound"] == "hbm" and abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    assert abs(d["value"] - 134217728 * 20 / (160.0 * 1e6)) < 1e-9
    assert d["fp64"]["roofline"]["bound"] == "alu" and 0 < d["fp64"]["roofline"]["frac"] < 1
    assert 0 < r["fp32_frac"] < 1 and 0 < r["smooth"]["frac"] < 1
    assert d["e2e"]["h2d_bytes_per_step"] == 6.5e9 / 20
