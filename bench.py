#!/usr/bin/env python3
"""Benchmark of the particle-in-cell step on one GB300 (or N replicas).

Default workload: 3D3V periodic thermal pair plasma, 128^3 cells, 32
particles per cell per species (134,217,728 particles), theta = 1, n_x = 1,
rho_sp0 = 64, dt = 0.5.  A step is one full main-loop step of App. A.3.1:
field half advances, gather + Boris + move + charge-conserving deposit,
e advance with the current, and the amortised re-sort.  The metric is
particle-steps per nanosecond of the mixed-precision path; the FP64 path is
timed on the same workload next to it.

--impl reference times the FP64 CPU oracle on the host cores instead, on a
bounded sample of the same workload (a 32^3 box with the same particles per
cell and temperature).  Multi-GPU: the runs are independent replicas, one per
rank, with no collective on the data path.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "thermal3d_128": dict(name="3D3V thermal pair plasma 128^3, 32 ppc/species, theta=1", ndim=3, nx=128, ny=128,
                          nz=128, ppc=32, theta=1.0, n_x=1.0, rho_sp0=64.0, dt=0.5),
    "thermal2d_1024": dict(name="2D3V thermal pair plasma 1024^2, 50 ppc/species, theta=0.01", ndim=2, nx=1024,
                           ny=1024, nz=1, ppc=50, theta=0.01, n_x=20.0, rho_sp0=100.0, dt=0.5),
    "thermal3d_64": dict(name="3D3V thermal pair plasma 64^3, 32 ppc/species, theta=1", ndim=3, nx=64, ny=64,
                         nz=64, ppc=32, theta=1.0, n_x=1.0, rho_sp0=64.0, dt=0.5),
    "thermal2d_512": dict(name="2D3V thermal pair plasma 512^2, 50 ppc/species, theta=0.01", ndim=2, nx=512,
                          ny=512, nz=1, ppc=50, theta=0.01, n_x=20.0, rho_sp0=100.0, dt=0.5),
    "ensemble256": dict(name="256 independent 2D3V thermal pair plasmas, grids 32^2..256^2, ppc/species in {4..256}, "
                             "theta in [0.01, 1]", ndim=2, nx=0, ny=0, nz=1, ppc=0, theta=0.0, n_x=0.0, rho_sp0=0.0,
                        dt=0.5, ensemble=256),
    "ensemble16": dict(name="16 independent 2D3V thermal pair plasmas (the first 16 runs of ensemble256; profiling "
                            "size)", ndim=2, nx=0, ny=0, nz=1, ppc=0, theta=0.0, n_x=0.0, rho_sp0=0.0, dt=0.5,
                       ensemble=16),
    "thermal2d_64": dict(name="2D3V thermal pair plasma 64^2, 16 ppc/species, theta=0.1", ndim=2, nx=64, ny=64, nz=1,
                         ppc=16, theta=0.1, n_x=0.1 ** -0.5, rho_sp0=32.0, dt=0.5),
}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def ensemble_members(count, seed=4):
    """The ensemble's runs: N_x, N_y uniform in [32, 256], particles per cell
    per species from {4, 8, ..., 256}, log theta uniform in [log 0.01, 0],
    n_x = theta^-1/2 (Debye length = cell), rho_sp0 = 2 ppc."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        nx, ny = (int(v) for v in rng.integers(32, 257, 2))
        ppc = int(rng.choice([4, 8, 16, 32, 64, 128, 256]))
        theta = float(np.exp(rng.uniform(np.log(0.01), 0.0)))
        out.append(dict(nx=nx, ny=ny, ppc=ppc, theta=theta, n_x=theta ** -0.5, rho_sp0=2.0 * ppc))
    return out


def _load(ctx, w, seed):
    """Seeded synthetic state through the library's own Maxwell-Juttner loader:
    co-located electron-positron pairs (rho = 0), uniform positions, rest-frame
    Maxwell-Juttner momenta of temperature theta, zero fields."""
    ctx.load_maxwell_juttner(0, 0, w["ppc"], w["theta"], (0.0, 0.0, 0.0), seed=seed)
    ctx.load_maxwell_juttner(0, 1, w["ppc"], w["theta"], (0.0, 0.0, 0.0), colocate_with=0, seed=seed + 1)


def _oracle_state(w, seed, nx, ny, nz):
    """The same kind of state built by the oracle's own loader (for the CPU leg)."""
    import oracle
    from oracle import mj
    ncell = nx * ny * (nz if w["ndim"] == 3 else 1)
    n = int(round(w["ppc"] * ncell))
    st = oracle.State.empty(w["ndim"], nx, ny, nz, w["dt"], w["n_x"], w["rho_sp0"],
                            smooth_passes=w.get("smooth", 0))
    pos, u0 = mj.load(seed, 0, n, w["theta"], (0.0, 0.0, 0.0), w["ndim"], nx, ny, nz)
    _, u1 = mj.load(seed + 1, 1, n, w["theta"], (0.0, 0.0, 0.0), w["ndim"], nx, ny, nz)
    st.species.append(oracle.Species(np.ascontiguousarray(pos), np.ascontiguousarray(u0), -1.0, 1.0))
    st.species.append(oracle.Species(np.ascontiguousarray(pos.copy()), np.ascontiguousarray(u1), 1.0, 1.0))
    return st, 2 * n


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def _time_oracle_sample(w, steps, seed, parallel=False):
    """FP64 oracle on a 32^3 (3D) or 64^2 (2D) box with the workload's ppc and
    temperature, serial (the parity reference build) or with the particle loop
    on all host cores (its OpenMP build); returns (particle-steps/ns, seconds,
    particles, steps, sizes, threads)."""
    import oracle
    sw = dict(w)
    if w.get("ensemble"):   # one representative member of the ensemble
        w = sw = dict(ndim=2, nx=64, ny=64, nz=1, ppc=32, theta=0.1, n_x=0.1 ** -0.5, rho_sp0=64.0, dt=0.5,
                      name=w["name"], smooth=w.get("smooth", 0))
    elif w["ndim"] == 3:
        sw.update(nx=32, ny=32, nz=32)
    else:
        sw.update(nx=min(w["nx"], 64), ny=min(w["ny"], 64), nz=1)
    st, npart = _oracle_state(w, seed, sw["nx"], sw["ny"], sw["nz"])
    threads = oracle.lib_parallel().orc_threads(os.cpu_count() or 1) if parallel else 1
    t0 = time.perf_counter()
    if parallel:
        oracle.step_parallel(st, steps, threads)
    else:
        oracle.step(st, steps)
    dt = time.perf_counter() - t0
    return npart * steps / (dt * 1e9), dt, npart, steps, sw, threads


def _oracle_sample_text(w, sw, npart, threads):
    return ("FP64 oracle, 1 step per timed step on a %dx%dx%d box, %d ppc/species, theta=%g (%d particles), "
            "particle loop on %d host thread%s" % (sw["nx"], sw["ny"], sw["nz"] if w["ndim"] == 3 else 1, w["ppc"],
                                                   w["theta"], npart, threads, "" if threads == 1 else "s"))


def rank_env():
    """(rank, world size, local rank) of this process, as torch.distributed.run sets them."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def replica_seed(rank):
    """Seed of the replica on `rank`: every GPU advances its own independent run."""
    return 2 + 1000 * rank


def max_over_ranks(x, dist, device):
    """The slowest rank's time: the job is done when every replica is."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(npart_rank, steps, ms_max, world):
    """Whole-job particle-steps/ns: each of `world` replicas advances npart_rank
    particles (weak scaling) and the job takes the slowest rank's ms_max."""
    return npart_rank * steps * world / (ms_max * 1e6)


def run_reference(args, w):
    rank, _, _ = rank_env()
    if rank != 0:
        return 0
    times = []
    for k in range(args.warmup + args.steps):
        v, dt, npart, nst, sw, threads = _time_oracle_sample(w, 1, seed=1000 + k, parallel=True)
        if k >= args.warmup:
            times.append(dt)
    npart_steps = npart * args.steps
    total = sum(times)
    val = npart_steps / (total * 1e9)
    sample = _oracle_sample_text(w, sw, npart, threads)
    v1, dt1, _, _, _, _ = _time_oracle_sample(w, 1, seed=999)   # the plain build on one core, for context
    out = {"impl": "reference", "metric": "particle-steps/ns", "value": val, "unit": "particle-steps/ns",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": w["name"], "sample": sample},
           "cpu_baseline": {"value": val, "unit": "particle-steps/ns", "cores": threads, "kind": "oracle",
                            "sample": sample, "host_cores": os.cpu_count(),
                            "single_core": {"value": v1, "cores": 1, "seconds_per_step": dt1}},
           "e2e": {"value": val, "unit": "particle-steps/ns", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def run_ours(args, w):
    import torch
    import paper_1308_5892_gb300 as pic

    rank, world, local = rank_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    seed = replica_seed(rank)
    # measured FMA throughput, the ALU denominators (the FP64 path is bound by the FP64 pipe)
    alu = {"fp32_fma_tflops": pic.alu_peak(pic.PIC_PEAK_FP32_FMA),
           "fp64_fma_tflops": pic.alu_peak(pic.PIC_PEAK_FP64_FMA)}
    if w.get("ensemble"):
        members = ensemble_members(w["ensemble"])
        descs = []
        npart = 0
        for m in members:
            n = m["ppc"] * m["nx"] * m["ny"]
            npart += 2 * n
            descs.append(pic.run_desc(2, m["nx"], m["ny"], 1, m["n_x"], m["rho_sp0"], w["dt"],
                                      [(-1.0, 1.0, n), (1.0, 1.0, n)], smooth_passes=args.smooth))
    else:
        members = None
        nz = 1 if w["ndim"] == 2 else w["nz"]
        n = int(round(w["ppc"] * w["nx"] * w["ny"] * nz))
        descs = [pic.run_desc(w["ndim"], w["nx"], w["ny"], nz, w["n_x"], w["rho_sp0"], w["dt"],
                              [(-1.0, 1.0, n), (1.0, 1.0, n)], smooth_passes=args.smooth)]
        npart = 2 * n

    def load_all(ctx):
        if members is None:
            _load(ctx, w, seed)
        else:
            for r, m in enumerate(members):
                ctx.load_maxwell_juttner(r, 0, m["ppc"], m["theta"], (0.0, 0.0, 0.0), seed=seed + 2 * r)
                ctx.load_maxwell_juttner(r, 1, m["ppc"], m["theta"], (0.0, 0.0, 0.0), colocate_with=0,
                                         seed=seed + 2 * r + 1)
    results = {}
    legs = ((pic.PIC_MIXED, "mixed"),) if args.no_fp64 else ((pic.PIC_MIXED, "mixed"), (pic.PIC_FP64, "fp64"))
    for prec, name in legs:
        steps = args.steps if prec == pic.PIC_MIXED else max(1, min(args.steps, args.fp64_steps))
        ctx = pic.Context(descs, precision=prec, flags=pic.PIC_FLAG_TIMING, tile=tuple(args.tile),
                          sort_interval=args.sort_interval)
        load_all(ctx)
        tuned = None
        if prec == pic.PIC_MIXED and not args.no_autotune and args.tile == (0, 0, 0) and args.sort_interval == 0:
            tuned = ctx.autotune(max_steps=args.autotune_steps)
        ctx.step(args.warmup)
        stream = torch.cuda.current_stream()
        K = int(ctx.tuning()["sort_interval"]) if prec == pic.PIC_MIXED else 1

        def align():
            # align the sort phase so that the first timed step sorts: the window then
            # holds ceil(steps / K) sorts, never fewer than the amortised share
            ctx.set_flags(pic.PIC_FLAG_TIMING)
            _, n0 = ctx.kernel_time(pic.PIC_KERNEL_SORT)
            for _ in range(K):
                ctx.step(1)
                if ctx.kernel_time(pic.PIC_KERNEL_SORT)[1] > n0:
                    break
            if K > 1:
                ctx.step(K - 1)

        def window(flags, sample_clocks):
            ctx.set_flags(flags)
            ctx.kernel_time(pic.PIC_KERNEL_PUSH, reset=True)
            barrier()
            clocks = ClockSampler(local)
            if sample_clocks:
                clocks.start()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.step(steps)
            e1.record(stream)
            barrier()
            return e0.elapsed_time(e1), (clocks.stop() if sample_clocks else None), ctx.counters()

        if prec == pic.PIC_MIXED:
            # headline window: the step as a user runs it, one CUDA graph per period
            # of 2K steps (captured beforehand, outside the timed region)
            align()
            ctx.set_flags(0)
            ctx.step(2 * K)
            ms, clk, cnt = window(0, True)
            # breakdown window: the same steps launched directly with per-class events
            align()
            ms_t, _, _ = window(pic.PIC_FLAG_TIMING, False)
        else:
            ms, clk, cnt = window(pic.PIC_FLAG_TIMING, False)
            ms_t = ms
        push_ms, push_n = ctx.kernel_time(pic.PIC_KERNEL_PUSH)
        field_ms, field_n = ctx.kernel_time(pic.PIC_KERNEL_FIELD)
        smooth_ms, smooth_n = ctx.kernel_time(pic.PIC_KERNEL_SMOOTH)
        sort_ms, sort_n = ctx.kernel_time(pic.PIC_KERNEL_SORT, reset=True)
        diag = ctx.diagnostics(0)
        ms = max_over_ranks(ms, dist, "cuda")
        ncell = sum(d.nx * d.ny * d.nz for d in descs)
        results[name] = dict(ms=ms, ms_direct=ms_t, steps=steps, push_ms=push_ms, push_n=push_n, field_ms=field_ms,
                             smooth_ms=smooth_ms, ncell=ncell, sort_ms=sort_ms, counters=cnt, clocks=clk, diag=diag,
                             tuning=dict(ctx.tuning(), autotune=tuned) if prec == pic.PIC_MIXED else None)
        ctx.close()
        del ctx
        torch.cuda.empty_cache()

    # end-to-end through the C ABI with host buffers: upload the state, run the
    # timed steps, read the state back; all copies inside the timed region
    e2e_s = None
    h2d = d2h = 0
    if not args.no_e2e and members is None:
        e2e_s, h2d, d2h = _e2e(pic, torch, descs[0], w, seed, args, barrier)
        e2e_s = max_over_ranks(e2e_s, dist, "cuda")
    if args.no_fp64:
        results["fp64"] = None
    ens = None
    if members is None and not args.no_ensemble:
        ens = _ensemble_leg(pic, torch, args, seed, barrier, dist)
    return _report(args, w, results, npart, world, rank, e2e_s, h2d, d2h, dist, len(descs), alu, ens)


def _ensemble_leg(pic, torch, args, seed, barrier, dist):
    """The batched ensemble of 256 uneven 2D3V runs (ensemble256) as a second leg
    of the default line: autotuned, then a window of graph-replayed steps (the
    value) and a window of direct launches with CUDA events around the batched
    push kernel (its roofline)."""
    w = WORKLOADS["ensemble256"]
    members = ensemble_members(w["ensemble"])
    descs, npart = [], 0
    for m in members:
        n = m["ppc"] * m["nx"] * m["ny"]
        npart += 2 * n
        descs.append(pic.run_desc(2, m["nx"], m["ny"], 1, m["n_x"], m["rho_sp0"], w["dt"],
                                  [(-1.0, 1.0, n), (1.0, 1.0, n)]))
    ctx = pic.Context(descs, precision=pic.PIC_MIXED)
    for r, m in enumerate(members):
        ctx.load_maxwell_juttner(r, 0, m["ppc"], m["theta"], (0.0, 0.0, 0.0), seed=seed + 2 * r)
        ctx.load_maxwell_juttner(r, 1, m["ppc"], m["theta"], (0.0, 0.0, 0.0), colocate_with=0, seed=seed + 2 * r + 1)
    tuned = None if args.no_autotune else ctx.autotune(max_steps=args.autotune_steps)
    steps = args.ensemble_steps
    K = int(ctx.tuning()["sort_interval"])
    ctx.set_flags(0)
    ctx.step(max(args.warmup, 2 * K))
    stream = torch.cuda.current_stream()

    def window(flags):
        ctx.set_flags(flags)
        ctx.kernel_time(pic.PIC_KERNEL_PUSH, reset=True)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.step(steps)
        e1.record(stream)
        barrier()
        return e0.elapsed_time(e1)

    ms = max_over_ranks(window(0), dist, "cuda")
    launches = ctx.counters()["launches_per_step"]
    # per-kernel events need the phase launches: the step walker runs every phase in one launch
    window(pic.PIC_FLAG_TIMING)
    push_ms, push_n = ctx.kernel_time(pic.PIC_KERNEL_PUSH)
    ctx.close()
    del ctx
    torch.cuda.empty_cache()
    world = dist.get_world_size() if dist is not None else 1
    peak, peak_kind = _peaks()
    push_step = push_ms / max(push_n, 1) if push_n else None
    ach = 48.0 * npart / (push_step * 1e-3) / 1e9 if push_step else None
    return {"workload": w["name"], "runs": len(members), "particles_per_gpu": npart, "steps": steps,
            "value": job_value(npart, steps, ms, world), "unit": "particle-steps/ns", "ms_per_step": ms / steps,
            "tuning": tuned, "launches_per_step": launches,
            "roofline": None if ach is None else {
                "bound": "hbm", "kernel": "k_push_mixed_multi (all runs, one persistent launch; timed in the "
                "phase-launch form of the step, the value window runs the step walker)", "achieved": ach,
                "peak": peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": ach / peak,
                "push_ms_per_step": push_step, "bytes_per_particle_step": 48.0}}


def _e2e(pic, torch, desc, w, seed, args, barrier):
    """End to end through the C ABI with host buffers: the timed region uploads
    the whole state from pinned host memory, runs the steps and reads the whole
    state back into pinned host memory."""
    ctx = pic.Context([desc], precision=pic.PIC_MIXED, tile=tuple(args.tile), sort_interval=args.sort_interval)
    _load(ctx, w, seed)
    if not args.no_autotune and args.tile == (0, 0, 0) and args.sort_interval == 0:
        ctx.autotune(max_steps=args.autotune_steps)   # the process-wide cache answers for this workload
    fields, parts, _ = ctx.get_state(0)
    pin_f = torch.from_numpy(fields).pin_memory().numpy()
    pin_p = [torch.from_numpy(p).pin_memory().numpy() for p in parts]
    out_f = torch.empty(fields.shape, dtype=torch.float64).pin_memory().numpy()
    out_p = [torch.empty(p.shape, dtype=torch.float64).pin_memory().numpy() for p in parts]
    del fields, parts
    ctx.step(args.warmup)
    barrier()
    t0 = time.perf_counter()
    ctx.set_state(0, pin_f, pin_p)
    ctx.step(args.steps)
    ctx.get_state(0, out=(out_f, out_p))
    barrier()
    e2e_s = time.perf_counter() - t0
    ctx.close()
    nbytes = pin_f.nbytes + sum(p.nbytes for p in pin_p)
    return e2e_s, nbytes, nbytes


# FP64 path: particle state read + written per particle-step (x, u as doubles)
FP64_BYTES_PER_PARTICLE = {2: 80.0, 3: 96.0}
# FP64 flops per particle-step of k_push_fp64 (dadd + dmul + 2 dfma) and FP64
# instructions (dadd + dmul + dfma), from ncu instruction counts on the 64^3 and 512^2
# thermal workloads divided by the particles pushed: 3D 108 + 80 + 86, 2D 58 + 50 + 62
FP64_FLOPS_PER_PARTICLE = {3: 360.0, 2: 232.0}
FP64_INST_PER_PARTICLE = {3: 274.0, 2: 170.0}
# FP32 flops per particle-step of the mixed 3D push (fadd + fmul + 2 ffma: 32.4 + 92.8 +
# 103.3 per particle, ncu on the 64^3 workload)
MIXED_FP32_FLOPS_PER_PARTICLE = {3: 331.8}
# DRAM bytes (read + written) per particle-step of the 3D push kernel, from one
# ncu capture of the same kernel and tiling (16x8x4, sort interval 3) on the
# 64^3 case (profiles/push_mixed_thermal3d_64.md: 917.2 MB for 16,777,216
# particles), scaled to a launch by the particles it processes.  None where no
# capture exists.
PUSH_TRAFFIC_B_PER_PARTICLE = {3: 917.2e6 / 16777216}
PUSH_TRAFFIC_TILING = {3: ([16, 8, 4], 3)}   # (tile, sort interval) of that capture


def _fp64_roofline(w, f64, npart, alu, peak_hbm):
    """The FP64 path's push against the measured FP64 FMA peak: FP64 flops per
    particle-step from ncu instruction counts of k_push_fp64 (dadd + dmul +
    2 dfma), times the particles, over the push time per step (CUDA events)."""
    if f64 is None or f64["push_n"] == 0:
        return None
    out = {"bound": "alu", "unit": "TFLOP/s", "peak": alu["fp64_fma_tflops"], "peak_kind": "measured (pic_alu_peak)",
           "push_ms_per_step": f64["push_ms"] / f64["steps"],
           "hbm_frac": (FP64_BYTES_PER_PARTICLE[w["ndim"]] * npart / (f64["push_ms"] / f64["steps"] * 1e-3) / 1e9
                        / peak_hbm)}
    flops = FP64_FLOPS_PER_PARTICLE.get(w["ndim"])
    if flops is not None:
        ach = flops * npart / (f64["push_ms"] / f64["steps"] * 1e-3) / 1e12
        inst = FP64_INST_PER_PARTICLE[w["ndim"]] * npart / (f64["push_ms"] / f64["steps"] * 1e-3) / 1e12
        out.update(achieved=ach, frac=ach / alu["fp64_fma_tflops"], flops_per_particle_step=flops,
                   flops_source="ncu FP64 instruction counts of k_push_fp64 (dadd + dmul + 2 dfma)",
                   fp64_pipe_frac=inst / (0.5 * alu["fp64_fma_tflops"]))
    return out


def _report(args, w, results, npart, world, rank, e2e_s, h2d, d2h, dist, nruns=1, alu=None, ensemble=None):
    m = results["mixed"]
    value = job_value(npart, m["steps"], m["ms"], world)
    f64 = results["fp64"]
    peak, peak_kind = _peaks()
    push_launch_ms = m["push_ms"] / max(m["push_n"], 1)
    bytes_per_launch = m["counters"]["bytes_per_particle_step"] * npart
    achieved = bytes_per_launch / (push_launch_ms * 1e-3) / 1e9
    if rank == 0:
        out = {
            "metric": "particle-steps/ns", "value": value, "unit": "particle-steps/ns", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": m["ms"] / m["steps"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+i32 (mixed); f64",
            "data": "synthetic",
            "config": {"workload": w["name"], "particles_per_gpu": npart, "runs": nruns,
                       "parallelism": "replicas" if world > 1 else "single", "l2": "inputs larger than L2 (%.1f GB particle state)" % (npart * 28 / 1e9),
                       "tuning": m["tuning"]},
            "fp64": None if f64 is None else {"value": npart * f64["steps"] / (f64["ms"] * 1e6) * world,
                                              "unit": "particle-steps/ns", "ms_per_step": f64["ms"] / f64["steps"],
                                              "steps": f64["steps"],
                                              "roofline": _fp64_roofline(w, f64, npart, alu, peak)},
            "alu_peaks": alu,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         # counters of another tiling do not describe this kernel: null then
                         "traffic": (PUSH_TRAFFIC_B_PER_PARTICLE[w["ndim"]] * npart
                                     if w.get("ndim") in PUSH_TRAFFIC_B_PER_PARTICLE and nruns == 1
                                     and PUSH_TRAFFIC_TILING[w["ndim"]] == (list(m["tuning"]["tile"]),
                                                                            m["tuning"]["sort_interval"]) else None),
                         "traffic_source": "ncu dram bytes of the same kernel and tiling (16x8x4) at 64^3, scaled by particles",
                         "kernel": "k_push_mixed (gather+push+deposit, both species)",
                         "peak_kind": peak_kind, "push_ms_per_step": push_launch_ms,
                         "field_ms_per_step": m["field_ms"] / m["steps"], "sort_ms_total": m["sort_ms"],
                         "sort_interval": m["tuning"]["sort_interval"],
                         "ms_per_step_direct_launches": m["ms_direct"] / m["steps"],
                         "sorts_timed": -(-m["steps"] // m["tuning"]["sort_interval"]),
                         "fp32_frac": (MIXED_FP32_FLOPS_PER_PARTICLE[w["ndim"]] * npart / (push_launch_ms * 1e-3)
                                       / 1e12 / alu["fp32_fma_tflops"]
                                       if alu and w.get("ndim") in MIXED_FP32_FLOPS_PER_PARTICLE and nruns == 1
                                       else None)},
            "cpu_baseline": None,
            "e2e": None if e2e_s is None else {
                "value": npart * args.steps / (e2e_s * 1e9) * world, "unit": "particle-steps/ns",
                "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
                "note": "set_state from pinned host + steps + get_state to pinned host"},
            "gpu_launches": int(m["counters"]["launches_per_step"] * m["steps"]),
            "clocks": m["clocks"],
            "diag": {"gauss_max": m["diag"]["gauss_max"], "rho_max": m["diag"]["rho_max"],
                     "gauss_over_rho_max": m["diag"]["gauss_max"] / max(m["diag"]["rho_max"], 1e-300),
                     "steps_since_load": int(m["diag"]["step"])},
        }
        if ensemble is not None:
            out["ensemble"] = ensemble
        if args.smooth > 0:
            # current smoothing: each pass reads and writes 3 x 8 B per interior cell (the in-place
            # fold of the ghost images touches only the boundary layers and is not counted)
            bytes_step = 48.0 * m["ncell"] * args.smooth
            sm_ms = m["smooth_ms"] / m["steps"]
            ach = bytes_step / (sm_ms * 1e-3) / 1e9 if sm_ms > 0 else None
            out["config"]["smooth_passes"] = args.smooth
            out["roofline"]["smooth"] = {
                "kernels": "k_fold_shell + %d x k_smooth_cols" % args.smooth if nruns == 1 else
                           "k_smooth_multi (fold + %d passes)" % args.smooth, "passes": args.smooth, "ms_per_step": sm_ms,
                "algorithmic_bytes_per_step": bytes_step, "achieved": ach, "unit": "GB/s",
                "frac": None if ach is None else ach / peak}
        if not args.no_cpu_baseline:
            v, dt, npp, nst, sw, threads = _time_oracle_sample(w, 1, seed=77, parallel=True)
            v1, dt1, _, _, _, _ = _time_oracle_sample(w, 1, seed=78)
            out["cpu_baseline"] = {"value": v, "unit": "particle-steps/ns", "cores": threads, "kind": "oracle",
                                   "sample": _oracle_sample_text(w, sw, npp, threads) + " (%.2f s)" % dt,
                                   "host_cores": os.cpu_count(),
                                   "single_core": {"value": v1, "cores": 1, "seconds_per_step": dt1}}
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="thermal3d_128", choices=sorted(WORKLOADS))
    ap.add_argument("--fp64-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison leg")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg")
    ap.add_argument("--tile", type=int, nargs=3, default=(0, 0, 0))
    ap.add_argument("--sort-interval", type=int, default=0)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--smooth", type=int, default=0, help="current smoothing passes per step (0..4, default off)")
    ap.add_argument("--autotune-steps", type=int, default=120)
    ap.add_argument("--no-ensemble", action="store_true", help="skip the 256-run ensemble leg of the default line")
    ap.add_argument("--ensemble-steps", type=int, default=12)
    args = ap.parse_args()
    args.tile = tuple(args.tile)
    w = dict(WORKLOADS[args.workload])
    if not 0 <= args.smooth <= 4:
        ap.error("--smooth takes 0..4 passes")
    w["smooth"] = args.smooth
    if args.smooth:
        w["name"] += ", current smoothing %d pass%s" % (args.smooth, "es" if args.smooth > 1 else "")
    if args.impl == "reference":
        return run_reference(args, w)
    return run_ours(args, w)


if __name__ == "__main__":
    sys.exit(main())
