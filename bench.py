#!/usr/bin/env python
"""Throughput of the SIPF-W step on the 128^3-grid / 2^22-particle workload.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl sipf|reference]
                    [--workload headline|large|ensemble|serve [--rate R | --rates a,b,..]]

One step = one pass of the whole hot path (the particle step: deposit,
gather, push, mass update and binning; the bucket plan; three spectral
passes) over the synthetic headline workload (three Gaussian
tumour seeds at seeded centres, sigma 0.04, unit periodic cube, dt 5e-4);
the FP64 diagnostics are read back every 100 steps inside the timed region.
Prints one JSON line on rank 0.  Under torchrun (N > 1) every rank runs an
independent replica on its own GPU (no data-path collective); the timed
region is bracketed by a barrier and the slowest rank's time is used.

--workload large times the 256^3-grid / 2^25-particle run the same way
(chi 0.02, dt 2.5e-4; no CPU baseline);
--workload ensemble instead times 64 uneven independent runs advanced
together (one stream each) against the same runs one at a time (runs/s);
--workload serve times continuous batching of Poisson-arriving requests
(p50/p99 time-to-result).

--impl reference times the FP64 oracle on the host cores (the paper ships
no code; the oracle is the reference arm), each step on a bounded sample of
the same workload recipe.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "particle-steps/s at 128^3 grid, 4M particles"
UNIT = "particle-steps/s"
WORKLOAD = "headline: 128^3 grid, 2^22 particles, 3 Gaussian seeds (sigma 0.04), dt 5e-4"
METRIC_LARGE = "particle-steps/s at 256^3 grid, 32M particles"
WORKLOAD_LARGE = ("large: 256^3 grid, 2^25 particles, 3 Gaussian seeds (sigma 0.04), chi 0.02, "
                  "dt 2.5e-4")
# Algorithmic bytes (what the method must move): per particle-step read X
# (12 B) + log a (8 B), write X' (12 B) + log a' (8 B); per node-step the 15
# float32 field touches of the reaction, solve, gather and deposit.
ALGO_B_PER_PARTICLE = 40
ALGO_B_PER_NODE = 60
# share of the per-node bytes that belongs to the particle-step kernel
# (gather of dv/dx, dv/dy, dv/dz, w: 16 B; deposit of u: 4 B)
SCATTER_B_PER_NODE = 20


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def _dist_init(n_gpus):
    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local = _env_int("LOCAL_RANK", 0)
    if world > 1:
        import torch
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return rank, world, local


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# DRAM bytes (read + write) of one launch from an ncu capture of the same
# workload (profiles/k_step_and_spectral_passes_headline_128cube_4M.md),
# valid only while the kernel's source is the one captured.
_STEP_SOURCES = ("paper_2605_20140_gb300/csrc/particles.cu",
                 "paper_2605_20140_gb300/csrc/sipf_internal.cuh")
# (kernel group, H, N) -> (sources, their digest, DRAM bytes per launch from
# the ncu captures summarised under profiles/)
NCU_TRAFFIC = {("particle_step", 128, 1 << 22): (_STEP_SOURCES, "9fe946df0af00a12", 151.4e6),
               ("particle_step", 256, 1 << 25): (_STEP_SOURCES, "9fe946df0af00a12", 1650.8e6)}


def _ncu_traffic(group, H, N):
    """DRAM bytes per launch from the committed ncu capture of this workload,
    or None when the kernel's sources changed since (sha256 over the files,
    first 16 hex)."""
    import hashlib
    entry = NCU_TRAFFIC.get((group, H, N))
    if not entry:
        return None
    paths, digest, traffic = entry
    h = hashlib.sha256()
    try:
        for path in paths:
            with open(os.path.join(ROOT, path), "rb") as f:
                h.update(f.read())
    except OSError:
        return None
    return traffic if h.hexdigest()[:16] == digest else None


def _host_cpu():
    """Core count and CPU model of this host (reported beside the CPU numbers)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                model = line.split(":", 1)[1].strip()
                if not model.isdigit():
                    break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"nproc": os.cpu_count(), "model": model}


def _cpu_baseline(wl_fn, n_sample_steps=1):
    """The FP64 oracle as it stands on this host: one full step of the
    workload (about 10-30 s of CPU work)."""
    from oracle import sipf_oracle as O
    wl = wl_fn()
    st = O.make_state(wl.H, wl.L, wl.origin, wl.params, wl.x, wl.mass, wl.ids, wl.v, wl.m, wl.w)
    t0 = time.perf_counter()
    for _ in range(n_sample_steps):
        st = O.step(st, wl.dt)
    dt = time.perf_counter() - t0
    return {"value": wl.N * n_sample_steps / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n_sample_steps} full step(s) of the 128^3 / 2^22 workload, "
                      f"NumPy FP64, single thread, {dt:.1f} s",
            "host": _host_cpu()}


def run_reference(args, rank, world):
    """The FP64 oracle on the host cores.  Each step is one oracle step of the
    headline recipe on a bounded sample, sized from --steps and --warmup so
    the whole run takes about two minutes: the full 128^3 grid with 2^16
    particles when the budget allows (~1.4 s per step), else a 64^3 or 32^3
    grid with fewer particles."""
    if rank != 0:
        return 0
    from oracle import sipf_oracle as O
    from sipf_inputs import workload
    budget = 120.0 / max(args.steps + args.warmup, 1)
    if budget >= 2.0:
        H, n_sample = 128, 1 << 16
    elif budget >= 0.3:
        H, n_sample = 64, 1 << 15
    else:
        H, n_sample = 32, 1 << 14
    wl = workload("headline", H=H, N=n_sample)
    st = O.make_state(wl.H, wl.L, wl.origin, wl.params, wl.x, wl.mass, wl.ids, wl.v, wl.m, wl.w)
    for _ in range(args.warmup):
        st = O.step(st, wl.dt)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        st = O.step(st, wl.dt)
    el = time.perf_counter() - t0
    value = n_sample * args.steps / el
    sample = (f"each step: one FP64 oracle step of the headline recipe on a {H}^3 grid with "
              f"{n_sample} particles ({el / args.steps:.3f} s/step, NumPy, single thread)")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": WORKLOAD + " (sampled)", "H": H, "N": n_sample},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": sample, "host": _host_cpu()},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


DIAG_EVERY = 100      # FP64 diagnostics (mass, minima, non-finite count) read back this often
DIAG_LAUNCHES = 4     # compact, deposit, partial sums, final sums


def _advance(sim, dt, steps):
    """`steps` calls' worth of sipf_step, with the diagnostics read back to
    the host every DIAG_EVERY steps as part of the timed work.  Returns the
    number of diagnostics calls."""
    done = calls = 0
    while done < steps:
        k = min(DIAG_EVERY - done % DIAG_EVERY, steps - done)
        sim.step(dt, k)
        done += k
        if done % DIAG_EVERY == 0:
            d = sim.diagnostics()
            calls += 1
            if d["nonfinite"]:
                raise SystemExit(f"non-finite values after step {d['step']}")
    return calls


def run_sipf(args, rank, world, local):
    import torch
    from paper_2605_20140_gb300 import sipf
    from sipf_inputs import workload

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the SIPF-W path has no CPU fallback)")
    torch.cuda.set_device(local)
    if not os.path.exists(sipf.LIB_PATH):
        from paper_2605_20140_gb300 import build
        build.build()
    sipf.load()
    large = args.workload == "large"
    wl = workload("large" if large else "headline", seed=rank)
    N, H, dt = wl.N, wl.H, wl.dt
    stream = torch.cuda.Stream()
    sim = sipf.Simulation(H, wl.L, wl.origin, N, wl.params, stream=stream.cuda_stream)
    sim.set_state(wl.x, wl.mass, wl.ids, wl.v, wl.m, wl.w)

    # ---- device-resident timed region: the public sipf_step (pairs of steps
    # replayed as the context's captured CUDA graph, captured during warm-up)
    sim.step(dt, args.warmup)
    sipf.sipf_sync(sim.ctx)
    clocks = ClockSampler(local)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    clocks.start()
    time.sleep(0.3)
    # `repeats` timed regions of --steps steps each (CUDA events on the
    # launching stream, barrier and synchronisation on both sides); the line
    # reports the median region and the spread of all of them
    reps = []
    n_diag = 0
    for r in range(args.repeats):
        if r:
            # every region times the same trajectory: back to the initial
            # state and the same warm-up (untimed), so the repeats differ
            # only by measurement noise
            sim.set_state(wl.x, wl.mass, wl.ids, wl.v, wl.m, wl.w)
            sim.step(dt, args.warmup)
        _barrier(world)
        torch.cuda.synchronize()
        e0.record(stream)
        n_diag += _advance(sim, dt, args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        _barrier(world)
        reps.append(_max_over_ranks(e0.elapsed_time(e1), world))
    ms_total = statistics.median(reps)
    # ---- per-kernel-group times over the timed region's own steps: the same
    # trajectory again (initial state, the same warm-up), traced with CUDA
    # events between the groups on the launching stream (tracing enqueues
    # launch by launch); the particle step's cost grows as the seeds spread,
    # so tracing later steps would describe other states than the ones timed
    n_prof = min(args.steps, 1000)
    sim.set_state(wl.x, wl.mass, wl.ids, wl.v, wl.m, wl.w)
    sim.step(dt, args.warmup)
    sipf.sipf_sync(sim.ctx)
    sipf.sipf_profile(sim.ctx, True)
    sim.step(dt, n_prof)
    torch.cuda.synchronize()
    sipf.sipf_profile(sim.ctx, False)
    clk = clocks.stop()
    prof = sipf.sipf_profile_read(sim.ctx)
    sipf.sipf_sync(sim.ctx)
    ms_step = ms_total / args.steps
    value = world * N * args.steps / (ms_total * 1e-3)

    # ---- roofline of the dominant kernel group (CUDA events on the launching stream)
    hbm, peak_kind = _peaks()
    dom = max(prof, key=lambda k: prof[k][0])
    dom_ms, dom_launches = prof[dom]
    per_launch_s = dom_ms * 1e-3 / max(dom_launches, 1)
    algo = {"particle_step": ALGO_B_PER_PARTICLE * N + SCATTER_B_PER_NODE * H ** 3}
    algo_bytes = algo.get(dom)
    roofline = None
    if algo_bytes is not None:
        achieved = algo_bytes / per_launch_s / 1e9
        roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm,
                    "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / hbm,
                    "traffic": _ncu_traffic(dom, H, N), "algorithmic_bytes": algo_bytes}
    step_bytes = ALGO_B_PER_PARTICLE * N + ALGO_B_PER_NODE * H ** 3
    step_roofline = {"algorithmic_bytes": step_bytes,
                     "achieved": step_bytes / (ms_step * 1e-3) / 1e9,
                     "frac": step_bytes / (ms_step * 1e-3) / 1e9 / hbm, "unit": "GB/s"}
    kernels = {k: {"ms_per_step": v[0] / max(n_prof, 1), "launches": v[1],
                   "share": v[0] / max(sum(x[0] for x in prof.values()), 1e-12)}
               for k, v in prof.items()}
    # per step: the traced groups' launches, plus the bucket-layout plan kernel
    # on the context's second stream
    launches = int(round((sum(v[1] for v in prof.values()) / max(n_prof, 1) + 1) * args.steps))
    launches += DIAG_LAUNCHES * n_diag // max(args.repeats, 1)
    sim.close()

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
        hx = pin(wl.x.T)
        hm, hid = pin(wl.mass), pin(wl.ids)
        hv, hmm, hw = pin(wl.v), pin(wl.m), pin(wl.w)
        out = torch.empty(4 * H ** 3, dtype=torch.float32).pin_memory().numpy()
        sim2 = sipf.Simulation(H, wl.L, wl.origin, N, wl.params, stream=stream.cuda_stream)
        sim2.set_state(hx.T, hm, hid, hv, hmm, hw)          # first call: device set-up
        sim2.step(dt, 2)
        sipf.sipf_sync(sim2.ctx)
        _barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sipf.sipf_set_state(sim2.ctx, hx, hm, hid, hv, hmm, hw, sipf.SIPF_HOST)
        t1 = time.perf_counter()
        _advance(sim2, dt, args.steps)
        sipf.sipf_sync(sim2.ctx)
        t2 = time.perf_counter()
        sipf.sipf_fields(sim2.ctx, sipf.FIELD_U | sipf.FIELD_V | sipf.FIELD_M | sipf.FIELD_W,
                         out, sipf.SIPF_HOST)
        t3 = time.perf_counter()
        el = _max_over_ranks(t3 - t0, world)
        sim2.close()
        h2d = hx.nbytes + hm.nbytes + hid.nbytes + hv.nbytes + hmm.nbytes + hw.nbytes
        d2h = out.nbytes
        e2e = {"value": world * N * args.steps / el, "unit": UNIT,
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "job": f"set_state from pinned host + {args.steps} steps (diagnostics every "
                      f"{DIAG_EVERY}) + u,v,m,w to host",
               # the one-off upload and download against the steps: a short run
               # is dominated by the upload, not by a slow step path
               "split_ms": {"upload_set_state": 1e3 * (t1 - t0),
                            "steps": 1e3 * (t2 - t1), "download_fields": 1e3 * (t3 - t2)},
               "steps_only_value": world * N * args.steps / (t2 - t1)}

    if rank != 0:
        return 0
    cpu = None if (args.no_cpu_baseline or large) else _cpu_baseline(lambda: workload("headline"))
    out = {"metric": METRIC_LARGE if large else METRIC, "value": value, "unit": UNIT,
           "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32 (f64 log-mass and reductions)", "data": "synthetic",
           "repeats": {"n": len(reps), "ms_per_step": [r / args.steps for r in reps],
                       "spread": (max(reps) - min(reps)) / ms_total,
                       "value_is": "median of the timed regions"},
           "config": {"workload": WORKLOAD_LARGE if large else WORKLOAD, "H": H, "N": N, "dt": dt,
                      "parallelism": f"replicas x{world}",
                      "l2": f"no flush: the step's working set (~{step_bytes / 1e6:.0f} MB of "
                            "algorithmic traffic) exceeds the 129 MB L2",
                      "diagnostics": f"FP64 diagnostics read back every {DIAG_EVERY} steps, "
                                     "inside the timed region"},
           "roofline": roofline, "step_roofline": step_roofline, "kernels": kernels,
           "kernels_traced_steps": n_prof,
           "gpu_launches": launches, "clocks": clk, "e2e": e2e, "cpu_baseline": cpu}
    print(json.dumps(out), flush=True)
    return 0


def run_ensemble(args, rank, world, local):
    """64 uneven independent runs (H in {32, 48, 64, 96}, N = 2^U[14, 20],
    chi, alpha, Du drawn per run, one Philox key each) advanced together:
    batched (one particle-step launch over all runs' work list, one launch per
    spectral pass and grid size, replayed as a CUDA graph), against the same
    runs one stream each, and one at a time.  Every arm starts from the same
    initial states; the batched and per-stream members must end bit for bit
    equal."""
    import torch
    from paper_2605_20140_gb300 import sipf
    from sipf_inputs import ensemble_workloads

    torch.cuda.set_device(local)
    count, K, W = 64, args.steps, args.warmup
    runs = ensemble_workloads(count, seed=rank)
    dts = np.array([w.dt for w in runs])
    specs = [(w.H, w.L, w.origin, w.N, w.params) for w in runs]

    def timed(mode):
        ens = sipf.Ensemble(specs, mode=mode)
        try:
            for sim, w in zip(ens.members, runs):
                sim.set_state(w.x, w.mass, w.ids, w.v, w.m, w.w)
            ens.step(dts, W)
            ens.sync()
            for sim, w in zip(ens.members, runs):
                sim.set_state(w.x, w.mass, w.ids, w.v, w.m, w.w)
            _barrier(world)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ens.step(dts, K)
            ens.sync()
            el = time.perf_counter() - t0
            path = ens.last_path()
            fields = [sim.fields(sipf.FIELD_U | sipf.FIELD_M) for sim in ens.members[:8]]
        finally:
            ens.close()
        return el, path, fields

    clocks = ClockSampler(local)
    clocks.start()
    t_batched, path_b, f_b = timed(sipf.SIPF_ENSEMBLE_BATCHED)
    t_streams, path_s, f_s = timed(sipf.SIPF_ENSEMBLE_STREAMS)
    # one at a time: the same runs, each alone on one stream (its own graphs)
    stream = torch.cuda.Stream()
    sims = [sipf.Simulation(*spec, stream=stream.cuda_stream) for spec in specs]
    try:
        for sim, w in zip(sims, runs):
            sim.set_state(w.x, w.mass, w.ids, w.v, w.m, w.w)
            sim.step(w.dt, W)
            sim.set_state(w.x, w.mass, w.ids, w.v, w.m, w.w)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for sim, dt in zip(sims, dts):
            sim.step(dt, K)
            sipf.sipf_sync(sim.ctx)
        t_alone = time.perf_counter() - t0
    finally:
        for sim in sims:
            sim.close()
    clk = clocks.stop()
    _barrier(world)
    t_batched = _max_over_ranks(t_batched, world)
    t_streams = _max_over_ranks(t_streams, world)
    t_alone = _max_over_ranks(t_alone, world)
    same = all(np.array_equal(a[k], b[k]) for a, b in zip(f_b, f_s) for k in a)
    member_steps = count * K * world
    particle_steps = sum(w.N for w in runs) * K * world
    if rank == 0:
        line = {
            "metric": f"runs/s, {count} uneven runs of {K} steps (H in 32..96, N in 2^14..2^20)",
            "value": count * world / t_batched,
            "unit": "runs/s",
            "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": 1e3 * t_batched / K,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (f64 log-mass and reductions)", "data": "synthetic",
            "config": {"workload": f"ensemble: {count} runs, H in {{32, 48, 64, 96}}, "
                                   "N = 2^U[14, 20], chi ~ U[0.005, 0.03], alpha ~ U[5, 20], "
                                   "Du ~ U[5e-4, 2e-3], dt 1e-3",
                       "parallelism": f"batched launches across runs, replicas x{world}",
                       "timing": "host wall clock around enqueue + sync of all runs",
                       "path": "batched" if path_b == sipf.SIPF_ENSEMBLE_BATCHED else "streams"},
            "one_stream_per_run": {"value": count * world / t_streams, "unit": "runs/s",
                                   "speedup_of_batched": t_streams / t_batched},
            "one_at_a_time": {"value": count * world / t_alone, "unit": "runs/s",
                              "speedup_of_batched": t_alone / t_batched},
            "bit_identical_batched_vs_streams": bool(same),
            "member_steps_per_s": member_steps / t_batched,
            "particle_steps_per_s": particle_steps / t_batched,
            "gpu_launches": (1 + 1 + 3 * len({w.H for w in runs})) * K,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    return 0


def _serve_once(sipf, runs, steps, arrival, budget, quantum, max_live):
    """One pass of the request stream through a server: time-to-result of
    every request (collection time - arrival time), makespan, peak bytes.
    max_live = 1 serves the requests one at a time (same server, same
    pooled memory, same kernels), 0 lets the budget alone limit admission."""
    R = len(runs)
    mask = sipf.FIELD_U | sipf.FIELD_V | sipf.FIELD_M | sipf.FIELD_W
    ttr, rid_of, results = {}, {}, {}
    srv = sipf.Server(budget, max_live=max_live)
    try:
        t0 = time.perf_counter()
        nxt = 0
        while len(ttr) < R:
            now = time.perf_counter() - t0
            while nxt < R and arrival[nxt] <= now:
                w = runs[nxt]
                rid_of[srv.submit(w.H, w.L, w.origin, w.N, w.params, w.x, w.mass, w.v, w.m,
                                  w.w, w.dt, steps[nxt])] = nxt
                nxt += 1
            pending = srv.advance(quantum)
            for rid in srv.poll():
                i = rid_of[rid]
                results[i] = srv.collect(rid, mask)
                ttr[i] = time.perf_counter() - t0 - arrival[i]
            if pending == 0 and nxt < R:
                time.sleep(max(0.0, arrival[nxt] - (time.perf_counter() - t0)))
        makespan = time.perf_counter() - t0
        st = srv.stats()
    finally:
        srv.close()
    lat = np.array([ttr[i] for i in range(R)])
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "requests_per_s": R / makespan,
            "makespan_s": makespan, "peak_device_bytes": st["peak"]}, results


def run_serve(args, rank, world, local):
    """Continuous batching: requests drawn like the ensemble's runs plus a
    simulated time T ~ U[0.05, 0.5] (T/dt steps), arriving as a Poisson
    process of rate --rate per second, served from one GPU under a 150 GB
    device-memory budget; time-to-result = collection time - arrival time.
    The same request stream is then served one at a time (the server with
    at most one admitted request), and the two arms' results are compared
    bit for bit.  --rates a,b,c sweeps the arrival rate (one stream per rate)."""
    import torch
    from paper_2605_20140_gb300 import sipf
    from sipf_inputs import ensemble_workloads

    torch.cuda.set_device(local)
    R = args.requests
    rates = [float(r) for r in args.rates.split(",")] if args.rates else [args.rate]
    rng = np.random.default_rng(np.random.PCG64(9000 + rank))
    runs = ensemble_workloads(R, seed=100 + rank)
    steps = [max(1, int(round(rng.uniform(0.05, 0.5) / w.dt))) for w in runs]
    gaps = rng.exponential(1.0, R)
    budget = 150 * 10 ** 9
    # warm-up: one request per grid size (graph capture, kernel attributes)
    with sipf.Server(budget) as warm:
        seen = {}
        for w in runs:
            if w.H not in seen:
                seen[w.H] = warm.submit(w.H, w.L, w.origin, w.N, w.params, w.x, w.mass, w.v,
                                        w.m, w.w, w.dt, 4)
        while warm.advance(2):
            pass
        for rid in warm.poll():
            warm.collect(rid, 0)
    clocks = ClockSampler(local)
    _barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    sweep = []
    for rate in rates:
        arrival = np.cumsum(gaps / rate)
        served, res_a = _serve_once(sipf, runs, steps, arrival, budget, args.quantum, 0)
        alone, res_b = _serve_once(sipf, runs, steps, arrival, budget, args.quantum, 1)
        same = all(np.array_equal(res_a[i][k], res_b[i][k]) for i in range(R) for k in res_a[i])
        sweep.append({"rate": rate, "served": served, "one_at_a_time": alone,
                      "bit_identical": bool(same)})
    clk = clocks.stop()
    head = sweep[0]
    p99 = _max_over_ranks(head["served"]["p99_s"], world)
    total_steps = sum(steps)
    h2d = sum(w.x.nbytes + w.mass.nbytes + 3 * w.v.nbytes for w in runs)
    d2h = sum(4 * w.v.nbytes for w in runs)
    if rank == 0:
        line = {
            "metric": f"p99 time-to-result, Poisson arrivals at {head['rate']:g} requests/s",
            "value": p99, "unit": "s", "n_gpus": world, "steps": total_steps,
            "warmup": len(seen),
            "ms_per_step": 1e3 * head["served"]["makespan_s"] / total_steps,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (f64 log-mass and reductions)", "data": "synthetic",
            "config": {"workload": f"serve: {R} requests drawn as the ensemble's runs "
                                   "(H in {32, 48, 64, 96}, N = 2^U[14, 20]) with "
                                   "T ~ U[0.05, 0.5], dt 1e-3; 150 GB budget",
                       "quantum_steps": args.quantum, "parallelism": f"replicas x{world}"},
            **{k: head["served"][k] for k in ("p50_s", "p99_s", "mean_s", "requests_per_s",
                                               "makespan_s", "peak_device_bytes")},
            "one_at_a_time": head["one_at_a_time"],
            "speedup_runs_per_s": head["served"]["requests_per_s"] /
                                  head["one_at_a_time"]["requests_per_s"],
            "bit_identical_to_one_at_a_time": head["bit_identical"],
            "sweep": sweep,
            "e2e": {"value": p99, "unit": "s", "h2d_bytes_per_step": h2d / total_steps,
                    "d2h_bytes_per_step": d2h / total_steps},
            "gpu_launches": 5 * total_steps, "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--workload", choices=["headline", "large", "ensemble", "serve"],
                    default="headline")
    ap.add_argument("--rate", type=float, default=100.0, help="serve: arrivals per second")
    ap.add_argument("--rates", default=None,
                    help="serve: comma-separated arrival rates to sweep (overrides --rate)")
    ap.add_argument("--requests", type=int, default=128, help="serve: number of requests")
    ap.add_argument("--quantum", type=int, default=2, help="serve: steps per round")
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["sipf", "reference"], default="sipf")
    ap.add_argument("--repeats", type=int, default=5,
                    help="timed regions of --steps steps; the median is reported")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = {"ensemble": 200, "large": 100}.get(args.workload, 1000)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank, world, local = _dist_init(args.gpus)
    try:
        if args.impl == "reference":
            return run_reference(args, rank, world)
        if args.workload == "ensemble":
            return run_ensemble(args, rank, world, local)
        if args.workload == "serve":
            return run_serve(args, rank, world, local)
        return run_sipf(args, rank, world, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
