"""Autotuner of the step's launch choices.

For each target (grid size H, a particle-count class [N_min, N_max] and a
representative N), it times every candidate tuning (radix plan of the
spectral passes: two Stockham plans of the plane passes, or the per-axis
pipeline of lane-group transforms; particle-step blocks per SM; bucket
slack) on the GPU:
the seeded workload of that size is set up, the tuning applied, a few
warm-up steps taken, and `steps` steps timed with CUDA events on the
context's stream; the fastest candidate wins.  The choices are written as
the text table the library reads (sipf_tuning.txt next to libsipf.so, or
the file SIPF_TUNING names): one line per target,

    H  N_min  N_max  radix_plan  step_blocks_per_sm  bucket_slack_div  bucket_slack_add

    python -m paper_2605_20140_gb300.autotune [--out PATH] [--steps K]

Tuning changes speed only: slack and blocks per SM leave every result bit
for bit unchanged, the radix plans differ by float32 rounding (both are
checked against the FP64 oracle by the tests).
"""

from __future__ import annotations

import argparse
import itertools
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

RADIX_PLANS = (0, 1, 2)
WARP_PIPELINE_H = (64, 128, 256)             # grid sizes with radix plan 2
STEP_BLOCKS = (0, 4, 3)                      # 0: the occupancy limit
SLACKS = ((8, 32), (16, 16), (32, 8))        # (bucket_slack_div, bucket_slack_add)

# (H, N_min, N_max, representative N, workload recipe): the headline and
# large runs, and the ensemble's grid sizes in three particle-count classes
TARGETS = [(128, 1 << 21, 1 << 23, 1 << 22, "headline"),
           (256, 1 << 24, 1 << 26, 1 << 25, "large")]
for _H in (32, 48, 64, 96):
    for _lo, _hi, _rep in ((1 << 14, (1 << 16) - 1, 1 << 15), (1 << 16, (1 << 18) - 1, 1 << 17),
                           (1 << 18, 1 << 20, 1 << 19)):
        TARGETS.append((_H, _lo, _hi, _rep, "headline"))


def candidates(H=None):
    """Candidate tunings (for grid size H: without plan 2 where H has none)."""
    plans = [p for p in RADIX_PLANS if p != 2 or H is None or H in WARP_PIPELINE_H]
    return [dict(radix_plan=p, step_blocks_per_sm=b, bucket_slack_div=d, bucket_slack_add=a)
            for p, b, (d, a) in itertools.product(plans, STEP_BLOCKS, SLACKS)]


def time_candidate(sim, stream, wl, tuning, steps, warmup):
    """ms per step of `steps` steps after `warmup` (CUDA events on the
    context's stream `stream`, a torch stream)."""
    import torch
    from paper_2605_20140_gb300 import sipf
    sipf.sipf_set_tuning(sim.ctx, **tuning)
    sim.set_state(wl.x, wl.mass, wl.ids, wl.v, wl.m, wl.w)
    sim.step(wl.dt, warmup)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    sipf.sipf_sync(sim.ctx)
    e0.record(stream)
    sim.step(wl.dt, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    sipf.sipf_sync(sim.ctx)
    return e0.elapsed_time(e1) / steps


def tune_target(H, N, recipe, steps=20, warmup=4, log=None):
    """Best tuning for (H, N): (tuning dict, ms per step, all timings)."""
    import torch
    from paper_2605_20140_gb300 import sipf
    from sipf_inputs import workload
    wl = workload(recipe, H=H, N=N)
    stream = torch.cuda.Stream()
    with sipf.Simulation(wl.H, wl.L, wl.origin, wl.N, wl.params,
                         stream=stream.cuda_stream) as sim:
        timings = []
        for cand in candidates(H):
            ms = time_candidate(sim, stream, wl, cand, steps, warmup)
            timings.append((ms, cand))
            if log:
                log(f"H={H} N={N} {cand} {ms:.4f} ms/step")
    timings.sort(key=lambda x: x[0])
    return timings[0][1], timings[0][0], timings


def table_line(H, lo, hi, best, ms, ms_default):
    return (f"{H} {lo} {hi} {best['radix_plan']} {best['step_blocks_per_sm']} "
            f"{best['bucket_slack_div']} {best['bucket_slack_add']}"
            f"   # {ms:.4f} ({ms_default:.4f})\n")


def write_table(path, rows, keep=()):
    """Write the table: the lines of `rows`, and before them the lines of
    the existing file at `path` whose grid size is in `keep` (a partial
    run re-tunes some sizes and keeps the others)."""
    kept = []
    if keep and os.path.exists(path):
        for line in open(path):
            fields = line.split("#", 1)[0].split()
            if fields and int(fields[0]) in keep:
                kept.append(line if line.endswith("\n") else line + "\n")
    with open(path, "w") as f:
        f.write("# sipf tuning table, written by paper_2605_20140_gb300/autotune.py on "
                f"{time.strftime('%Y-%m-%d')}\n")
        f.write("# H  N_min  N_max  radix_plan  step_blocks_per_sm  bucket_slack_div  "
                "bucket_slack_add   # ms/step at the representative N (default tuning)\n")
        for line in kept:
            f.write(line)
        for row in rows:
            f.write(table_line(*row))


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    here = os.path.dirname(os.path.abspath(__file__))
    ap.add_argument("--out", default=os.path.join(here, "sipf_tuning.txt"))
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=4)
    ap.add_argument("--max-h", type=int, default=512, help="skip targets above this grid size")
    ap.add_argument("--only", type=str, default="",
                    help="comma-separated grid sizes to re-tune; the table keeps the other lines")
    args = ap.parse_args(argv)
    import torch
    from paper_2605_20140_gb300 import sipf
    if not torch.cuda.is_available():
        raise SystemExit("the autotuner times candidates on a CUDA GPU")
    sipf.load()
    sipf.sipf_tuning_load(None)           # tune from the defaults, not an older table
    rows = []
    default = dict(radix_plan=0, step_blocks_per_sm=0, bucket_slack_div=8, bucket_slack_add=32)
    only = {int(h) for h in args.only.split(",") if h}
    for H, lo, hi, rep, recipe in TARGETS:
        if H > args.max_h or (only and H not in only):
            continue
        best, ms, timings = tune_target(H, rep, recipe, args.steps, args.warmup, log=print)
        ms_default = next(t for t, c in timings if c == default)
        rows.append((H, lo, hi, best, ms, ms_default))
        print(f"H={H} N={rep}: {best} {ms:.4f} ms/step (default {ms_default:.4f})", flush=True)
    keep = {t[0] for t in TARGETS} - only if only else ()
    write_table(args.out, rows, keep)
    print(f"wrote {args.out}")


if __name__ == "__main__":
    main()
