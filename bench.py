"""Benchmark of the flow-map / FTLE hot path on one GB300 (per rank).

Workload (default): the 3D time-modulated ABC flow on a periodic 128^3 grid with
64 FP32 frames over [0, 8]; a 256^3 periodic seed lattice (16.7M tracers); RK4,
dt = 0.02, T = 8 (400 steps); grad F by finite differences, the full 3x3
Cauchy-Green tensor (FP64) and the FTLE field.  Synthetic seeded data.

A timed step = lcs_advect + lcs_ftle (FTLE and C written to device memory) with
the field and the seed lattice resident.  `e2e` adds, every step, the upload of
the frames from pinned host memory (lcs_update_frames into a ring of fields, from
a loader thread with its own context and stream) and the read-back of C and the
FTLE into pinned host memory, each overlapping other steps' advection as a
serving loop would run them.

The default line also carries `other_configs`: the bench lines of the other
workloads (c3, c4, tri, c5, next; 3 timed steps each, no CPU baseline), each run
as a child process after the default workload's measurement.

`--impl reference` times the FP64 CPU oracle on a bounded sample of the same
workload on the host cores (the baseline arm).  Under torchrun every rank runs
its own independent copy of the workload (weak scaling, no data exchange);
`value` is the total over ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FTLE seeds/s & tracer-steps/s on 1 GB300; surrogate/mixed vs plain at stated err"
WORKLOAD = ("3D time-modulated ABC flow, periodic 128^3 FP32 velocity grid, 64 frames on [0,8]; "
            "256^3 seed grid (16.7M tracers); RK4 dt=0.02, T=8 (400 steps); FD grad F, 3x3 Cauchy-Green "
            "(FP64) and FTLE")
L = 2 * math.pi
N_SIDE, N_GRID, N_FRAMES, T_END, DT = 256, 128, 64, 8.0, 0.02
# fields the end-to-end leg keeps in flight (uploads run up to E2E_FIELDS - 1 steps ahead)
E2E_FIELDS = 3
NSTEPS = int(round(T_END / DT))
# algorithmic FP32 work of one RK4 tracer-step on trilinear, linear-in-time data (the per-unit figure
# of the measurement plan): per stage evaluation 7 lerps x 3 components x 2 frames = 84, the time
# blend 6 and the weights ~10, about 100; 4 evaluations + ~40 for the RK4 stage points and update = 440
FLOP_PER_TRACER_STEP = 440
# DRAM read + write bytes per tracer-step of the episode kernel, from the ncu capture of the small case
# with the same tracer density (profiles/ep_advect3_traffic.md)
TRAFFIC_BYTES_PER_TRACER_STEP = 23.2


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16"])
    p.add_argument("--e2e-steps", type=int, default=6,
                   help="steps of the end-to-end leg from host buffers (0 = none)")
    p.add_argument("--storage-passes", type=int, default=3,
                   help="c2 with f32: steps of the FP32/FP16/BF16 storage passes after the timed region (0 = none)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--seeds-side", type=int, default=N_SIDE,
                   help="seed lattice side (default 256; smaller only for profiling captures)")
    p.add_argument("--config", default="c2", choices=["c2", "c3", "c3x", "c4", "c5", "tri", "next", "peaks"],
                   help="c2: the 3D ABC workload (default, the headline); c3: the batched sliding-window "
                        "workload; c3x: its full cross product of horizons from multi-horizon snapshots; "
                        "c4: adaptive DP5(4) on the tetrahedral pipe; c5: the learned surrogate; tri: RK4 on "
                        "the triangulated stenosis; next: the eigenvectors, early Cauchy-Green, auxiliary-point "
                        "and variational passes; peaks: plain-loop FMA and read rates")
    p.add_argument("--train-epochs", type=int, default=4, help="c5: training epochs over the 50M samples")
    p.add_argument("--c5-side", type=int, default=16384,
                   help="c5: seed lattice side along x (y is half; default 16384, smaller only for profiling)")
    p.add_argument("--grid", type=int, default=N_GRID,
                   help="velocity grid side (default 128; smaller only for profiling captures)")
    p.add_argument("--tri-side", type=int, default=TRI_N[0],
                   help="tri: seed lattice side along x (y is a quarter; default 4096, smaller only for profiling)")
    p.add_argument("--c4-nz", type=int, default=C4_N[2],
                   help="c4: seed lattice size along the pipe axis (default 512, smaller only for profiling)")
    p.add_argument("--no-other-configs", dest="other_configs", action="store_false",
                   help="c2: skip the other workloads (c3, c4, tri, c5, next) that the default line summarises")
    p.add_argument("--c3-t0s", type=int, default=32,
                   help="c3: t0 values per direction (default 32, i.e. 64 jobs; fewer only for profiling)")
    p.add_argument("--mesh-T", type=float, default=None,
                   help="c4 / tri: integration time (default the workload's T = 1; shorter only for profiling "
                        "captures, which keeps the seed density and the caches' behaviour)")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples (every 200 ms) while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.out = tempfile.TemporaryFile(mode="w+")

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()

    def summary(self):
        self.out.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------- reference arm

def oracle_sample_run(g, side, threads=0, want_ftle=False):
    """Oracle FTLE on a side^3 block of the 256^3 lattice (its stencils included); returns (seeds, s,
    threads, tracers integrated), and with want_ftle also (lattice ids of the block's seeds, their FTLE)."""
    import oracle

    oracle.build()
    nthreads = oracle.set_threads(threads)
    n = (N_SIDE, N_SIDE, N_SIDE)
    h = L / N_SIDE
    # block of side^3 seeds at the lattice origin plus a 2-seed halo (stencil neighbours, periodic): a
    # halo seed across the wrap starts at its lattice seed's FP32 position minus the period, as the
    # library's differences shift it, so the block's central differences are the lattice's
    idx = np.arange(-2, side + 2)
    xs = (idx % N_SIDE * h).astype(np.float32).astype(np.float64) - np.where(idx < 0, L, 0.0)
    Z, Y, X = np.meshgrid(xs, xs, xs, indexing="ij")
    x0 = np.stack([X.ravel(), Y.ravel(), Z.ravel()])
    F = oracle.RectField(g.frames, g.times, g.origin, g.spacing, g.periodic)
    t = time.perf_counter()
    xT, st, _ = oracle.rk4(F, x0, 0.0, T_END, DT)
    m = side + 4
    # the halo block is a non-periodic lattice of its own; FTLE of its interior side^3 seeds
    G = oracle.flowmap_gradient(3, (m, m, m), (h, h, h), (0, 0, 0), (0, 0, 0), xT, st)
    C = oracle.cauchy_green(G)
    lam, sig = oracle.ftle(C, 3, T_END)
    dt = time.perf_counter() - t
    if not want_ftle:
        return side ** 3, dt, nthreads, x0.shape[1]
    # interior seeds (i, j, k) in [0, side)^3 of the halo block: their central differences are those of
    # the full periodic lattice
    b = np.arange(2, side + 2)
    K, J, I = np.meshgrid(b, b, b, indexing="ij")
    inner = (I + m * (J + m * K)).ravel()
    i0 = np.arange(side)
    K0, J0, I0 = np.meshgrid(i0, i0, i0, indexing="ij")
    ids = (I0 + N_SIDE * (J0 + N_SIDE * K0)).ravel()
    return side ** 3, dt, nthreads, x0.shape[1], ids, sig[inner]


def reference_arm(args, rank, world):
    if rank != 0:
        return
    from paper_2209_13775_gb300 import inputs

    g = inputs.abc(n=N_GRID, nframes=N_FRAMES, t_end=T_END)
    # calibrate: a small block first, then one sized for about 5 s per step
    s_small, dt_small, _, _ = oracle_sample_run(g, 4)
    per_seed = dt_small / ((4 + 4) ** 3)
    side = int(max(4, min(72, (5.0 / max(per_seed, 1e-9)) ** (1 / 3) - 4)))
    if args.warmup > 0:
        oracle_sample_run(g, 4)
    times = []
    for _ in range(args.steps):
        s, dt, nth, integrated = oracle_sample_run(g, side)
        times.append(dt)
    tmean = sum(times) / len(times)
    value = s / tmean            # FTLE seeds/s of the sample (halo integration included in the time)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "seeds/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tmean * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": "%d^3-seed block (+2-seed halo, %d integrated)" % (side, integrated)},
        "tracer_steps_per_s": value * NSTEPS,
        "cpu_baseline": {"value": value, "unit": "seeds/s", "cores": nth, "kind": "oracle",
                         "sample": "%d^3 seeds of the 256^3 lattice with their stencil halo, all 400 steps" % side},
        "e2e": {"value": value, "unit": "seeds/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm

def max_over_ranks(x, world, device="cuda"):
    """MAX of a per-rank float over all ranks (the timing rule: the slowest rank sets the time);
    the value itself for one rank."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def our_arm(args, rank, world, local):
    import torch

    from paper_2209_13775_gb300 import inputs, lcs

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    storage = {"f32": lcs.F32, "f16": lcs.F16, "bf16": lcs.BF16}[args.storage]
    stream = torch.cuda.current_stream()
    ctx = lcs.lcs_create(local, stream)
    g = inputs.abc(n=args.grid, nframes=N_FRAMES, t_end=T_END)
    desc = lcs.field_desc(3, g.n, g.origin, g.spacing, g.periodic, g.times, storage=storage)
    frames_dev = torch.from_numpy(g.frames).cuda()
    field = lcs.lcs_load_field(ctx, desc, frames_dev)
    sd = lcs.seed_desc(3, (args.seeds_side,) * 3, (0.0,) * 3, (L,) * 3, (1, 1, 1))
    seeds = lcs.lcs_seed_grid(ctx, sd)
    N = lcs.lcs_seeds_count(seeds)
    fm = lcs.lcs_flowmap_create(ctx, seeds, 1)
    opts = lcs.advect_opts(lcs.RK4, t0=0.0, T=T_END, dt=DT)
    ftle = torch.empty(N, dtype=torch.float32, device="cuda")
    C = torch.empty((N, 6), dtype=torch.float64, device="cuda")
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def step(rec=None):
        if rec is not None:
            rec[0].record(stream)
        lcs.lcs_advect(ctx, field, seeds, opts, fm)
        if rec is not None:
            rec[1].record(stream)
        lcs.lcs_ftle(ctx, fm, 0, ftle, None, C)

    for _ in range(args.warmup):
        step()
    lcs.lcs_synchronize(ctx)

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()
        torch.cuda.synchronize()

    adv_events = [(ev(), ev()) for _ in range(args.steps)]
    t_start, t_stop = ev(), ev()
    for ph in range(4):
        lcs.lcs_timing_read(ctx, ph)            # drop anything recorded before
    lcs.lcs_timing_enable(ctx, True)
    with ClockSampler(local) as clk:
        barrier()
        t_start.record(stream)
        for k in range(args.steps):
            step(adv_events[k])
        t_stop.record(stream)
        barrier()
    lcs.lcs_synchronize(ctx)
    phase = {name: lcs.lcs_timing_read(ctx, ph) for ph, name in
             enumerate(("advect", "rebundle", "slices", "cg_ftle"))}
    lcs.lcs_timing_enable(ctx, False)
    elapsed = max_over_ranks(t_start.elapsed_time(t_stop) / 1e3, world)
    adv_ms = [a.elapsed_time(b) for a, b in adv_events]
    ms_per_step = elapsed / args.steps * 1e3
    value = world * N * args.steps / elapsed
    clocks = clk.summary()

    # end to end through the C ABI from host buffers, pipelined as a serving loop runs it: every
    # step uploads its 1.61 GB of frames from pinned memory and reads C and the FTLE back into
    # pinned memory.  A loader thread with its own context and stream uploads frames
    # (lcs_update_frames) into a ring of E2E_FIELDS fields, up to E2E_FIELDS - 1 steps ahead of the
    # advection, each upload waiting for the step that last read its field; read-backs run on a
    # third stream behind each step's lcs_ftle (double-buffered device outputs, the next use of a
    # buffer waiting for its read-back).  The first upload and the last read-back are not hidden and
    # are counted; the fields, the lattice (made on the device from its descriptor), the flow map
    # and the output buffers are allocated before timing.
    frames_pin = torch.from_numpy(g.frames).pin_memory()
    load_stream = torch.cuda.Stream(device=local)
    d2h_stream = torch.cuda.Stream(device=local)
    ctx_load = lcs.lcs_create(local, load_stream)
    nf = E2E_FIELDS if args.e2e_steps > 0 else 0
    fbuf = [lcs.lcs_load_field(ctx_load, desc, frames_pin) for _ in range(nf)]
    no = 2 if nf else 0
    ftle_d = [torch.empty(N, dtype=torch.float32, device="cuda") for _ in range(no)]
    C_d = [torch.empty((N, 6), dtype=torch.float64, device="cuda") for _ in range(no)]
    ftle_h = [torch.empty(N, dtype=torch.float32).pin_memory() for _ in range(no)]
    C_h = [torch.empty((N, 6), dtype=torch.float64).pin_memory() for _ in range(no)]
    s_e = lcs.lcs_seed_grid(ctx, sd) if nf else None
    m_e = lcs.lcs_flowmap_create(ctx, s_e, 1) if nf else None
    up_ms = []   # host time of each upload of the timed run (lcs_update_frames returns once it is complete)

    def e2e_run(k_steps):
        ready = [threading.Event() for _ in range(k_steps)]
        used = [torch.cuda.Event() for _ in range(k_steps)]      # after step k's lcs_ftle
        used_rec = [threading.Event() for _ in range(k_steps)]   # used[k] has been recorded
        err = []
        up_ms.clear()

        def loader():
            try:
                torch.cuda.set_device(local)
                for k in range(k_steps):
                    if k >= nf:   # the field's previous reader, step k - nf, must be done with it
                        used_rec[k - nf].wait()
                        used[k - nf].synchronize()
                    t = time.perf_counter()
                    lcs.lcs_update_frames(ctx_load, fbuf[k % nf], frames_pin)
                    up_ms.append(round((time.perf_counter() - t) * 1e3, 1))
                    ready[k].set()
            except BaseException as e:   # surfaced by the main thread
                err.append(e)
                for r in ready:
                    r.set()

        th = threading.Thread(target=loader, daemon=True)
        th.start()
        copied = [None] * no   # read-back of the step that last wrote each output buffer
        for k in range(k_steps):
            ready[k].wait()
            if err:
                break
            b = k % no
            if copied[b] is not None:
                stream.wait_event(copied[b])
            lcs.lcs_advect(ctx, fbuf[k % nf], s_e, opts, m_e)
            lcs.lcs_ftle(ctx, m_e, 0, ftle_d[b], None, C_d[b])
            used[k].record(stream)
            used_rec[k].set()
            with torch.cuda.stream(d2h_stream):
                d2h_stream.wait_event(used[k])
                ftle_h[b].copy_(ftle_d[b], non_blocking=True)
                C_h[b].copy_(C_d[b], non_blocking=True)
                copied[b] = torch.cuda.Event()
                copied[b].record(d2h_stream)
        if err:   # let the loader see every step as recorded so that it ends
            for r in used_rec:
                r.set()
        th.join()
        torch.cuda.synchronize()
        if err:
            raise err[0]

    e2e_t = []
    if args.e2e_steps > 0:
        e2e_run(3)                          # warm-up of the allocator, copy and thread paths
        barrier()
        t0 = time.perf_counter()
        e2e_run(args.e2e_steps)
        barrier()
        e2e_t.append((time.perf_counter() - t0) / args.e2e_steps)
    for fb in fbuf:
        lcs.lcs_free_field(fb)
    if nf:
        lcs.lcs_free_flowmap(m_e)
        lcs.lcs_free_seeds(s_e)
    lcs.lcs_destroy(ctx_load)
    e2e_el = max_over_ranks(sum(e2e_t) / len(e2e_t) if e2e_t else float("nan"), world)
    h2d = g.frames.nbytes
    d2h = N * 4 + N * 6 * 8     # FTLE (FP32) and C (6 FP64 entries) per seed

    pk, pk_kind = peaks()
    # dominant kernel: the RK4 advection launches (episodes of the re-bundled path); their summed
    # event time over the timed steps, divided by their count, is the average launch duration
    adv_ms_total, adv_launches = phase["advect"]
    adv_launch_s = adv_ms_total / max(adv_launches, 1) / 1e3
    steps_per_launch = NSTEPS * args.steps / max(adv_launches, 1)
    flops = float(N) * steps_per_launch * FLOP_PER_TRACER_STEP
    sm_mhz = pk.get("sm_max_mhz", 2070.0)
    fp32_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12          # TFLOP/s at the maximum SM clock
    achieved = flops / adv_launch_s / 1e12
    # DRAM traffic per launch: the small case's bytes per tracer-step (ncu, 64^3 field, 128^3 seeds, the
    # same 8 tracers per cell) times the tracer-steps of this launch (profiles/ep_advect3_traffic.md)
    traffic = TRAFFIC_BYTES_PER_TRACER_STEP * N * steps_per_launch if args.storage == "f32" else None
    n_ep = adv_launches / max(args.steps, 1)
    line = {
        "metric": METRIC, "value": value, "unit": "seeds/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"f32": "f32", "f16": "f32 (f16 storage)", "bf16": "f32 (bf16 storage)"}[args.storage],
        "data": "synthetic",
        "config": {"workload": WORKLOAD if (args.seeds_side, args.grid) == (N_SIDE, N_GRID) else
                   WORKLOAD.replace("256^3 seed grid (16.7M tracers)", "%d^3 seed grid" % args.seeds_side)
                   .replace("128^3 FP32 velocity grid", "%d^3 FP32 velocity grid" % args.grid),
                   "seeds": N, "steps_per_tracer": NSTEPS, "storage": args.storage,
                   "parallelism": "independent replica per GPU" if world > 1 else "single GPU",
                   "l2": "no flush needed: each step writes 872 MB of outputs (C + FTLE) > 129 MB L2"},
        "tracer_steps_per_s": value * NSTEPS,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": achieved / fp32_peak, "traffic": traffic,
                     "kernel": "ep_advect3_kernel (RK4 episode of %d steps)" % round(steps_per_launch),
                     "flop_per_launch": flops, "avg_launch_ms": adv_launch_s * 1e3, "launches": adv_launches,
                     "peak_basis": "152 SMs x 128 FP32 lanes x 2 x %.0f MHz (%s sm_max_mhz)" % (sm_mhz, pk_kind),
                     "traffic_note": "ncu DRAM bytes per tracer-step of the small case (64^3 field, 128^3 "
                                     "seeds) scaled by this launch's tracer-steps "
                                     "(profiles/ep_advect3_traffic.md)",
                     "limiter": "the L1 data stage (ncu, small case: 79% of its one-wavefront-per-cycle peak; "
                                "7.7 wavefronts per 16-byte gather request against 4 when a quarter warp's "
                                "lanes read at most 4 lines: the re-bundled tracers spread over 5-8 rows of "
                                "cells within a few steps); issue 69%, 470 instructions per warp-step"},
        "phases_ms_per_step": {k: v[0] / args.steps for k, v in phase.items()},
        "clocks": clocks,
        "e2e": {"value": world * N / e2e_el if e2e_t else None, "unit": "seeds/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_el * 1e3,
                "upload_call_ms": list(up_ms), "fields_in_flight": E2E_FIELDS,
                "note": "upload_call_ms: host time of each lcs_update_frames of the timed run, issued by a "
                        "loader thread up to %d steps ahead of the advection" % (E2E_FIELDS - 1)},
        # ours per step: schedule, init, finalize, FD/CG/FTLE, and per episode 3 scan + permutation +
        # gather + slice table + slice fill + advection
        "gpu_launches": int(round(args.steps * 4 + adv_launches * 8)),
    }
    if args.storage != "f32":
        # reduced-precision storage against FP32 storage on the same lattice (outside the timed region)
        d32 = lcs.field_desc(3, g.n, g.origin, g.spacing, g.periodic, g.times, storage=lcs.F32)
        f32 = lcs.lcs_load_field(ctx, d32, frames_dev)
        ftle32 = torch.empty(N, dtype=torch.float32, device="cuda")
        lcs.lcs_advect(ctx, f32, seeds, opts, fm)
        lcs.lcs_ftle(ctx, fm, 0, ftle32)
        lcs.lcs_advect(ctx, field, seeds, opts, fm)
        lcs.lcs_ftle(ctx, fm, 0, ftle)
        lcs.lcs_synchronize(ctx)
        lcs.lcs_free_field(f32)
        a, b = ftle.cpu().double().numpy(), ftle32.cpu().double().numpy()
        ok = np.isfinite(a) & np.isfinite(b)
        dd = np.abs(a[ok] - b[ok])
        line["ftle_err_vs_f32_storage"] = {"median": float(np.median(dd)), "p99.9": float(np.quantile(dd, 0.999)),
                                           "max": float(dd.max()), "ftle_range": [float(b[ok].min()),
                                                                                  float(b[ok].max())]}
    # the same workload with FP32, FP16 and BF16 velocity storage (FP32 tracers and arithmetic),
    # outside the timed region: step time, and the FTLE of every pass kept for its error below
    passes, pass_ftle = {}, {}
    if args.storage_passes > 0 and args.storage == "f32":
        for name, st in (("f32", lcs.F32), ("f16", lcs.F16), ("bf16", lcs.BF16)):
            dsc = lcs.field_desc(3, g.n, g.origin, g.spacing, g.periodic, g.times, storage=st)
            fp = lcs.lcs_load_field(ctx, dsc, frames_dev)
            fo = torch.empty(N, dtype=torch.float32, device="cuda")
            lcs.lcs_advect(ctx, fp, seeds, opts, fm)
            lcs.lcs_ftle(ctx, fm, 0, fo)
            a, b = ev(), ev()
            torch.cuda.synchronize()
            a.record(stream)
            for _ in range(args.storage_passes):
                lcs.lcs_advect(ctx, fp, seeds, opts, fm)
                lcs.lcs_ftle(ctx, fm, 0, fo)
            b.record(stream)
            lcs.lcs_synchronize(ctx)
            ms = a.elapsed_time(b) / args.storage_passes
            passes[name] = {"ms_per_step": ms, "seeds_per_s": N / (ms / 1e3),
                            "field_bytes": int(g.frames.nbytes // (1 if st == lcs.F32 else 2))}
            pass_ftle[name] = fo
            lcs.lcs_free_field(fp)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        _, dts, _, _ = oracle_sample_run(g, 4)                 # calibration: 8^3 tracers
        side = int(max(4, min(96, (10.0 / max(dts / 512.0, 1e-9)) ** (1 / 3) - 4)))
        s, dt, nth, integrated, ids, sig = oracle_sample_run(g, side, want_ftle=True)
        line["cpu_baseline"] = {"value": s / dt, "unit": "seeds/s", "cores": nth, "kind": "oracle",
                                "sample": "%d^3-seed block of the 256^3 lattice with its 2-seed stencil halo "
                                          "(%d tracers integrated, 400 steps each), FD/CG/FTLE; %.1f s"
                                          % (side, integrated, dt)}
        # FTLE error of each storage pass against the FP64 oracle (on the FP32-sampled field) at the
        # baseline's seeds
        idt = torch.from_numpy(ids).cuda()
        for name, fo in pass_ftle.items():
            got = fo[idt].cpu().double().numpy()
            ok = np.isfinite(got) & np.isfinite(sig)
            d = np.abs(got[ok] - sig[ok])
            passes[name]["ftle_err_vs_oracle"] = {"median": float(np.median(d)), "p99.9": float(np.quantile(d, 0.999)),
                                                  "max": float(d.max()), "seeds": int(ok.sum())}
    if passes:
        line["storage_passes"] = passes
        line["storage_passes_note"] = ("the default workload with each velocity storage type, %d untimed-region "
                                       "steps each after one warm-up (CUDA events); FTLE error against the FP64 "
                                       "oracle on the FP32-sampled frames at the cpu_baseline block's seeds"
                                       % args.storage_passes)
    lcs.lcs_free_flowmap(fm)
    lcs.lcs_free_seeds(seeds)
    lcs.lcs_free_field(field)
    lcs.lcs_destroy(ctx)
    if rank == 0 and world == 1 and args.other_configs and (args.seeds_side, args.grid) == (N_SIDE, N_GRID):
        line["other_configs"] = other_configs()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


# ------------------------------------------------ the other workloads in the default line

OTHER_CONFIGS = ("c3", "c4", "tri", "c5", "next")
OTHER_KEYS = ("value", "unit", "ms_per_step", "tracer_steps_per_s", "roofline", "clocks", "phases_ms",
              "phases_ms_per_step", "surrogate", "passes", "gpu_launches")


def other_configs(timeout_s=300):
    """Each other workload's own bench line (3 timed steps after 3 warm-up steps, no CPU baseline), run
    as a child process after the default workload's measurement, summarised by its workload and
    measured keys; a child that fails or runs out of time is recorded as such."""
    out = {}
    for cfg in OTHER_CONFIGS:
        cmd = [sys.executable, os.path.abspath(__file__), "--config", cfg, "--steps", "3", "--warmup", "3",
               "--no-cpu-baseline"]
        t0 = time.perf_counter()
        try:
            r = subprocess.run(cmd, capture_output=True, text=True, timeout=timeout_s)
            lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
            if r.returncode != 0 or not lines:
                rec = {"error": "exit %d: %s" % (r.returncode, (r.stderr.strip().splitlines() or [""])[-1][:300])}
            else:
                d = json.loads(lines[-1])
                rec = {"workload": d.get("config", {}).get("workload")}
                rec.update({k: d[k] for k in OTHER_KEYS if k in d})
        except subprocess.TimeoutExpired:
            rec = {"error": "timed out after %d s" % timeout_s}
        except ValueError as e:   # a line that is not JSON
            rec = {"error": "unreadable line: %s" % str(e)[:200]}
        rec["wall_s"] = round(time.perf_counter() - t0, 1)
        out[cfg] = rec
    return out


# ------------------------------------------------ batched sliding-window arm

C3_WORKLOAD = ("batched sliding-window FTLE on the double gyre (129x65 FP32, 101 frames): 32 t0 spaced 0.25, "
               "forward and backward, T in {2,4,8} (64 jobs), 2048x1024 seeds each (2^21), RK4 dt=0.05; "
               "one persistent launch in a CUDA graph with autotuned block/tile; FP64 FD + eigenvalue + FTLE")
# algorithmic FP32 work of one RK4 tracer-step on bilinear, linear-in-time data (the per-unit figure of
# the measurement plan): per evaluation bilinear 24 + time 4 + weights ~6 = 34; 4 evaluations + ~28 for
# the RK4 combination = 164
FLOP_PER_TRACER_STEP_2D = 164


def c3_arm(args, rank, world, local):
    import torch

    from paper_2209_13775_gb300 import inputs, lcs

    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    ctx = lcs.lcs_create(local, stream)
    g = inputs.double_gyre()
    field = lcs.lcs_load_field(ctx, lcs.field_desc(2, g.n, g.origin, g.spacing, g.periodic, g.times,
                                                   g.time_periodic, g.period), g.frames)
    sd = lcs.seed_desc(2, (2048, 1024), (0.0, 0.0), (2.0, 1.0))
    seeds = lcs.lcs_seed_grid(ctx, sd)
    N = lcs.lcs_seeds_count(seeds)
    nt = args.c3_t0s
    t0s = [0.25 * k for k in range(nt)] * 2
    Ts = [(2.0, 4.0, 8.0)[k % 3] for k in range(nt)] + [-(2.0, 4.0, 8.0)[k % 3] for k in range(nt)]
    nj = len(t0s)
    tracer_steps = N * sum(int(round(abs(T) / 0.05)) for T in Ts)
    fm = lcs.lcs_flowmap_create(ctx, seeds, nj)
    opts = lcs.advect_opts(lcs.RK4, dt=0.05, job_t0=t0s, job_T=Ts, use_graph=True)
    cache = os.path.join(tempfile.gettempdir(), "lcs_tune_%d.txt" % os.getpid())
    lcs.lcs_autotune(ctx, field, seeds, opts, cache)
    ftle = torch.empty((nj, N), dtype=torch.float32, device="cuda")
    lam = torch.empty((nj, N), dtype=torch.float64, device="cuda")

    def step():
        lcs.lcs_advect(ctx, field, seeds, opts, fm)
        lcs.lcs_ftle(ctx, fm, -1, ftle, lam)

    for _ in range(args.warmup):
        step()
    lcs.lcs_synchronize(ctx)
    for ph in range(4):
        lcs.lcs_timing_read(ctx, ph)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(args.steps):
            step()
        b.record(stream)
        torch.cuda.synchronize()
    el = a.elapsed_time(b) / 1e3
    # kernel-only time of the advection launches: one untimed-graph pass with phase events
    lcs.lcs_timing_enable(ctx, True)
    o2 = lcs.advect_opts(lcs.RK4, dt=0.05, job_t0=t0s, job_T=Ts, variant=opts.variant,
                         block_threads=opts.block_threads, tracers_per_thread=opts.tracers_per_thread)
    lcs.lcs_advect(ctx, field, seeds, o2, fm)
    lcs.lcs_ftle(ctx, fm, -1, ftle, lam)
    lcs.lcs_synchronize(ctx)
    adv_ms, adv_n = lcs.lcs_timing_read(ctx, 0)
    cg_ms, _ = lcs.lcs_timing_read(ctx, 3)
    lcs.lcs_timing_enable(ctx, False)
    pk, pk_kind = peaks()
    sm_mhz = pk.get("sm_max_mhz", 2070.0)
    fp32_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
    flops = float(tracer_steps) * FLOP_PER_TRACER_STEP_2D
    achieved = flops / (adv_ms / 1e3) / 1e12
    line = {
        "metric": METRIC, "value": nj * N * args.steps / el, "unit": "seeds/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": C3_WORKLOAD, "jobs": nj, "seeds_per_job": N, "tracer_steps": tracer_steps,
                   "tuned": {"variant": opts.variant, "block_threads": opts.block_threads,
                             "tracers_per_thread": opts.tracers_per_thread}},
        "tracer_steps_per_s": tracer_steps * args.steps / el,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": achieved / fp32_peak, "traffic": None,
                     "kernel": {1: "rk4_gather_kernel", 2: "rk4_ring2d_kernel", 4: "rk4_ring2d_kernel (persistent)",
                                5: "rk4_slice2d_kernel (with slice2d_fill_kernel)"}.get(opts.variant, "?")
                               + " (variant %d)" % opts.variant, "flop_per_launch": flops,
                     "avg_launch_ms": adv_ms / max(adv_n, 1), "launches": adv_n,
                     "peak_basis": "152 SMs x 128 FP32 lanes x 2 x %.0f MHz (%s sm_max_mhz)" % (sm_mhz, pk_kind)},
        "phases_ms": {"advect": adv_ms, "cg_ftle": cg_ms},
        "clocks": clk.summary(),
    }
    lcs.lcs_free_flowmap(fm)
    lcs.lcs_free_seeds(seeds)
    lcs.lcs_free_field(field)
    lcs.lcs_destroy(ctx)
    try:
        os.remove(cache)
    except OSError:
        pass
    print(json.dumps(line), flush=True)


# ------------------------------------- sliding windows, every horizon, snapshots

C3X_WORKLOAD = ("sliding-window FTLE on the double gyre (129x65 FP32, 101 frames): 32 t0 spaced 0.25, forward and "
                "backward, every horizon T in {2,4,8} (192 FTLE fields), 2048x1024 seeds each (2^21), RK4 dt=0.05; "
                "one T=8 integration per (t0, direction) with snapshots at |T| = 2 and 4; FP64 FD + eigenvalue + FTLE")


def c3x_arm(args, rank, world, local):
    """The C3 field and lattice with the full cross product of horizons: 64 integrations of |T| = 8 whose
    snapshots at |T| = 2 and 4 give the other 128 flow maps, against 192 separate integrations."""
    import torch

    from paper_2209_13775_gb300 import inputs, lcs

    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    ctx = lcs.lcs_create(local, stream)
    g = inputs.double_gyre()
    field = lcs.lcs_load_field(ctx, lcs.field_desc(2, g.n, g.origin, g.spacing, g.periodic, g.times,
                                                   g.time_periodic, g.period), g.frames)
    seeds = lcs.lcs_seed_grid(ctx, lcs.seed_desc(2, (2048, 1024), (0.0, 0.0), (2.0, 1.0)))
    N = lcs.lcs_seeds_count(seeds)
    t0s = [0.25 * k for k in range(32)] * 2
    Ts = [8.0] * 32 + [-8.0] * 32
    nj, snaps = len(t0s), [2.0, 4.0]
    nslot = nj * (1 + len(snaps))
    fm = lcs.lcs_flowmap_create(ctx, seeds, nslot)
    cache = os.path.join(tempfile.gettempdir(), "lcs_tune_x_%d.txt" % os.getpid())
    opts = lcs.advect_opts(lcs.RK4, dt=0.05, job_t0=t0s, job_T=Ts, snap_T=snaps)
    lcs.lcs_autotune(ctx, field, seeds, opts, cache)
    opts = lcs.advect_opts(lcs.RK4, dt=0.05, job_t0=t0s, job_T=Ts, snap_T=snaps, variant=opts.variant,
                           block_threads=opts.block_threads, tracers_per_thread=opts.tracers_per_thread,
                           use_graph=True)
    ftle = torch.empty((nslot, N), dtype=torch.float32, device="cuda")

    def step():
        lcs.lcs_advect(ctx, field, seeds, opts, fm)
        lcs.lcs_ftle(ctx, fm, -1, ftle)

    for _ in range(args.warmup):
        step()
    lcs.lcs_synchronize(ctx)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(args.steps):
            step()
        b.record(stream)
        torch.cuda.synchronize()
    el = a.elapsed_time(b) / 1e3
    tracer_steps = N * nj * 160
    # the same 192 FTLE fields as 192 separate integrations (one warm-up, one timed)
    Ta = [sgn * h for sgn in (1.0, -1.0) for _ in range(32) for h in (2.0, 4.0, 8.0)]
    t0a = [0.25 * k for k in range(32) for _ in range(3)] * 2
    fm2 = lcs.lcs_flowmap_create(ctx, seeds, len(t0a))
    o2 = lcs.advect_opts(lcs.RK4, dt=0.05, job_t0=t0a, job_T=Ta, variant=opts.variant,
                         block_threads=opts.block_threads, tracers_per_thread=opts.tracers_per_thread)
    ftle2 = torch.empty((len(t0a), N), dtype=torch.float32, device="cuda")
    lcs.lcs_advect(ctx, field, seeds, o2, fm2)
    lcs.lcs_ftle(ctx, fm2, -1, ftle2)
    torch.cuda.synchronize()
    a.record(stream)
    lcs.lcs_advect(ctx, field, seeds, o2, fm2)
    lcs.lcs_ftle(ctx, fm2, -1, ftle2)
    b.record(stream)
    torch.cuda.synchronize()
    el2 = a.elapsed_time(b) / 1e3
    # the snapshot fields are the separate runs' fields bit for bit (slot order differs)
    same = True
    for j in range(nj):
        sgn = 1.0 if Ts[j] > 0 else -1.0
        k = j % 32
        base = (0 if sgn > 0 else 96) + 3 * k
        pairs = [(j, base + 2), (nj + 2 * j, base), (nj + 2 * j + 1, base + 1)]
        for p, q in pairs:
            same = same and bool(torch.equal(ftle[p].nan_to_num(-7.0), ftle2[q].nan_to_num(-7.0)))
    line = {
        "metric": METRIC, "value": nslot * N * args.steps / el, "unit": "seeds/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": C3X_WORKLOAD, "integrations": nj, "ftle_fields": nslot, "seeds_per_field": N,
                   "tracer_steps": tracer_steps,
                   "tuned": {"variant": opts.variant, "block_threads": opts.block_threads,
                             "tracers_per_thread": opts.tracers_per_thread}},
        "tracer_steps_per_s": tracer_steps * args.steps / el,
        "separate_runs": {"ms_per_step": el2 * 1e3, "seeds_per_s": nslot * N / el2,
                          "tracer_steps": N * sum(int(round(abs(T) / 0.05)) for T in Ta),
                          "snapshot_speedup": el2 / (el / args.steps), "bit_identical_ftle": same},
        "clocks": clk.summary(),
    }
    lcs.lcs_free_flowmap(fm2)
    lcs.lcs_free_flowmap(fm)
    lcs.lcs_free_seeds(seeds)
    lcs.lcs_free_field(field)
    lcs.lcs_destroy(ctx)
    try:
        os.remove(cache)
    except OSError:
        pass
    print(json.dumps(line), flush=True)


# ------------------------------------------------------ tetrahedral RK45 arm

C4_WORKLOAD = ("pipe on tetrahedra: Delaunay tets of a jittered lattice in a cylinder R=1, L=10 (h=0.0466), "
               "pulsatile Poiseuille flow + 5% random-phase swirl, 50 FP32 frames per period 1 (time-periodic); "
               "64x64x512 seed lattice on [-1,1]^2x[0,10] (2,097,152 seeds); DP5(4) rtol=atol=1e-6, t0=0, T=1, "
               "cell walk per stage; FD grad F, 3x3 Cauchy-Green (FP64) and FTLE")
C4_N = (64, 64, 512)
C4_LO, C4_HI = (-1.0, -1.0, 0.0), (1.0, 1.0, 10.0)
C4_T, C4_TOL, C4_H0 = 1.0, 1e-6, 0.01
# algorithmic bytes of one stage evaluation on tets: one walk step (48 B inverse map + 16 B neighbours),
# 16 B connectivity, 4 vertices x 2 frames x 3 components x 4 B = 96 B of velocity; 6 new stages per
# accepted DP5(4) step (the first stage is the previous step's last)
C4_BYTES_PER_STAGE = 48 + 16 + 16 + 96
C4_STAGES_PER_STEP = 6


def c4_oracle_block(mesh, side, nz, threads=0):
    """Oracle DP5(4) (32-lane groups) + FD/CG/FTLE on a side x side x nz block of the C4 lattice
    centred in the pipe, with a 2-seed stencil halo; returns (interior seeds, seconds, threads, integrated)."""
    import oracle

    oracle.build()
    nth = oracle.set_threads(threads)
    h = [(C4_HI[a] - C4_LO[a]) / (C4_N[a] - 1) for a in range(3)]
    c = [C4_N[0] // 2 - side // 2, C4_N[1] // 2 - side // 2, C4_N[2] // 2 - nz // 2]
    m = (side + 4, side + 4, nz + 4)
    axes = [(C4_LO[a] + (c[a] - 2 + np.arange(m[a])) * h[a]).astype(np.float32) for a in range(3)]
    Z, Y, X = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    x0 = np.stack([X.ravel(), Y.ravel(), Z.ravel()])
    F = oracle.TetField(mesh.xyz, mesh.tets, mesh.nbrs, mesh.frames, mesh.times, True, mesh.period)
    t = time.perf_counter()
    cells = F.locate_seeds(x0)
    xT, st, _, _ = oracle.dp45(F, x0.astype(np.float64), 0.0, C4_T, h0=C4_H0, rtol=C4_TOL, atol=C4_TOL,
                               group=32, cells=cells)
    G = oracle.flowmap_gradient(3, m, h, (0, 0, 0), (0, 0, 0), xT, st)
    lam, sig = oracle.ftle(oracle.cauchy_green(G), 3, C4_T)
    return side * side * nz, time.perf_counter() - t, nth, x0.shape[1]


def c4_arm(args, rank, world, local):
    import torch

    from paper_2209_13775_gb300 import inputs, lcs

    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    ctx = lcs.lcs_create(local, stream)
    t_mesh = time.perf_counter()
    mesh = inputs.pipe_frames(inputs.pipe_mesh(), nframes=50, period=1.0)
    t_mesh = time.perf_counter() - t_mesh
    desc = lcs.field_desc(3, times=mesh.times, time_periodic=True, period=mesh.period, kind=lcs.TET,
                          mesh=(mesh.xyz, mesh.tets, mesh.nbrs))
    t_load = time.perf_counter()
    field = lcs.lcs_load_field(ctx, desc, mesh.frames)
    lcs.lcs_synchronize(ctx)
    t_load = time.perf_counter() - t_load
    t_seed = time.perf_counter()
    n_lat = (C4_N[0], C4_N[1], args.c4_nz)
    seeds = lcs.lcs_seed_grid(ctx, lcs.seed_desc(3, n_lat, C4_LO, C4_HI), field)
    lcs.lcs_synchronize(ctx)
    t_seed = time.perf_counter() - t_seed
    N = lcs.lcs_seeds_count(seeds)
    fm = lcs.lcs_flowmap_create(ctx, seeds, 1)
    T_run = args.mesh_T if args.mesh_T else C4_T
    opts = lcs.advect_opts(lcs.RK45, t0=0.0, T=T_run, rtol=C4_TOL, atol=C4_TOL, h0=C4_H0)
    ftle = torch.empty(N, dtype=torch.float32, device="cuda")
    C = torch.empty((N, 6), dtype=torch.float64, device="cuda")

    def step():
        lcs.lcs_advect(ctx, field, seeds, opts, fm)
        lcs.lcs_ftle(ctx, fm, 0, ftle, None, C)

    for _ in range(args.warmup):
        step()
    lcs.lcs_synchronize(ctx)
    for ph in range(4):
        lcs.lcs_timing_read(ctx, ph)
    lcs.lcs_timing_enable(ctx, True)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(args.steps):
            step()
        b.record(stream)
        torch.cuda.synchronize()
    el = a.elapsed_time(b) / 1e3
    adv_ms, adv_n = lcs.lcs_timing_read(ctx, 0)
    cg_ms, _ = lcs.lcs_timing_read(ctx, 3)
    lcs.lcs_timing_enable(ctx, False)
    steps = np.empty(N, dtype=np.int32)
    status = np.empty(N, dtype=np.uint8)
    lcs.lcs_flowmap_steps(ctx, fm, 0, steps)
    lcs.lcs_flowmap_get(ctx, fm, 0, None, status, None)
    tracer_steps = int(steps.astype(np.int64).sum())
    counts = {name: int((status == v).sum()) for name, v in
              (("ok", lcs.TRACER_OK), ("left", lcs.TRACER_LEFT), ("outside", lcs.TRACER_OUTSIDE),
               ("maxsteps", lcs.TRACER_MAXSTEPS), ("walkfail", lcs.TRACER_WALKFAIL))}
    live = status != lcs.TRACER_OUTSIDE
    pk, pk_kind = peaks()
    launch_s = adv_ms / max(adv_n, 1) / 1e3
    alg_bytes = float(tracer_steps) * C4_STAGES_PER_STEP * C4_BYTES_PER_STAGE
    achieved = alg_bytes / launch_s / 1e9
    hbm = pk.get("hbm_gbs", 6800.0)
    l2, l2_basis = l2_peak(local)
    line = {
        "metric": METRIC, "value": N * args.steps / el, "unit": "seeds/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": C4_WORKLOAD, "lattice": list(n_lat), "T": T_run, "seeds": N, "nodes": int(mesh.xyz.shape[0]),
                   "tets": int(mesh.tets.shape[0]), "mesh_build_s": round(t_mesh, 1),
                   "field_load_ms": round(t_load * 1e3, 1), "seed_location_ms": round(t_seed * 1e3, 1),
                   "status": counts, "accepted_steps_per_live_tracer": float(steps[live].mean()),
                   "l2": "no flush: the mesh store (geometry + 50 slabs, %.0f MB) exceeds the 129 MB L2"
                         % ((mesh.tets.shape[0] * (16 + 16 + 48) + mesh.xyz.shape[0] * 16
                             + 50 * mesh.xyz.shape[0] * 32) / 1e6)},
        "tracer_steps_per_s": tracer_steps * args.steps / el,
        "roofline": {"bound": "l2", "achieved": achieved, "peak": l2, "unit": "GB/s", "frac": achieved / l2,
                     "traffic": None, "kernel": "dp45_kernel<TetEval<F32>>",
                     "bytes_per_launch": alg_bytes, "avg_launch_ms": launch_s * 1e3, "launches": adv_n,
                     "peak_basis": l2_basis,
                     "basis": "%d B per stage x 6 stages per accepted step x accepted tracer-steps; the mesh "
                              "gathers stay in L1/L2 (DRAM reads under 1 GB per launch)" % C4_BYTES_PER_STAGE,
                     "frac_of_hbm_copy": achieved / hbm},
        "phases_ms_per_step": {"advect": adv_ms / args.steps, "cg_ftle": cg_ms / args.steps},
        "clocks": clk.summary(),
        # per step: the per-job values kernel, the DP5(4) kernel, FD/CG/FTLE
        "gpu_launches": 3 * args.steps,
    }
    if not args.no_cpu_baseline:
        _, dts, _, _ = c4_oracle_block(mesh, 12, 12)           # calibration: 16^3 tracers
        per = dts / 16 ** 3
        nz = int(max(4, min(500, (12.0 / max(per, 1e-9)) / (44 * 44) - 4)))
        s, dt, nth, integrated = c4_oracle_block(mesh, 40, nz)
        line["cpu_baseline"] = {"value": s / dt, "unit": "seeds/s", "cores": nth, "kind": "oracle",
                                "sample": "40x40x%d block of the 64x64x512 lattice at the pipe centre with its "
                                          "2-seed halo (%d tracers, DP5(4) in 32-lane groups), FD/CG/FTLE; %.1f s"
                                          % (nz, integrated, dt)}
    lcs.lcs_free_flowmap(fm)
    lcs.lcs_free_seeds(seeds)
    lcs.lcs_free_field(field)
    lcs.lcs_destroy(ctx)
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ triangle-mesh arm

TRI_WORKLOAD = ("stenosis on triangles: body-fitted triangulation of a channel 0<=x<=10, |y|<=1-0.5exp(-((x-3)/0.75)^2) "
                "(2000x400 jittered quads, 1.6M triangles), pulsatile flux-conserving Poiseuille flow + travelling "
                "wall wave, 40 FP32 frames per period 1 (time-periodic); 4096x1024 seed lattice on [0,10]x[-1,1] "
                "(4,194,304 seeds, those beside the constriction outside the mesh); RK4 dt=0.002, t0=0, T=1 "
                "(500 steps), cell walk per stage; FD grad F, 2x2 Cauchy-Green (FP64) and FTLE")
TRI_N, TRI_LO, TRI_HI = (4096, 1024), (0.0, -1.0), (10.0, 1.0)
TRI_T, TRI_DT, TRI_H = 1.0, 0.002, 0.005
# algorithmic bytes of one stage evaluation on triangles: one walk step (16 B inverse map + 8 B vertex 0),
# 16 B connectivity, 3 vertices x 16 B frame pairs (u_k, v_k, u_k+1, v_k+1)
TRI_BYTES_PER_STAGE = 16 + 8 + 16 + 48
# FP32 flops of one RK4 step on triangles: per stage the barycentric coordinates (10), the P1 and time
# blend of 3 vertices x 2 components (30 + 1), the stage point (4, stages 2-4); the update (12 + 2)
TRI_FLOP_PER_STEP = 4 * (10 + 31) + 3 * 4 + 14


def l2_peak(device):
    """Read rate of an L2-resident buffer on this GPU (bench_peaks.cu, median of 3), the denominator of
    the gather-bound mesh kernels."""
    runs = [probe_peaks(device)["l2_read_gbs"] for _ in range(3)]
    return float(np.median(runs)), "bench_peaks.cu: 16-byte loads re-reading a 32 MB buffer, median of 3"


def alu_peak():
    """FP32 ALU peak (TFLOP/s) at the measured maximum SM clock, and its basis."""
    pk, pk_kind = peaks()
    sm_mhz = pk.get("sm_max_mhz", 2070.0)
    return (152 * 128 * 2 * sm_mhz * 1e6 / 1e12,
            "152 SMs x 128 FP32 lanes x 2 x %.0f MHz (%s sm_max_mhz)" % (sm_mhz, pk_kind))


def tri_oracle_block(mesh, ni, nj, threads=0):
    """Oracle RK4 + FD/CG/FTLE on an ni x nj block of the triangle lattice at the channel centre
    downstream of the constriction, with a 2-seed stencil halo; returns (interior seeds, seconds,
    threads, integrated)."""
    import oracle

    oracle.build()
    nth = oracle.set_threads(threads)
    h = [(TRI_HI[a] - TRI_LO[a]) / (TRI_N[a] - 1) for a in range(2)]
    c = [int(TRI_N[0] * 0.6) - ni // 2, TRI_N[1] // 2 - nj // 2]
    m = (ni + 4, nj + 4)
    axes = [(TRI_LO[a] + (c[a] - 2 + np.arange(m[a])) * h[a]).astype(np.float32) for a in range(2)]
    Y, X = np.meshgrid(axes[1], axes[0], indexing="ij")
    x0 = np.stack([X.ravel(), Y.ravel()])
    F = oracle.TriField(mesh.xyz, mesh.tets, mesh.nbrs, mesh.frames, mesh.times, True, mesh.period)
    t = time.perf_counter()
    cells = F.locate_seeds(x0)
    xT, st, _ = oracle.rk4(F, x0.astype(np.float64), 0.0, TRI_T, TRI_DT, cells=cells)
    G = oracle.flowmap_gradient(2, m, h, (0, 0), (0, 0), xT, st)
    lam, sig = oracle.ftle(oracle.cauchy_green(G), 2, TRI_T)
    return ni * nj, time.perf_counter() - t, nth, x0.shape[1]


def tri_arm(args, rank, world, local):
    import torch

    from paper_2209_13775_gb300 import inputs, lcs

    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    ctx = lcs.lcs_create(local, stream)
    t_mesh = time.perf_counter()
    mesh = inputs.stenosis_frames(inputs.stenosis_mesh(h=TRI_H), nframes=40, period=1.0)
    t_mesh = time.perf_counter() - t_mesh
    st_kind = {"f32": lcs.F32, "f16": lcs.F16, "bf16": lcs.BF16}[args.storage]
    desc = lcs.field_desc(2, times=mesh.times, time_periodic=True, period=mesh.period, kind=lcs.TRI,
                          storage=st_kind, mesh=(mesh.xyz, mesh.tets, mesh.nbrs))
    t_load = time.perf_counter()
    field = lcs.lcs_load_field(ctx, desc, mesh.frames)
    lcs.lcs_synchronize(ctx)
    t_load = time.perf_counter() - t_load
    t_seed = time.perf_counter()
    n_lat = (args.tri_side, args.tri_side // 4)
    seeds = lcs.lcs_seed_grid(ctx, lcs.seed_desc(2, n_lat, TRI_LO, TRI_HI), field)
    lcs.lcs_synchronize(ctx)
    t_seed = time.perf_counter() - t_seed
    N = lcs.lcs_seeds_count(seeds)
    fm = lcs.lcs_flowmap_create(ctx, seeds, 1)
    T_run = args.mesh_T if args.mesh_T else TRI_T
    opts = lcs.advect_opts(lcs.RK4, t0=0.0, T=T_run, dt=TRI_DT)
    ftle = torch.empty(N, dtype=torch.float32, device="cuda")
    C = torch.empty((N, 3), dtype=torch.float64, device="cuda")

    def step():
        lcs.lcs_advect(ctx, field, seeds, opts, fm)
        lcs.lcs_ftle(ctx, fm, 0, ftle, None, C)

    for _ in range(args.warmup):
        step()
    lcs.lcs_synchronize(ctx)
    for ph in range(4):
        lcs.lcs_timing_read(ctx, ph)
    lcs.lcs_timing_enable(ctx, True)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(args.steps):
            step()
        b.record(stream)
        torch.cuda.synchronize()
    el = a.elapsed_time(b) / 1e3
    adv_ms, adv_n = lcs.lcs_timing_read(ctx, 0)
    cg_ms, _ = lcs.lcs_timing_read(ctx, 3)
    lcs.lcs_timing_enable(ctx, False)
    status = np.empty(N, dtype=np.uint8)
    te = np.empty(N, dtype=np.float32)
    lcs.lcs_flowmap_get(ctx, fm, 0, None, status, te)
    counts = {name: int((status == v).sum()) for name, v in
              (("ok", lcs.TRACER_OK), ("left", lcs.TRACER_LEFT), ("outside", lcs.TRACER_OUTSIDE))}
    nsteps = int(round(T_run / TRI_DT))
    # steps actually taken: all for OK tracers, up to the exit for LEFT ones
    taken = np.where(status == lcs.TRACER_OK, nsteps,
                     np.where(status == lcs.TRACER_LEFT, np.rint(te / TRI_DT), 0)).astype(np.int64)
    tracer_steps = int(taken.sum())
    launch_s = adv_ms / max(adv_n, 1) / 1e3
    alg_bytes = float(tracer_steps) * 4 * TRI_BYTES_PER_STAGE
    flop = float(tracer_steps) * TRI_FLOP_PER_STEP
    achieved = flop / launch_s / 1e12
    fp32_peak, peak_basis = alu_peak()
    l2, l2_basis = l2_peak(local)
    gbs = alg_bytes / launch_s / 1e9
    line = {
        "metric": METRIC, "value": N * args.steps / el, "unit": "seeds/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": TRI_WORKLOAD, "lattice": list(n_lat), "T": T_run, "seeds": N, "nodes": int(mesh.xyz.shape[0]),
                   "triangles": int(mesh.tets.shape[0]), "storage": args.storage,
                   "mesh_build_s": round(t_mesh, 1), "field_load_ms": round(t_load * 1e3, 1),
                   "seed_location_ms": round(t_seed * 1e3, 1), "status": counts,
                   "l2": "no flush: each step writes %.0f MB of outputs (C + FTLE) > 129 MB L2" % (N * 28 / 1e6)},
        "tracer_steps_per_s": tracer_steps * args.steps / el,
        "roofline": {"bound": "l2", "achieved": gbs, "peak": l2, "unit": "GB/s", "frac": gbs / l2,
                     "traffic": None, "kernel": "rk4_tri_kernel<%s>" % args.storage,
                     "bytes_per_launch": alg_bytes, "avg_launch_ms": launch_s * 1e3, "launches": adv_n,
                     "peak_basis": l2_basis,
                     "basis": "%d B of gathers per stage x 4 stages x tracer-steps taken (map, vertex 0, "
                              "connectivity, three frame pairs), served by L1/L2" % TRI_BYTES_PER_STAGE,
                     "alu": {"achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                             "peak_basis": peak_basis,
                             "basis": "%d FP32 flops per tracer-step" % TRI_FLOP_PER_STEP}},
        "phases_ms_per_step": {"advect": adv_ms / args.steps, "cg_ftle": cg_ms / args.steps},
        "clocks": clk.summary(),
        # per step: the schedule kernel, the RK4 kernel, FD/CG/FTLE
        "gpu_launches": 3 * args.steps,
    }
    if not args.no_cpu_baseline:
        _, dts, _, _ = tri_oracle_block(mesh, 16, 16)           # calibration
        per = dts / 400
        nj = int(max(4, min(400, (12.0 / max(per, 1e-9)) / 104 - 4)))
        s, dt, nth, integrated = tri_oracle_block(mesh, 100, nj)
        line["cpu_baseline"] = {"value": s / dt, "unit": "seeds/s", "cores": nth, "kind": "oracle",
                                "sample": "100x%d block of the 4096x1024 lattice at x = 6 with its 2-seed halo "
                                          "(%d tracers, RK4), FD/CG/FTLE; %.1f s" % (nj, integrated, dt)}
    lcs.lcs_free_flowmap(fm)
    lcs.lcs_free_seeds(seeds)
    lcs.lcs_free_field(field)
    lcs.lcs_destroy(ctx)
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ surrogate arm

C5_WORKLOAD = ("learned surrogate on the double gyre (129x65 FP32, 101 frames, period 10): MLP 7->128x4->3 (SiLU, "
               "BF16 weights/activations, FP32 accumulate, tcgen05) trained on 50,331,648 RK4 (dt=0.05) "
               "displacements over tau=0.5 from (x0,y0,t0) ~ U([0,2]x[0,1]x[0,10)); FTLE from K=16 gated "
               "surrogate steps (T=8, t0=0) on a 16384x8192 seed lattice (2^27 seeds), audit threshold 1e-3 with "
               "RK4 fallback; FTLE error against plain RK4 on the same lattice")
C5_N = (16384, 8192)
C5_TAU, C5_K, C5_DT, C5_TOL = 0.5, 16, 0.05, 1e-3
C5_FEAT = dict(center=(1.0, 0.5), kx=math.pi, ky=math.pi, omega=2 * math.pi / 10)
C5_SAMPLES, C5_BATCH = 768 * 65536, 65536
# algorithmic work of one network evaluation: 2 (7*128 + 3*128*128 + 128*3) FLOP
C5_FLOP_PER_EVAL = 2 * (7 * 128 + 3 * 128 * 128 + 128 * 3)


def c5_oracle_block(gyre, params, side, threads=0):
    """Oracle gated surrogate (FP64 network on the trained parameters) + FD/CG/FTLE on a side x side block
    of the C5 lattice with a 2-seed halo; returns (interior seeds, seconds, threads, integrated)."""
    import oracle
    from oracle import mlp as omlp

    oracle.build()
    nth = oracle.set_threads(threads)
    h = [2.0 / (C5_N[0] - 1), 1.0 / (C5_N[1] - 1)]
    c0 = [C5_N[0] // 3, C5_N[1] // 3]
    m = side + 4
    xs = (0.0 + (c0[0] - 2 + np.arange(m)) * h[0]).astype(np.float32)
    ys = (0.0 + (c0[1] - 2 + np.arange(m)) * h[1]).astype(np.float32)
    Y, X = np.meshgrid(ys, xs, indexing="ij")
    x0 = np.stack([X.ravel(), Y.ravel()]).astype(np.float64)
    F = oracle.RectField(gyre.frames, gyre.times, gyre.origin, gyre.spacing, gyre.periodic, gyre.time_periodic,
                         gyre.period)
    t = time.perf_counter()
    xT, _, _ = omlp.surrogate_advect(params.astype(np.float64), F, x0, 0.0, C5_K, C5_TAU, C5_DT, C5_TOL,
                                     **C5_FEAT, out_scale=0.1)
    st = np.zeros(x0.shape[1], dtype=np.uint8)
    G = oracle.flowmap_gradient(2, (m, m), h, (0, 0), (0, 0), xT, st)
    lam, sig = oracle.ftle(oracle.cauchy_green(G), 2, C5_K * C5_TAU)
    return side * side, time.perf_counter() - t, nth, x0.shape[1]


def c5_arm(args, rank, world, local):
    import torch

    from paper_2209_13775_gb300 import inputs, lcs

    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    ctx = lcs.lcs_create(local, stream)
    g = inputs.double_gyre()
    field = lcs.lcs_load_field(ctx, lcs.field_desc(2, g.n, g.origin, g.spacing, g.periodic, g.times,
                                                   g.time_periodic, g.period), g.frames)
    desc = lcs.mlp_desc(C5_FEAT["center"], C5_FEAT["kx"], C5_FEAT["ky"], C5_FEAT["omega"], C5_TAU, 0.1)
    mlp = lcs.lcs_mlp_create(ctx, desc, inputs.mlp_init())
    samples = torch.from_numpy(inputs.surrogate_samples(C5_SAMPLES)).cuda()
    torch.cuda.synchronize()
    t_train = time.perf_counter()
    hist = lcs.lcs_surrogate_train(ctx, field, mlp, lcs.train_desc(batch=C5_BATCH, epochs=args.train_epochs,
                                                                   lr=2e-3, lr_min=1e-5, rho_weight=0.01,
                                                                   dt=C5_DT), samples)
    t_train = time.perf_counter() - t_train
    del samples
    c5n = (args.c5_side, args.c5_side // 2)
    seeds = lcs.lcs_seed_grid(ctx, lcs.seed_desc(2, c5n, (0.0, 0.0), (2.0, 1.0)))
    N = lcs.lcs_seeds_count(seeds)
    T = C5_K * C5_TAU
    fm = lcs.lcs_flowmap_create(ctx, seeds, 1)
    sur = lcs.advect_opts(lcs.SURROGATE, t0=0.0, T=T, dt=C5_DT, surrogate=mlp, gate_tol=C5_TOL)
    plain = lcs.advect_opts(lcs.RK4, t0=0.0, T=T, dt=C5_DT)
    ftle = torch.empty(N, dtype=torch.float32, device="cuda")
    ftle_p = torch.empty(N, dtype=torch.float32, device="cuda")

    def step(opts, out):
        lcs.lcs_advect(ctx, field, seeds, opts, fm)
        lcs.lcs_ftle(ctx, fm, 0, out)

    def timed(opts, out, k):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(k):
            step(opts, out)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1e3 / k

    for _ in range(args.warmup):
        step(sur, ftle)
    step(plain, ftle_p)
    lcs.lcs_synchronize(ctx)
    for ph in range(4):
        lcs.lcs_timing_read(ctx, ph)
    lcs.lcs_timing_enable(ctx, True)
    with ClockSampler(local) as clk:
        el = timed(sur, ftle, args.steps)
    mlp_ms, mlp_n = lcs.lcs_timing_read(ctx, 0)
    gate_ms, gate_n = lcs.lcs_timing_read(ctx, 1)
    cg_ms, _ = lcs.lcs_timing_read(ctx, 3)
    lcs.lcs_timing_enable(ctx, False)
    counts = np.empty(N, dtype=np.int32)
    lcs.lcs_flowmap_steps(ctx, fm, 0, counts)
    fb_frac = float(counts.astype(np.int64).sum()) / (N * C5_K)
    el_plain = timed(plain, ftle_p, max(1, args.steps // 2))
    a, b = ftle.cpu().double().numpy(), ftle_p.cpu().double().numpy()
    ok = np.isfinite(a) & np.isfinite(b)
    d = np.abs(a[ok] - b[ok])
    pk, pk_kind = peaks()
    peak = pk.get("bf16_tflops", 1900.0)
    launch_s = mlp_ms / max(mlp_n, 1) / 1e3
    flops = float(N) * C5_FLOP_PER_EVAL
    achieved = flops / launch_s / 1e12
    line = {
        "metric": METRIC, "value": N * 1.0 / el, "unit": "seeds/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": el * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16 (network), f32 (integrator)", "data": "synthetic",
        "config": {"workload": C5_WORKLOAD if c5n == C5_N else
                   C5_WORKLOAD.replace("16384x8192 seed lattice (2^27 seeds)", "%dx%d seed lattice" % c5n),
                   "seeds": N, "K": C5_K, "tau": C5_TAU, "gate_tol": C5_TOL,
                   "train_samples": C5_SAMPLES, "train_batch": C5_BATCH, "train_epochs": args.train_epochs,
                   "l2": "no flush: each step writes 2.7 GB of flow map and FTLE (> 129 MB L2)"},
        "surrogate": {"train_s": round(t_train, 2), "loss_per_epoch": [float(x) for x in hist],
                      "fallback_fraction": fb_frac,
                      "ftle_err_vs_plain": {"median": float(np.median(d)), "p99.9": float(np.quantile(d, 0.999)),
                                            "max": float(d.max())},
                      "plain_rk4_ms_per_step": el_plain * 1e3, "plain_rk4_seeds_per_s": N / el_plain,
                      "speedup_vs_plain": el_plain / el},
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None, "kernel": "mlp_step_kernel (tcgen05, 5 layers)",
                     "flop_per_launch": flops, "avg_launch_ms": launch_s * 1e3, "launches": mlp_n,
                     "peak_basis": "bf16_tflops (%s, burst)" % pk_kind},
        "phases_ms_per_step": {"network": mlp_ms / args.steps, "audit_and_fallback": gate_ms / args.steps,
                               "cg_ftle": cg_ms / args.steps},
        "clocks": clk.summary(),
        # per step: schedule, state init (3), K x (network, audit, apply), FD/CG/FTLE
        "gpu_launches": args.steps * (1 + 3 + 3 * C5_K + 1),
    }
    if not args.no_cpu_baseline:
        params = np.empty(lcs.MLP_NPARAMS, dtype=np.float32)
        lcs.lcs_mlp_get_params(ctx, mlp, params)
        _, dts, _, _ = c5_oracle_block(g, params, 4)
        per = dts / 64.0
        side = int(max(4, min(64, math.sqrt(10.0 / max(per, 1e-9)) - 4)))
        s, dt, nth, integrated = c5_oracle_block(g, params, side)
        line["cpu_baseline"] = {"value": s / dt, "unit": "seeds/s", "cores": nth, "kind": "oracle",
                                "sample": "%dx%d block of the 16384x8192 lattice with its 2-seed halo (%d tracers, "
                                          "FP64 network + audits + RK4 fallback), FD/CG/FTLE; %.1f s"
                                          % (side, side, integrated, dt)}
    lcs.lcs_free_flowmap(fm)
    lcs.lcs_free_seeds(seeds)
    lcs.lcs_mlp_free(mlp)
    lcs.lcs_free_field(field)
    lcs.lcs_destroy(ctx)
    print(json.dumps(line), flush=True)


# ------------------------------------- eigenvectors, early CG, auxiliary points

def next_arm(args, rank, world, local):
    """Times of the passes that widen the pipeline: all eigenpairs of C on the 3D ABC lattice (256^3),
    the early Cauchy-Green evaluation on the double gyre cut to x in [0, 1.5] (2^21 seeds, T = 6),
    and the auxiliary-point FTLE of a 1024x512 gyre lattice (4 points per seed)."""
    import torch

    from paper_2209_13775_gb300 import inputs, lcs
    from dataclasses import replace

    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    ctx = lcs.lcs_create(local, stream)
    ev = lambda: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))

    def timed(fn, k):
        fn()
        torch.cuda.synchronize()
        a, b = ev()
        a.record(stream)
        for _ in range(k):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / k

    out = {}
    # 1. eigenpairs of C on the ABC lattice (the flow map of one C2 step)
    g = inputs.abc(n=N_GRID, nframes=N_FRAMES, t_end=T_END)
    field = lcs.lcs_load_field(ctx, lcs.field_desc(3, g.n, g.origin, g.spacing, g.periodic, g.times),
                               torch.from_numpy(g.frames).cuda())
    seeds = lcs.lcs_seed_grid(ctx, lcs.seed_desc(3, (N_SIDE,) * 3, (0.0,) * 3, (L,) * 3, (1, 1, 1)))
    N = lcs.lcs_seeds_count(seeds)
    fm = lcs.lcs_flowmap_create(ctx, seeds, 1)
    lcs.lcs_advect(ctx, field, seeds, lcs.advect_opts(lcs.RK4, t0=0.0, T=T_END, dt=DT), fm)
    eigval = torch.empty((N, 3), dtype=torch.float64, device="cuda")
    eigvec = torch.empty((N, 3, 3), dtype=torch.float64, device="cuda")
    ftle = torch.empty(N, dtype=torch.float32, device="cuda")
    ms_eig = timed(lambda: lcs.lcs_cg_eigen(ctx, fm, 0, eigval, eigvec), max(args.steps, 3))
    ms_ftle = timed(lambda: lcs.lcs_ftle(ctx, fm, 0, ftle), max(args.steps, 3))
    out["eigen_abc_256cubed"] = {"ms": ms_eig, "seeds_per_s": N / ms_eig * 1e3, "ftle_pass_ms": ms_ftle,
                                 "bytes_written": N * 96, "write_gbs": N * 96 / ms_eig / 1e6}
    # grad F by the variational equations on the same lattice, against the default finite-difference step
    ov = lcs.advect_opts(lcs.RK4, t0=0.0, T=T_END, dt=DT, variational=True)
    od = lcs.advect_opts(lcs.RK4, t0=0.0, T=T_END, dt=DT)

    def var_step():
        lcs.lcs_advect(ctx, field, seeds, ov, fm)
        lcs.lcs_ftle_variational(ctx, fm, 0, ftle)

    def fd_step():
        lcs.lcs_advect(ctx, field, seeds, od, fm)
        lcs.lcs_ftle(ctx, fm, 0, ftle)

    ms_var = timed(var_step, 3)
    ms_fd = timed(fd_step, 3)
    out["variational_abc_256cubed"] = {"ms": ms_var, "seeds_per_s": N / ms_var * 1e3, "fd_step_ms": ms_fd,
                                       "note": "re-bundled episodes carrying the 3x3 M per tracer (time slices, "
                                               "127 registers, 2 blocks of 256 per SM); fd_step = the default "
                                               "re-bundled path + FD"}
    lcs.lcs_free_flowmap(fm)
    lcs.lcs_free_seeds(seeds)
    lcs.lcs_free_field(field)
    # 2. early CG on the truncated gyre
    g2 = inputs.double_gyre()
    g2 = replace(g2, frames=np.ascontiguousarray(g2.frames[:, :, :97]))
    f2 = lcs.lcs_load_field(ctx, lcs.field_desc(2, g2.n, g2.origin, g2.spacing, g2.periodic, g2.times,
                                                g2.time_periodic, g2.period), g2.frames)
    s2 = lcs.lcs_seed_grid(ctx, lcs.seed_desc(2, (2048, 1024), (0.0, 0.0), (1.5, 1.0)))
    N2 = lcs.lcs_seeds_count(s2)
    fm2 = lcs.lcs_flowmap_create(ctx, s2, 1)
    o2 = lcs.advect_opts(lcs.RK4, t0=0.0, T=6.0, dt=0.05)
    lcs.lcs_advect(ctx, f2, s2, o2, fm2)
    fe = torch.empty(N2, dtype=torch.float32, device="cuda")
    te = torch.empty(N2, dtype=torch.float32, device="cuda")
    ms_early = timed(lambda: lcs.lcs_ftle_early(ctx, f2, s2, o2, fm2, 0, fe, te), max(args.steps, 3))
    ms_adv2 = timed(lambda: lcs.lcs_advect(ctx, f2, s2, o2, fm2), 2)
    n_early = int(((te > 0) & (te < 6.0)).sum().item())
    out["early_cg_gyre_2M"] = {"ms": ms_early, "early_seeds": n_early, "seeds": N2, "advect_ms": ms_adv2,
                               "note": "the early seeds' stencils (5 tracers each) are re-integrated"}
    lcs.lcs_free_flowmap(fm2)
    # 3. auxiliary-point FTLE on a 1024x512 gyre lattice (full gyre box)
    lat = lcs.lcs_seed_grid(ctx, lcs.seed_desc(2, (1024, 512), (0.0, 0.0), (2.0, 1.0)))
    aux = lcs.lcs_seed_aux(ctx, lat, [2.0 / 1023 / 8, 1.0 / 511 / 8])
    M = lcs.lcs_seeds_count(aux)
    g3 = inputs.double_gyre()
    f3 = lcs.lcs_load_field(ctx, lcs.field_desc(2, g3.n, g3.origin, g3.spacing, g3.periodic, g3.times,
                                                g3.time_periodic, g3.period), g3.frames)
    fm3 = lcs.lcs_flowmap_create(ctx, aux, 1)
    o3 = lcs.advect_opts(lcs.RK4, t0=0.0, T=10.0, dt=0.05)
    fa = torch.empty(1024 * 512, dtype=torch.float32, device="cuda")

    def aux_step():
        lcs.lcs_advect(ctx, f3, aux, o3, fm3)
        lcs.lcs_ftle(ctx, fm3, 0, fa)

    ms_aux = timed(aux_step, max(args.steps, 3))
    out["aux_points_gyre_1024x512"] = {"ms": ms_aux, "points": M, "ftle_seeds_per_s": 1024 * 512 / ms_aux * 1e3,
                                       "tracer_steps_per_s": M * 200 / ms_aux * 1e3}
    # 4. the same seeds' grad F by the variational equations (one tracer per seed)
    fm4 = lcs.lcs_flowmap_create(ctx, lat, 1)
    o4 = lcs.advect_opts(lcs.RK4, t0=0.0, T=10.0, dt=0.05, variational=True)

    def var2_step():
        lcs.lcs_advect(ctx, f3, lat, o4, fm4)
        lcs.lcs_ftle_variational(ctx, fm4, 0, fa)

    ms_var2 = timed(var2_step, max(args.steps, 3))
    out["variational_gyre_1024x512"] = {"ms": ms_var2, "ftle_seeds_per_s": 1024 * 512 / ms_var2 * 1e3,
                                        "aux_points_ms": ms_aux}
    for h in (fm3, fm4):
        lcs.lcs_free_flowmap(h)
    for h in (aux, lat, s2):
        lcs.lcs_free_seeds(h)
    for h in (f2, f3):
        lcs.lcs_free_field(h)
    lcs.lcs_destroy(ctx)
    line = {"metric": METRIC, "value": out["eigen_abc_256cubed"]["seeds_per_s"], "unit": "seeds/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 (eigen), f32 (tracers)", "data": "synthetic",
            "config": {"workload": "widening passes: eigenpairs of C (ABC 256^3 after the C2 integration), early "
                                   "CG (gyre cut to x<=1.5, 2048x1024 seeds, T=6), auxiliary-point FTLE "
                                   "(gyre 1024x512, delta = 1/8 lattice step, T=10), variational grad F "
                                   "(ABC 256^3 T=8 and gyre 1024x512 T=10)"},
            "passes": out}
    print(json.dumps(line), flush=True)


PROBE_SRC = os.path.join(ROOT, "bench_peaks.cu")
PROBE_LIB = os.path.join(ROOT, "_build", "libbench_peaks.so")


def build_probes() -> str:
    """Compile bench_peaks.cu (the measurement probes; not part of liblcs) for sm_103a when stale."""
    if not os.path.exists(PROBE_LIB) or os.path.getmtime(PROBE_LIB) < os.path.getmtime(PROBE_SRC):
        os.makedirs(os.path.dirname(PROBE_LIB), exist_ok=True)
        nvcc = "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else "nvcc"
        tmp = PROBE_LIB + ".tmp.%d" % os.getpid()
        subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-Xcompiler", "-fPIC", "-shared",
                        "-o", tmp, PROBE_SRC], check=True, capture_output=True)
        os.replace(tmp, PROBE_LIB)
    return PROBE_LIB


def probe_peaks(device):
    """FP32 and FP64 FMA TFLOP/s, L2-resident and HBM read GB/s measured with plain loops."""
    import ctypes

    lib = ctypes.CDLL(build_probes())
    out = np.zeros(4)
    rc = lib.bench_probe_peaks(int(device), ctypes.c_void_p(out.ctypes.data))
    if rc != 0:
        raise RuntimeError("bench_probe_peaks: CUDA error %d" % rc)
    return {"fp32_tflops": out[0], "fp64_tflops": out[1], "l2_read_gbs": out[2], "hbm_read_gbs": out[3]}


L1_PATTERNS = ["1 line per quarter warp", "2 lines, distinct bank groups", "4 lines, distinct bank groups",
               "8 lines, distinct bank groups", "8 lines, one bank group", "2 lines, one bank group"]


def probe_l1(device):
    """SM cycles per warp-wide 16-byte gather request for lane patterns of the L1 data stage."""
    import ctypes

    lib = ctypes.CDLL(build_probes())
    out = np.zeros(len(L1_PATTERNS))
    rc = lib.bench_probe_l1(int(device), ctypes.c_void_p(out.ctypes.data))
    if rc != 0:
        raise RuntimeError("bench_probe_l1: CUDA error %d" % rc)
    return dict(zip(L1_PATTERNS, [float(v) for v in out]))


def peaks_arm(args, rank, world, local):
    """The rates plain loops reach on this GPU (FP32/FP64 FMA, L2-resident and HBM reads, the L1 gather
    patterns), next to the measured copy bandwidth and the FP32 ALU figure the advection
    rooflines use."""
    import torch

    torch.cuda.set_device(local)
    runs = [probe_peaks(local) for _ in range(max(args.steps, 3))]
    med = {k: float(np.median([r[k] for r in runs])) for k in runs[0]}
    l1 = probe_l1(local)
    alu, basis = alu_peak()
    pk, pk_kind = peaks()
    line = {"metric": "plain-loop peaks on 1 GB300", "value": med["fp32_tflops"], "unit": "TFLOP/s (FP32 FMA)",
            "n_gpus": 1, "steps": len(runs), "warmup": 1, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32/f64", "data": "synthetic",
            "config": {"workload": "FMA chains (8 per thread, 16 blocks of 256 per SM); reads of a 32 MB buffer "
                                   "x256 and of a 4 GiB buffer x1 (16-byte loads, grid-stride); 16-byte gathers "
                                   "from a 128 KB buffer per lane pattern"},
            "peaks": med, "l1_gather_clk_per_request": l1, "fp32_alu_formula_tflops": alu,
            "fp32_alu_formula": basis, "driver_hbm_copy_gbs": pk.get("hbm_gbs"), "driver_peaks": pk_kind}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    if args.config == "c3":
        c3_arm(args, rank, world, local)
        return
    if args.config == "c3x":
        c3x_arm(args, rank, world, local)
        return
    if args.config == "c4":
        c4_arm(args, rank, world, local)
        return
    if args.config == "next":
        next_arm(args, rank, world, local)
        return
    if args.config == "tri":
        tri_arm(args, rank, world, local)
        return
    if args.config == "peaks":
        peaks_arm(args, rank, world, local)
        return
    if args.config == "c5":
        c5_arm(args, rank, world, local)
        return
    our_arm(args, rank, world, local)


if __name__ == "__main__":
    main()
