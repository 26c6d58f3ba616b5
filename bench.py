#!/usr/bin/env python3
"""Throughput of the scattered-field PIC step (arXiv 2310.11393) on GB300.

One step = push + incident-field evaluation + gather + Boris + Esirkepov deposit for every
macro-electron, the particle re-sort by tile, and the Yee update of the scattered field.
Default workload: the largest single-GPU configuration, the 3D tightly focused RP case
(512 x 256 x 256 cells, dx = lambda/24, RP pulse w0 = 0.7 lambda, a0 = 20, 5 fs,
256 x 128 x 128-cell slab at 0.01 n_c with 4 ppc = 16 777 216 electrons).  The K timed steps
are the window of the run centred on the step at which the pulse peak crosses the focus
(the simulation is first advanced to the window's start, untimed); --window start times
the first K steps instead; without --steps the whole run is timed.  Metric:
particle-pushes/s (each push includes the incident-field evaluation and the deposit),
counted exactly: an electron alive at the end counts every timed step, one that left the
box counts the timed steps up to the one in which it left (its exit record).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload 3d|2d|1d]

N > 1: one process per GPU (when WORLD_SIZE is not set, bench.py starts the N ranks itself
under torch.distributed.run); every rank advances its own replica of the workload
(independent simulations: no data-path collective), timing is max over ranks and the value
sums all ranks' pushes (weak scaling).  --impl reference times the FP64 CPU oracle on all
host cores (one single-threaded oracle process per core, each on its own seeded sample box
of the same workload).
"""
import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "particle-pushes/s incl. incident-field eval+deposit"
UNIT = "pushes/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=0, help="timed steps (default: the workload's full run)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="3d", choices=["1d", "2d", "3d", "2d_gauss", "batch", "serve"])
    ap.add_argument("--window", default="focus", choices=["focus", "start"],
                    help="timed steps centred on the pulse crossing the focus (default) or from t = 0")
    ap.add_argument("--scale", type=int, default=1, help="1d/2d/3d: box divided by this per axis (profiling)")
    ap.add_argument("--slab-cells", type=int, default=0,
                    help="1d/2d/3d: electron slab cut to this many cells per axis (profiling the field solve)")
    ap.add_argument("--tile", default="", help="particle tile, e.g. 16,8,4 (skips the autotuner's tile search)")
    ap.add_argument("--chunk", type=int, default=0, help="particles per push work item (skips its autotuning)")
    ap.add_argument("--autotune", type=int, default=10,
                    help="trial steps per candidate of the tile/work-item autotuner before timing (0: defaults)")
    ap.add_argument("--incident", default="particle", choices=["particle", "grid"],
                    help="incident field at every particle (Sec. 2) or on the Yee nodes, gathered")
    ap.add_argument("--sort-every", type=int, default=0,
                    help="steps between cell sorts within the tiles (<= 0: none)")
    ap.add_argument("--sims", type=int, default=256, help="batch: number of simulations")
    ap.add_argument("--requests", type=int, default=100, help="serve: number of requests per stream")
    ap.add_argument("--rate", type=float, default=20.0, help="serve: mean arrival rate (1/s)")
    ap.add_argument("--profile-steps", type=int, default=0, help="steps timed kernel by kernel (default: --steps)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


SCALE = 1
INCIDENT_GRID = 0
SLAB_CELLS = 0

# dram__bytes_read.sum + dram__bytes_write.sum of one launch of the dominant kernel, from the
# ncu capture summarised in profiles/ (kept in step with the kernel: set to None when the
# kernel changes and until it is captured again)
PROFILED_TRAFFIC = {
    ("2d_lp_1024sq", "k_push1<2,float>"): (108.4e6, "profiles/k_push_2d_lp_1024sq.md, step 762 (focus)"),
    # the full 3D state (14 GB) is too large for a multi-pass capture: the box halved per axis
    # (2.1 M electrons, step 233 at the focus), scaled by the electrons (x8): the push's traffic
    # is per particle (record read and written) plus the grid per cell, both x8
    ("3d_rp_512x256x256", "k_push1<3,float>"): (8 * 161.3e6, "profiles/k_push_3d_rp_256x128x128.md, box halved per "
                                                             "axis at the focus, scaled x8 by electrons and cells"),
}


def workload(name):
    w = {"1d": synth.c1_1d_plane, "2d": synth.c2_2d_lp, "3d": synth.c3_3d_rp, "2d_gauss": synth.c6_2d_gauss}[name]()
    w = w if SCALE == 1 else synth.scaled(w, SCALE)
    if SLAB_CELLS > 0:
        # profiling: the electron slab cut to SLAB_CELLS cells per axis at its low corner
        # (the grid and the field solve unchanged, the device state a few GB)
        hi = tuple(min(w.slab_hi[d], w.slab_lo[d] + SLAB_CELLS) if d < w.dim else w.slab_hi[d] for d in range(3))
        w = w.with_(slab_hi=hi, name=w.name + f"_slab{SLAB_CELLS}")
    return w.with_(incident_grid=INCIDENT_GRID, name=w.name + ("_incgrid" if INCIDENT_GRID else ""))


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), float(m.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region (SM clock, reasons)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if parts[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if sm:
            out = {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return out


def flops_per_push(w):
    """Algorithmic FP32 operations of one push (add/mul = 1, FMA = 2, each transcendental call = 1),
    counted from the formulas the kernel evaluates, with BOTH terms tau_+ and tau_- of the
    closed form evaluated (the kernel drops a term below e^-36 of the peak; that saving is not
    subtracted, so the fraction reported is an upper bound of the pipe use)."""
    D = w.dim
    gather = {1: 6 * 6 + 12, 2: 6 * 24 + 24, 3: 6 * 78 + 36}[D]
    boris = 60
    # Esirkepov on four-node windows: per axis two order-2 shapes; along the current's own axis
    # three partial sums per transverse node, 2D Jz / 3D every component over 4^(D-1) nodes
    deposit = {1: 40, 2: 300, 3: 970}[D]
    incident = {synth.BEAM_LP: 280, synth.BEAM_RP: 270, synth.BEAM_PLANE: 25, synth.BEAM_GAUSS2D: 45}.get(w.beam, 0)
    if w.incident_grid:       # one evaluation per distinct stagger pattern per cell, shared by ppc
        incident = incident * {1: 2, 2: 4, 3: 6}[D] / max(w.ppc, 1)
    move = 5 * D
    return gather + boris + deposit + incident + move


def bytes_per_push(w):
    """Algorithmic HBM bytes of one push: the particle record (cell, offsets, momenta, weight,
    id) read from one buffer set and written into its destination tile of the other, plus
    the field and current grid traffic shared by the ppc particles of a cell (E, B read
    once; J read-modify-write once)."""
    es = 4 if w.precision == synth.FP32 else 8
    part = 2 * (4 + w.dim * es + 3 * es + es + 4)
    grid = (6 * es + 2 * 3 * es) / max(w.ppc, 1)
    return part + grid


def shard(n, rank, world):
    """Items of a batch taken by one rank (round robin): independent simulations need no
    exchange between ranks, so the ranks are replicas over disjoint shares."""
    return list(range(rank, n, world))


def pushes_of(sim, s0, steps, n_end):
    """Pushes in the steps s0 .. s0+steps-1: every electron alive at the end was pushed in
    each of them, and one that left the box in step e (its exit record) in steps s0 .. e."""
    ex = sim.exits()["step"]
    ex = ex[(ex >= s0) & (ex < s0 + steps)]
    return float(n_end) * steps + float(np.sum(ex - s0 + 1))


def job_totals(pushes, secs, world, device=None):
    """Whole-job pushes (sum over ranks) and time (max over ranks)."""
    if world <= 1:
        return pushes, secs
    import torch

    t = torch.tensor([secs], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    p = torch.tensor([pushes], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(p)
    return float(p.item()), float(t.item())


def window_start(w, k, mode):
    """First timed step: the K-step window centred on the step at which the pulse peak
    crosses the focus (focused beams: t_focus; plane wave: the envelope centre at the slab
    centre), kept inside the run; 0 for mode "start" or when K covers the run."""
    if mode == "start" or k >= w.steps:
        return 0
    if w.beam == synth.BEAM_PLANE:
        t_c = w.duration + 0.5 * (w.slab_lo[0] + w.slab_hi[0]) * w.dx - w.focus[0]
    else:
        t_c = w.t_focus
    centre = int(round(t_c / w.dt))
    return max(0, min(w.steps - k, centre - k // 2))


def run_ours(args, rank, world, local_rank):
    import torch

    from paper_2310_11393_gb300 import _build, pic

    _build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = workload(args.workload)
    tile = [int(v) for v in args.tile.split(",")] if args.tile else None
    cfg = pic.config_from(w, tile=tile, sort_every=args.sort_every, chunk=args.chunk)
    stream = torch.cuda.current_stream(dev).cuda_stream
    alloc = pic.torch_allocator(local_rank)
    s0 = window_start(w, args.steps, args.window)
    # tile and work-item size: measured by the autotuner (untimed set-up)
    tune = {"trial_steps": args.autotune}
    if args.autotune > 0:
        t0 = time.perf_counter()
        tune["ms_per_step_trial"] = round(pic.pic_autotune(cfg, args.autotune, stream), 4)
        tune["seconds"] = round(time.perf_counter() - t0, 2)
    prm = pic.pic_derive_params(cfg)
    tune["push_tile"] = list(prm.tile)[: w.dim]
    tune["chunk"] = prm.chunk
    tune["field_solver_tile"] = list(prm.yee_tile)[: w.dim]
    tune["cell_sort_every"] = prm.sort_every
    # measured issue rates of this GPU (the fused push's arithmetic roofline)
    pk = pic.pic_probe_peaks(stream)
    # warm-up: W steps on a throw-away instance (clocks, caches, graph, launch attributes)
    warm = pic.Simulation(cfg, allocator=alloc, stream=stream)
    warm.step(args.warmup)
    torch.cuda.synchronize()
    warm.close()
    # the job: a fresh simulation (inputs resident in HBM), advanced untimed to the window's
    # first step, then K timed steps
    sim = pic.Simulation(cfg, allocator=alloc, stream=stream)
    if s0:
        sim.step(s0)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local_rank)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(torch.cuda.current_stream(dev))
    sim.step(args.steps)
    e1.record(torch.cuda.current_stream(dev))
    torch.cuda.synchronize()
    secs = e0.elapsed_time(e1) * 1e-3
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    n_b = sim.info().n_alive
    pushes = pushes_of(sim, s0, args.steps, n_b)
    tot_pushes, t_max = job_totals(pushes, secs, world, dev)
    info = sim.info()
    sim.close()
    # live per-kernel timing over the same window: another fresh instance advanced to the
    # same step, then K steps with CUDA events between the kernels of every step
    psim = pic.Simulation(cfg, allocator=alloc, stream=stream)
    if s0:
        psim.step(s0)
    snap = None
    if not args.no_e2e:      # the state at the window's start, for the end-to-end run
        # held as a user keeps a checkpoint: one contiguous host array per quantity
        parts = {k: np.ascontiguousarray(v) for k, v in psim.particles().items()}
        snap = (parts, np.ascontiguousarray(psim.fields()))
    nsteps_prof = args.steps if args.profile_steps <= 0 else min(args.steps, args.profile_steps)
    nwin = 10 if nsteps_prof >= 10 else 1
    prof = np.zeros(5)
    windows = []
    done = 0
    n_p0 = psim.info().n_alive
    for k in range(nwin):
        m = nsteps_prof * (k + 1) // nwin - done
        pw = pic.pic_profile_step(psim.h, m, stream)
        prof += pw
        windows.append({"steps": [s0 + done, s0 + done + m], "n_alive": int(psim.info().n_alive),
                        "ms_per_step": [round(x / m * 1e3, 4) for x in pw]})
        done += m
    n_c = psim.info().n_alive
    psim.close()
    push_s = prof[0] / nsteps_prof
    yee_s = prof[3] / nsteps_prof

    hbm, sm_max, src = peaks()
    npush = 0.5 * (n_p0 + n_c)
    fl = flops_per_push(w) * npush
    es = 4 if w.precision == synth.FP32 else 8
    if es == 4:
        alu_peak, alu_name = pk.fp32_tflops, "FP32"
    else:
        alu_peak, alu_name = pk.fp64_tflops, "FP64"
    alu_frac = fl / push_s / 1e12 / alu_peak
    by = bytes_per_push(w) * npush
    hbm_frac = by / push_s / 1e9 / hbm
    cells = w.n_cells
    yee_bytes = cells * (9 * es + 6 * es + 3 * es)           # read E, B, J; write E, B; clear J
    kname = "k_push1<%d,%s>" % (w.dim, "float" if es == 4 else "double")   # one simulation: k_push1
    traffic = PROFILED_TRAFFIC.get((w.name, kname))
    roof = {"bound": "alu", "achieved": round(fl / push_s / 1e12, 3), "peak": round(alu_peak, 2),
            "unit": "TFLOP/s", "frac": round(alu_frac, 4), "traffic": traffic[0] if traffic else None,
            "traffic_source": traffic[1] if traffic else None, "kernel": kname,
            "peak_source": f"measured: {alu_name} FMA-chain probe (pic_probe_peaks) over {pk.sms} SMs at "
                           f"{pk.sm_clock_mhz:.0f} MHz",
            "flop_per_push": flops_per_push(w),
            "probe": {"sms": pk.sms, "fp32_tflops": round(pk.fp32_tflops, 2), "fp64_tflops": round(pk.fp64_tflops, 3),
                      "sfu_gops": round(pk.sfu_gops, 1), "sm_clock_mhz": round(pk.sm_clock_mhz, 1),
                      "fp32_flop_per_clk_sm": round(pk.fp32_flop_per_clk_sm, 1)},
            "push_ms": round(push_s * 1e3, 4),
            "hbm_view": {"achieved_gbs": round(by / push_s / 1e9, 1), "peak_gbs": hbm, "peak_source": src,
                         "frac": round(hbm_frac, 4), "bytes_per_push": round(bytes_per_push(w), 2)},
            "yee": {"ms": round(yee_s * 1e3, 4), "achieved_gbs": round(yee_bytes / yee_s / 1e9, 1),
                    "frac_of_hbm": round(yee_bytes / yee_s / 1e9 / hbm, 4), "bytes_per_cell": 18 * es},
            "phases_ms": [round(x / nsteps_prof * 1e3, 4) for x in prof],
            "phases": ["push+deposit+placement", "tile scan", "cell-sort placement", "field solve", "step end"],
            "windows": windows}

    e2e = None
    if snap is not None:
        e2e = run_e2e(args, w, cfg, pic, torch, stream, alloc, snap, s0)
    out = {"metric": METRIC, "value": tot_pushes / t_max, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": t_max / args.steps * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32" if es == 4 else "f64", "data": "synthetic",
           "config": {"workload": w.name, "dim": w.dim, "grid": list(w.n[: w.dim]), "particles": w.n_particles,
                      "ppc": w.ppc, "beam": {1: "plane", 2: "LP", 3: "RP", 5: "Gaussian 2D"}[w.beam],
                      "precision": "fp32 body, fp64 phase" if es == 4 else "fp64",
                      "window": {"mode": args.window, "steps": [s0, s0 + args.steps], "run_steps": w.steps,
                                 "focus_step": int(round(w.t_focus / w.dt)) if w.beam != synth.BEAM_PLANE else None,
                                 "advanced_untimed": s0},
                      "cell_updates_per_s": cells * args.steps * world / t_max,
                      "l2": "inputs larger than L2 (device state %.2f GB > 129 MB)" % (info.params.device_bytes / 1e9),
                      "parallelism": f"replicas x{world}" if world > 1 else "single GPU", "tiles": tune},
           # kernels launched by the timed run: per step push, tile scan, field solve, step end
           # (+ the incident field on the grid; + cell count, cell scan and scatter on cell-sort
           # steps), and one k_prefix before the first step
           "roofline": roof, "clocks": clk, "gpu_launches": (5 if w.incident_grid else 4) * args.steps + 1
           + (3 * (args.steps // prm.sort_every) if prm.sort_every > 0 else 0), "e2e": e2e}
    return out


def run_e2e(args, w, cfg, pic, torch, stream, alloc, snap, s0):
    """Through the C-ABI with HOST buffers: the state at the window's first step (every
    particle and the six field components, as a user restores a checkpoint) goes host ->
    device, the K steps run, the energies and every particle's state come back device ->
    host, all inside the timed region."""
    parts, fields = snap
    x, u, wt, ids = parts["x"], parts["u"], parts["w"], parts["id"]
    sim = pic.Simulation(cfg, allocator=alloc, stream=stream)
    n = len(ids)
    es = 4 if w.precision == synth.FP32 else 8
    rec = 4 + 4 + w.dim * es + 3 * es + es          # cell, id, offsets, momenta, weight
    ext = [w.n[d] + 1 if d < w.dim else 1 for d in range(3)]
    npts = ext[0] * ext[1] * ext[2]
    h2d = n * rec + 6 * npts * es
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim.set_particles(x, u, wt, ids)
    sim.set_fields(fields)
    pic.pic_set_step(sim.h, s0, stream)
    sim.step(args.steps)
    en = sim.energies()
    out = sim.particles()
    t1 = time.perf_counter()
    n_end = len(out["id"])
    d2h = n_end * rec + 64
    pushes = pushes_of(sim, s0, args.steps, n_end)
    sim.close()
    return {"value": pushes / (t1 - t0), "unit": UNIT, "h2d_bytes_per_step": int(h2d / args.steps),
            "d2h_bytes_per_step": int(d2h / args.steps), "seconds": t1 - t0,
            "what": f"restore the state at step {s0} from host arrays (particles, E and B), {args.steps} steps, "
                    "energies and every particle back to the host",
            "energies": [float(v) for v in en[:4]]}


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform

    return platform.processor() or platform.machine()


def _oracle_worker(job):
    """One single-threaded oracle process: the sample workload with its own seed, `warm`
    untimed steps, then `steps` timed steps; returns (pushes, seconds)."""
    w, warm, steps = job
    sys.path.insert(0, ROOT)
    import oracle

    sim = oracle.Sim(oracle.config_from(w))
    if warm:
        sim.step(warm)
    t0 = time.perf_counter()
    sim.step(steps)
    t1 = time.perf_counter()
    # counted like the device runs: the electrons alive at the end every step, the ones that
    # left in steps warm .. e
    ex = sim.exits()["step"]
    ex = ex[ex >= warm]
    return float(sim.num_particles()) * steps + float(np.sum(ex - warm + 1)), t1 - t0


def oracle_all_cores(w, warm, steps):
    """The oracle as it stands on every host core at once: nproc single-threaded processes
    (spawned), each on its own seeded copy of the sample box w.  Returns (pushes/s of the
    whole host, per-process pushes/s, cores)."""
    import multiprocessing as mp

    import oracle

    oracle.build()
    cores = os.cpu_count() or 1
    jobs = [(w.with_(seed=w.seed + 7919 * k), warm, steps) for k in range(cores)]
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_worker, jobs)
    pushes = sum(r[0] for r in res)
    secs = max(r[1] for r in res)
    return pushes / secs, [r[0] / r[1] for r in res], cores


def cpu_baseline(w, nsteps=None):
    """The oracle on all host cores: one single-threaded process per core, each advancing
    its own seeded sample box of the workload (same physics and cell size) for nsteps
    steps from t = 0."""
    ws, f = reference_sample(w)
    if nsteps is None:
        nsteps = max(2, min(40, int(1.5e6 / max(ws.n_particles, 1))))
    v, per, cores = oracle_all_cores(ws, 0, nsteps)
    what = f"full {w.name} workload" if f == 1 else f"{w.name} box divided by {f} per axis"
    return {"value": v, "unit": UNIT, "cores": cores, "nproc": os.cpu_count(), "cpu_model": cpu_model(),
            "kind": "oracle",
            "sample": f"{cores} single-threaded oracle processes at once, each on its own seeded copy of the "
                      f"{what} ({ws.n_particles} electrons), {nsteps} steps from t = 0, FP64",
            "per_core_pushes_per_s": round(float(np.mean(per)), 1)}


def reference_sample(w, max_particles=80_000):
    """The workload on a box shrunk per axis (same cell size, physics and layout, slab and
    focus scaled with the box) until its electrons fit max_particles: one oracle step of it
    takes about 0.1 s, so --steps K of the full run's K stays within a few minutes."""
    f = 1
    while synth.scaled(w, f).n_particles > max_particles and f < 64:
        f += 1
    return synth.scaled(w, f) if f > 1 else w, f


def run_reference(args, rank, world):
    full = workload(args.workload)
    w, f = reference_sample(full)
    v, per, cores = oracle_all_cores(w, args.warmup, args.steps)
    what = f"full {w.name} workload" if f == 1 else f"{full.name} box divided by {f} per axis ({w.n_particles} electrons)"
    cb = {"value": v, "unit": UNIT, "cores": cores, "nproc": os.cpu_count(), "cpu_model": cpu_model(),
          "kind": "oracle",
          "sample": f"{cores} single-threaded oracle processes at once, each on its own seeded copy of the {what}, "
                    f"{args.steps} steps after {args.warmup} warm-up steps, FP64",
          "per_core_pushes_per_s": round(float(np.mean(per)), 1)}
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": cores * w.n_particles / v * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": full.name, "dim": full.dim, "grid": list(full.n[: full.dim]),
                       "particles": full.n_particles, "sample_grid": list(w.n[: w.dim]),
                       "sample_particles": w.n_particles, "sample_copies": cores},
            "cpu_baseline": cb, "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_batch(args, rank=0, world=1, local_rank=0):
    """Batched 2D workload: `--sims` independent runs of uneven size (LP/RP mix).  The same
    K steps of every simulation are timed (a) one simulation after another, each through its
    own step graph, and (b) all together through pic_batch_step (one persistent launch per
    phase over every simulation's work, one graph)."""
    import torch

    from paper_2310_11393_gb300 import _build, pic

    _build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    ws_all = synth.c4_batch(args.sims)
    ws = [ws_all[i] for i in shard(len(ws_all), rank, world)]
    stream = torch.cuda.current_stream().cuda_stream
    K = args.steps
    out = {}
    c0 = pic.config_from(ws[0])
    if args.autotune > 0:
        pic.pic_autotune(c0, args.autotune, stream)
    tile, chunk = list(c0.tile), c0.chunk
    chunk_of = {"plain": chunk, "batched": chunk}

    def cfg_of(w, mode):
        tuned = args.autotune > 0
        return pic.config_from(w, tile=tile if tuned else None, chunk=chunk_of[mode] if tuned else 0)

    if args.autotune > 0:
        # the work-item size of each arm, measured the same way on the batch itself (untimed
        # set-up): the tuner's choice for one small member is not the best for the batch,
        # and both arms get the same search
        for mode in ("plain", "batched"):
            trial = []
            for ch in sorted({chunk, 512, 1024, 2048}):
                chunk_of[mode] = ch
                sims = [pic.Simulation(cfg_of(w, mode), stream=stream) for w in ws]
                if mode == "plain":
                    for s in sims:
                        s.step(max(args.warmup, 2))
                else:
                    pic.pic_batch_step([s.h for s in sims], max(args.warmup, 2), stream)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                if mode == "plain":
                    for s in sims:
                        s.step(5)
                else:
                    pic.pic_batch_step([s.h for s in sims], 5, stream)
                torch.cuda.synchronize()
                trial.append((time.perf_counter() - t0, ch))
                for s in sims:
                    s.close()
            chunk_of[mode] = min(trial)[1]

    for mode in ("plain", "batched"):
        sims = [pic.Simulation(cfg_of(w, mode), stream=stream) for w in ws]
        n0 = sum(s.info().n_alive for s in sims)
        # warm-up (graphs, attributes, batch graph capture)
        if mode == "plain":
            for s in sims:
                s.step(args.warmup)
        else:
            pic.pic_batch_step([s.h for s in sims], args.warmup, stream)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        if mode == "plain":
            for s in sims:
                s.step(K)
        else:
            pic.pic_batch_step([s.h for s in sims], K, stream)
        e1.record()
        torch.cuda.synchronize()
        secs = e0.elapsed_time(e1) * 1e-3
        n1 = sum(s.info().n_alive for s in sims)
        pushes, secs = job_totals(0.5 * (n0 + n1) * K, secs, world, dev)
        # the same K steps once more, phase by phase (events between the phases; every
        # phase launched on its own, so the sum exceeds the graph's step time)
        if mode == "plain":
            ph = np.zeros(5)
            for s in sims:
                ph += pic.pic_profile_step(s.h, K, stream)
        else:
            ph = pic.pic_batch_profile_step([s.h for s in sims], K, stream)
        n2 = sum(s.info().n_alive for s in sims)
        out[mode] = {"pushes_per_s": pushes / secs, "seconds": secs,
                     "phases_ms_per_step": [round(x / K * 1e3, 4) for x in ph],
                     "push_phase_pushes_per_s": 0.5 * (n1 + n2) * K / ph[0] if ph[0] > 0 else None}
        for s in sims:
            s.close()
    cells = sum(w.n_cells for w in ws_all)
    ratio = out["batched"]["pushes_per_s"] / out["plain"]["pushes_per_s"]
    return {"metric": "batched particle-pushes/s (256 uneven 2D runs)", "value": out["batched"]["pushes_per_s"],
            "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "strong", "parallelism": f"replicas x{world}, simulations round robin" if world > 1 else "single GPU",
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"batch2d_{len(ws_all)}", "sims": len(ws_all), "cells": cells,
                       "tiles": {"push_tile": tile[:2], "chunk_plain": chunk_of["plain"],
                                 "chunk_batched": chunk_of["batched"], "tile_autotuned_on": ws[0].name,
                                 "chunks_measured_on": "the batch, both arms (512..2048)"}
                       if args.autotune > 0 else "defaults",
                       "particles": int(sum(w.n_particles for w in ws_all)),
                       "sample": f"steps {args.warmup}..{args.warmup + K} of each 500-step run"},
            "phases": ["push+deposit+placement", "tile scan", "cell-sort placement", "field solve", "step end"],
            "plain": out["plain"], "batched": out["batched"], "batched_over_plain": ratio}


def _serve_stream(args, pic, torch, reqs, plain=True):
    """The request stream `reqs` ((arrival s, Workload) pairs) through pic_serve_*, and (plain)
    the same requests back to back on one stream, arrival times honoured in both."""
    out = {}
    if plain:
        stream = torch.cuda.current_stream().cuda_stream
        t0 = time.perf_counter()
        lat_plain, pushes = [], 0
        for (ta, w) in reqs:
            now = time.perf_counter() - t0
            if now < ta:
                time.sleep(ta - now)
            s = pic.Simulation(pic.config_from(w), stream=stream)
            done = 0
            while done < w.steps:          # electrons leave the box: count them as the server does
                k = min(50, w.steps - done)
                pushes += s.info().n_alive * k
                s.step(k)
                done += k
            s.energies()
            s.close()
            lat_plain.append(time.perf_counter() - t0 - ta)
        plain_secs = time.perf_counter() - t0
        out["plain"] = {"p50_s": float(np.percentile(lat_plain, 50)), "p99_s": float(np.percentile(lat_plain, 99)),
                        "pushes_per_s": pushes / plain_secs, "makespan_s": plain_secs}
    srv = pic.pic_serve_open(quantum=50)
    t0 = pic.pic_serve_clock(srv)
    w0 = time.perf_counter()
    tickets = []
    for (ta, w) in reqs:
        now = time.perf_counter() - w0
        if now < ta:
            time.sleep(ta - now)
        tickets.append(pic.pic_serve_submit(srv, pic.config_from(w), w.steps))
    res = {}
    while len(res) < len(tickets):
        for t in tickets:
            if t in res:
                continue
            st, r = pic.pic_serve_poll(srv, t)
            if st != pic.PIC_EBUSY:
                res[t] = (st, r)
        time.sleep(0.005)
    served_secs = pic.pic_serve_clock(srv) - t0
    pic.pic_serve_close(srv)
    lat = [r.finish_time - r.submit_time for (st, r) in res.values()]
    spushes = sum(r.pushes for (st, r) in res.values())
    out["served"] = {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                     "pushes_per_s": spushes / served_secs,
                     "completed": sum(1 for (st, r) in res.values() if st == pic.PIC_OK), "makespan_s": served_secs,
                     "requests_per_s": len(reqs) / served_secs,
                     "steps_done": int(sum(r.steps_done for (st, r) in res.values())),
                     "steps_requested": int(sum(w.steps for _, w in reqs))}
    if plain:
        out["served_over_plain"] = out["served"]["pushes_per_s"] / out["plain"]["pushes_per_s"]
    return out


def run_serve(args):
    """Served parameter scan: a Poisson stream of 2D (256-1024^2) and 3D (128-256^3) RP runs of
    500-2000 steps submitted to pic_serve, time-to-result p50/p99 and aggregate pushes/s, next
    to the same requests run back to back on one stream.  First at the configured mean rate
    (20/s, far above the device's capacity: the queue grows for the whole run), then at 0.7
    times the capacity that run measured (requests completed per second), where time to
    result is the service time plus a finite wait."""
    import torch

    from paper_2310_11393_gb300 import _build, pic

    _build.build()
    torch.cuda.set_device(0)
    reqs = synth.c5_requests(args.requests, rate_hz=args.rate, steps_range=(500, 2000))
    over = _serve_stream(args, pic, torch, reqs)
    cap = over["served"]["requests_per_s"]
    rate2 = 0.7 * cap
    reqs2 = synth.c5_requests(args.requests, rate_hz=rate2, steps_range=(500, 2000))
    under = _serve_stream(args, pic, torch, reqs2)
    n3 = sum(1 for _, w in reqs if w.dim == 3)
    return {"metric": "served time-to-result p50/p99 and pushes/s", "value": over["served"]["pushes_per_s"],
            "unit": UNIT, "higher_is_better": True, "n_gpus": 1, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "served_scan", "requests": len(reqs), "requests_3d": n3,
                       "sizes": "2D 256-1024^2 or 3D 128-256^3 (clipped log-normal), RP a0 = 20, 500-2000 steps",
                       "rates_hz": [args.rate, rate2]},
            "at_configured_rate": over, "at_0.7_capacity": under, "capacity_requests_per_s": cap}


def relaunch_ranks(args):
    """--gpus N > 1 without a launcher: start N ranks of this command under
    torch.distributed.run on this node (127.0.0.1) and return its exit code."""
    import socket

    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        port = so.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={args.gpus}",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__)] + sys.argv[1:]
    return subprocess.call(cmd)


def main():
    args = parse()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        sys.exit(relaunch_ranks(args))
    global SCALE, INCIDENT_GRID, SLAB_CELLS
    SCALE = max(1, args.scale)
    SLAB_CELLS = max(0, args.slab_cells)
    INCIDENT_GRID = 1 if args.incident == "grid" else 0
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if args.steps <= 0:
            args.steps = workload(args.workload).steps
        if rank == 0:
            print(json.dumps(run_reference(args, rank, world)))
        return
    if world > 1:
        import torch

        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    if args.workload in ("batch", "serve"):
        if args.workload == "batch":
            args.steps = args.steps if args.steps > 0 else 100
            out = run_batch(args, rank, world, local_rank)
        else:
            out = run_serve(args)
        if rank == 0:
            print(json.dumps(out))
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    if args.steps <= 0:
        args.steps = workload(args.workload).steps
    out = run_ours(args, rank, world, local_rank)
    if rank == 0:
        run_cb = world == 1 and not args.no_cpu_baseline
        out["cpu_baseline"] = cpu_baseline(workload(args.workload)) if run_cb else None
        print(json.dumps(out))
    if world > 1:
        import torch

        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
