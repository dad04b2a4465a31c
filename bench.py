"""Benchmark of the hybrid nodal-staggered PSATD PIC step on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl libpic|reference] [--workload NAME]

Default workload: the beam-driven wakefield box, the largest single-GPU workload (256 x 256 x 1024
cells, dx = dy = 0.1, dz = 0.02, dt = dz/c, averaged Galilean PSATD with v_gal = the beam velocity,
spectral order 16, centering (8, 8, 16), cubic shape; a cold plasma at 1 electron per cell
(67,108,864) plus a 1,000,000-particle Gaussian driver at gamma = 1000).  One step = one full hybrid
cycle (gather, push, deposit, centering, FFTs, PSATD update) through pic_step32 (FP32 form, the
headline value) and, in the same run, pic_step (plain FP64 form, reported beside it with the
FP32/FP64 ratio).  The other workloads (thermal plasma 32^3, laser wakefield 128 x 128 x 512,
drifting pair plasma 64 x 64 x 256, and the differentiable probe problem 64^3: forward plus
gradient) are timed after it and reported under "workloads".  Prints one JSON line.

--impl libpic (default): K steps of pic_step timed with CUDA events on the library's stream after
W warm-up steps; value = particle-steps/s over all ranks.  Under torchrun each rank runs an
independent replica of the workload (replicas only: the single-GPU periodic step has no data
exchange).
--impl reference: the FP64 CPU oracle on every core of this host (one process per core, each on
its own bounded sample box of the same workload), rank 0 only.
"""
import argparse
import datetime
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2106_12919_gb300 import workloads  # noqa: E402

METRIC = "particle-steps/s (full hybrid PIC step) vs plain FP64 form; % of HBM roofline"
UNIT = "particle-steps/s"
DEFAULT_WORKLOAD = "beam_wakefield"
HBM_PEAK_FALLBACK = 6800.0
# FP64 FMA units: 152 SMs x 4 FP64 flop/clk/SM x 2.070 GHz (nominal 1.25 TFLOP/s class figure)
FP64_PEAK_TFLOPS = 152 * 4 * 2.070e9 / 1e12
# DRAM bytes (read + write) of the push stage per step (every species' push32_tile launch), from one
# ncu capture of the current kernel version: at the full laser-wakefield size, and for the
# beam-driven box on a 128 x 128 x 512 box of the same physics scaled by 8 (particles and cells);
# other workloads / forms report null
MEASURED_TRAFFIC = {("beam_wakefield", (256, 256, 1024), "fp32"): 7.611e9,
                    ("laser_wakefield", (128, 128, 512), "fp32"): 1.4945e9}
# LSU data-pipe wavefronts (shared memory, L1, global) of the push stage per step, same captures:
# the pipe that bounds the particle kernel on chip issues one wavefront per SM per cycle
MEASURED_LSU_WAVEFRONTS = {("beam_wakefield", (256, 256, 1024), "fp32"): 2.073e9,
                           ("laser_wakefield", (128, 128, 512), "fp32"): 4.761e8}
N_SM = 152
# CPU-oracle samples: the same workload on a smaller box (same dx, dt, physics)
SAMPLE_SHAPE = {"laser_wakefield": (32, 32, 128), "beam_wakefield": (32, 32, 128),
                "thermal_plasma": (16, 16, 32), "galilean_drift": (32, 32, 64), "seed_wave": (32, 32, 32)}
FULL_SHAPE = {"laser_wakefield": (128, 128, 512), "beam_wakefield": (256, 256, 1024),
              "thermal_plasma": (32, 32, 32), "galilean_drift": (64, 64, 256), "seed_wave": (64, 64, 64)}
# particle tile per workload (pic_ext.tile), from sweeps on one GB300 with the final kernels: at 1
# particle per cell (beam-driven box) 8 x 16 x 8 beats 8 x 8 x 8 (push 8.70 against 8.94 ms per
# step; 16 x 8 x 8 9.01, 16 x 16 x 8 9.84); at 2 per cell (laser-wakefield box) 8 x 8 x 8 is best
TILE = {"beam_wakefield": (8, 16, 8)}
# the other workloads, timed after the headline one: (name, forms)
EXTRA_WORKLOADS = (("thermal_plasma", ("fp64", "fp32")), ("laser_wakefield", ("fp32", "fp64")),
                   ("galilean_drift", ("fp32", "fp64")))


def push_flops_per_particle(order):
    """Algorithmic FP64 flops of the gather + Boris + move + deposit of one particle.

    gather 12 S^3 (6 fields x S^3 nodes x FMA) + S^3 weight products, J deposit
    7 S^3 (weight, 3 products, 3 adds), rho deposit 2 S^3, shapes/Boris/move 250;
    S = order + 1.
    """
    S3 = (order + 1) ** 3
    return 22 * S3 + 250


def make_workload(name, shape=None, seed=None):
    f = workloads.WORKLOADS[name]
    kw = {}
    if shape is not None:
        kw["shape"] = tuple(shape)
        if name == "beam_wakefield":
            kw["n_beam"] = max(1000, int(1_000_000 * np.prod(shape) / np.prod(FULL_SHAPE[name])))
    if seed is not None:
        kw["seed"] = seed
    return f(**kw)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return None


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 50 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,timestamp")

    def __init__(self, device):
        self.device = device
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self, window=None):
        """Median SM clock and the throttle reasons seen; with window = (t0, t1) (host wall
        clock of the timed region) only the samples taken inside it, when there are any."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        rows = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(f[9], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        inside = [r for r in rows if window and window[0] - 0.025 <= r[0] <= window[1] + 0.025]
        use = inside or rows
        reasons = {n for r in use for n, v in zip(names, r[3]) if v.lower().startswith("active")}
        sm = [r[1] for r in use]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(r[2] for r in use) if use else None, "reasons": sorted(reasons),
                "samples": len(sm), "in_timed_region": bool(inside)}


def max_over_ranks(x, world, device="cuda"):
    """The largest value of x over the ranks of the job (replicas: the slowest rank sets the
    time); x itself when running alone."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, steps, world, ms_max):
    """Whole-job units per second: every rank processed units_per_rank per step (weak scaling,
    independent replicas) and the job took the slowest rank's time."""
    return units_per_rank * steps * world / (ms_max * 1e-3)


# ---------------------------------------------------------------------------------------------
# the oracle on the host's cores (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------------------------

def run_oracle_sample(name, warmup, steps, seed, barrier, results):
    """One worker process: the oracle (FP64 CPU, single-threaded) on its own sample box of the
    workload; warm-up steps, then the timed steps once every worker is ready.  Puts (particles,
    steps, seconds) on the results queue."""
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    from oracle import step
    w = make_workload(name, SAMPLE_SHAPE[name], seed=seed)
    p = step.Params(**w["params"])
    st = {"E": w["E"], "B": w["B"], "species": w["species"]}
    st["rho"] = step.initial_rho(p, st["species"])
    npart = sum(s["x"].size for s in w["species"])
    for _ in range(warmup):
        step.hybrid_step(p, st)
    barrier.wait()
    t0 = time.perf_counter()
    for _ in range(steps):
        step.hybrid_step(p, st)
    results.put((npart, steps, time.perf_counter() - t0))


def oracle_on_host(name, warmup, steps, cores=None):
    """The oracle on `cores` worker processes (default: every core this process may run on), each
    on an independent sample box (own seed) of the workload.  Returns (particle-steps/s of all
    workers together over the slowest worker's time, seconds, cores, sample description)."""
    import multiprocessing as mp
    cores = cores or len(os.sched_getaffinity(0))
    ctx = mp.get_context("spawn")          # never fork a process that may hold a CUDA context
    barrier = ctx.Barrier(cores)
    results = ctx.Queue()
    procs = [ctx.Process(target=run_oracle_sample, args=(name, warmup, steps, 7000 + i, barrier, results))
             for i in range(cores)]
    for pr in procs:
        pr.start()
    out = [results.get() for _ in procs]
    for pr in procs:
        pr.join()
    secs = max(o[2] for o in out)
    total = sum(o[0] * o[1] for o in out)
    shape = SAMPLE_SHAPE[name]
    desc = ("%d worker processes (one per host core), each %d step(s) of the oracle (FP64, single-threaded "
            "numpy) on its own %dx%dx%d sample box of the workload (%d particles, same dx/dt/physics, own "
            "seed), after %d warm-up step(s); value = all workers' particle-steps / the slowest worker's time"
            % (cores, steps, shape[0], shape[1], shape[2], out[0][0], warmup))
    return total / secs, secs, cores, desc


# particles per cell of each generator's default (the drifting pair plasma: 2 electrons + 2 positrons)
PPC = {"thermal_plasma": 8, "laser_wakefield": 2, "galilean_drift": 4, "seed_wave": 4, "beam_wakefield": 1}


def workload_config(name, world, shape=None):
    """The config block of a workload's bench line (its full size unless shape is given), without
    generating its particles."""
    shape = tuple(shape) if shape else FULL_SHAPE[name]
    ncell = int(np.prod(shape))
    npart = PPC[name] * ncell + (max(1000, int(1_000_000 * ncell / np.prod(FULL_SHAPE[name])))
                                 if name == "beam_wakefield" else 0)
    small = make_workload(name, (16, 16, 16))["params"]
    return {"workload": name, "grid": list(shape), "particles": npart, "shape_order": small["shape_order"],
            "centering_order": list(small["centering_order"]), "variant": small["variant"],
            "parallelism": "replicas" if world > 1 else "single"}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    value, secs, cores, desc = oracle_on_host(args.workload, args.warmup, args.steps)
    config = workload_config(args.workload, world, args.grid)
    config["form"] = "fp64"
    config["note"] = "the oracle is FP64; the libpic arm's headline value is its FP32 form on this config"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------------
# the library on the GPU
# ---------------------------------------------------------------------------------------------

def cufft_reference(shape, dtype, libpic_ms):
    """cuFFT (through torch.fft) on the step's transform load, timed as a reference only:
    4 forward R2C (J, rho) and 6 inverse C2R (nodal E, B) 3D transforms of the grid."""
    import torch
    x = torch.randn((4,) + tuple(shape), dtype=dtype, device="cuda")
    y = torch.randn((6,) + tuple(shape), dtype=dtype, device="cuda")
    dims = (1, 2, 3)
    Ys = torch.fft.rfftn(y, dim=dims)
    del y
    for _ in range(3):
        torch.fft.rfftn(x, dim=dims)
        torch.fft.irfftn(Ys, s=tuple(shape), dim=dims)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    e0.record()
    for _ in range(reps):
        torch.fft.rfftn(x, dim=dims)
        torch.fft.irfftn(Ys, s=tuple(shape), dim=dims)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / reps
    del x, Ys
    torch.cuda.empty_cache()
    return {"cufft_ms_per_step": ms, "libpic_fft_ms_per_step": libpic_ms,
            "note": "cuFFT via torch.fft: 4 R2C + 6 C2R 3D transforms of the grid per step, reference only"}


def setup_form(form, w, stream, tile=(8, 8, 8)):
    """Context and device state of one form on the workload (inputs resident in HBM)."""
    import torch
    from paper_2106_12919_gb300 import pic
    p = w["params"]
    ncell = int(np.prod(p["shape"]))
    fp32 = form == "fp32"
    ctx = pic.Context(p["shape"], p["dx"], p["dt"], p["shape_order"], p["centering_order"], p["variant"], p["v_gal"],
                      p["spectral_order"], p["c"], p["eps0"], stream=stream, tile=tuple(tile),
                      precision=pic.PIC_FP32 if fp32 else pic.PIC_FP64)
    tdt = torch.float32 if fp32 else torch.float64
    with torch.cuda.stream(stream):
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda", tdt).reshape(-1)
        E = [dev(a) for a in w["E"]]
        B = [dev(a) for a in w["B"]]
        J = [torch.zeros(ncell, dtype=tdt, device="cuda") for _ in range(3)]
        rho = torch.zeros(ncell, dtype=tdt, device="cuda")
        sp = []
        for s in w["species"]:
            if fp32:
                sp.append(pic.Species32.from_positions(ctx, s["x"], s["y"], s["z"], s["ux"], s["uy"], s["uz"], s["w"],
                                                       s["q"], s["m"]))
            else:
                d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
                sp.append(pic.Species(d(s["x"]), d(s["y"]), d(s["z"]), d(s["ux"]), d(s["uy"]), d(s["uz"]), d(s["w"]),
                                      s["q"], s["m"]))
    torch.cuda.synchronize()
    return ctx, E, B, J, rho, sp


def time_steps(ctx, step, E, B, J, rho, sp, steps, warmup, world, local):
    """W warm-up steps, then K steps in one call timed with CUDA events on the library's stream
    (barrier + synchronize on both sides), with the clocks sampled during the timed region."""
    import torch
    import torch.distributed as dist
    step(E, B, J, rho, sp, warmup)
    ctx.sync()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ctx.timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    w0 = time.time()
    e0.record(ctx.stream)
    step(E, B, J, rho, sp, steps)
    e1.record(ctx.stream)
    e1.synchronize()
    torch.cuda.synchronize()
    w1 = time.time()
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    clocks = sampler.stop((w0, w1))
    stage = {s: ctx.timing_read(s) for s in ("push", "fft", "update", "bin", "other", "all")}
    ctx.timing(False)
    return max_over_ranks(ms, world), clocks, stage


def e2e_roundtrip(ctx, fp32, E, B, rho, sp, steps, world, use_graph=True, copy_streams=1, nbuf=3):
    """End to end through the public API with host buffers: every step copies its whole input
    state (E, B, rho and every particle array) from pinned host memory, runs pic_step(1) and copies
    the whole advanced state (E, B, rho, particles) back into pinned host memory.  nbuf device
    copies of the state rotate, so that the input copy of the next step and the output copy of the
    previous one (own streams) overlap a step."""
    import torch
    from paper_2106_12919_gb300 import pic
    stream = ctx.stream
    devs = E + B + [rho] + [a for s in sp for a in s.arrays()]
    host_in = [t.cpu().pin_memory() for t in devs]
    host_out = [torch.empty(h.shape, dtype=h.dtype, pin_memory=True) for h in host_in]
    nbytes = sum(h.numel() * h.element_size() for h in host_in)
    sets = [(E, B, rho, sp)]
    for _ in range(nbuf - 1):
        E2 = [torch.empty_like(t) for t in E]
        B2 = [torch.empty_like(t) for t in B]
        rho2 = torch.empty_like(rho)
        sp2 = []
        for s in sp:
            arrs = [torch.empty_like(a) for a in s.arrays()]
            sp2.append(pic.Species32(*arrs[:8], s.q, s.m) if fp32 else pic.Species(*arrs[:7], s.q, s.m))
        sets.append((E2, B2, rho2, sp2))
    bufs = [Eb + Bb + [rb] + [a for s in spb for a in s.arrays()] for Eb, Bb, rb, spb in sets]
    h2d_streams = [torch.cuda.Stream() for _ in range(copy_streams)]
    d2h_stream = torch.cuda.Stream()
    copied = [[torch.cuda.Event() for _ in h2d_streams] for _ in range(nbuf)]
    done = [torch.cuda.Event() for _ in range(nbuf)]        # step on set b finished
    read = [torch.cuda.Event() for _ in range(nbuf)]        # set b copied back to the host

    def enqueue_h2d(k):
        b = k % nbuf
        for i, cs in enumerate(h2d_streams):
            with torch.cuda.stream(cs):
                cs.wait_event(read[b])                     # set b's previous result has left the device
                for d, h in list(zip(bufs[b], host_in))[i::len(h2d_streams)]:
                    d.copy_(h, non_blocking=True)
                copied[b][i].record(cs)

    def enqueue_d2h(k):
        b = k % nbuf
        with torch.cuda.stream(d2h_stream):
            d2h_stream.wait_event(done[b])
            for d, h in zip(bufs[b], host_out):
                h.copy_(d, non_blocking=True)
            read[b].record(d2h_stream)

    step = ctx.step32 if fp32 else ctx.step
    graphs = []
    if use_graph:
        capture = ctx.capture_step32 if fp32 else ctx.capture_step
        for b in range(nbuf):
            for d, h in zip(bufs[b], host_in):
                d.copy_(h)
            Eb, Bb, rb, spb = sets[b]
            graphs.append(capture(Eb, Bb, None, rb, spb, 1))
    for ev in done + read:
        ev.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    enqueue_h2d(0)
    for k in range(steps):
        if k + 1 < steps:
            enqueue_h2d(k + 1)
        b = k % nbuf
        Eb, Bb, rb, spb = sets[b]
        for ev in copied[b]:
            stream.wait_event(ev)
        if graphs:
            with torch.cuda.stream(stream):
                graphs[b].replay()                          # pic_step(1) on set b, J = NULL
        else:
            step(Eb, Bb, None, rb, spb, 1)                  # J^{n+1/2} is not part of the result: J = NULL
        done[b].record(stream)
        enqueue_d2h(k)
    stream.wait_stream(d2h_stream)
    t1.record(stream)
    t1.synchronize()
    ms = max_over_ranks(t0.elapsed_time(t1), world)
    npart = sum(s.n for s in sp)
    out = {"value": job_throughput(npart, steps, world, ms), "unit": UNIT, "h2d_bytes_per_step": nbytes,
           "d2h_bytes_per_step": nbytes, "steps": steps,
           "note": "per step: pinned H2D of E, B, rho and every particle array, pic_step(1) (%s), D2H of the "
                   "whole advanced state (E, B, rho, particles) into pinned host memory; %d device copies of "
                   "the state rotate so that the copies overlap the neighbouring steps" %
                   ("replayed as a CUDA graph, pic.StepGraph" if graphs else "direct call", nbuf)}
    del graphs, sets, bufs, host_in, host_out
    return out


def push_roofline(w, fp32, stage, steps, npart, ncell, clocks, hbm):
    """Roofline of the push stage (gather + Boris + move + deposit: per species and step one push
    launch in the FP64 form; in the FP32 form two, of which the one matching the species' tile-frame
    velocity works and the other returns at once) against its algorithmic bytes (FP32) or flops
    (FP64) per step."""
    p = w["params"]
    shape = tuple(p["shape"])
    push_ms, push_n = stage["push"]
    push_s_per_step = push_ms * 1e-3 / steps
    per_launch_s = push_ms * 1e-3 / max(push_n, 1)
    name = w["name"].rsplit("_", 1)[0]
    if fp32:
        # 32 B read + 28 B written per particle; nodal E, B read (24 B) and J, rho deposited (16 B) per cell
        nbytes = 60 * npart + 40 * ncell
        achieved = nbytes / push_s_per_step / 1e9
        traffic = MEASURED_TRAFFIC.get((name, shape, "fp32"))
        roof = {"kernel": "push32_tile_kernel (gather + Boris + deposit), all species' launches of a step",
                "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": traffic, "algorithmic_bytes": "60 B/particle + 40 B/cell per step (%.4g B)" % nbytes,
                "launches_per_step": push_n / steps, "working_launches_per_step": push_n / steps / 2,
                "avg_working_launch_ms": 2 * per_launch_s * 1e3}
        wf = MEASURED_LSU_WAVEFRONTS.get((name, shape, "fp32"))
        if wf is not None:
            mhz = clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or 2070.0
            peak_wf = N_SM * mhz * 1e6
            roof["onchip"] = {"bound": "lsu", "unit": "wavefronts/s", "achieved": wf / push_s_per_step,
                              "peak": peak_wf, "frac": wf / push_s_per_step / peak_wf, "wavefronts_per_step": wf,
                              "note": "LSU data-pipe wavefronts of the push stage per step from one ncu capture; "
                                      "peak = 152 SMs x 1 wavefront/cycle x median SM clock in the timed region"}
        return roof
    flops = push_flops_per_particle(p["shape_order"]) * npart
    achieved = flops / push_s_per_step / 1e12
    return {"kernel": "push_kernel (gather + Boris + deposit), all species' launches of a step", "bound": "alu",
            "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
            "traffic": None, "algorithmic_flops": "22 (p+1)^3 + 250 per particle",
            "hbm_frac": 104 * npart / push_s_per_step / 1e9 / hbm}


def run_form(form, w, args, world, rank, local, full=True):
    """Time K steps of one form (fp32 | fp64) of the step on the workload; with full=True also the
    end-to-end round trip, the push roofline and cuFFT on the same transform load."""
    import torch
    p = w["params"]
    ncell = int(np.prod(p["shape"]))
    fp32 = form == "fp32"
    stream = torch.cuda.Stream()
    tile = args.tile or TILE.get(w["name"].rsplit("_", 1)[0], (8, 8, 8))
    ctx, E, B, J, rho, sp = setup_form(form, w, stream, tile)
    npart = sum(s.n for s in sp)
    step = ctx.step32 if fp32 else ctx.step
    (ctx.deposit_rho32 if fp32 else ctx.deposit_rho)(sp, rho)
    ms, clocks, stage = time_steps(ctx, step, E, B, J, rho, sp, args.steps, args.warmup, world, local)
    out = {"value": job_throughput(npart, args.steps, world, ms), "ms": ms, "npart": npart, "clocks": clocks,
           "stage_ms": {k: v[0] / args.steps for k, v in stage.items() if k != "all"},
           "launches": stage["all"][1],
           "cell_updates_per_s": job_throughput(ncell, args.steps, world, ms)}
    if full:
        peaks = measured_peaks()
        hbm = (peaks or {}).get("hbm_gbs", HBM_PEAK_FALLBACK)
        out["roofline"] = push_roofline(w, fp32, stage, args.steps, npart, ncell, clocks, hbm)
        ke = args.e2e_steps or (max(3, min(args.steps, 10)) if fp32 else 3)
        out["e2e"] = e2e_roundtrip(ctx, fp32, E, B, rho, sp, ke, world, not args.e2e_no_graph,
                                   args.e2e_copy_streams, args.e2e_buffers)
        esz = 4 if fp32 else 8
        resident = (10 * ncell * esz + sum(sum(a.numel() * a.element_size() for a in s.arrays()) for s in sp)
                    + 40 * ncell * esz) / 1e9
        out["bytes_resident"] = resident
        out["fft_reference"] = cufft_reference(p["shape"], torch.float32 if fp32 else torch.float64,
                                               stage["fft"][0] / args.steps)
    ctx.close()
    del E, B, J, rho, sp
    torch.cuda.empty_cache()
    return out


def run_adjoint(args, world):
    """The differentiable probe problem (64^3, 1M particles, CIC, 50 steps, checkpoint every 10):
    one forward pass and one gradient of the probe energy w.r.t. the seed amplitude's field and all
    initial momenta (torch.autograd over pic_step / pic_adjoint_step), timed with CUDA events."""
    import torch
    from paper_2106_12919_gb300 import adjoint as gadj
    from paper_2106_12919_gb300 import pic
    w = make_workload("seed_wave")
    p = w["params"]
    ctx = pic.Context(p["shape"], p["dx"], p["dt"], p["shape_order"], p["centering_order"], p["variant"], p["v_gal"],
                      p["spectral_order"], p["c"], p["eps0"], sort_interval=0)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda().reshape(-1)
    s = w["species"][0]
    sp = pic.Species(d(s["x"]), d(s["y"]), d(s["z"]), d(s["ux"]), d(s["uy"]), d(s["uz"]), d(s["w"]), s["q"], s["m"])
    lo, hi = w["probe"]
    run = gadj.Rollout(ctx, [sp], w["steps"], lo, hi, checkpoint=10)
    E0 = torch.stack([d(a) for a in w["E"]]).requires_grad_(True)
    B0 = torch.stack([d(a) for a in w["B"]]).requires_grad_(True)
    u = [sp.ux.clone().requires_grad_(True), sp.uy.clone().requires_grad_(True), sp.uz.clone().requires_grad_(True)]

    def once():
        loss = gadj.ProbeEnergy.apply(E0, B0, u[0], u[1], u[2], run)
        loss.backward()
        return loss

    once()                                           # warm-up (allocations, first binning)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    reps = 2
    for _ in range(reps):
        once()
    e1.record()
    e1.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1) / reps, world)
    n = sp.n
    ctx.close()
    del E0, B0, u, sp, run
    torch.cuda.empty_cache()
    return {"forward_plus_gradient_ms": ms, "steps": w["steps"], "checkpoint": 10, "particles": n,
            "grid": list(p["shape"]),
            "forward_particle_steps_per_s": job_throughput(n, w["steps"], world, ms),
            "note": "one forward pass of 50 FP64 steps plus the reverse pass (segments recomputed from "
                    "checkpoints every 10 steps, pic_adjoint_step per step) per gradient"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="libpic", choices=["libpic", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(workloads.WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="time the headline workload only")
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--e2e-copy-streams", type=int, default=1,
                    help="streams the per-step host-to-device input copies are spread over")
    ap.add_argument("--e2e-buffers", type=int, default=3,
                    help="device copies of the state that rotate in the end-to-end loop")
    ap.add_argument("--e2e-no-graph", action="store_true",
                    help="end-to-end loop with direct pic_step calls instead of their CUDA graphs")
    ap.add_argument("--form", default="both", choices=["both", "fp32", "fp64"],
                    help="both: FP32 form timed as the headline, FP64 form beside it")
    ap.add_argument("--tile", type=int, nargs=3, default=None, metavar=("TX", "TY", "TZ"),
                    help="particle tile edge in cells (pic_ext.tile); default: the workload's (TILE)")
    ap.add_argument("--grid", type=int, nargs=3, default=None, metavar=("NX", "NY", "NZ"),
                    help="run the workload's generator on a smaller box (same dx, dt, physics), e.g. for profiling")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return reference_arm(args)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__
    __graft_entry__.build()

    w = make_workload(args.workload, args.grid)
    p = w["params"]
    shape = p["shape"]
    forms = ["fp32", "fp64"] if args.form == "both" else [args.form]
    res = {f: run_form(f, w, args, world, rank, local) for f in forms}
    head = res[forms[0]]
    value = head["value"]
    peaks = measured_peaks()
    hbm = (peaks or {}).get("hbm_gbs", HBM_PEAK_FALLBACK)
    config = workload_config(args.workload, world, shape)
    config["form"] = forms[0]
    config["particles"] = head["npart"]
    config["tile"] = list(args.tile or TILE.get(args.workload, (8, 8, 8)))
    config["cache"] = "working set (%.1f GB) > L2 (129 MB); no flush needed" % head["bytes_resident"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms"] / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if forms[0] == "fp32" else "f64", "data": "synthetic",
        "config": config,
        "cell_updates_per_s": head["cell_updates_per_s"],
        "stage_ms_per_step": head["stage_ms"],
        "gpu_launches": head["launches"],
        "clocks": head["clocks"],
        "e2e": head["e2e"],
        "roofline": head["roofline"],
        "fft_reference": head["fft_reference"],
    }
    if "fp64" in res and forms[0] != "fp64":
        r64 = res["fp64"]
        line["fp64_form"] = {"value": r64["value"], "ms_per_step": r64["ms"] / args.steps,
                             "cell_updates_per_s": r64["cell_updates_per_s"], "stage_ms_per_step": r64["stage_ms"],
                             "roofline": r64["roofline"], "clocks": r64["clocks"], "e2e": r64["e2e"],
                             "gpu_launches": r64["launches"]}
        line["fp32_over_fp64"] = value / r64["value"]
    line["roofline"]["peak_note"] = "HBM %.0f GB/s %s; FP64 peak derived: 152 SMs x 4 flop/clk x 2.07 GHz" % (
        hbm, "of measured" if peaks else "of fallback")
    del w
    if not args.no_extra and args.grid is None:
        extra = {}
        for name, ex_forms in EXTRA_WORKLOADS:
            if name == args.workload:
                continue
            wx = make_workload(name)
            ent = {"grid": list(wx["params"]["shape"]), "particles": sum(s["x"].size for s in wx["species"]),
                   "variant": wx["params"]["variant"], "shape_order": wx["params"]["shape_order"]}
            for f in ex_forms:
                r = run_form(f, wx, args, world, rank, local, full=False)
                ent[f] = {"particle_steps_per_s": r["value"], "cell_updates_per_s": r["cell_updates_per_s"],
                          "ms_per_step": r["ms"] / args.steps, "stage_ms_per_step": r["stage_ms"],
                          "clocks": r["clocks"]}
            if "fp32" in ent and "fp64" in ent:
                ent["fp32_over_fp64"] = ent["fp32"]["particle_steps_per_s"] / ent["fp64"]["particle_steps_per_s"]
            extra[name] = ent
            del wx
        extra["seed_wave"] = run_adjoint(args, world)
        line["workloads"] = extra
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, _, cores, desc = oracle_on_host(args.workload, 1, 2)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
