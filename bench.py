"""Benchmark of the hybrid nodal-staggered PSATD PIC step on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl libpic|reference] [--workload NAME]

Default workload: the laser-wakefield box (128 x 128 x 512 cells, dx = dy = 0.2,
dz = 0.04, dt = dz/c, standard PSATD at infinite order, centering (8, 8, 16),
cubic shape, 2 electrons per cell = 16,777,216 particles, Gaussian a0 = 2
laser).  One step = one full hybrid cycle (gather, push, deposit, centering,
FFTs, PSATD update) through pic_step32 (FP32 form, the headline value) and,
in the same run, pic_step (plain FP64 form, reported beside it with the
FP32/FP64 ratio).  Prints one JSON line.

--impl libpic (default): K steps of pic_step timed with CUDA events on the
library's stream after W warm-up steps; value = particle-steps/s over all ranks.
Under torchrun each rank runs an independent replica of the workload
(replicas only: the single-GPU periodic step has no data exchange).
--impl reference: the FP64 CPU oracle on this host's cores, one bounded sample
of the same workload per step (rank 0 only).
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
HBM_PEAK_FALLBACK = 6800.0
# FP64 FMA units: 152 SMs x 4 FP64 flop/clk/SM x 2.070 GHz (nominal 1.25 TFLOP/s class figure)
FP64_PEAK_TFLOPS = 152 * 4 * 2.070e9 / 1e12
# DRAM bytes (read + write) per steady-state launch of the dominant kernel, from one ncu capture of
# the current kernel version at the full bench size
# (profiles/push32_tile_laser_wakefield_128x128x512_dram.md); other workloads / forms report null
MEASURED_TRAFFIC = {("laser_wakefield", (128, 128, 512), "fp32"): 1.490e9}
# LSU data-pipe wavefronts (shared memory, L1, global) per steady-state launch of the same kernel,
# same capture size (profiles/push32_tile_laser_wakefield_128x128x512_lsu.md): the pipe that bounds
# the particle kernel on chip issues one wavefront per SM per cycle
MEASURED_LSU_WAVEFRONTS = {("laser_wakefield", (128, 128, 512), "fp32"): 4.953e8}
N_SM = 152
# CPU-oracle sample: the same workload on a 1/64-volume box (same dx, dt, physics)
SAMPLE_SHAPE = {"laser_wakefield": (32, 32, 128), "beam_wakefield": (64, 64, 128),
                "thermal_plasma": (32, 32, 32), "galilean_drift": (32, 32, 64), "seed_wave": (32, 32, 32)}
FULL_SHAPE = {"laser_wakefield": (128, 128, 512), "beam_wakefield": (256, 256, 1024),
              "thermal_plasma": (32, 32, 32), "galilean_drift": (64, 64, 256), "seed_wave": (64, 64, 64)}


def push_flops_per_particle(order):
    """Algorithmic FP64 flops of the gather + Boris + move + deposit of one particle.

    gather 12 S^3 (6 fields x S^3 nodes x FMA) + S^3 weight products, J deposit
    7 S^3 (weight, 3 products, 3 adds), rho deposit 2 S^3, shapes/Boris/move 250;
    S = order + 1.
    """
    S3 = (order + 1) ** 3
    return 22 * S3 + 250


def make_workload(name, shape=None):
    f = workloads.WORKLOADS[name]
    kw = {}
    if shape is not None:
        kw["shape"] = shape
        if name == "beam_wakefield":
            kw["n_beam"] = max(1000, int(1_000_000 * np.prod(shape) / np.prod(FULL_SHAPE[name])))
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


def run_oracle_sample(name, steps):
    """Oracle (FP64 CPU) on the 1/64-volume sample box: returns (particle-steps/s, description)."""
    from oracle import step
    w = make_workload(name, SAMPLE_SHAPE[name])
    p = step.Params(**w["params"])
    st = {"E": w["E"], "B": w["B"], "species": w["species"]}
    st["rho"] = step.initial_rho(p, st["species"])
    npart = sum(s["x"].size for s in w["species"])
    t0 = time.perf_counter()
    for _ in range(steps):
        step.hybrid_step(p, st)
    dt = time.perf_counter() - t0
    desc = "%d step(s) of the oracle on a %dx%dx%d sample of the workload (%d particles, same dx/dt/physics)" % (
        (steps,) + tuple(SAMPLE_SHAPE[name]) + (npart,))
    return npart * steps / dt, desc, dt, w["params"], npart


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # warm-up samples are run too (untimed) so that the timed steps see warm caches
    run_oracle_sample(args.workload, max(1, min(args.warmup, 1)))
    value, desc, secs, prm, n_sample = run_oracle_sample(args.workload, args.steps)
    # the libpic arm's config: the full workload (the oracle times a bounded sample of it)
    shape = tuple(args.grid) if args.grid else FULL_SHAPE[args.workload]
    scale = float(np.prod(shape)) / float(np.prod(SAMPLE_SHAPE[args.workload]))
    config = {"workload": args.workload, "grid": list(shape), "particles": int(round(n_sample * scale)),
              "form": "fp64" if args.form == "fp64" else "fp32", "shape_order": prm["shape_order"],
              "centering_order": list(prm["centering_order"]), "variant": prm["variant"],
              "parallelism": "replicas" if args.gpus > 1 else "single"}
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="libpic", choices=["libpic", "reference"])
    ap.add_argument("--workload", default="laser_wakefield", choices=sorted(workloads.WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--e2e-copy-streams", type=int, default=1,
                    help="streams the per-step host-to-device input copies are spread over "
                         "(one measured fastest: 2.45e9 vs 2.28e9 particle-steps/s with four)")
    ap.add_argument("--e2e-no-graph", action="store_true",
                    help="end-to-end loop with direct pic_step calls instead of their CUDA graphs")
    ap.add_argument("--form", default="both", choices=["both", "fp32", "fp64"],
                    help="both: FP32 form timed as the headline, FP64 form beside it")
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


    w = make_workload(args.workload, tuple(args.grid) if args.grid else None)
    p = w["params"]
    shape = p["shape"]
    ncell = shape[0] * shape[1] * shape[2]
    forms = ["fp32", "fp64"] if args.form == "both" else [args.form]
    res = {f: run_form(f, w, args, world, rank, local) for f in forms}
    head = res[forms[0]]
    value = head["value"]
    peaks = measured_peaks()
    hbm = (peaks or {}).get("hbm_gbs", HBM_PEAK_FALLBACK)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms"] / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if forms[0] == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": args.workload, "grid": list(shape), "particles": head["npart"], "form": forms[0],
                   "shape_order": p["shape_order"], "centering_order": list(p["centering_order"]),
                   "variant": p["variant"],
                   "cache": "working set (%.1f GB) > L2 (129 MB); no flush needed" % head["bytes_resident"],
                   "parallelism": "replicas" if world > 1 else "single"},
        "cell_updates_per_s": ncell * args.steps * world / (head["ms"] * 1e-3),
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
                             "stage_ms_per_step": r64["stage_ms"], "roofline": r64["roofline"],
                             "clocks": r64["clocks"], "e2e": r64["e2e"]}
        line["fp32_over_fp64"] = value / r64["value"]
    line["roofline"]["peak_note"] = "HBM %.0f GB/s %s; FP64 peak derived: 152 SMs x 4 flop/clk x 2.07 GHz" % (
        hbm, "of measured" if peaks else "of fallback")
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, desc, _, _, _ = run_oracle_sample(args.workload, 4)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def cufft_reference(shape, dtype, libpic_ms):
    """cuFFT (through torch.fft) on the step's transform load, timed as a reference only:
    4 forward R2C (J, rho) and 6 inverse C2R (nodal E, B) 3D transforms of the grid."""
    import torch
    x = torch.randn((4,) + tuple(shape), dtype=dtype, device="cuda")
    y = torch.randn((6,) + tuple(shape), dtype=dtype, device="cuda")
    dims = (1, 2, 3)

    Ys = torch.fft.rfftn(y, dim=dims)
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
    del x, y, Ys
    torch.cuda.empty_cache()
    return {"cufft_ms_per_step": ms, "libpic_fft_ms_per_step": libpic_ms,
            "note": "cuFFT via torch.fft: 4 R2C + 6 C2R 3D transforms of the grid per step, reference only"}


def run_form(form, w, args, world, rank, local):
    """Time K steps of one form (fp32 | fp64) of the step on the workload; returns a dict of results."""
    import torch
    import torch.distributed as dist
    from paper_2106_12919_gb300 import pic

    p = w["params"]
    shape = p["shape"]
    ncell = shape[0] * shape[1] * shape[2]
    fp32 = form == "fp32"
    stream = torch.cuda.Stream()
    ctx = pic.Context(shape, p["dx"], p["dt"], p["shape_order"], p["centering_order"], p["variant"], p["v_gal"],
                      p["spectral_order"], p["c"], p["eps0"], stream=stream,
                      precision=pic.PIC_FP32 if fp32 else pic.PIC_FP64)
    fdt = np.float32 if fp32 else np.float64
    tdt = torch.float32 if fp32 else torch.float64
    with torch.cuda.stream(stream):
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=fdt)).cuda()
        E = [dev(a) for a in w["E"]]
        B = [dev(a) for a in w["B"]]
        J = [torch.zeros(ncell, dtype=tdt, device="cuda") for _ in range(3)]
        rho = torch.zeros(ncell, dtype=tdt, device="cuda")
        if fp32:
            sp = [pic.Species32.from_positions(ctx, s["x"], s["y"], s["z"], s["ux"], s["uy"], s["uz"], s["w"],
                                               s["q"], s["m"]) for s in w["species"]]
        else:
            sp = [pic.Species(dev(s["x"]), dev(s["y"]), dev(s["z"]), dev(s["ux"]), dev(s["uy"]), dev(s["uz"]),
                              dev(s["w"]), s["q"], s["m"]) for s in w["species"]]
    torch.cuda.synchronize()
    npart = sum(s.n for s in sp)
    step = ctx.step32 if fp32 else ctx.step
    (ctx.deposit_rho32 if fp32 else ctx.deposit_rho)(sp, rho)
    step(E, B, J, rho, sp, args.warmup)
    ctx.sync()

    # ---- timed region: K steps of pic_step, inputs resident in HBM ----
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ctx.timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    w0 = time.time()
    e0.record(stream)
    step(E, B, J, rho, sp, args.steps)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    w1 = time.time()
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    clocks = sampler.stop((w0, w1))
    stage = {s: ctx.timing_read(s) for s in ("push", "fft", "update", "bin", "other", "all")}
    ctx.timing(False)
    ms = max_over_ranks(ms, world)
    value = job_throughput(npart, args.steps, world, ms)

    # ---- end to end: host (pinned) state -> device, one pic_step, field energy back ----
    # Every step copies its whole input state (E, B, rho and all particle arrays) from pinned host
    # memory and reads the field energy back.  Two device copies of the state alternate, so the
    # copy of step k+1 (on its own stream) overlaps the step k computation.
    ke = args.e2e_steps or max(3, min(args.steps, 10))
    devs = E + B + [rho] + [a for s in sp for a in s.arrays()]
    host = [t.cpu().pin_memory() for t in devs]
    h2d = sum(h.numel() * h.element_size() for h in host)
    energy = ctx.field_energy32 if fp32 else ctx.field_energy
    sets = [(E, B, rho, sp)]
    E2 = [torch.empty_like(t) for t in E]
    B2 = [torch.empty_like(t) for t in B]
    rho2 = torch.empty_like(rho)
    sp2 = []
    for s in sp:
        arrs = [torch.empty_like(a) for a in s.arrays()]
        if fp32:
            sp2.append(pic.Species32(*arrs[:8], s.q, s.m))
        else:
            sp2.append(pic.Species(*arrs[:7], s.q, s.m))
    sets.append((E2, B2, rho2, sp2))
    bufs = [E + B + [rho] + [a for s in sp for a in s.arrays()],
            E2 + B2 + [rho2] + [a for s in sp2 for a in s.arrays()]]
    # the per-step input copies may be spread over several streams
    copy_streams = [torch.cuda.Stream() for _ in range(args.e2e_copy_streams)]
    copied = [[torch.cuda.Event() for _ in copy_streams] for _ in range(2)]
    done = [torch.cuda.Event(), torch.cuda.Event()]

    def enqueue_copy(k):
        b = k % 2
        for i, cs in enumerate(copy_streams):
            with torch.cuda.stream(cs):
                cs.wait_event(done[b])             # the step that last used this buffer has finished
                for d, h in list(zip(bufs[b], host))[i::len(copy_streams)]:
                    d.copy_(h, non_blocking=True)
                copied[b][i].record(cs)

    # the one-step call on each buffer set, captured as a CUDA graph (pic.StepGraph: the library
    # takes every decision on the device, so the call replays exactly without its host launches)
    graphs = []
    if not args.e2e_no_graph:
        capture = ctx.capture_step32 if fp32 else ctx.capture_step
        for b in range(2):
            for d, h in zip(bufs[b], host):
                d.copy_(h)
            Eb, Bb, rb, spb = sets[b]
            graphs.append(capture(Eb, Bb, None, rb, spb, 1))
    for ev in done:
        ev.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    enqueue_copy(0)
    for k in range(ke):
        if k + 1 < ke:
            enqueue_copy(k + 1)
        b = k % 2
        Eb, Bb, rb, spb = sets[b]
        for ev in copied[b]:
            stream.wait_event(ev)
        if graphs:
            with torch.cuda.stream(stream):
                graphs[b].replay()                  # pic_step(1) on set b, J = NULL
        else:
            step(Eb, Bb, None, rb, spb, 1)         # J^{n+1/2} is not part of the result: J = NULL
        done[b].record(stream)
        energy(Eb, Bb)                              # host reads the result back (synchronous)
    t1.record(stream)
    t1.synchronize()
    e2e_ms = t0.elapsed_time(t1)
    del E2, B2, rho2, sp2, bufs, sets, graphs
    e2e_ms = max_over_ranks(e2e_ms, world)
    e2e = {"value": job_throughput(npart, ke, world, e2e_ms), "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": 8, "steps": ke,
           "note": "per step: pinned H2D of E, B, rho and all particles (double-buffered: the copy of "
                   "step k+1 overlaps step k), pic_step(1) (%s), field energy read back" %
                   ("replayed as a CUDA graph, pic.StepGraph" if not args.e2e_no_graph else "direct call")}

    # ---- roofline of the dominant kernel (gather + push + deposit) ----
    push_ms, push_n = stage["push"]
    push_avg_s = push_ms * 1e-3 / max(push_n, 1)
    per_launch = npart / max(1, len(sp))
    peaks = measured_peaks()
    hbm = (peaks or {}).get("hbm_gbs", HBM_PEAK_FALLBACK)
    if fp32:
        # 32 B read + 28 B written per particle; nodal E, B read (24 B) and J, rho deposited (16 B) per cell
        nbytes = 60 * per_launch + 40 * ncell
        achieved = nbytes / push_avg_s / 1e9
        traffic = MEASURED_TRAFFIC.get((w["name"].rsplit("_", 1)[0], tuple(shape), form))
        roofline = {"kernel": "push32_tile_kernel (gather + Boris + deposit)", "bound": "hbm", "achieved": achieved,
                    "peak": hbm, "unit": "GB/s", "frac": achieved / hbm, "traffic": traffic,
                    "algorithmic_bytes": "60 B/particle + 40 B/cell per launch (%.3g B)" % nbytes}
        wf = MEASURED_LSU_WAVEFRONTS.get((w["name"].rsplit("_", 1)[0], tuple(shape), form))
        if wf is not None:
            # the on-chip bound: the LSU data pipe (one wavefront per SM per cycle at the sampled clock)
            mhz = clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or 2070.0
            peak_wf = N_SM * mhz * 1e6
            roofline["onchip"] = {"bound": "lsu", "unit": "wavefronts/s", "achieved": wf / push_avg_s,
                                  "peak": peak_wf, "frac": wf / push_avg_s / peak_wf,
                                  "wavefronts_per_launch": wf,
                                  "note": "LSU data-pipe wavefronts per launch from one ncu capture at this size; "
                                          "peak = 152 SMs x 1 wavefront/cycle x median SM clock sampled in the "
                                          "timed region"}
    else:
        flops = push_flops_per_particle(p["shape_order"]) * per_launch
        achieved = flops / push_avg_s / 1e12
        roofline = {"kernel": "push_kernel (gather + Boris + deposit)", "bound": "alu", "achieved": achieved,
                    "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                    "traffic": None, "algorithmic_flops": "22 (p+1)^3 + 250 per particle",
                    "hbm_frac": 104 * per_launch / push_avg_s / 1e9 / hbm}
    esz = 4 if fp32 else 8
    resident = (10 * ncell * esz + sum(sum(a.numel() * a.element_size() for a in s.arrays()) for s in sp)
                + 40 * ncell * esz) / 1e9
    fft_ref = cufft_reference(shape, tdt, stage["fft"][0] / args.steps)
    out = {"value": value, "ms": ms, "npart": npart, "clocks": clocks, "e2e": e2e, "roofline": roofline,
           "fft_reference": fft_ref,
           "stage_ms": {k: v[0] / args.steps for k, v in stage.items() if k != "all"},
           "launches": stage["all"][1], "bytes_resident": resident}
    ctx.close()
    del E, B, J, rho, sp, host, devs
    torch.cuda.empty_cache()
    return out


if __name__ == "__main__":
    main()
