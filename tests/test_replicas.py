"""The N > 1 path of bench.py on CPU: the step has no data exchange ("replicas only"), so the
only multi-rank logic is the timing reduction (the slowest rank sets the job time) and the
whole-job throughput; checked here with two gloo ranks.  The reference arm runs on rank 0 only."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = 10.0 + 5.0 * rank                      # rank 1 is the slower one
    ms = bench.max_over_ranks(ms_local, world, device="cpu")
    out.put((rank, ms, bench.job_throughput(1000, 4, world, ms)))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29600 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in res:
        assert ms == 15.0
        assert value == pytest.approx(1000 * 4 * 2 / 15.0e-3)


def test_single_rank_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.job_throughput(10, 2, 1, 4.0) == pytest.approx(5000.0)


def test_reference_arm_prints_nothing_on_other_ranks():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference"], env=env,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_reference_arm_line_on_rank_zero():
    """The reference arm (the oracle on the host cores) prints one JSON line with the contract's
    keys and the libpic arm's config of the same workload."""
    import json
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1"],
                       env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["warmup"] >= 3
    cfg = dict(d["config"])
    cfg.pop("note")
    assert cfg == {"workload": "beam_wakefield", "grid": [256, 256, 1024], "particles": 68108864,
                   "form": "fp64", "shape_order": 3, "centering_order": [8, 8, 16], "variant": 2,
                   "parallelism": "single"}
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] == len(os.sched_getaffinity(0))
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_clock_sampler_keeps_the_samples_of_the_timed_region():
    """bench.ClockSampler: nvidia-smi lines are parsed and only those stamped inside the timed
    region enter the median and the throttle reasons (all of them when none falls inside)."""
    import datetime
    sys.path.insert(0, ROOT)
    import bench

    def stamp(t):
        return datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]

    t0 = 1_800_000_000.0
    lines = [
        "0, 900, 2070, 150.0, 0x0, Not Active, Not Active, Not Active, Not Active, %s" % stamp(t0 - 0.2),
        "0, 2070, 2070, 900.0, 0x4, Not Active, Not Active, Not Active, Active, %s" % stamp(t0 + 0.01),
        "0, 2055, 2070, 910.0, 0x0, Not Active, Not Active, Not Active, Not Active, %s" % stamp(t0 + 0.05),
        "0, 600, 2070, 150.0, 0x0, Active, Not Active, Not Active, Not Active, %s" % stamp(t0 + 0.4),
    ]

    class FakeProc:
        def terminate(self):
            pass

        def communicate(self, timeout=None):
            return "\n".join(lines) + "\n", ""

    s = bench.ClockSampler(0)
    s.proc = FakeProc()
    c = s.stop((t0, t0 + 0.06))
    assert c["in_timed_region"] and c["samples"] == 2
    assert c["sm_mhz"] == (2070 + 2055) / 2 and c["sm_max_mhz"] == 2070
    assert c["reasons"] == ["sw_power_cap"]          # the hw_slowdown sample lies outside the region
    s.proc = FakeProc()
    c = s.stop((t0 + 10, t0 + 11))                  # no sample inside: all of them
    assert not c["in_timed_region"] and c["samples"] == 4
    assert "hw_slowdown" in c["reasons"]
