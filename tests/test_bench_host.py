"""Host-side logic of bench.py that needs no GPU: the reference arm (the CPU
oracle timed on a bounded sample) and the multi-rank reduction of timings
(replicas only: one process per GPU, max over ranks), run as two gloo ranks."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--cells", "6", "--steps", "2",
                          "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    j = json.loads(lines[0])
    assert j["impl"] == "reference" and j["unit"] == "atom-timesteps/s" and j["value"] > 0
    assert j["cpu_baseline"]["kind"] == "oracle" and j["cpu_baseline"]["cores"] >= 1
    assert j["e2e"]["h2d_bytes_per_step"] == 0 and j["higher_is_better"] is True


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist = bench.dist_init(world)
    bench.barrier(dist)
    m = bench.max_over_ranks(dist, float(rank + 1) * 1.5)
    q.put((rank, m))
    dist.destroy_process_group()


def test_two_rank_max_over_ranks_with_gloo():
    import multiprocessing as mp
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(2))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == {0: 3.0, 1: 3.0}


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--cells", "6", "--steps", "1",
                          "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=300, env=env)
    assert out.returncode == 0 and not out.stdout.strip()


def _bench():
    sys.path.insert(0, ROOT)
    import bench
    return bench


def test_clock_summary_prefers_the_timed_region():
    b = _bench()
    c = b.ClockSampler(0)
    row = lambda t, mhz, cap="Not Active": [t, "0", str(mhz), "2070", "900.0", "0x0", "Not Active", "Not Active",
                                             "Not Active", cap]
    c.rows = [row(1.0, 1500), row(2.0, 2070), row(2.1, 2055), row(3.0, 1600, "Active")]
    inside = c.summary(1.9, 2.2)
    assert inside["region"] == "timed steps" and inside["samples"] == 2 and inside["sm_mhz"] == 2062.5
    assert inside["reasons"] == []
    # a timed region between two samples: the whole window, labelled as such
    w = c.summary(2.2, 2.3, window="the window")
    assert w["region"] == "the window" and w["samples"] == 4 and w["reasons"] == ["sw_power_cap"]
    c.rows = []
    assert c.summary(0, 1)["reasons"] == ["unsampled"]


def test_nve_drift_is_the_least_squares_slope():
    # a fake system whose total energy per atom rises linearly with steps plus
    # a bounded oscillation: the slope, not the end points, is reported
    b = _bench()

    class Fake:
        def __init__(self):
            self.t = 0

        def step(self, k):
            self.t += k

    fake = Fake()
    n = 1000
    orig = b.total_energy
    b.total_energy = lambda s: n * (2e-8 * s.t + 1e-6 * np.sin(s.t / 7.0))
    try:
        r = b.nve_drift(fake, n, steps=1000, every=50)
    finally:
        b.total_energy = orig
    assert fake.t == 1000
    assert abs(r["drift_per_atom_per_1000_steps"] - 2e-5) < 2e-6
    assert r["steps"] == 1000 and r["sampled_every"] == 50


def test_roofline_names_the_binding_ceiling():
    b = _bench()
    ceil = {"l2_gather_gps": 500.0, "fp32_fma_tflops": 80.0, "hbm_copy_gbs": 6500.0, "fp64_fma_tflops": 1.2}
    r = b.roofline_of(0.1, 300e6, 60e6, 0.09, ceil, 6800.0, "measured", None)
    assert r["achieved"] == pytest.approx(3000.0) and r["frac"] == pytest.approx(3000.0 / 6800.0)
    assert r["ceilings"]["l2_gather"]["achieved_Ggathers_s"] == pytest.approx(600.0)
    assert r["ceilings"]["access_pattern_twin"]["frac"] == pytest.approx(0.9)
    assert r["binding"] == "access_pattern_twin"
    assert "note" in r["ceilings"]["l2_gather"]  # 1.2 of the random-gather probe: not a ceiling of this pattern
    r = b.roofline_of(0.1, 300e6, 60e6, None, ceil, 6800.0, "measured", None)
    assert r["binding"] == "hbm"  # l2_gather exceeded, fp32 0.2, hbm 0.44
    assert r["traffic"] is None and r["traffic_source"] is None
