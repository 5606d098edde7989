"""The DRAM traffic bench.py reports beside each roofline comes from the
committed ncu summary (profiles/ncu_traffic.txt), keyed by a hash of the
kernel's sources and by its launch shape: every line parses, and the kernels
and shapes the bench runs on its default workloads have a line taken on the
current sources (a kernel edited without a new capture fails here, not as a
silent null in the bench line)."""
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lines():
    for ln in open(os.path.join(ROOT, "profiles", "ncu_traffic.txt")):
        if ln.startswith("#") or not ln.strip():
            continue
        yield dict(t.split("=", 1) for t in ln.split() if "=" in t)


def test_every_line_parses():
    n = 0
    for kv in _lines():
        assert kv["kernel"].startswith("k_") and kv["workload"] and len(kv["src_sha"]) == 12
        b = float(kv.get("dram_bytes_per_launch", kv.get("dram_bytes_per_step", "nan")))
        assert b > 1e8, kv
        n += 1
    assert n > 0


def test_current_sources_have_traffic():
    # the ring kernel the autotuner keeps at 4096^2 and the register kernel at 512^3 (the bench's cfg 2 and cfg 3)
    assert bench.ncu_traffic("k_kinetic_ring", "2d_tmz_4096_kinetic", (16, 16, 3)) is not None
    assert bench.ncu_traffic("k_kinetic", "2d_tmz_4096_kinetic", (8, 32, 0)) is not None
    for shape in ((2, 2, 0), (4, 1, 0), (1, 4, 0)):
        assert bench.ncu_traffic("k_kinetic", "3d_512_kinetic_bf16", shape) is not None, shape
    for w in ("batch1d_256_f32", "batch1d_256_bf16"):
        t = bench.batch_traffic(w, 4)
        assert t is not None and t > 1e9, w


def test_traffic_close_to_algorithmic_bytes():
    # cfg 2: 823 473 plasma rows x 1024 FP32 nodes, delta f read and written once a step
    alg = 8 * 823473 * 1024
    t = bench.ncu_traffic("k_kinetic_ring", "2d_tmz_4096_kinetic", (16, 16, 3))
    assert 0.95 * alg < t < 1.05 * alg


def test_step_launches_counts_remainder_graphs():
    """32-step chunks, then one graph per set bit of the remainder (16, 8, 4,
    2, 1 steps); a sequence of n steps launches H_0, (middle, E, H) per step
    less the last H, one counter advance, and fused transitions merge E + H."""
    import bench
    seq = lambda n, mid, f: mid * n + 2 * n - (((n - 1) - (n - 1) % 2) if f else 0) + 1
    assert bench.step_launches(20, 1, False) == seq(16, 1, False) + seq(4, 1, False)
    assert bench.step_launches(64, 1, True) == 2 * seq(32, 1, True)
    assert bench.step_launches(2000, 1, True) == 62 * seq(32, 1, True) + seq(16, 1, True)
    assert bench.step_launches(7, 2, False) == seq(4, 2, False) + seq(2, 2, False) + seq(1, 2, False)
    assert bench.step_launches(1, 0, True) == 3
