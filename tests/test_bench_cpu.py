"""The benchmark's host-side contract on CPU: the reference arm (the oracle on a bounded
sample) prints one JSON line with the keys the driver reads, and the algorithmic-byte
accounting of every kernel class is defined and consistent."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--size", "32"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "GB/s"
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == os.cpu_count()
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0


def test_class_bytes_defined_for_bandwidth_classes():
    n = 1 << 20
    tot = {"items": 1000, "launches": 10, "ms": 1.0, "timed": 10,
           "work": {"edit": 100, "refresh": 200, "cpass": 300}}
    for cls in ("dense", "cpass", "edit", "refresh", "rebuild", "sep_init", "sep_seed", "sep_update", "rounds"):
        b = bench.class_bytes(cls, tot, n, 1, 3)
        assert b is not None and b > 0, cls
    # the persistent round kernel counts the bytes of the work it did, as the classes do
    r = bench.class_bytes("rounds", tot, n, 1, 3)
    assert r == 1000 * n / 8192.0 + 16.0 * 300 + 22.0 * 100 + 36.0 * 200
    assert set(bench.CLASS_KERNELS) >= {"dense", "cpass", "edit", "refresh", "rebuild", "sep_seed", "rounds"}


def test_configs_cover_the_workloads():
    """Every configuration names its generator, bound and tier; --size shrinks 3D sides and
    2D grids alike."""
    import argparse
    assert set(bench.CONFIGS) == {1, 2, 3, 4}
    for k, c in bench.CONFIGS.items():
        a = argparse.Namespace(config=k, size=None, rel=None, tier=None)
        cfg = bench.config_of(a)
        assert cfg["tier"] in (3, 4) and cfg["rel"] in (1e-3, 1e-4)
        d = bench.workload_desc(cfg, (64, 64) if k < 3 else (8, 8, 8))
        assert "%g" not in d and "%d" not in d and "xi=" in d
    a = argparse.Namespace(config=2, size=100, rel=None, tier=None)
    assert bench.config_of(a)["size"] == (100, 200)
    # a run at another size says so: the description keeps the named size and adds the run's
    a = argparse.Namespace(config=4, size=256, rel=None, tier=None)
    d = bench.workload_desc(bench.config_of(a), (256, 256, 256))
    assert "512x512x512" in d and d.endswith("(run at 256x256x256)")
    assert "run at" not in bench.workload_desc(bench.config_of(argparse.Namespace(
        config=4, size=None, rel=None, tier=None)), (512, 512, 512))
    assert bench.CONFIGS[3]["batch"] == 8
