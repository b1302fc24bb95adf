#!/usr/bin/env python3
"""Benchmark of the MSC fix loop on one synthetic workload.

One step = the whole hot path on one field: the original-side preparation (discrete
gradient of f, separatrix seeds) and the fix loop (re-clamp, gradient of g, C- and
S-passes with quantised edits until the MSC of g equals f's), through the C ABI.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Default workload: 512^3 Kolmogorov-spectrum field with a 5% block of constant plateaus,
base compressor emulated by U[-xi, xi] noise, xi = 1e-4 * range, tier 4 (geometry).
value = field bytes (4 B x N) per second of a step with f and f_hat resident on the GPU;
e2e = the same metric with host buffers (host->device and device->host copies timed).
With --gpus N (torchrun, one rank per GPU) every rank fixes its own field (seed + rank):
replicas, no collective on the data path; value = all ranks' bytes / max step time.
--impl reference times the CPU oracle (single thread) on a bounded sample of the same
workload instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fix-loop GB/s of field & %HBM roofline at 1 GB300; serving p50/p99 latency, batched vs plain"
WORKLOAD = "kolmogorov3d"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", type=int, default=512)
    ap.add_argument("--rel", type=float, default=1e-4)
    ap.add_argument("--tier", type=int, default=4)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock samples (200 ms) during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx = float(parts[2])
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
            os.unlink(self.path)
        except Exception:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def workload(size, rel, rank):
    from paper_2409_17346_gb300 import synth
    f, fh, xi, tier = synth.config_case(WORKLOAD, seed=4 + rank, size=size, rel=rel)
    return f, fh, xi


def cpu_baseline(f, fh, rel, budget_s=12.0):
    """The oracle (single thread, as it stands) on sub-blocks of the same fields with the
    same xi; returns field GB/s over the sample."""
    import oracle
    from paper_2409_17346_gb300 import synth
    xi = synth.xi_from_range(f, rel)
    side = 12
    n_done, t_done, blocks = 0, 0.0, 0
    rng = np.random.default_rng(0)
    t_start = time.perf_counter()
    while time.perf_counter() - t_start < budget_s and blocks < 64:
        o = [int(rng.integers(0, s - side)) for s in f.shape]
        sl = tuple(slice(a, a + side) for a in o)
        fb, fhb = np.ascontiguousarray(f[sl]), np.ascontiguousarray(fh[sl])
        t0 = time.perf_counter()
        r = oracle.fix(fb, fhb, xi, tier=4)
        t_done += time.perf_counter() - t0
        assert r["status"] == 0
        n_done += fb.size
        blocks += 1
    return dict(value=4.0 * n_done / t_done / 1e9, unit="GB/s", cores=1, kind="oracle",
                sample="%d blocks of %d^3 vertices cut from the same f / f_hat (xi as the workload), "
                       "fixed to tier 4 by the single-threaded oracle, %.1f s" % (blocks, side, t_done))


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    f, fh, xi = workload(args.size, args.rel, 0)
    for _ in range(args.warmup):
        cpu_baseline(f, fh, args.rel, budget_s=2.0)
    vals = []
    base = None
    for _ in range(args.steps):
        base = cpu_baseline(f, fh, args.rel, budget_s=8.0)
        vals.append(base["value"])
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GB/s", "n_gpus": 0, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "%s %d^3, xi=%g*range, tier 4 (oracle on 12^3 sub-blocks)" % (WORKLOAD, args.size, args.rel)},
            "cpu_baseline": dict(base, value=v),
            "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2409_17346_gb300 import msc

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    f, fh, xi = workload(args.size, args.rel, rank)
    n = f.size
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    fd = torch.from_numpy(f).cuda()
    fhd = torch.from_numpy(fh).cuda()
    gd = torch.empty_like(fd)

    def step(profile=False, stats=None):
        h = msc.Handle(fd, opts=msc.options(stream=sp, profile=profile))
        _, ed = h.fix(fhd, xi, g_out=gd, tier=args.tier, stream=sp, profile=profile)
        if stats is not None:
            stats.append((h.stats(), ed))
        h.close()
        return ed

    for _ in range(args.warmup):
        ed = step()
    torch.cuda.synchronize()
    # correctness of the timed configuration (not timed)
    h = msc.Handle(fd)
    rep = h.verify(gd, xi)
    h.close()

    stats = []
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            ed = step(profile=True, stats=stats)
        e1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms_step = e0.elapsed_time(e1) / args.steps
    if dist is not None:
        t = torch.tensor([ms_step], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step = float(t.item())
    clocks = clk.summary()

    # per-class device time over the timed steps; the dominant class sets the roofline
    cls_ms = {k: sum(s[k]["ms"] for s, _ in stats) for k in msc.KERNEL_CLASSES}
    cls_launch = {k: sum(s[k]["timed"] for s, _ in stats) for k in msc.KERNEL_CLASSES}
    cls_items = {k: sum(s[k]["items"] for s, _ in stats) for k in msc.KERNEL_CLASSES}
    launches = sum(s[k]["launches"] for s, _ in stats for k in msc.KERNEL_CLASSES)
    dom = max(cls_ms, key=cls_ms.get)
    peak, peak_kind = peaks()
    roof = None
    if dom == "dense" and cls_launch["dense"]:
        # algorithmic bytes of one dense launch: read the field once (4 B) and write one
        # 8-byte gradient code per vertex
        per_launch = 12.0 * n
        avg_s = cls_ms["dense"] / cls_launch["dense"] / 1e3
        ach = per_launch / avg_s / 1e9
        roof = {"bound": "hbm", "kernel": "k_eval_dense (dense discrete gradient)", "achieved": ach, "peak": peak,
                "unit": "GB/s", "frac": ach / peak, "traffic": None, "peak_source": peak_kind,
                "algorithmic_bytes_per_launch": per_launch, "avg_launch_ms": avg_s * 1e3}
    else:
        roof = {"bound": "hbm", "kernel": dom, "achieved": None, "peak": peak, "unit": "GB/s", "frac": None,
                "traffic": None, "peak_source": peak_kind}

    value = world * 4.0 * n / (ms_step / 1e3) / 1e9
    iters = (ed["n_iters_c"], ed["n_iters_s"])

    # end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        g_host = np.empty_like(f)
        t_e2e = []
        for _ in range(max(1, min(args.steps, 3))):
            barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h = msc.Handle(f)
            _, ed2 = h.fix(fh, xi, g_out=g_host, tier=args.tier)
            h.close()
            t_e2e.append(time.perf_counter() - t0)
        te = statistics.median(t_e2e)
        if dist is not None:
            t = torch.tensor([te], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            te = float(t.item())
        d2h = 4 * n + n + 12 * ed2["n_lossless"]
        e2e = {"value": world * 4.0 * n / te / 1e9, "unit": "GB/s", "h2d_bytes_per_step": 8 * n,
               "d2h_bytes_per_step": d2h}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "%s %dx%dx%d float32, 5%% constant-plateau block, base = U[-xi,xi] noise, "
                                   "xi=%g*range, tier %d, q_max 6" % (WORKLOAD, *f.shape[::-1], args.rel, args.tier),
                       "n_vertices": n, "xi": xi, "iters_c": iters[0], "iters_s": iters[1],
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs (%d MB each) exceed L2; no flush" % (4 * n >> 20),
                       "verify_passed": rep["passed"],
                       "kernel_ms_per_step": {k: v / args.steps for k, v in cls_ms.items()},
                       "kernel_launches_per_step": {k: v / args.steps for k, v in cls_launch.items()},
                       "kernel_items_per_step": {k: v / args.steps for k, v in cls_items.items()},
                       "launches_per_step": launches / args.steps},
            "roofline": roof, "clocks": clocks, "gpu_launches": launches, "e2e": e2e,
        }
        if not args.no_cpu and world == 1:
            line["cpu_baseline"] = cpu_baseline(f, fh, args.rel)
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
