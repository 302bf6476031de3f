"""Benchmark: one 2^28 x 2^28-bit GF(2)[x] product per step on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload c1_2^28] [--no-cpu-baseline]

Prints ONE JSON line (rank 0).  A step is one whole product (Alg. 5: Split,
BasisCvt, changeRepr, FFT_LCH x2, pointmul, iFFT_LCH, iBasisCvt,
changeRepr^-1, InterleavedCombine) with inputs resident in HBM; `value` is ms
per product (lower is better).  `e2e` times the same product through the
C-ABI call with HOST buffers (gf2x_mul_host: H2D copies, product, D2H copy).
The L2 is flushed (a 256 MiB write) between timed steps, outside the timed
events.  With N > 1 (torchrun) every rank runs independent products (the
single product does not shard: replicas only) and value = max elapsed over
ranks / (N * K) products.

`--impl reference` times the CPU oracle (the plain Karatsuba carry-less
product) on the host cores on a bounded sample of the same workload, scaled to
ms per product.
"""
import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("ms per 2^28-bit GF(2)[x] product (% HBM roofline); "
          "batched products/s vs one-by-one")
PAPER_MS_2_28 = 2302.0  # Table 2, F~_{2^128} tower row, 2^28-bit operands (Haswell)


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="c1_2^28")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-depth", type=int, default=6,
                   help="Karatsuba depth of the CPU-baseline sample (3^d sub-products)")
    return p.parse_args()


def _dist_init(n):
    rank, world, local = 0, 1, 0
    if n > 1 or int(os.environ.get("WORLD_SIZE", "1")) > 1:
        import torch.distributed as dist
        rank = int(os.environ.get("RANK", "0"))
        world = int(os.environ.get("WORLD_SIZE", "1"))
        local = int(os.environ.get("LOCAL_RANK", "0"))
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        import torch
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", rank=rank, world_size=world)
    return rank, world, local


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", "clocks_bench_%d.csv" % os.getpid())

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def cpu_sample(a, na, b, nb, depth, reps=1):
    """Time the oracle on one depth-`depth` Karatsuba sub-product of the
    workload (the product of the lowest 2^-depth parts of a and b) on all
    host cores and scale by 3^depth to ms per full product.  The linear
    recombination work of the upper levels is not included."""
    from oracle import product as P
    nw = max((na + 63) // 64, (nb + 63) // 64)
    sub_w = max(1, nw >> depth)
    sa, sb = a[:sub_w].copy(), b[:sub_w].copy()
    best = None
    for _ in range(reps):
        t0 = time.perf_counter()
        P.mul(sa, 64 * sub_w, sb, 64 * sub_w)
        dt = time.perf_counter() - t0
        best = dt if best is None else min(best, dt)
    scale = 3 ** depth
    return {"value": best * 1e3 * scale, "unit": "ms", "cores": P.num_threads(),
            "kind": "oracle",
            "sample": "1 of 3^%d Karatsuba sub-products (%d x %d bits: the low "
                      "parts of a and b), all cores, x%d; upper-level linear "
                      "recombination not included" % (depth, 64 * sub_w, 64 * sub_w, scale),
            "sample_s": best}


def run_reference(args):
    rank, world, _ = int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), 0
    if rank != 0:
        return
    import workloads as W
    from oracle import build as ob
    ob.build()
    a, na, b, nb = W.make_workload(args.workload)
    for _ in range(args.warmup):
        cpu_sample(a, na, b, nb, args.cpu_depth)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_sample(a, na, b, nb, args.cpu_depth))
    wall = time.perf_counter() - t0
    v = sum(x["value"] for x in vals) / len(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "ms",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": wall * 1e3 / args.steps, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": v / PAPER_MS_2_28, "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": "single %d x %d-bit product (%s)" % (na, nb, args.workload),
                   "na_bits": na, "nb_bits": nb},
        "cpu_baseline": {"kind": "oracle", "cores": vals[0]["cores"],
                         "sample": vals[0]["sample"], "value": v, "unit": "ms"},
        "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = _dist_init(args.gpus)
    from paper_1708_09746_gb300 import build as gb
    gb.build()
    import paper_1708_09746_gb300 as G
    import workloads as W

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    a, na, b, nb = W.make_workload(args.workload)
    ow = G.gf2x_out_words(na, nb)
    N = G.gf2x_fft_points(na, nb)
    da = torch.from_numpy(a.view(np.int64)).to(dev)
    db = torch.from_numpy(b.view(np.int64)).to(dev)
    out = torch.empty(ow, dtype=torch.int64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)

    def step():
        G.gf2x_mul_async(da, na, db, nb, out, stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.zero_()
            step()
    stream.synchronize()

    clocks = ClockSampler(local)
    G.gf2x_profile_reset()
    G.gf2x_profile_enable(1)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    _barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            flush.zero_()
            evs[i][0].record(stream)
            step()
            evs[i][1].record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    _barrier(world)
    clk = clocks.stop()
    G.gf2x_profile_enable(0)
    stages = G.profile_all()
    per_step = [e0.elapsed_time(e1) for e0, e1 in evs]
    dev_ms = sum(per_step)
    dev_ms_max = _max_over_ranks(dev_ms, world)
    ms_per_product = dev_ms_max / (args.steps * world)

    # end to end through the host-buffer C-ABI call
    ha = torch.from_numpy(a.view(np.int64).copy()).pin_memory().numpy()
    hb = torch.from_numpy(b.view(np.int64).copy()).pin_memory().numpy()
    hout = torch.empty(ow, dtype=torch.int64).pin_memory().numpy()
    G.gf2x_mul_host(ha, na, hb, nb, hout)
    e2e = []
    for _ in range(max(2, args.steps // 2)):
        flush.zero_()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        G.gf2x_mul_host(ha, na, hb, nb, hout)
        e2e.append((time.perf_counter() - t1) * 1e3)
    e2e_ms = _max_over_ranks(sum(e2e) / len(e2e), world) / world

    if rank != 0:
        return
    peaks = _peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    # dominant stage by device time; its kernels are the roofline subject
    dom = max(stages.items(), key=lambda kv: kv[1][0])
    dom_name, (dom_ms, dom_launches, _) = dom
    # algorithmic bytes per launch of the dominant kernel: a one-layer FFT
    # pass reads and writes the N-point array of 16-byte elements
    per_launch_bytes = {"fft": 32 * N, "ifft": 32 * N}.get(dom_name)
    roof = None
    if per_launch_bytes and dom_launches:
        avg_s = dom_ms / 1e3 / dom_launches
        ach = per_launch_bytes / avg_s / 1e9
        roof = {"bound": "hbm", "kernel": "k_fft_layer (%s stage)" % dom_name,
                "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "traffic": None, "bytes_per_launch": per_launch_bytes,
                "avg_launch_ms": avg_s * 1e3, "peak_source": "MEASURED_PEAKS.json hbm_gbs"}
    plan_bytes = 240 * N
    path_frac = plan_bytes / (ms_per_product / 1e3) / 1e9 / hbm
    launches = sum(v[1] for v in stages.values())
    line = {
        "metric": METRIC, "value": ms_per_product, "unit": "ms", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dev_ms_max / args.steps, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": ms_per_product / PAPER_MS_2_28,
        "dtype": "u64", "data": "synthetic",
        "config": {"workload": "single %d x %d-bit product (%s), uniform random bits"
                   % (na, nb, args.workload), "na_bits": na, "nb_bits": nb,
                   "fft_points": N, "l2": "flushed between steps (256 MiB write)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "path_hbm_roofline": {"plan_bytes": plan_bytes, "frac_of_measured_hbm": path_frac},
        "roofline": roof,
        "stages_ms_per_product": {k: v[0] / args.steps for k, v in stages.items()},
        "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": int(a.nbytes + b.nbytes),
                "d2h_bytes_per_step": int(8 * ow)},
        "gpu_launches": launches,
        "clocks": clk,
        "wall_s_timed": wall,
    }
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_sample(a, na, b, nb, args.cpu_depth)
    print(json.dumps(line))


def main():
    args = _args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
