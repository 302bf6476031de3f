"""Benchmark: one 2^28 x 2^28-bit GF(2)[x] product per step on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload c1_2^28] [--no-cpu-baseline] [--no-systems]

Prints ONE JSON line (rank 0).  A step is one whole product (Alg. 5: Split,
BasisCvt, changeRepr, FFT_LCH x2, pointmul, iFFT_LCH, iBasisCvt,
changeRepr^-1, InterleavedCombine) with inputs resident in HBM; `value` is ms
per product (lower is better).  `e2e` times the same product through the
C-ABI call with HOST buffers (gf2x_mul_host: H2D copies, product, D2H copy).
The L2 is flushed (a 256 MiB write) between timed steps, outside the timed
events.  With N > 1 (torchrun) every rank runs independent products (the
single product does not shard: replicas only) and value = max elapsed over
ranks / (N * K) products.

Beside the headline line, `batched` measures 4096 products of log-uniform
lengths in [2^12, 2^22] bits (one batch, CUDA-graph replay, against the same
products one by one) and `serving` a Poisson stream of 2000 requests/s with
lengths log-uniform in [2^10, 2^26] bits and 10% 2^24 x 2^12 pairs, through
the continuous-batching server and a one-at-a-time server.

`--impl reference` times the CPU oracle (the plain Karatsuba carry-less
product) on the host cores on a bounded sample of the same workload, scaled to
ms per product.
"""
import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("ms per 2^28-bit GF(2)[x] product (% HBM roofline); "
          "batched products/s vs one-by-one")
PAPER_MS_2_28 = 2302.0  # Table 2, F~_{2^128} tower row, 2^28-bit operands (Haswell)
# warp shuffles per F~_{2^32} limb product (5-bit windows): seven in the strided
# FFT passes, six in the bottom passes (the 2-bit window on the integer pipe)
SHFL_STRIDED, SHFL_BOTTOM, FFT_TILE_LOG = 7, 6, 12


def shfl_per_limb_mul(M, la, lb):
    """Average shuffles per limb product over the computed layers of one
    product: the layers below 2^12 of each transform run in the bottom pass."""
    bottom = min(la, FFT_TILE_LOG) + min(lb, FFT_TILE_LOG) + min(M, FFT_TILE_LOG)
    strided = (la + lb + M) - bottom
    return (SHFL_BOTTOM * bottom + SHFL_STRIDED * strided) / max(1, bottom + strided)


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="c1_2^28")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-tune", action="store_true",
                   help="use the default plan parameters instead of autotuning the shape")
    p.add_argument("--no-sizes", action="store_true",
                   help="skip the ms-per-product line for 2^29, 2^30 and 2^32 bits")
    p.add_argument("--no-systems", action="store_true",
                   help="skip the batched and serving measurements")
    p.add_argument("--serve-seconds", type=float, default=10.0)
    p.add_argument("--cpu-depth", type=int, default=6,
                   help="Karatsuba depth of the CPU-baseline sample (3^d sub-products)")
    return p.parse_args()


def _dist_init(n):
    rank, world, local = 0, 1, 0
    if n > 1 or int(os.environ.get("WORLD_SIZE", "1")) > 1:
        import torch
        import torch.distributed as dist
        rank = int(os.environ.get("RANK", "0"))
        world = int(os.environ.get("WORLD_SIZE", "1"))
        local = int(os.environ.get("LOCAL_RANK", "0"))
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
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
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        # raw samples go to a scratch file (GF2X_CLOCKS_DIR, else the system's
        # temporary directory); the JSON line carries their summary
        self.path = os.path.join(os.environ.get("GF2X_CLOCKS_DIR", tempfile.gettempdir()),
                                 "gf2x_clocks_bench_%d.csv" % os.getpid())

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.f, stderr=subprocess.DEVNULL)
            # the timed region starts once the sampler is producing lines
            t0 = time.time()
            while time.time() - t0 < 3.0 and os.path.getsize(self.path) == 0:
                time.sleep(0.02)
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


def cpu_sample(a, na, b, nb, depth, reps=1, single_thread=False):
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
    out = {"value": best * 1e3 * scale, "unit": "ms", "cores": P.num_threads(),
           "kind": "oracle",
           "sample": "1 of 3^%d Karatsuba sub-products (%d x %d bits: the low "
                     "parts of a and b), all cores, x%d; upper-level linear "
                     "recombination not included" % (depth, 64 * sub_w, 64 * sub_w, scale),
           "sample_s": best}
    if single_thread:
        # the same estimate on one core, from a sub-product two levels deeper
        d1 = depth + 2
        w1 = max(1, nw >> d1)
        t0 = time.perf_counter()
        P.mul(a[:w1].copy(), 64 * w1, b[:w1].copy(), 64 * w1, threads=1)
        dt1 = time.perf_counter() - t0
        out["one_core"] = {"value": dt1 * 1e3 * 3 ** d1, "unit": "ms", "cores": 1,
                           "sample": "1 of 3^%d sub-products (%d x %d bits), one core, x%d"
                                     % (d1, 64 * w1, 64 * w1, 3 ** d1),
                           "sample_s": dt1}
    out["host"] = _host_cpu()
    return out


def _host_cpu():
    model = ""
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part", "hardware")):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    import platform
    return {"machine": platform.machine(), "model": model, "nproc": os.cpu_count()}


def cpu_whole(a, na, b, nb):
    """The oracle's whole product of the workload on all host cores (the
    Karatsuba carry-less product over the host's fastest word product), one
    run, in ms."""
    from oracle import product as P
    t0 = time.perf_counter()
    P.mul(a, na, b, nb)
    dt = time.perf_counter() - t0
    return {"value": dt * 1e3, "unit": "ms", "cores": P.num_threads(), "kind": "oracle",
            "sample": "one whole %d x %d-bit product, all cores, word product %s"
                      % (na, nb, P.clmul_kind()),
            "clmul": P.clmul_kind(), "host": _host_cpu()}


def pick_cpu_depth(a, na, b, nb, budget_s):
    """Karatsuba depth of a sub-product sample that takes about budget_s
    seconds on all cores (each level deeper is about 3x less work)."""
    from oracle import product as P
    nw = max((na + 63) // 64, (nb + 63) // 64)
    d = 8
    while d > 0:
        w = max(1, nw >> d)
        t0 = time.perf_counter()
        P.mul(a[:w].copy(), 64 * w, b[:w].copy(), 64 * w)
        dt = time.perf_counter() - t0
        if dt * 3 > budget_s or (nw >> (d - 1)) < 64:
            return d
        d -= 1
    return 0


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import workloads as W
    from oracle import build as ob
    ob.build()
    a, na, b, nb = W.make_workload(args.workload)
    # each step is a bounded sample: about 150 s of CPU work over the whole run
    depth = pick_cpu_depth(a, na, b, nb, max(0.05, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_sample(a, na, b, nb, depth)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_sample(a, na, b, nb, depth))
    wall = time.perf_counter() - t0
    v = sum(x["value"] for x in vals) / len(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "ms",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": wall * 1e3 / args.steps, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": v / PAPER_MS_2_28, "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": "single %d x %d-bit product (%s), uniform random bits"
                   % (na, nb, args.workload), "na_bits": na, "nb_bits": nb},
        "cpu_baseline": {"kind": "oracle", "cores": vals[0]["cores"],
                         "sample": vals[0]["sample"], "value": v, "unit": "ms"},
        "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def fft_work(na, nb):
    """F~_{2^32} limb products of FFT(a), FFT(b) and iFFT: 4 per butterfly,
    N/2 butterflies per computed layer (the fan-out layers above log2 P
    multiply by zero and are not computed)."""
    def lg(x):
        return max(0, (x - 1).bit_length())
    na_w, nb_w = (na + 63) // 64, (nb + 63) // 64
    M = lg(max(2, na_w + nb_w - 1))
    N = 1 << M
    return 4 * (N // 2) * (lg(na_w) + lg(nb_w) + M), N, M, lg(na_w), lg(nb_w)


def fft_plan_bytes(N, la, lb):
    """Algorithmic HBM bytes of the FFT passes of one product in the minimal
    pass plan of the path's byte model: FFT(a) = changeRepr'd blocks in (I_a)
    + one global pass (W out) + one local pass (2W); FFT(b) the same, its local
    pass also reading FFT(a) and running pointmul and the bottom inverse layers
    (I_b + W + 3W); the inverse global pass 2W.  I_x = 8 P_x padded input bytes,
    W = 16 N transform bytes: I_a + I_b + 9W (2I + 9W for equal operands)."""
    W = 16 * N
    return 8 * (1 << la) + 8 * (1 << lb) + 9 * W


def fft_hbm_bytes(N, M, la, lb, depth=7):
    """Bytes the FFT passes (k_fft_pass) of one product move at least: each
    pass a tile in and a tile out (the first strided pass reading only the P
    elements changeRepr staged, a lone bottom pass the P blocks), the fused
    pass also reading the other transform.  Passes: layers 12 .. log2 P
    (forward) or M (inverse) in strided passes of at most `depth` layers,
    then the 4096-element bottom pass."""
    def strided(layers):
        return max(0, -(-(layers - 12) // depth))
    b = 0
    for L in (la, lb):
        P = 1 << L
        s = strided(L)
        if s:
            b += 16 * P + 16 * N                     # first strided pass
            b += (s - 1) * 32 * N + 32 * N           # other strided passes, bottom pass
        else:
            b += 8 * P + 16 * N                      # bottom pass converts the blocks
    b += 16 * N                                      # fused pass reads FA
    b += strided(M) * 32 * N                         # inverse top passes
    return b


FFT_KERNEL_SOURCES = ("fft_pass.cu", "fft_pass.h", "gf2x_mul.cuh", "gf2x_dev.cuh", "tma.cuh")
FFT_PROFILE = os.path.join(ROOT, "profiles", "k_fft_pass_2^28.md")


def fft_sources_sha256():
    """sha256 over the sources of k_fft_pass, in a fixed order."""
    h = hashlib.sha256()
    for name in FFT_KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1708_09746_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def fft_traffic_per_launch():
    """DRAM bytes (read + write) per k_fft_pass launch from the committed ncu
    summary, if it was taken on the current kernel sources; else None."""
    try:
        text = open(FFT_PROFILE).read()
    except OSError:
        return None
    mb = re.search(r"^traffic_bytes_per_launch: (\d+)$", text, re.M)
    mh = re.search(r"^kernel_sources_sha256: ([0-9a-f]{64})$", text, re.M)
    if not mb or not mh or mh.group(1) != fft_sources_sha256():
        return None
    return {"bytes": int(mb.group(1)), "source": "profiles/k_fft_pass_2^28.md (ncu, sources sha256 %s)"
            % mh.group(1)[:12]}


def measure_sizes(G, torch, W, dev, stream, flush):
    """ms per product (device time, autotuned plan, L2 flushed between
    products) for the larger single-product workloads."""
    import numpy as np
    res = {}
    for name in ("c1_2^29", "c1_2^28x2^16", "c1_2^28+64", "c1_2^28x64", "c2_2^30", "c2_2^32"):
        a, na, b, nb = W.make_workload(name)
        da = torch.from_numpy(a.view(np.int64)).to(dev)
        db = torch.from_numpy(b.view(np.int64)).to(dev)
        del a, b
        out = torch.empty(G.gf2x_out_words(na, nb), dtype=torch.int64, device=dev)
        # unbalanced operands run by chunks of the long one (their own plan,
        # default parameters), a short operand directly, a length just past a
        # power of two by the tail split; the others with the shape's
        # autotuned plan
        path, ma, mb = G.gf2x_product_path(na, nb)
        if path == 1:
            chunking = G.gf2x_chunking(na, nb)
            tuned = ("chunked product (%d chunks of %d words, %d-point transforms), default plan "
                     "parameters" % (chunking[1], chunking[0], chunking[2]))
        elif path == 2:
            tuned = "direct product by the short operand (no transform)"
        elif path == 3:
            tuned = ("tail split: main product of %d x %d words (%d-point transform) plus the "
                     "direct tail products" % (ma, mb, G.gf2x_fft_points(64 * ma, 64 * mb)))
        else:
            tuned = G.gf2x_autotune(na, nb, 2)
        evs = []
        with torch.cuda.stream(stream):
            for i in range(4):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                G.gf2x_mul_async(da, na, db, nb, out, stream)
                e1.record(stream)
                evs.append((e0, e1))
        stream.synchronize()
        ms = [e0.elapsed_time(e1) for e0, e1 in evs[1:]]
        N = G.gf2x_fft_points(na, nb)
        # the whole-path byte model (240 N) describes one transform of N points;
        # chunked, direct and split products move other amounts
        frac = (240 * N / (sum(ms) / len(ms) / 1e3) / 1e9 / _peaks().get("hbm_gbs", 6800.0)
                if path == 0 else None)
        res[name] = {"bits": [na, nb], "ms": sum(ms) / len(ms), "fft_points": N,
                     "path": ["one transform", "chunked", "direct", "tail split"][path],
                     "path_hbm_frac": frac, "plan": tuned}
        del da, db, out
        torch.cuda.empty_cache()
    return res


def measure_variants(G, torch, dev, stream, flush, da, na, db, nb, out, ref_ms):
    """The paper's other forms of the product on the headline workload, each
    through its own C-ABI call (device time, L2 flushed between products,
    3 timed runs after one untimed), checked word for word against the
    headline product's output."""
    import numpy as np
    ref = out.clone()
    res = {}
    forms = [("tower256_w128", G.gf2x_mul_tower256_async,
              "F~_{2^256} tower field, 128-bit blocks (Sec. 4.3, Table 2 F~_{2^256} row), %d points"
              % G.gf2x_tower256_fft_points(na, nb)),
             ("simple_gf2_128_poly", G.gf2x_mul_simple_async,
              "GF(2^128) polynomial basis, Cantor-basis points, general products by emulated "
              "carry-less multiply (Alg. 4, Table 2 simple row), %d points"
              % G.gf2x_fft_points(na, nb)),
             ("frobenius_truncated", G.gf2x_mul_frobenius_async,
              "Frobenius partition / truncated additive FFT, GF(2^128) polynomial basis, "
              "BasisCvt on bits, 7-layer encoding (Appendix C, Table 3), %d points"
              % (1 << G.gf2x_frobenius_points(na, nb)))]
    for name, fn, desc in forms:
        try:
            evs = []
            with torch.cuda.stream(stream):
                for i in range(4):
                    flush.zero_()
                    out.zero_()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    fn(da, na, db, nb, out, stream)
                    e1.record(stream)
                    evs.append((e0, e1))
            stream.synchronize()
            G.gf2x_stream_status(stream)
            ms = [e0.elapsed_time(e1) for e0, e1 in evs[1:]]
            v = sum(ms) / len(ms)
            res[name] = {"ms": v, "vs_f2_128_form": v / ref_ms, "form": desc,
                         "same_product": bool(torch.equal(out, ref))}
        except Exception as e:  # report, keep the headline line
            res[name] = {"error": repr(e)}
    out.copy_(ref)
    return res


def measure_batched(G, torch, W, dev, stream):
    """4096 products, lengths floor(2^U) with U ~ U[12, 22] per side (seed 7);
    operands are slices of one seeded random-word pool (seed 7)."""
    lens = W.log_uniform_lengths(7, 2 * 4096, 12, 22)
    na = [int(x) for x in lens[0::2]]
    nb = [int(x) for x in lens[1::2]]
    words = [((x + 63) // 64) for x in na + nb]
    pool_n = sum(words)
    pool = torch.from_numpy(W.random_words(7, pool_n).view("int64")).to(dev)
    offs, o = [], 0
    for w in words:
        offs.append(o)
        o += w
    A = [pool[offs[i]:offs[i] + words[i]] for i in range(4096)]
    B = [pool[offs[4096 + i]:offs[4096 + i] + words[4096 + i]] for i in range(4096)]
    outs = [torch.empty(G.gf2x_out_words(na[i], nb[i]), dtype=torch.int64, device=dev)
            for i in range(4096)]
    # one by one: gf2x_mul_async per product on one stream (plans cached)
    for i in range(4096):
        G.gf2x_mul_async(A[i], na[i], B[i], nb[i], outs[i], stream)
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(4096):
        G.gf2x_mul_async(A[i], na[i], B[i], nb[i], outs[i], stream)
    e1.record(stream)
    stream.synchronize()
    t_loop = e0.elapsed_time(e1) / 1e3
    # batched: one batch, captured once and replayed
    def run_batch():
        batch = G.gf2x_batch_create(na, nb, 8 << 30)
        try:
            G.gf2x_batch_execute(batch, A, B, outs, stream)
            stream.synchronize()
            reps = 3
            e0.record(stream)
            for _ in range(reps):
                G.gf2x_batch_execute(batch, A, B, outs, stream)
            e1.record(stream)
            stream.synchronize()
            return e0.elapsed_time(e1) / 1e3 / reps
        finally:
            G.gf2x_batch_destroy(batch)
    t_default = run_batch()
    # tune the batch in batch context (each shape group on its own grouped
    # launch), then replay it
    batch = G.gf2x_batch_create(na, nb, 8 << 30)
    try:
        G.gf2x_batch_execute(batch, A, B, outs, stream)
        stream.synchronize()
        t0 = time.perf_counter()
        groups_before, groups_after = G.gf2x_batch_tune(batch, 2)
        t_tune = time.perf_counter() - t0
        G.gf2x_batch_execute(batch, A, B, outs, stream)  # captures the tuned graph
        stream.synchronize()
        reps = 3
        e0.record(stream)
        for _ in range(reps):
            G.gf2x_batch_execute(batch, A, B, outs, stream)
        e1.record(stream)
        stream.synchronize()
        G.gf2x_batch_status(batch)
        t_batch = e0.elapsed_time(e1) / 1e3 / reps
    finally:
        G.gf2x_batch_destroy(batch)
    shapes = {"groups_ms_before": groups_before, "groups_ms_after": groups_after}
    del pool, A, B, outs
    torch.cuda.empty_cache()
    return {"workload": "4096 products, per-side lengths log-uniform in [2^12, 2^22] bits, "
                        "seed 7", "products": 4096,
            "batched_products_per_s": 4096 / t_batch,
            "batched_default_params_products_per_s": 4096 / t_default,
            "one_by_one_products_per_s": 4096 / t_loop,
            "speedup": t_loop / t_batch, "unit": "products/s",
            "batch_tune": dict(shapes, seconds=t_tune),
            "method": "gf2x_batch_execute (shape-grouped launches, direct products by short "
                      "operands in one launch, CUDA graph replay) tuned in batch context "
                      "(gf2x_batch_tune) vs gf2x_mul_async in a loop, device-timed"}


def measure_serving(G, torch, W, dev, seconds):
    """Poisson arrivals at 2000/s for `seconds` (seed 8); per-side lengths
    floor(2^U), U ~ U[10, 26], except 10% 2^24 x 2^12 pairs; operands are
    slices of a seeded random pool, outputs a ring of 256 buffers."""
    import numpy as np
    t_arr = W.poisson_arrivals(8, 2000.0, seconds)
    n = len(t_arr)
    lens = W.log_uniform_lengths(8, 2 * n, 10, 26)
    pick = W.random_words(9, n)
    na, nb = [], []
    for i in range(n):
        if int(pick[i]) % 10 == 0:
            na.append(1 << 24)
            nb.append(1 << 12)
        else:
            na.append(int(lens[2 * i]))
            nb.append(int(lens[2 * i + 1]))
    pool_words = 1 << 21  # 16 MiB: operands start at seeded offsets in it
    pool = torch.from_numpy(W.random_words(10, 2 * pool_words).view("int64")).to(dev)
    starts = [int(x) % pool_words for x in W.random_words(11, 2 * n)]
    ring = 512  # one output buffer per request in flight
    max_out = (1 << 21) + 2
    outs = torch.empty((ring, max_out), dtype=torch.int64, device=dev)
    res = {}
    for label, slots, batch in (("continuous_batching", 16, 64), ("one_at_a_time", 1, 1)):
        sv = G.gf2x_server_create(16 << 30, slots, batch)
        try:
            tickets = []
            t0 = time.perf_counter()
            for i in range(n):
                while time.perf_counter() - t0 < t_arr[i]:
                    pass
                if i >= ring:
                    G.gf2x_server_wait(sv, tickets[i - ring], 120_000_000)
                a = pool[starts[2 * i]:starts[2 * i] + (na[i] + 63) // 64]
                b = pool[starts[2 * i + 1]:starts[2 * i + 1] + (nb[i] + 63) // 64]
                tickets.append(G.gf2x_server_submit(sv, a, na[i], b, nb[i], outs[i % ring]))
            for i in range(max(0, n - ring), n):
                G.gf2x_server_wait(sv, tickets[i], 120_000_000)
            wall = time.perf_counter() - t0
            p50, p99, thr, done = G.gf2x_server_stats(sv)
            res[label] = {"p50_ms": p50, "p99_ms": p99, "throughput_per_s": thr,
                          "completed": done, "wall_s": wall, "slots": slots,
                          "max_batch": batch}
        finally:
            G.gf2x_server_destroy(sv)
    # saturated: a closed loop keeping `depth` requests in flight (the same
    # request sequence, cycled) for the same duration: the completed requests
    # per second show what each server can carry, not the offered load
    depth = 512
    sat = {}
    for label, slots, batch in (("continuous_batching", 16, 64), ("one_at_a_time", 1, 1)):
        sv = G.gf2x_server_create(16 << 30, slots, batch)
        try:
            tickets = []
            t0 = time.perf_counter()
            i = 0
            while time.perf_counter() - t0 < seconds:
                if len(tickets) >= depth:
                    G.gf2x_server_wait(sv, tickets[i - depth], 120_000_000)
                k = i % n
                a = pool[starts[2 * k]:starts[2 * k] + (na[k] + 63) // 64]
                b = pool[starts[2 * k + 1]:starts[2 * k + 1] + (nb[k] + 63) // 64]
                tickets.append(G.gf2x_server_submit(sv, a, na[k], b, nb[k], outs[i % ring]))
                i += 1
            for t in tickets[max(0, len(tickets) - depth):]:
                G.gf2x_server_wait(sv, t, 120_000_000)
            wall = time.perf_counter() - t0
            p50, p99, thr, done = G.gf2x_server_stats(sv)
            sat[label] = {"requests": i, "wall_s": wall, "throughput_per_s": i / wall,
                          "p50_ms": p50, "p99_ms": p99, "slots": slots, "max_batch": batch}
        finally:
            G.gf2x_server_destroy(sv)
    sat["in_flight"] = depth
    sat["throughput_ratio"] = (sat["continuous_batching"]["throughput_per_s"] /
                               sat["one_at_a_time"]["throughput_per_s"])
    res["saturated"] = sat
    del pool, outs
    torch.cuda.empty_cache()
    res["workload"] = ("Poisson 2000 req/s for %.1f s (%d requests), per-side lengths "
                       "log-uniform in [2^10, 2^26] bits, 10%% 2^24 x 2^12, seed 8; saturated: "
                       "the same requests cycled with %d in flight for %.1f s"
                       % (seconds, n, depth, seconds))
    res["requests"] = n
    return res


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

    # plan parameters for this shape from the autotuner (not timed)
    tuned = G.gf2x_autotune(na, nb, 3) if not args.no_tune else G.gf2x_tune_get(na, nb)

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
    # the dominant kernel: k_fft_pass runs every FFT stage
    fft_stages = ["fft_a", "fft_b", "fft_pointmul_ifft_bottom", "ifft_top"]
    fft_ms = sum(stages[k][0] for k in fft_stages) / args.steps
    fft_launches = sum(stages[k][1] for k in fft_stages) / args.steps
    total_stage_ms = sum(v[0] for v in stages.values()) / args.steps
    work, _, M, la, lb = fft_work(na, nb)
    sm_mhz = clk.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    # the shuffle issue rate measured on this device (gf2x_probe_pipes); the
    # nominal one shuffle per SM per clock if the probe fails
    try:
        probe = G.gf2x_probe_pipes()
    except Exception as e:  # report the failure, keep the nominal peak
        probe = {"error": str(e)}
    shfl_rate = probe.get("shfl_per_clk_sm") or 1.0
    sms = probe.get("sms") or 152
    spl = shfl_per_limb_mul(M, la, lb)
    peak_lmul = sms * shfl_rate * 32 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / spl
    ach_lmul = work / (fft_ms / 1e3)
    traffic = fft_traffic_per_launch()
    # The dominant kernel against the HBM roofline, bytes from the path's byte
    # model (I_a + I_b + 9W for the FFT passes), per launch over the measured
    # average launch time, against the measured copy bandwidth.
    n_launch = max(1, fft_launches)
    alg_bytes = fft_plan_bytes(N, la, lb)
    alg_per_launch = alg_bytes / n_launch
    avg_launch_s = fft_ms / 1e3 / n_launch
    roof = {"bound": "hbm", "kernel": "k_fft_pass (all FFT_LCH / iFFT_LCH passes)",
            "achieved": alg_per_launch / avg_launch_s / 1e9, "peak": hbm, "unit": "GB/s",
            "frac": alg_per_launch / avg_launch_s / 1e9 / hbm,
            "traffic": traffic["bytes"] if traffic else None,
            "traffic_unit": "bytes per launch (DRAM read + write, ncu)",
            "traffic_source": traffic["source"] if traffic else
            "none for these kernel sources (captured for other sources, or no capture)",
            "algorithmic_bytes_per_launch": alg_per_launch,
            "algorithmic_bytes_per_product": alg_bytes,
            "traffic_over_algorithmic": (traffic["bytes"] / alg_per_launch) if traffic else None,
            "launches_per_product": fft_launches,
            "avg_launch_ms": avg_launch_s * 1e3,
            "share_of_step": fft_ms / max(1e-9, total_stage_ms),
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured copy bandwidth, burst)",
            "bytes_model": "I_a + I_b + 9 W (I_x = 8 P_x, W = 16 N): changeRepr'd blocks in, "
                           "one global + one local pass per forward transform, the local pass "
                           "of b also reading FFT(a), one inverse global pass"}
    roof_alu = {"bound": "alu", "kernel": "k_fft_pass",
            "note": "ceiling of the current butterfly method (%.2f warp shuffles per "
                    "F~_{2^32} limb product: 7 in strided passes, 6 in bottom passes), not of "
                    "the chip or the algorithm" % spl,
            "achieved": ach_lmul / 1e9, "peak": peak_lmul / 1e9,
            "unit": "G limb-mult/s", "frac": ach_lmul / peak_lmul,
            "work_per_launch": work / n_launch,
            "peak_source": ("measured shuffle issue rate (gf2x_probe_pipes: %.3f warp shuffles "
                            "per SM clock) x %d SMs x 32 lanes x max SM clock / %.2f shuffles per "
                            "F~_{2^32} limb product" % (shfl_rate, sms, spl))
            if "shfl_per_clk_sm" in probe else
            "derived: 152 SMs x 32 lanes x max SM clock / %.2f warp shuffles per F~_{2^32} "
            "limb product (probe failed: %s)" % (spl, probe.get("error")),
            "pipe_probe": probe}
    plan_depth = max(1, min(7, int(tuned.get("fft_depth", 7))))
    fbytes = fft_hbm_bytes(N, M, la, lb, plan_depth)
    # the same kernel against the bytes its actual pass schedule moves
    roof_sched = {"bound": "hbm", "kernel": "k_fft_pass",
                  "achieved": fbytes / (fft_ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                  "frac": fbytes / (fft_ms / 1e3) / 1e9 / hbm, "bytes_per_product": fbytes,
                  "note": "bytes of the pass schedule the plan runs (strided passes of at most "
                          "%d layers + 4096-element bottom passes), not the minimal plan"
                          % plan_depth}
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
        "roofline_schedule_bytes": roof_sched,
        "roofline_alu_method": roof_alu,
        "stages_ms_per_product": {k: v[0] / args.steps for k, v in stages.items()},
        "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": int(a.nbytes + b.nbytes),
                "d2h_bytes_per_step": int(8 * ow)},
        "gpu_launches": launches,
        "clocks": clk,
        "wall_s_timed": wall,
    }
    line["config"]["plan"] = tuned
    if world == 1:
        line["variants_ms"] = measure_variants(G, torch, dev, stream, flush, da, na, db, nb, out,
                                               ms_per_product)
    if not args.no_sizes and world == 1:
        line["sizes_ms"] = measure_sizes(G, torch, W, dev, stream, flush)
    if not args.no_systems and world == 1:
        try:
            line["batched"] = measure_batched(G, torch, W, dev, stream)
        except Exception as e:  # report, keep the headline line
            line["batched"] = {"error": repr(e)}
        try:
            line["serving"] = measure_serving(G, torch, W, dev, args.serve_seconds)
        except Exception as e:
            line["serving"] = {"error": repr(e)}
    if not args.no_cpu_baseline and world == 1:
        from oracle import build as ob
        from oracle import product as P
        ob.build()
        if P.clmul_kind() == "pmull" or max(na, nb) <= (1 << 24):
            # the whole product on all cores; the one-core figure from a sample
            cb = cpu_whole(a, na, b, nb)
            samp = cpu_sample(a, na, b, nb, args.cpu_depth, single_thread=True)
            cb["one_core"] = samp.get("one_core")
            cb["all_cores_sample_estimate"] = {k: samp[k] for k in ("value", "sample")}
        else:
            cb = cpu_sample(a, na, b, nb, args.cpu_depth, single_thread=True)
        line["cpu_baseline"] = cb
        line["vs_oracle"] = cb["value"] / ms_per_product
    print(json.dumps(line))


def main():
    args = _args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
