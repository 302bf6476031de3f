"""Multiply two seeded random operands on cuda:0 and print the time per product.

    python -m paper_1708_09746_gb300 --log-bits 28 --reps 2 [--plan 7 2 11 256]
                                     [--form tower|tower256|simple|frobenius]

Each operand has 2^log_bits bits (top bit set, uniform otherwise, seed 1).  The
first product is a warm-up (it builds the plan and the tables); the command
prints the duration of each product.  It is the small driver used for launch
lists and kernel captures: a fixed, short launch sequence (one product = the
same launches every time).
"""
import argparse
import time

import numpy as np
import torch

from . import build as _build


def main():
    p = argparse.ArgumentParser(prog="python -m paper_1708_09746_gb300")
    p.add_argument("--log-bits", type=int, default=28)
    p.add_argument("--log-bits-b", type=int, default=None,
                   help="log2 of b's length (default: the same as a)")
    p.add_argument("--reps", type=int, default=2)
    p.add_argument("--plan", type=int, nargs=4, metavar=("DEPTH", "BUFFERS", "TILE_LOG", "THREADS"),
                   help="plan parameters of the shape (gf2x_tune_set) instead of the defaults")
    p.add_argument("--autotune", action="store_true",
                   help="run gf2x_autotune for the shape first and print its choice")
    p.add_argument("--form", default="tower", choices=["tower", "tower256", "simple", "frobenius"],
                   help="the form of the method: tower field F~_{2^128} with 64-bit blocks "
                        "(gf2x_mul), F~_{2^256} with 128-bit blocks, the simple polynomial-"
                        "basis form, or the Frobenius partition")
    args = p.parse_args()
    _build.build()
    import paper_1708_09746_gb300 as G
    import workloads as W

    na = 1 << args.log_bits
    nb = 1 << (args.log_bits if args.log_bits_b is None else args.log_bits_b)
    a, b = W.operand_pair(1, na, nb)
    da = torch.from_numpy(a.view(np.int64)).cuda()
    db = torch.from_numpy(b.view(np.int64)).cuda()
    out = torch.empty(G.gf2x_out_words(na, nb), dtype=torch.int64, device="cuda")
    if args.plan:
        G.gf2x_tune_set(na, nb, *args.plan)
    if args.autotune:
        print("autotune:", G.gf2x_autotune(na, nb))
    torch.cuda.synchronize()
    fn = {"tower": G.gf2x_mul, "tower256": G.gf2x_mul_tower256, "simple": G.gf2x_mul_simple,
          "frobenius": G.gf2x_mul_frobenius}[args.form]
    for i in range(args.reps):
        t0 = time.perf_counter()
        fn(da, na, db, nb, out)
        torch.cuda.synchronize()
        print("product %d (%s): %d x %d bits, %.3f ms" % (i, args.form, na, nb,
                                                      1e3 * (time.perf_counter() - t0)))


if __name__ == "__main__":
    main()
