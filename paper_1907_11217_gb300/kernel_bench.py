"""Time one kernel of the library on a given shape (CUDA events, after
warm-up) and print one JSON line. Used to tune the kernels and as a small,
self-contained target for profiler captures.

    python -m paper_1907_11217_gb300.kernel_bench --op cgemm --precision tf32x3 \\
        --batch 2 --m 16384 --n 1024 --k 2048
    python -m paper_1907_11217_gb300.kernel_bench --op permute --rank 28
"""
import argparse
import json

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--op", choices=["cgemm", "permute"], default="cgemm")
    ap.add_argument("--precision", default="tf32x3", choices=["c64", "tf32x3", "bf16x3", "fp16x3", "c128"])
    ap.add_argument("--batch", type=int, default=1)
    ap.add_argument("--m", type=int, default=4096)
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--k", type=int, default=256)
    ap.add_argument("--rank", type=int, default=26)
    ap.add_argument("--iters", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--pairs", type=int, default=-1, choices=[-1, 0, 1],
                    help="split BF16/FP16 products: 1 pairs of CTAs, 0 single CTAs, -1 default")
    ap.add_argument("--prefetch", type=int, default=-1,
                    help="L2 prefetch distance of A tiles in k-blocks (0 off, -1 default)")
    a = ap.parse_args()
    import torch
    import paper_1907_11217_gb300 as tz
    tz.tz_tune_tc_pairs(a.pairs)
    tz.tz_tune_tc_prefetch(a.prefetch)
    dev = "cuda"
    if a.op == "permute":
        x = torch.randn(2 << a.rank, device=dev)
        y = torch.empty_like(x)
        perm = list(np.random.default_rng(0).permutation(a.rank))
        run = lambda: tz.tz_op_permute(x, y, perm)
        flops, nbytes, shape = 0.0, 2 * 8.0 * (1 << a.rank), {"rank": a.rank}
    else:
        dt = torch.float64 if a.precision == "c128" else torch.float32
        esz = 16 if a.precision == "c128" else 8
        A = torch.randn(a.batch * a.m * a.k * 2, device=dev, dtype=dt)
        B = torch.randn(a.batch * a.n * a.k * 2, device=dev, dtype=dt)
        C = torch.empty(a.batch * a.m * a.n * 2, device=dev, dtype=dt)
        scratch = None
        if a.precision in ("tf32x3", "bf16x3", "fp16x3"):
            nb = tz.tz_op_cgemm_scratch_bytes(a.precision, a.batch, a.m, a.n, a.k)
            scratch = torch.empty(nb // 4 + 64, device=dev, dtype=torch.float32)
        run = lambda: tz.tz_op_cgemm(a.precision, a.batch, a.m, a.n, a.k, A, a.m * a.k, B, a.n * a.k, C, a.m * a.n,
                                     scratch=scratch)
        flops = 8.0 * a.batch * a.m * a.n * a.k
        nbytes = esz * a.batch * (a.m * a.k + a.n * a.k + a.m * a.n)
        shape = {"batch": a.batch, "m": a.m, "n": a.n, "k": a.k}
    for _ in range(a.warmup):
        run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.iters):
        run()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.iters
    print(json.dumps({"op": a.op, "precision": a.precision, **shape, "pairs": a.pairs, "prefetch": a.prefetch, "ms": ms,
                      "useful_tflops": flops / ms / 1e9, "algorithmic_gbs": nbytes / ms / 1e6}))


if __name__ == "__main__":
    main()
