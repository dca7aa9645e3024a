"""Single-step micro-benchmarks: one step of the round through the C ABI on
synthetic uint32 tuples, timed with CUDA events on the launching stream,
reported as algorithmic GB/s (the bytes the step must move / its time).

  python -m paper_2501_13051_gb300.microbench --step diff_merge --n 50000000
  python -m paper_2501_13051_gb300.microbench --step sort --n 16777216
  python -m paper_2501_13051_gb300.microbench --step join --n 16777216

Steps: hash (build the index of n sorted keys), join (three-pass join of n
probe rows against n build rows, two head columns), sort (sort + unique of n
pairs with 18-bit columns), diff_merge (n sorted full pairs against n/8
sorted new pairs, half of them already in full), scan (n counts).  Inputs
exceed the 129 MB L2 for n >= 2^24, and each timed repeat is preceded by an
L2-sized write.  Used for the ncu captures of single kernels.
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def _pairs(rng, n, bits=18):
    keys = np.unique(rng.integers(0, 1 << (2 * bits), size=int(n * 1.05), dtype=np.uint64))
    rng.shuffle(keys)
    keys = np.sort(keys[:n])
    return (keys >> np.uint64(bits)).astype(np.uint32), (keys & np.uint64((1 << bits) - 1)).astype(np.uint32)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--step", required=True, choices=["hash", "join", "sort", "diff_merge", "scan"])
    ap.add_argument("--n", type=int, default=1 << 24)
    ap.add_argument("--repeat", type=int, default=5)
    ap.add_argument("--seed", type=int, default=1)
    args = ap.parse_args()

    import torch

    from . import cdl

    rng = np.random.default_rng(args.seed)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    n = args.n
    if args.step == "diff_merge":
        f0, f1 = _pairs(rng, n)
        nu = max(1, n // 8)
        pick = np.sort(rng.choice(n, size=nu // 2, replace=False))
        u0 = np.concatenate([f0[pick], rng.integers(0, 1 << 18, size=nu - nu // 2).astype(np.uint32)])
        u1 = np.concatenate([f1[pick], rng.integers(0, 1 << 18, size=nu - nu // 2).astype(np.uint32)])
        o = np.lexsort((u1, u0))
        F, U = [dev(f0), dev(f1)], [dev(u0[o]), dev(u1[o])]
        run = lambda: cdl.diff_merge(F, U)
        nd = len(run()[0][0])
        algo = 8 * (n + nu) + 8 * (n + nd) + 8 * nd
    elif args.step == "sort":
        c0 = rng.integers(0, 1 << 18, size=n).astype(np.uint32)
        c1 = rng.integers(0, 1 << 18, size=n).astype(np.uint32)
        C = [dev(c0), dev(c1)]
        run = lambda: cdl.sort_unique(C)
        algo = None  # reported per kernel class by the engine profiler instead
    elif args.step == "scan":
        c = dev(rng.integers(0, 100, size=n).astype(np.uint32))
        run = lambda: cdl.exclusive_scan(c)
        algo = 4 * n + 4 * n + 8 * n
    elif args.step == "hash":
        k = dev(np.sort(rng.integers(0, n // 2, size=n).astype(np.uint32)))
        run = lambda: cdl.hash_build(k)
        algo = 4 * n + 16 * (n // 2)
    else:
        b0 = np.sort(rng.integers(0, n, size=n).astype(np.uint32))
        b1 = rng.integers(0, 1 << 30, size=n).astype(np.uint32)
        p0 = rng.integers(0, n, size=n).astype(np.uint32)
        p1 = rng.integers(0, 1 << 30, size=n).astype(np.uint32)
        P, B = [dev(p0), dev(p1)], [dev(b0), dev(b1)]
        run = lambda: cdl.join(P, 0, B, 0, [(0, 1), (1, 1)])
        total = len(run()[0])
        algo = (4 + 16 + 4 + 12) * n + 4 * n + 4 * n + (4 + 8) * total
    run()  # warm-up
    times = []
    for _ in range(args.repeat):
        flush.fill_(1)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        run()
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    ms = float(np.median(times))
    out = {"step": args.step, "n": n, "ms": ms}
    if algo:
        out["algo_GBps"] = algo / (ms * 1e-3) / 1e9
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
