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

--fixpoint NAME runs whole fixpoints of one of the benchmark programs in the
engine's default form (sg-200k, tc-1000, points-to at scale 2^-9,
owl-20m), --repeat times, one JSON line each: the command the ncu captures
of a kernel inside a fixpoint run.

--dist zipf draws the keys Zipf(1.1) over the same domain (the join's probe
keys against unique build keys, so the output stays n rows).  --sweep runs
every step at 2^24, 2^26 and 2^28 (diff_merge and the Zipf cases up to
2^26) for both distributions and prints one JSON line per case.
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


def _zipf(rng, n, universe, s=1.1):
    """Zipf(s) ranks over [0, universe) by inverse CDF, scattered by a
    permutation so hot keys are not the small ones."""
    w = np.arange(1, universe + 1, dtype=np.float64) ** -s
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    r = np.searchsorted(cdf, rng.random(n), side="right")
    return rng.permutation(universe).astype(np.uint32)[np.minimum(r, universe - 1)]


def _bits(v):
    return int(v.max()).bit_length() if v.size else 0


def make_case(step, n, dist, rng, dev, cdl):
    """(run, algorithmic bytes) of one step on n synthetic tuples."""
    keys = (lambda m, u: _zipf(rng, m, u)) if dist == "zipf" else \
        (lambda m, u: rng.integers(0, u, size=m).astype(np.uint32))
    if step == "diff_merge":
        f0, f1 = _pairs(rng, n)
        nu = max(1, n // 8)
        pick = np.sort(rng.choice(n, size=nu // 2, replace=False))
        u0 = np.concatenate([f0[pick], keys(nu - nu // 2, 1 << 18)])
        u1 = np.concatenate([f1[pick], keys(nu - nu // 2, 1 << 18)])
        o = np.lexsort((u1, u0))
        F, U = [dev(f0), dev(f1)], [dev(u0[o]), dev(u1[o])]
        run = lambda: cdl.diff_merge(F, U)
        nd = len(run()[0][0])
        return run, 8 * (n + nu) + 8 * (n + nd) + 8 * nd
    if step == "sort":
        c0, c1 = keys(n, 1 << 18), keys(n, 1 << 18)
        C = [dev(c0), dev(c1)]
        b0, b1 = _bits(c0), _bits(c1)
        total = b0 + b1
        # the library's digit width: 9 where 9-bit digits take one pass fewer
        p8 = (total + 7) // 8
        width = 9 if p8 > 1 and total <= 9 * (p8 - 1) else 8
        npass = (total + width - 1) // width
        # upsweep: 4 B per column holding bits of the pass's digit; scatter:
        # both columns read and written
        up = sum(4 * ((lo < b1) + (lo + width > b1)) for lo in range(0, total, width))
        return (lambda: cdl.sort_unique(C)), (up + 16 * npass) * n
    if step == "scan":
        c = dev(rng.integers(0, 100, size=n).astype(np.uint32))
        return (lambda: cdl.exclusive_scan(c)), 16 * n
    if step == "hash":
        k = dev(np.sort(keys(n, n // 2)))
        return (lambda: cdl.hash_build(k)), 4 * n + 16 * (n // 2)
    # join: build keys unique and sorted, probe keys over the same domain
    b0 = np.sort(rng.permutation(2 * n)[:n].astype(np.uint32))
    b1 = rng.integers(0, 1 << 30, size=n).astype(np.uint32)
    p0 = b0[keys(n, n)]
    p1 = rng.integers(0, 1 << 30, size=n).astype(np.uint32)
    P, B = [dev(p0), dev(p1)], [dev(b0), dev(b1)]
    run = lambda: cdl.join(P, 0, B, 0, [(0, 1), (1, 1)])
    total = len(run()[0])
    return run, (4 + 16 + 4 + 12) * n + 4 * n + 4 * n + (4 + 8) * total


def time_case(run, repeat, flush):
    import torch
    run()  # warm-up
    times = []
    for _ in range(repeat):
        flush.fill_(1)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        run()
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    return float(np.median(times))


FIXPOINTS = {
    "sg-200k": lambda W: W.sg_program(W.random_forest(200_000, 2)),
    "tc-1000": lambda W: W.tc_program(W.er_graph(1000, 1500, 1)),
    "points-to": lambda W: W.points_to_program(W.points_to_edb(1 / 512, 3)),
    "owl-20m": lambda W: W.owl_program(*W.owl_triples(20_000_000, 4)),
}


def run_fixpoints(name, repeat, **opts):
    import time

    import torch

    from . import cdl
    from . import workloads as W

    prog = FIXPOINTS[name](W)
    dev = {nm: [torch.from_numpy(np.ascontiguousarray(r[:, k]).view(np.int32)).cuda()
                for k in range(prog.arity[nm])] for nm, r in prog.edb.items()}
    for i in range(repeat):
        torch.cuda.synchronize()
        t = time.perf_counter()
        with cdl.Engine(**opts) as e:
            for nm, ar in prog.arity.items():
                e.relation(nm, ar)
            e.load_many(dev)
            for r in prog.rules:
                e.rule(r.head, r.body, r.neq)
            st = e.run()
        torch.cuda.synchronize()
        print(json.dumps({"fixpoint": name, "opts": opts, "run": i,
                          "ms": (time.perf_counter() - t) * 1e3,
                          "iterations": st.iterations, "derived": st.derived_tuples,
                          "kernel_launches": st.kernel_launches}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--step", choices=["hash", "join", "sort", "diff_merge", "scan"])
    ap.add_argument("--fixpoint", choices=sorted(FIXPOINTS))
    ap.add_argument("--n", type=int, default=1 << 24)
    ap.add_argument("--repeat", type=int, default=5)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--dist", default="uniform", choices=["uniform", "zipf"])
    ap.add_argument("--sweep", action="store_true")
    ap.add_argument("--dedup", type=int, default=0, choices=[0, 1, 2],
                    help="fixpoints: step (d) as merge (0) or Algorithm 2 (1 hybrid, 2 hash-only)")
    args = ap.parse_args()
    if args.fixpoint:
        run_fixpoints(args.fixpoint, args.repeat, dedup=args.dedup)
        return

    import torch

    from . import cdl

    rng = np.random.default_rng(args.seed)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    if args.sweep:
        cases = [(st, 1 << e, d) for st in ("hash", "join", "sort", "scan", "diff_merge")
                 for e in (24, 26, 28) for d in ("uniform", "zipf")
                 if not ((st == "diff_merge" or d == "zipf") and e > 26)
                 and not (st == "scan" and d == "zipf")]
    else:
        if not args.step:
            ap.error("--step or --sweep")
        cases = [(args.step, args.n, args.dist)]
    for step, n, dist in cases:
        run, algo = make_case(step, n, dist, rng, dev, cdl)
        ms = time_case(run, args.repeat, flush)
        print(json.dumps({"step": step, "n": n, "dist": dist, "ms": ms,
                          "algo_GBps": algo / (ms * 1e-3) / 1e9}), flush=True)
        del run
        torch.cuda.empty_cache()


if __name__ == "__main__":
    main()
