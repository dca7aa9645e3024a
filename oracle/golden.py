"""Writes the stored expected values of the full-size fixpoint tests.

TEST INFRASTRUCTURE ONLY.  Run as ``python -m oracle.golden [name ...]`` from
the repository root; it calls only this package (the std::set evaluator of
oracle.cpp) and the seeded input generators, and writes
``tests/golden/fixpoint_<name>.json``.  Nothing here touches a GPU.

Each file holds, per relation, the size and the SHA-256 of the relation's
tuples as the oracle exports them (sorted lexicographically by unsigned
column value, unique, row-major little-endian uint32), the per-round delta
sizes, the iteration count, the derived total, and, for batched runs, every
instance's sizes and iteration count.  A batched relation's digest covers
the instances' results in instance order with the instance id as column 0,
which is the lexicographic order of the batched relation itself.

Digests let a test compare a GPU export with the oracle's result without
running the oracle on the GPU machine, which for these sizes takes minutes.
"""
from __future__ import annotations

import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")


def relation_digest(rows) -> str:
    """SHA-256 of an (n, k) tuple array as row-major little-endian uint32."""
    a = np.ascontiguousarray(np.asarray(rows, dtype="<u4"))
    return hashlib.sha256(a.tobytes()).hexdigest()


# Workloads at the sizes the benchmark times them (and one smaller SG with
# cross edges, where no closed form exists).  Each entry names the
# generator call; the test regenerates the same input from the same seed.
SPECS = {
    "points-to-2e-9": dict(kind="pt", scale=1 / 512, seed=3),
    "owl-rl-20m": dict(kind="owl", triples=20_000_000, seed=4, entities=5_000_000),
    "sg-forest-50k": dict(kind="sg", n=50_000, seed=2),
    "batched-512": dict(kind="batch", count=512, seed=5, lo=1e3, hi=5e5),
}


def make_program(spec):
    sys.path.insert(0, ROOT)
    from paper_2501_13051_gb300 import workloads as W
    k = spec["kind"]
    if k == "pt":
        return W.points_to_program(W.points_to_edb(spec["scale"], spec["seed"]))
    if k == "owl":
        return W.owl_program(*W.owl_triples(spec["triples"], spec["seed"],
                                            n_entities=spec["entities"]))
    if k == "sg":
        return W.sg_program(W.random_forest(spec["n"], spec["seed"]))
    raise ValueError(k)


def program_golden(spec) -> dict:
    from oracle import oracle as O
    prog = make_program(spec)
    t0 = time.time()
    res = O.run_program(prog)
    secs = time.time() - t0
    rels = {nm: dict(n=int(len(rows)), sha256=relation_digest(rows))
            for nm, rows in res.relations.items()}
    return dict(spec=spec, relations=rels, deltas=res.deltas, iterations=res.iterations,
                rounds=res.rounds, derived=int(res.derived(prog)), oracle_seconds=round(secs, 1))


def _instance(args):
    """One batched instance run alone: its relation rows and round data."""
    i, kind, edges = args
    sys.path.insert(0, ROOT)
    from oracle import oracle as O
    from paper_2501_13051_gb300 import workloads as W
    prog = W.tc_program(edges) if kind == "tc" else W.sg_program(edges)
    res = O.run_program(prog)
    name = "path" if kind == "tc" else "sg"
    return i, kind, res.relations[name], res.deltas[name], res.iterations


def batched_golden(spec, workers: int | None = None) -> dict:
    sys.path.insert(0, ROOT)
    from paper_2501_13051_gb300 import workloads as W
    graphs, kinds = W.batched_instances(spec["count"], spec["seed"], spec["lo"], spec["hi"])
    t0 = time.time()
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers or os.cpu_count()) as pool:
        # largest first, so the slowest instances do not start last
        order = sorted(range(len(graphs)), key=lambda i: -len(graphs[i]))
        out = {}
        for i, kind, rows, deltas, iters in pool.imap_unordered(
                _instance, [(i, kinds[i], graphs[i]) for i in order]):
            out[i] = (kind, rows, deltas, iters)
    secs = time.time() - t0
    rel_of = {"tc": "tc_path", "sg": "sg"}
    h = {"tc_path": hashlib.sha256(), "sg": hashlib.sha256()}
    n = {"tc_path": 0, "sg": 0}
    rounds = {"tc_path": [], "sg": []}
    inst = []
    for i in range(len(graphs)):
        kind, rows, deltas, iters = out[i]
        rel = rel_of[kind]
        full = np.concatenate([np.full((len(rows), 1), i, np.uint32), rows], axis=1)
        h[rel].update(np.ascontiguousarray(full.astype("<u4")).tobytes())
        n[rel] += len(rows)
        r = rounds[rel]
        for k, d in enumerate(deltas):
            if k == len(r):
                r.append(0)
            r[k] += int(d)
        inst.append(dict(kind=kind, n=int(len(rows)), iterations=int(iters)))
    its = max(x["iterations"] for x in inst)
    # every relation's per-round list covers the batched run's rounds
    for rel in rounds:
        rounds[rel] = (rounds[rel] + [0] * (its + 1))[:its + 1]
    rels = {rel: dict(n=int(n[rel]), sha256=h[rel].hexdigest()) for rel in h}
    return dict(spec=spec, relations=rels, deltas=rounds, iterations=its, rounds=its + 1,
                derived=int(sum(n.values())), instances=inst, oracle_seconds=round(secs, 1))


def golden_path(name: str) -> str:
    return os.path.join(GOLDEN, f"fixpoint_{name}.json")


def write(name: str) -> dict:
    spec = SPECS[name]
    g = batched_golden(spec) if spec["kind"] == "batch" else program_golden(spec)
    g["written_by"] = "python -m oracle.golden " + name
    with open(golden_path(name), "w") as f:
        json.dump(g, f, indent=1)
        f.write("\n")
    return g


if __name__ == "__main__":
    names = sys.argv[1:] or list(SPECS)
    for nm in names:
        t = time.time()
        g = write(nm)
        print(f"{nm}: derived {g['derived']}, {g['iterations']} iterations, "
              f"{time.time() - t:.1f} s", flush=True)
