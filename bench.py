#!/usr/bin/env python
"""Benchmark of the semi-naive Datalog fixpoint on GB300.

One step = one complete fixpoint (every round: hash index, three-pass join,
radix sort + dedup, difference + merge) of a workload whose input columns
are already resident in device memory.  The default workload is
same-generation on a seeded random forest of 200,000 nodes (each node's
parent uniform among the earlier nodes with probability 0.98, else a root)
plus 2% random cross edges.  Metric: derived tuples per second (the derived
relations' sizes summed over the steps / device time of the steps).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                  [--workload NAME] [--scale S]

Workloads: sg-forest-200k (default), tc-er-1000-1500, points-to (scale S of
2M variables / 4M assign / 1M dereference, Zipf 1.1; default 2^-9),
owl-rl-20m, batched-512 (512 TC / SG instances in one batched run).  Each
runs in the form it names: points-to and owl-rl-20m with the learned
join-size estimator (trained first, untimed, on another seed), batched-512
with the estimator and the autotuner (six tuning runs first, untimed).
tc-er-1000-1500 runs its rounds after the first semi-naive one as one CUDA
graph (a device-side loop).  Those lines also carry the plain form timed
the same way, and batched-512 the same instances run one after another.

Under torchrun each rank runs an independent instance (seed + rank): the
fixpoint has no exchange step here, so ranks are replicas and the value is
the tuples all ranks derived / the slowest rank's time.

Also reported: an end-to-end figure through the C ABI with host buffers
(input upload and export of every derived relation inside the timed
region), the roofline of the dominant kernel (its algorithmic bytes / its
CUDA-event time over the timed steps, against the measured HBM copy
bandwidth), and the CPU oracle timed on a bounded sample of the same
workload on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2501_13051_gb300 import workloads as W  # noqa: E402

WORKLOADS = {
    "sg-forest-200k": dict(kind="sg", n=200_000, seed=2,
                           desc="same-generation on a random forest, 200000 nodes, "
                                "p_parent 0.98, +2% cross edges",
                           sample=dict(kind="sg", n=10_000, seed=2),
                           learned_also=dict(est_max_rows=1 << 32),
                           train=[dict(kind="sg", n=20_000, seed=102),
                                  dict(kind="sg", n=60_000, seed=103)]),
    "tc-er-1000-1500": dict(kind="tc", n=1000, m=1500, seed=1, graph=True, rows_also=True,
                            desc="transitive closure on a directed Erdos-Renyi graph, "
                                 "1000 nodes, 1500 edges; rounds after the first semi-naive "
                                 "one captured as one CUDA graph with a device-side loop",
                            sample=dict(kind="tc", n=1000, m=1500, seed=1)),
    "points-to": dict(kind="pt", scale=1 / 32, seed=3, learned=True, base=dict(dense_bits=34),
                      desc="points-to analysis (valueFlow / memoryAlias / valueAlias), "
                           "Zipf(1.1) endpoints, 2M vars / 4M assign / 1M deref times scale "
                           "(2^-5: the largest power-of-two scale that fits; the full size "
                           "stops with CDL_E_CAPACITY); new tuples of a round as bitmaps of "
                           "tuple spaces up to 2^34; learned join-size estimator on, exact "
                           "count pass as fallback",
                      sample=dict(kind="pt", scale=1 / 1024, seed=3),
                      train=dict(kind="pt", scale=1 / 1024, seed=103)),
    "owl-rl-20m": dict(kind="owl", triples=20_000_000, seed=4, learned=True,
                       desc="OWL-2-RL-style rules over 20M synthetic triples, 5M entities, "
                            "500 classes, 200 properties, 193 rule instances; learned "
                            "join-size estimator on, exact count pass as fallback",
                       sample=dict(kind="owl", triples=1_000_000, seed=4),
                       train=dict(kind="owl", triples=2_000_000, seed=104)),
    "batched-512": dict(kind="batch", count=512, seed=5, lo=1e3, hi=5e5, tune=True, graph=True,
                        learned_also=dict(),
                        desc="512 independent fixpoints in one batched run (instance column "
                             "leading): TC on even, SG on odd instances, directed ER graphs "
                             "with log-uniform 1e3..5e5 edges, mean out-degree 0.9; launch "
                             "parameters from the autotuner; rounds after the first "
                             "semi-naive one in one captured CUDA graph, converged instances "
                             "retired on the device; the learned form (estimator + tuner, "
                             "host rounds) timed beside",
                        sample=dict(kind="batch", count=16, seed=5, lo=1e3, hi=2e4),
                        train=dict(kind="batch", count=64, seed=105, lo=1e3, hi=5e5)),
}
METRIC = "derived tuples/s per fixpoint"


def make_program(spec, seed_offset=0, scale=None):
    seed = spec["seed"] + seed_offset
    kind = spec["kind"]
    if kind == "sg":
        return W.sg_program(W.random_forest(spec["n"], seed))
    if kind == "tc":
        return W.tc_program(W.er_graph(spec["n"], spec["m"], seed))
    if kind == "pt":
        return W.points_to_program(W.points_to_edb(scale or spec["scale"], seed))
    if kind == "owl":
        t = spec["triples"]
        f = t / 20_000_000
        return W.owl_program(*W.owl_triples(t, seed, n_entities=max(1000, int(5_000_000 * f))))
    if kind == "batch":
        return W.batched_program(*W.batched_instances(spec["count"], seed, spec["lo"], spec["hi"]))
    raise ValueError(kind)


def train_estimator(spec, seed_offset=0):
    """Logs every join of a run of the workload's training instance (another
    seed, smaller), then trains the size network on the GPU with the
    library's own kernels.  Returns (parameters, samples, seconds)."""
    from paper_2501_13051_gb300 import cdl
    t0 = time.time()
    Xs, ys = [], []
    for tr in (spec["train"] if isinstance(spec["train"], list) else [spec["train"]]):
        prog = make_program(tr, seed_offset)
        ninst = tr["count"] if spec["kind"] == "batch" else 0
        with cdl.Engine(estimator=2, n_instances=ninst, **spec.get("base", {})) as e:
            e.load_program(prog)
            e.run()
            Xi, yi = e.estimator_log()
        Xs.append(Xi)
        ys.append(yi)
    X, y = np.concatenate(Xs), np.concatenate(ys)
    with cdl.Engine() as t:
        t.estimator_train(X, y, epochs=2000)
        params = t.estimator_params()
    return params, len(y), time.time() - t0


def sequential_baseline(spec, seed_offset=0):
    """The batched workload's instances run one after another, each as its
    own engine (the plain exact form): derived tuples and device seconds."""
    import torch

    from paper_2501_13051_gb300 import cdl
    graphs, kinds = W.batched_instances(spec["count"], spec["seed"] + seed_offset, spec["lo"],
                                        spec["hi"])
    progs = [W.tc_program(g) if k == "tc" else W.sg_program(g) for g, k in zip(graphs, kinds)]
    dev = [[torch.from_numpy(np.ascontiguousarray(p.edb["edge"][:, k]).view(np.int32)).cuda()
            for k in range(2)] for p in progs]
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    derived = 0
    for p, d in zip(progs, dev):
        with cdl.Engine() as e:
            for nm, ar in p.arity.items():
                e.relation(nm, ar)
            e.load("edge", d)
            for r in p.rules:
                e.rule(r.head, r.body, r.neq)
            derived += e.run().derived_tuples
    b.record()
    torch.cuda.synchronize()
    return derived, a.elapsed_time(b) * 1e-3


def describe_sample(spec, derived, secs):
    what = {"sg": lambda s: f"same-generation, forest {s['n']} nodes (+2% cross edges)",
            "tc": lambda s: f"transitive closure, ER {s['n']} nodes / {s['m']} edges",
            "pt": lambda s: f"points-to at scale {s['scale']:g}",
            "owl": lambda s: f"OWL-RL rules over {s['triples']} triples",
            "batch": lambda s: f"{s['count']} batched TC/SG instances, {s['lo']:g}..{s['hi']:g} "
                               f"edges"}[spec["kind"]](spec)
    return f"{what}, seed {spec['seed']}: {derived} tuples in {secs:.2f} s"


def over_ranks(secs, derived, dist, device):
    """Whole-job (seconds, derived tuples) of N replicas: the slowest rank's
    time and every rank's tuples (one rank: unchanged)."""
    if dist is None:
        return secs, derived
    import torch
    t = torch.tensor([secs, float(derived)], dtype=torch.float64, device=device)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(mx[0]), int(t[1])


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, STREAM-style copy)"
    except Exception:
        return 6800.0, "fallback (6.8 TB/s, one earlier GB300 measurement)"


def kernel_traffic(name):
    """DRAM bytes per algorithmic byte for a kernel class from the committed
    ncu summary, or None when its source changed since the capture."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(p))[name]
        src = os.path.join(ROOT, "paper_2501_13051_gb300", "csrc", d["source"])
        if hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] != d["source_sha"]:
            return None
        return d
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi SM clocks and throttle reasons while the timed steps run."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        # nvidia-smi's start-up takes driver locks: let it reach its polling
        # loop (first sample written) before the timed steps begin
        t0 = time.time()
        while time.time() - t0 < 5 and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.05)
        time.sleep(0.25)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def run_oracle_sample(spec):
    from oracle import oracle as orc
    prog = make_program(spec)
    t = time.perf_counter()
    res = orc.run_program(prog)
    dt = time.perf_counter() - t
    return res.derived(prog), dt


def bench_reference(args, rank, world):
    """Reference arm: the CPU oracle, as it stands, on a bounded sample of the
    workload per step, on this host's cores (rank 0 only)."""
    if rank != 0:
        return
    spec = WORKLOADS[args.workload]["sample"]
    for _ in range(args.warmup):
        run_oracle_sample(spec)
    derived, secs = 0, 0.0
    for _ in range(args.steps):
        d, dt = run_oracle_sample(spec)
        derived += d
        secs += dt
    v = derived / secs
    sample = describe_sample(spec, derived // max(args.steps, 1), secs / max(args.steps, 1))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "tuples/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * secs / max(args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": args.workload, "sample": sample},
        "cpu_baseline": {"value": v, "unit": "tuples/s", "cores": 1, "kind": "oracle",
                         "sample": sample + ", 1 thread"},
        "e2e": {"value": v, "unit": "tuples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def bench_gb300(args, rank, world, dist):
    import torch
    from paper_2501_13051_gb300 import cdl

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    spec = WORKLOADS[args.workload]
    prog = make_program(spec, seed_offset=rank, scale=args.scale)
    idb = prog.idb()
    host_cols = {nm: [np.ascontiguousarray(rows[:, k]) for k in range(prog.arity[nm])]
                 for nm, rows in prog.edb.items()}
    dev_edb = {nm: [torch.from_numpy(c.view(np.int32)).cuda() for c in cols]
               for nm, cols in host_cols.items()}
    in_tuples = sum(len(r) for r in prog.edb.values())
    ninst = spec["count"] if spec["kind"] == "batch" else 0
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def declare(e):
        for nm, ar in prog.arity.items():
            e.relation(nm, ar)

    def rules(e):
        for r in prog.rules:
            e.rule(r.head, r.body, r.neq)

    # the form the workload names: autotuned launch parameters (tuning runs
    # first, untimed) and / or the learned estimator (trained first, untimed)
    form = {}
    tune_dir = tempfile.mkdtemp(prefix="cdl_tune_")
    if spec.get("tune"):
        cache = os.path.join(tune_dir, "tune.txt")
        for _ in range(6):
            with cdl.Engine(n_instances=ninst, autotune=2, tune_cache=cache) as e:
                declare(e)
                e.load_many(dev_edb)  # one check of every relation's values
                rules(e)
                e.run()
        form.update(autotune=1, tune_cache=cache)
    if spec.get("graph"):
        form.update(graph=True)
    if args.dedup:
        form.update(dedup=args.dedup)
    if args.host_full:
        form.update(host_full=1)
    trained = None
    if spec.get("learned"):
        params, nsamp, tsec = train_estimator(spec, rank)
        form.update(estimator=1, est_params=params)
        trained = {"samples": nsamp, "seconds": round(tsec, 2),
                   "instance": describe_sample(spec["train"], 0, 0).split(":")[0]}

    base = spec.get("base", {})  # options of every form (the workload's size needs them)

    def step(timing, plain=False, extra=None):
        opts = dict(base, **(extra if extra is not None else ({} if plain else form)))
        with cdl.Engine(timing=timing, n_instances=ninst, **opts) as e:
            declare(e)
            e.load_many(dev_edb)  # one check of every relation's values
            rules(e)
            st = e.run()
            return st, (e.kernel_profile() if timing else None)

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):
        step(False)
    flush.fill_(0)  # the fill kernel's first launch loads its module: not in the timed region
    torch.cuda.synchronize()
    # ---- one untimed step with every kernel class timed: the breakdown, and
    # the dominant class, whose launches alone carry events in the timed steps
    # events cannot wrap the launches inside a captured graph: a graph form's
    # breakdown (and roofline) comes from a step of the same form in host rounds
    in_graph = bool(form.get("graph"))
    host_form = {k: v for k, v in form.items() if k != "graph"}
    _, pr = step(True, extra=host_form if in_graph else None)
    breakdown = {p["kernel"]: p for p in pr if p["launches"]}
    dominant = max(breakdown.values(), key=lambda p: p["ms"])["kernel"]
    total_ms = sum(p["ms"] for p in breakdown.values())
    # ---- timed steps (device resident input)
    barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    derived, launches, iters = 0, 0, 0
    dom = {"launches": 0, "ms": 0.0, "bytes": 0.0}
    for i in range(args.steps):
        if i:
            flush.fill_(i & 0xFF)  # evict L2 between steps
        # events wrap the dominant class's launches in the last timed step
        # only: around hundreds of small launches they would cost the other
        # steps their time
        st, pr = step([dominant] if i == args.steps - 1 and not in_graph else False)
        derived += st.derived_tuples
        launches += st.kernel_launches
        iters = st.iterations
        for p in pr or ():
            if p["kernel"] == dominant:
                for key in dom:
                    dom[key] += p[key]
    ev1.record()
    torch.cuda.synchronize()
    barrier()
    clocks = clk.stop()
    secs = ev0.elapsed_time(ev1) * 1e-3
    secs, derived = over_ranks(secs, derived, dist, "cuda")
    value = derived / secs
    per_step = st.derived_tuples

    # ---- the plain exact form (no estimator, no tuner, no graph), timed the same way
    plain = None
    if form:
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record()
        pd = 0
        for i in range(args.steps):
            if i:
                flush.fill_(i & 0xFF)
            # the same events as the form's timed steps (last step only)
            pd += step([dominant] if i == args.steps - 1 else False, plain=True)[0].derived_tuples
        p1.record()
        torch.cuda.synchronize()
        psecs = p0.elapsed_time(p1) * 1e-3
        plain = {"tuples_per_s": pd / psecs, "ms_per_step": 1e3 * psecs / args.steps}

    # ---- the learned form beside the plain one, where the workload's own
    # form is plain: the estimator trained first (untimed, another seed)
    learned = None
    if "learned_also" in spec:
        params, nsamp, tsec = train_estimator(spec, rank)
        # the estimator's checks are host decisions: the learned form runs host rounds
        lform = {k: v for k, v in form.items() if k != "graph"}
        lform.update(spec["learned_also"], estimator=1, est_params=params)
        torch.cuda.synchronize()
        l0, l1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0.record()
        ld, lpred, lfall = 0, 0, 0
        for i in range(args.steps):
            if i:
                flush.fill_(i & 0xFF)
            lst = step(False, extra=lform)[0]
            ld += lst.derived_tuples
            lpred += lst.est_predictions
            lfall += lst.est_overflows
        l1.record()
        torch.cuda.synchronize()
        lsecs = l0.elapsed_time(l1) * 1e-3
        learned = {"tuples_per_s": ld / lsecs, "ms_per_step": 1e3 * lsecs / args.steps,
                   "over_line_value": (ld / lsecs) / value,
                   "predictions_per_step": lpred / args.steps,
                   "fallbacks_per_step": lfall / args.steps,
                   "trained_on": {"samples": nsamp, "seconds": round(tsec, 2),
                                  "instances": [describe_sample(t, 0, 0).split(":")[0]
                                                for t in (spec["train"] if isinstance(
                                                    spec["train"], list) else [spec["train"]])]},
                   "form": "learned join-size estimator (count pass skipped where predicted, "
                           "build side by cost), exact fallback"}

    # ---- rounds in one captured graph (the tuner's choices, no estimator:
    # a predicted join's check is a host decision), retirement on the device
    graph_line = None
    if spec.get("graph_also"):
        gform = {k: v for k, v in form.items() if k not in ("estimator", "est_params")}
        gform["graph"] = True
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record()
        gd, grounds, gret = 0, 0, 0
        for i in range(args.steps):
            if i:
                flush.fill_(i & 0xFF)
            gst = step(False, extra=gform)[0]
            gd += gst.derived_tuples
            grounds += gst.graph_rounds
            gret += gst.graph_retirements
        g1.record()
        torch.cuda.synchronize()
        gsecs = g0.elapsed_time(g1) * 1e-3
        graph_line = {"tuples_per_s": gd / gsecs, "ms_per_step": 1e3 * gsecs / args.steps,
                      "graph_rounds_per_step": grounds / args.steps,
                      "device_retirements_per_step": gret / args.steps,
                      "form": "rounds after the first semi-naive one in one captured CUDA graph "
                              "(conditional while node), converged instances retired on the "
                              "device, autotuned launch parameters"}

    # ---- the round's new tuples as sorted rows (radix sort + unique) instead
    # of bitmaps, where the bitmap form is the default: timed the same way
    rows = None
    if spec.get("rows_also"):
        torch.cuda.synchronize()
        r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        r0.record()
        rd = 0
        for i in range(args.steps):
            if i:
                flush.fill_(i & 0xFF)
            rd += step(False, extra=dict(form, dense_bits=-1))[0].derived_tuples
        r1.record()
        torch.cuda.synchronize()
        rsecs = r0.elapsed_time(r1) * 1e-3
        rows = {"tuples_per_s": rd / rsecs, "ms_per_step": 1e3 * rsecs / args.steps,
                "form": "new tuples as sorted rows (LSD radix sort, unique folded into step d)"}

    # ---- end to end through the C ABI with host buffers
    pinned_in = {nm: [torch.from_numpy(c.view(np.int32)).pin_memory() for c in cols]
                 for nm, cols in host_cols.items()}
    sizes = {}
    with cdl.Engine(n_instances=ninst, **base, **form) as e:
        declare(e)
        e.load_many(dev_edb)  # one check of every relation's values
        rules(e)
        e.run()
        sizes = {nm: e.size(nm) for nm in idb}
    pinned_out = {nm: [torch.empty(max(sizes[nm], 1), dtype=torch.int32, pin_memory=True)
                       for _ in range(prog.arity[nm])] for nm in idb}

    def step_e2e():
        with cdl.Engine(n_instances=ninst, **base, **form) as e:
            declare(e)
            e.load_many(pinned_in)  # one check of every relation's values
            rules(e)
            s = e.run()
            for nm in idb:
                e.export(nm, out=[t.data_ptr() for t in pinned_out[nm]])
            return s

    step_e2e()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    d_e2e = 0
    for _ in range(args.steps):
        d_e2e += step_e2e().derived_tuples
    e1.record()
    torch.cuda.synchronize()
    barrier()
    secs_e2e, d_e2e = over_ranks(e0.elapsed_time(e1) * 1e-3, d_e2e, dist, "cuda")
    e2e = {"value": d_e2e / secs_e2e, "unit": "tuples/s",
           "h2d_bytes_per_step": int(sum(4 * c.size for cols in host_cols.values() for c in cols)),
           "d2h_bytes_per_step": int(sum(4 * sizes[nm] * prog.arity[nm] for nm in idb))}

    if rank != 0:
        return
    # ---- roofline of the dominant kernel class, from its timed-step launches
    name, d = dominant, (breakdown[dominant] if in_graph else dom)
    achieved = d["bytes"] / (d["ms"] * 1e-3) / 1e9
    peak, peak_src = measured_peak()
    tr = kernel_traffic(name)
    traffic = None
    if tr is not None:
        traffic = tr["dram_bytes_per_unit"] / tr["algo_bytes_per_unit"] * d["bytes"] / d["launches"]
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": name,
                "kernel_share": breakdown[name]["ms"] / total_ms, "launches": d["launches"],
                "timed": ("CUDA events around every launch of the kernel in a step of the same "
                          "form in host rounds (events cannot wrap launches inside a captured "
                          "graph)") if in_graph else
                         "CUDA events around every launch of the kernel in the last timed step",
                "peak_source": peak_src}
    # step (d) as a whole: its algorithmic bytes (New and Full read, Full and
    # delta written) over the count pass (with its tile scan) and the write
    # pass, from the step with every class timed
    if "diff_merge" in breakdown:
        dm, dc = breakdown["diff_merge"], breakdown.get("diff_count", {"ms": 0.0})
        sd = dm["bytes"] / ((dm["ms"] + dc["ms"]) * 1e-3) / 1e9
        roofline["step_d"] = {"achieved": sd, "peak": peak, "unit": "GB/s", "frac": sd / peak,
                              "bytes": dm["bytes"], "ms": dm["ms"] + dc["ms"],
                              "kernels": "count pass + tile scan + write pass (diff_count, "
                                         "diff_merge), the step with every class timed"}
    # ---- the oracle on a bounded sample, on this host's cores
    sspec = spec["sample"]
    od, osecs = run_oracle_sample(sspec)
    cpu = {"value": od / osecs, "unit": "tuples/s", "cores": 1, "kind": "oracle",
           "sample": describe_sample(sspec, od, osecs) + f", 1 thread of {os.cpu_count()} host cores"}
    config = {"workload": args.workload, "desc": spec["desc"], "input_tuples": int(in_tuples),
              "derived_per_step": int(per_step), "iterations": int(iters),
              "seed": spec["seed"] + rank,
              "l2": "256 MB buffer written between steps; working set > L2",
              "parallelism": f"replicas x{world}"}
    if spec["kind"] == "pt":
        config["scale"] = args.scale or spec["scale"]
    if spec.get("learned"):
        config["estimator"] = {"trained_on": trained, "predictions": int(st.est_predictions),
                               "fallbacks": int(st.est_overflows)}
    if spec.get("tune"):
        config["autotune"] = "6 tuning runs (untimed), then the cached choices"
    if spec.get("graph"):
        config["graph"] = "rounds after the first semi-naive one as one CUDA graph (conditional " \
                          "while node)"
        config["graph_rounds_per_step"] = int(st.graph_rounds)
    if args.host_full:
        config["host_full"] = ("Full of relations only step (d) reads in pinned host memory, "
                               "merged in place over the CPU-GPU link")
    if args.dedup:
        config["dedup"] = ("Algorithm 2, hybrid index (decomposed Full: per-column sorted ids "
                           "+ unique hashmap)" if args.dedup == 1 else
                           "Algorithm 2, hash-only index (multimap of column 0)")
    if graph_line is not None:
        config["graph_form"] = graph_line
    if learned is not None:
        config["learned_form"] = learned
    if rows is not None:
        config["rows_form"] = rows
    if base:
        config["options"] = base
    if plain is not None:
        config["plain_exact"] = plain
        config["form_over_plain_exact"] = value / plain["tuples_per_s"]
    if spec["kind"] == "batch":
        sd, ss = sequential_baseline(spec, seed_offset=rank)
        config["instances"] = spec["count"]
        config["max_iterations_per_instance"] = int(max(st.iters_per_instance))
        config["sequential_plain"] = {"tuples_per_s": sd / ss, "seconds": ss,
                                      "derived": int(sd)}
        config["batched_over_sequential"] = value / (sd / ss)
    line = {
        "metric": METRIC, "value": value, "unit": "tuples/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic", "config": config,
        "e2e": e2e, "gpu_launches": launches, "roofline": roofline, "cpu_baseline": cpu,
        "clocks": clocks,
        "kernels_one_step": {k: {"ms": round(v["ms"], 3), "launches": v["launches"],
                                 "GBps": round(v["bytes"] / max(v["ms"], 1e-9) / 1e6, 1)}
                             for k, v in sorted(breakdown.items(), key=lambda kv: -kv[1]["ms"])},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="sg-forest-200k", choices=sorted(WORKLOADS))
    ap.add_argument("--scale", type=float, default=None, help="points-to scale factor")
    ap.add_argument("--host-full", action="store_true",
                    help="keep Full of relations only step (d) reads in pinned host memory")
    ap.add_argument("--dedup", type=int, default=0, choices=[0, 1, 2],
                    help="step (d): 0 merge of sorted rows, 1 Algorithm 2 (hybrid index), "
                         "2 Algorithm 2 (hash-only index)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if args.impl == "reference":
        bench_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    try:
        bench_gb300(args, rank, world, dist)
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
