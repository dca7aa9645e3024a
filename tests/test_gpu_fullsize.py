"""Parity at the sizes the benchmark times (GPU, through the C ABI).

* Same generation on the 200,000-node forest without cross edges: the exact
  set follows from the closed form (oracle.closed_forms.sg_forest).  Each
  exported row is checked to be a pair x != y of one (tree, depth) group,
  rows strictly increasing, and every x to have exactly (group size - 1)
  partners: together that is set equality with the closed form.  Per-round
  delta sizes and the iteration count are compared too.
* Same generation on the benchmark's forest (200,000 nodes with 2 % cross
  edges), where no closed form exists: the exported relation is sorted,
  unique, holds every head of the non-recursive rule and is closed under
  the recursive rule (every derivation from it lands in it).  Leastness at
  this size rests on the oracle's agreement at 50,000 nodes (golden file).
* Points-to at scale 2^-9, OWL-RL-style rules over 20M triples, SG on a
  50,000-node forest with cross edges, and 512 batched TC / SG instances:
  the export of every relation against digests the oracle wrote
  (tests/golden/fixpoint_*.json, from ``python -m oracle.golden``), with
  sizes, per-round delta sizes and iteration counts, in the forms the
  benchmark runs them (plain, learned, tuned, graph rounds, bitmap or rows).
* Points-to at scale 2^-5, the benchmarked size, in the bitmap form:
  beyond the oracle, so sampled tuples are checked to have a derivation by
  a rule from the exports and sampled rule instances over the exports to
  land in them.  The full-size input stops with CDL_E_CAPACITY: a join of
  its valueAlias rule would exceed 2^32 outputs.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2501_13051_gb300 import workloads as W
from fixpoint_props import points_to_fixpoint_checks

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a GPU"
    from paper_2501_13051_gb300 import build as B
    B.build()
    from paper_2501_13051_gb300 import cdl
    return torch, cdl


def load_golden(name):
    with open(os.path.join(GOLDEN, f"fixpoint_{name}.json")) as f:
        return json.load(f)


def run_dev(cdl, prog, **opts):
    """Runs a program; returns (stats, {relation: device column list})."""
    e = cdl.Engine(**opts)
    e.load_program(prog)
    st = e.run()
    cols = {nm: e.export(nm, device=True) for nm in prog.idb()}
    e.close()
    return st, cols


# ------------------------------------------------------------------ SG-200K

CHUNK = 1 << 27


def sorted_unique(torch, c0, c1):
    """Rows strictly increasing in (c0, c1) (node ids below 2^31)."""
    n = c0.numel()
    prev = None
    for s in range(0, n, CHUNK):
        k = (c0[s:s + CHUNK].long() << 32) | c1[s:s + CHUNK].long()
        if prev is not None and not bool(prev < k[0]):
            return False
        if k.numel() > 1 and not bool((k[1:] > k[:-1]).all()):
            return False
        prev = k[-1]
    return True


def test_sg_forest_200k_equals_closed_form(env):
    torch, cdl = env
    from oracle import closed_forms as C
    n = 200_000
    f = W.random_forest(n, 2, cross_frac=0.0)
    cf = C.sg_forest(n, f)
    st, cols = run_dev(cdl, W.sg_program(f))
    c0, c1 = cols["sg"]
    assert c0.numel() == cf["size"] == st.derived_tuples
    assert st.iterations == cf["iterations"]
    assert st.delta_per_round == cf["deltas"] + [0]
    assert sorted_unique(torch, c0, c1)
    grp = torch.from_numpy(cf["group"]).cuda()
    gsz = torch.from_numpy(cf["group_size"]).cuda()
    deg = torch.zeros(n, dtype=torch.int64, device="cuda")
    for s in range(0, c0.numel(), CHUNK):
        a, b = c0[s:s + CHUNK].long(), c1[s:s + CHUNK].long()
        assert bool((a != b).all())
        assert bool((grp[a] == grp[b]).all())
        deg += torch.bincount(a, minlength=n)
    # unique within-group pairs, x != y, and each x with all its partners
    assert torch.equal(deg, gsz[grp] - 1)


def csr(torch, src, dst, n):
    """Out-neighbour lists: (offsets[n + 1], neighbours sorted by source)."""
    order = torch.argsort(src * n + dst)
    off = torch.zeros(n + 1, dtype=torch.int64, device=src.device)
    off[1:] = torch.cumsum(torch.bincount(src, minlength=n), 0)
    return off, dst[order]


def member(torch, x, y, row_off, col1, max_row):
    """(x, y) in the relation whose rows of x are col1[row_off[x]:row_off[x+1]],
    sorted: a lower-bound binary search per query."""
    lo, hi = row_off[x], row_off[x + 1]
    end = hi.clone()
    last = col1.numel() - 1
    for _ in range(int(math.ceil(math.log2(max_row + 1))) + 1):
        act = lo < hi
        mid = (lo + hi) // 2
        v = col1[mid.clamp(max=last)].long()
        right = act & (v < y)
        lo = torch.where(right, mid + 1, lo)
        hi = torch.where(act & ~right, mid, hi)
    return (lo < end) & (col1[lo.clamp(max=last)].long() == y)


def test_sg_forest_200k_cross_edges_closed_under_rules(env):
    """The benchmark's input: the result is sorted, unique, holds every
    sibling pair and is closed under sg(x,y) <- edge(a,x), sg(a,b), edge(b,y)."""
    torch, cdl = env
    n = 200_000
    edges = W.random_forest(n, 2)
    st, cols = run_dev(cdl, W.sg_program(edges))
    c0, c1 = cols["sg"]
    N = c0.numel()
    assert N == st.derived_tuples and N > 0
    assert sorted_unique(torch, c0, c1)
    row_off = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    for s in range(0, N, CHUNK):
        row_off[1:] += torch.bincount(c0[s:s + CHUNK].long(), minlength=n)
    row_off = torch.cumsum(row_off, 0)
    max_row = int((row_off[1:] - row_off[:-1]).max())
    e = torch.from_numpy(edges.astype(np.int64)).cuda()
    off, child = csr(torch, e[:, 0], e[:, 1], n)
    deg = off[1:] - off[:-1]
    # non-recursive rule: every pair of distinct children of one parent
    p = e[:, 0]
    cnt = deg[p]
    idx = torch.repeat_interleave(torch.arange(p.numel(), device="cuda"), cnt)
    start = torch.cumsum(cnt, 0) - cnt
    j = torch.arange(idx.numel(), device="cuda") - start[idx]
    x, y = e[idx, 1], child[off[p[idx]] + j]
    keep = x != y
    assert bool(member(torch, x[keep], y[keep], row_off, c1, max_row).all())
    # recursive rule, from every sg row (a, b)
    checked = 0
    for s in range(0, N, 1 << 25):
        a, b = c0[s:s + (1 << 25)].long(), c1[s:s + (1 << 25)].long()
        da, db = deg[a], deg[b]
        cnt = da * db
        live = cnt > 0
        a, b, da, db, cnt = a[live], b[live], da[live], db[live], cnt[live]
        if not a.numel():
            continue
        idx = torch.repeat_interleave(torch.arange(a.numel(), device="cuda"), cnt)
        start = torch.cumsum(cnt, 0) - cnt
        w = torch.arange(idx.numel(), device="cuda") - start[idx]
        x = child[off[a[idx]] + w // db[idx]]
        y = child[off[b[idx]] + w % db[idx]]
        assert bool(member(torch, x, y, row_off, c1, max_row).all()), s
        checked += idx.numel()
    assert checked > N // 2


# ------------------------------------------------------------ golden files

def check_against_golden(g, st, rels, digest):
    assert st.iterations == g["iterations"]
    assert st.derived_tuples == g["derived"]
    per_round = [sum(g["deltas"][nm][k] for nm in g["deltas"] if k < len(g["deltas"][nm]))
                 for k in range(g["rounds"])]
    assert st.delta_per_round == per_round
    for nm, want in g["relations"].items():
        rows = rels[nm]
        assert len(rows) == want["n"], nm
        assert digest(rows) == want["sha256"], nm


def export_all(e, prog):
    return {nm: e.export(nm) for nm in prog.arity}


def bench_module():
    import importlib
    import sys
    root = os.path.dirname(os.path.dirname(GOLDEN))
    if root not in sys.path:
        sys.path.insert(0, root)
    return importlib.import_module("bench")


@pytest.mark.parametrize("form", ["plain", "rows", "learned"])
def test_points_to_2e_9_matches_oracle(env, form):
    torch, cdl = env
    from oracle.golden import SPECS, make_program, relation_digest
    g = load_golden("points-to-2e-9")
    prog = make_program(SPECS["points-to-2e-9"])
    opts = {}
    if form == "rows":
        opts = dict(dense_bits=-1)
    if form == "learned":
        bench = bench_module()
        params, _, _ = bench.train_estimator(bench.WORKLOADS["points-to"])
        opts = dict(estimator=1, est_params=params)
    with cdl.Engine(**opts) as e:
        e.load_program(prog)
        st = e.run()
        check_against_golden(g, st, export_all(e, prog), relation_digest)


@pytest.mark.parametrize("form", ["plain", "learned"])
def test_owl_rl_20m_matches_oracle(env, form):
    torch, cdl = env
    from oracle.golden import SPECS, make_program, relation_digest
    g = load_golden("owl-rl-20m")
    prog = make_program(SPECS["owl-rl-20m"])
    opts = {}
    if form == "learned":
        bench = bench_module()
        params, _, _ = bench.train_estimator(bench.WORKLOADS["owl-rl-20m"])
        opts = dict(estimator=1, est_params=params)
    with cdl.Engine(**opts) as e:
        e.load_program(prog)
        st = e.run()
        check_against_golden(g, st, export_all(e, prog), relation_digest)


@pytest.mark.parametrize("form", ["plain", "graph", "alg2", "alg2-hash"])
def test_sg_forest_50k_matches_oracle(env, form):
    torch, cdl = env
    from oracle.golden import SPECS, make_program, relation_digest
    g = load_golden("sg-forest-50k")
    prog = make_program(SPECS["sg-forest-50k"])
    opts = {"graph": dict(graph=True), "alg2": dict(dedup=1), "alg2-hash": dict(dedup=2)}
    with cdl.Engine(**opts.get(form, {})) as e:
        e.load_program(prog)
        st = e.run()
        check_against_golden(g, st, export_all(e, prog), relation_digest)


@pytest.mark.parametrize("form", ["exact", "learned+tuned", "graph+tuned"])
def test_batched_512_matches_oracle(env, form, tmp_path):
    torch, cdl = env
    from oracle.golden import relation_digest
    g = load_golden("batched-512")
    sp = g["spec"]
    graphs, kinds = W.batched_instances(sp["count"], sp["seed"], sp["lo"], sp["hi"])
    prog = W.batched_program(graphs, kinds)
    opts = dict(n_instances=sp["count"])
    if form != "exact":
        cache = str(tmp_path / "tune.txt")
        with cdl.Engine(autotune=2, tune_cache=cache, **opts) as e:  # one tuning run
            e.load_program(prog)
            e.run()
        opts.update(autotune=1, tune_cache=cache)
    if form == "learned+tuned":
        bench = bench_module()
        params, _, _ = bench.train_estimator(bench.WORKLOADS["batched-512"])
        opts.update(estimator=1, est_params=params)
    if form == "graph+tuned":  # rounds in the captured graph, retirement on the device
        opts.update(graph=True)
    with cdl.Engine(**opts) as e:
        e.load_program(prog)
        st = e.run()
        rels = {nm: e.export(nm) for nm in ("tc_path", "sg")}
    check_against_golden(g, st, rels, relation_digest)
    if form == "graph+tuned":
        assert st.graph_rounds > 0 and st.graph_retirements > 0
    got_n = {}
    for nm, rows in rels.items():
        got_n.update({int(i): int(c) for i, c in
                      zip(*np.unique(rows[:, 0], return_counts=True))})
    for i, inst in enumerate(g["instances"]):
        assert got_n.get(i, 0) == inst["n"], i
        assert st.iters_per_instance[i] == inst["iterations"], i


def test_points_to_benched_size_is_a_fixpoint_of_its_rules(env):
    """Scale 2^-5, the size the benchmark times (62,500 variables; 3.5e8
    derived tuples), in its bitmap form: beyond the oracle (a std::set
    evaluator would visit ~1e12 join outputs).  The exports are sorted and
    unique; sampled tuples of each derived relation have a derivation from
    the exported relations by one of its rules (so nothing is made up), and
    sampled rule instances over the exports land in them (so nothing is
    missing there).  Together with the oracle's agreement at 2^-9 (golden
    file) this pins the fixpoint at the benchmarked size."""
    torch, cdl = env
    edb = W.points_to_edb(1 / 32, 3)
    prog = W.points_to_program(edb)
    with cdl.Engine(dense_bits=34) as e:
        e.load_program(prog)
        st = e.run()
        rel = {nm: e.export(nm) for nm in prog.idb()}
    assert st.derived_tuples == sum(len(r) for r in rel.values())
    assert st.derived_tuples > 10 ** 8
    points_to_fixpoint_checks(edb, rel, np.random.default_rng(20250123), 3000)


def test_points_to_as_written_stops_with_capacity_error(env):
    """The full-size points-to input (2M variables, 4M assign, 1M
    dereference): valueAlias's first join, over a Zipf hub of hundreds of
    thousands of assignments, counts more than 2^32 outputs, which the
    exact count pass reports before anything is written."""
    torch, cdl = env
    prog = W.points_to_program(W.points_to_edb(1.0, 3))
    with cdl.Engine() as e:
        e.load_program(prog)
        with pytest.raises(cdl.CdlError) as err:
            e.run()
    assert cdl.STATUS[err.value.status] == "CDL_E_CAPACITY"
    assert "2^32" in str(err.value)
