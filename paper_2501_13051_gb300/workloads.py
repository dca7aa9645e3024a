"""Seeded synthetic inputs and the Datalog programs that run on them.

This module only *makes inputs*: a counter-based random number generator,
graph / points-to / triple generators shaped like the workloads of the
paper's evaluation (Section 5: transitive closure and same-generation on
sparse graphs, knowledge-graph reasoning over RDF-style triples), and the
rule sets of those workloads written out as plain data.  It contains none of
the evaluation arithmetic (no join, sort, dedup or fixpoint) and is the one
module that the CUDA path, the benches and the CPU oracle's tests share.

Random numbers: SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used in its counter form:
draw ``i`` of stream ``s`` is the SplitMix64 finaliser applied to
``s + (i + 1) * golden_gamma``.  Written with numpy uint64 arithmetic so that
every machine produces the same inputs for the same seed.

Program representation (consumed by both bindings):

* a term is a ``str`` (variable name) or an ``int`` (constant, < 2**32 - 1);
* an atom is ``(relation_name, (term, ...))``;
* a rule is ``Rule(head, body, neq)`` with ``neq`` a tuple of variable pairs
  that must bind to different values (the ``x != y`` of the SG query,
  Section 5.2);
* a program is ``Program(arity, rules, edb)`` with ``edb`` mapping relation
  name -> ``(n, arity)`` uint32 array of input facts.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Rule", "Program", "splitmix64", "stream", "uniform_below", "uniform01",
    "er_graph", "random_forest", "zipf_ids", "points_to_edb", "owl_triples",
    "batched_graph_sizes", "tc_program", "sg_program", "sg_paper_program",
    "points_to_program", "owl_program", "batched_program", "random_program",
    "RESERVED",
]

RESERVED = 0xFFFFFFFF  # the one uint32 value no relation may hold

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, idx):
    """Counter-based SplitMix64: draw ``idx`` (uint64 array) of stream ``seed``."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (idx + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream(seed: int, purpose: int) -> int:
    """Derive an independent sub-stream seed for one purpose of one workload."""
    return int(splitmix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF), np.uint64(purpose)))


def uniform_below(z, m):
    """Map uint64 draws to integers in [0, m) (m may be an array), m < 2**32."""
    hi = (np.asarray(z, dtype=np.uint64) >> np.uint64(32))
    with np.errstate(over="ignore"):
        return ((hi * np.asarray(m, dtype=np.uint64)) >> np.uint64(32)).astype(np.uint64)


def uniform01(z):
    """Map uint64 draws to doubles in [0, 1)."""
    return (np.asarray(z, dtype=np.uint64) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def _first_distinct(keys: np.ndarray, want: int) -> np.ndarray:
    """Indices of the first ``want`` distinct keys, in stream order."""
    _, first = np.unique(keys, return_index=True)
    first.sort()
    return first[:want]


# --------------------------------------------------------------------------
# graphs
# --------------------------------------------------------------------------

def er_graph(n: int, m: int, seed: int) -> np.ndarray:
    """Directed Erdos-Renyi graph with exactly ``m`` distinct ordered pairs
    (u, v), u != v, over ``n`` nodes: draw uniform pairs from one stream,
    drop self-loops and repeats, keep the first ``m``.  Returns (m, 2) uint32."""
    if m > n * (n - 1):
        raise ValueError("more edges than ordered pairs")
    s = stream(seed, 1)
    batch = max(2 * m + 64, 1024)
    while True:
        i = np.arange(batch, dtype=np.uint64)
        u = uniform_below(splitmix64(s, 2 * i), n)
        v = uniform_below(splitmix64(s, 2 * i + np.uint64(1)), n)
        ok = u != v
        u, v = u[ok], v[ok]
        first = _first_distinct(u * np.uint64(n) + v, m)
        if len(first) == m:
            return np.stack([u[first], v[first]], axis=1).astype(np.uint32)
        batch *= 2


def random_forest(n: int, seed: int, p_parent: float = 0.98,
                  cross_frac: float = 0.02) -> np.ndarray:
    """Random recursive forest plus cross edges, as edge(parent, child) pairs.

    Node 0 is a root; node i >= 1 takes a parent drawn uniformly from the
    earlier nodes with probability ``p_parent`` and is a root otherwise.
    Then ``floor(cross_frac * n)`` extra ordered pairs (u, v), u != v, that are
    not already edges are drawn uniformly (first distinct ones in stream
    order).  Returns (E, 2) uint32: tree edges in node order, then cross edges.
    """
    s_root, s_par, s_cross = stream(seed, 11), stream(seed, 12), stream(seed, 13)
    i = np.arange(1, n, dtype=np.uint64)
    has_parent = uniform01(splitmix64(s_root, i)) < p_parent
    parent = uniform_below(splitmix64(s_par, i), i)
    child = i[has_parent]
    tree = np.stack([parent[has_parent], child], axis=1)
    n_cross = int(math.floor(cross_frac * n))
    if n_cross == 0:
        return tree.astype(np.uint32)
    tree_keys = tree[:, 0] * np.uint64(n) + tree[:, 1]
    batch = 4 * n_cross + 64
    while True:
        j = np.arange(batch, dtype=np.uint64)
        u = uniform_below(splitmix64(s_cross, 2 * j), n)
        v = uniform_below(splitmix64(s_cross, 2 * j + np.uint64(1)), n)
        keys = u * np.uint64(n) + v
        ok = (u != v) & ~np.isin(keys, tree_keys)
        u, v, keys = u[ok], v[ok], keys[ok]
        first = _first_distinct(keys, n_cross)
        if len(first) == n_cross:
            cross = np.stack([u[first], v[first]], axis=1)
            return np.concatenate([tree, cross]).astype(np.uint32)
        batch *= 2


def zipf_ids(count: int, universe: int, s: float, seed: int, purpose: int,
             perm: np.ndarray) -> np.ndarray:
    """``count`` ids in [0, universe) with P(rank r) proportional to r**-s,
    by inverse CDF over a table of ranks, mapped through ``perm`` so that the
    hot ids are scattered over the id space."""
    ranks = np.arange(1, universe + 1, dtype=np.float64)
    cdf = np.cumsum(ranks ** -s)
    cdf /= cdf[-1]
    u = uniform01(splitmix64(stream(seed, purpose), np.arange(count, dtype=np.uint64)))
    r = np.minimum(np.searchsorted(cdf, u, side="right"), universe - 1)
    return perm[r]


def _perm(universe: int, seed: int, purpose: int) -> np.ndarray:
    keys = splitmix64(stream(seed, purpose), np.arange(universe, dtype=np.uint64))
    return np.argsort(keys, kind="stable").astype(np.uint64)


def _dedup_pairs(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    pairs = np.stack([a, b], axis=1).astype(np.uint32)
    return np.unique(pairs, axis=0)


def points_to_edb(scale: float, seed: int, s: float = 1.1) -> dict:
    """Points-to EDB: 2M*scale variables, 4M*scale assign and 1M*scale
    dereference pairs, both endpoints Zipf(s) independently, repeats removed."""
    nv = max(2, int(round(2_000_000 * scale)))
    na = max(1, int(round(4_000_000 * scale)))
    nd = max(1, int(round(1_000_000 * scale)))
    perm = _perm(nv, seed, 21)
    assign = _dedup_pairs(zipf_ids(na, nv, s, seed, 22, perm), zipf_ids(na, nv, s, seed, 23, perm))
    deref = _dedup_pairs(zipf_ids(nd, nv, s, seed, 24, perm), zipf_ids(nd, nv, s, seed, 25, perm))
    return {"assign": assign, "dereference": deref}


# --------------------------------------------------------------------------
# OWL-2-RL-style triples (vertically partitioned)
# --------------------------------------------------------------------------

@dataclass
class OwlSchema:
    n_entities: int
    n_classes: int
    n_props: int
    class_base: int
    sub_class: list = field(default_factory=list)      # (C, D): C subClassOf D
    sub_prop: list = field(default_factory=list)       # (p, q): p subPropertyOf q
    transitive: list = field(default_factory=list)     # p
    domain: list = field(default_factory=list)         # (p, C)
    range_: list = field(default_factory=list)         # (p, C)
    inverse: list = field(default_factory=list)        # (p, q)


def owl_triples(n_triples: int, seed: int, n_entities: int = 5_000_000,
                n_classes: int = 500, n_props: int = 200, levels: int = 12,
                s: float = 1.1):
    """Synthetic triples and schema in the shape of an OWL 2 RL workload.

    Entities take ids [0, n_entities), classes [n_entities, n_entities +
    n_classes).  A quarter of the triples are ``type(x, C)`` (Zipf subject,
    uniform class); the rest are property triples spread uniformly over the
    properties with a Zipf subject and a uniform object.  Schema: a
    ``levels``-level subclass DAG (one parent with probability 0.8, else
    two, from the level above), 40 acyclic subproperty edges, 10 transitive
    properties, 60 domain and 60 range axioms, 10 inverse pairs.
    Returns ``(edb, schema)`` with edb relation names ``type``, ``sc`` and
    ``p<k>`` per property."""
    rnd = lambda purpose, k: splitmix64(stream(seed, purpose), np.arange(k, dtype=np.uint64))
    cb = n_entities
    sch = OwlSchema(n_entities, n_classes, n_props, cb)
    # subclass DAG by levels
    lvl = (np.arange(n_classes) * levels) // n_classes
    z1, z2, z3 = rnd(31, n_classes), rnd(32, n_classes), rnd(33, n_classes)
    for c in range(n_classes):
        if lvl[c] == 0:
            continue
        above = np.nonzero(lvl == lvl[c] - 1)[0]
        p1 = int(above[uniform_below(z1[c], len(above))])
        sch.sub_class.append((cb + c, cb + p1))
        if uniform01(z2[c]) >= 0.8 and len(above) > 1:
            p2 = int(above[uniform_below(z3[c], len(above))])
            if p2 != p1:
                sch.sub_class.append((cb + c, cb + p2))
    # subproperty edges (acyclic: lower index -> higher index)
    zs = rnd(34, 4 * 40 + 64)
    seen, k = set(), 0
    while len(sch.sub_prop) < 40:
        a = int(uniform_below(zs[k], n_props)); b = int(uniform_below(zs[k + 1], n_props)); k += 2
        a, b = min(a, b), max(a, b)
        if a != b and (a, b) not in seen:
            seen.add((a, b)); sch.sub_prop.append((a, b))
    props = np.argsort(rnd(35, n_props), kind="stable")
    sch.transitive = [int(p) for p in props[:10]]
    zd = rnd(36, 240)
    sch.domain = [(int(uniform_below(zd[2 * i], n_props)), cb + int(uniform_below(zd[2 * i + 1], n_classes))) for i in range(60)]
    sch.range_ = [(int(uniform_below(zd[120 + 2 * i], n_props)), cb + int(uniform_below(zd[121 + 2 * i], n_classes))) for i in range(60)]
    inv = props[10:30]
    sch.inverse = [(int(inv[2 * i]), int(inv[2 * i + 1])) for i in range(10)]
    # data
    perm = _perm(n_entities, seed, 37)
    n_type = n_triples // 4
    n_prop_tr = n_triples - n_type
    t_sub = zipf_ids(n_type, n_entities, s, seed, 38, perm)
    t_cls = cb + uniform_below(rnd(39, n_type), n_classes)
    edb = {"type": _dedup_pairs(t_sub, t_cls)}
    p_of = uniform_below(rnd(40, n_prop_tr), n_props)
    p_sub = zipf_ids(n_prop_tr, n_entities, s, seed, 41, perm)
    p_obj = uniform_below(rnd(42, n_prop_tr), n_entities)
    order = np.argsort(p_of, kind="stable")
    p_of, p_sub, p_obj = p_of[order], p_sub[order], p_obj[order]
    bounds = np.searchsorted(p_of, np.arange(n_props + 1))
    for p in range(n_props):
        lo, hi = bounds[p], bounds[p + 1]
        edb[f"p{p}"] = _dedup_pairs(p_sub[lo:hi], p_obj[lo:hi]) if hi > lo else np.zeros((0, 2), np.uint32)
    edb["sc"] = np.array(sorted(set(sch.sub_class)), dtype=np.uint32).reshape(-1, 2)
    return edb, sch


def batched_graph_sizes(count: int, seed: int, lo: float = 1e3, hi: float = 5e5):
    """Edge counts log-uniform in [lo, hi] for ``count`` instances."""
    u = uniform01(splitmix64(stream(seed, 51), np.arange(count, dtype=np.uint64)))
    return np.floor(np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))).astype(np.int64)


def batched_instances(count: int, seed: int, lo: float = 1e3, hi: float = 5e5,
                      degree: float = 0.9):
    """``count`` independent instances for batched fixpoints: instance i is
    transitive closure (even i) or same generation (odd i) on a directed
    Erdos-Renyi graph with E_i edges, E_i log-uniform in [lo, hi], over
    ceil(E_i / degree) nodes (mean out-degree ``degree``), graph seed
    1000 * seed + i.  Returns (graphs, kinds)."""
    sizes = batched_graph_sizes(count, seed, lo, hi)
    graphs, kinds = [], []
    for i, e in enumerate(sizes):
        e = int(e)
        n = int(math.ceil(e / degree))
        graphs.append(er_graph(n, e, 1000 * seed + i))
        kinds.append("tc" if i % 2 == 0 else "sg")
    return graphs, kinds


# --------------------------------------------------------------------------
# programs
# --------------------------------------------------------------------------

@dataclass(frozen=True)
class Rule:
    head: tuple
    body: tuple
    neq: tuple = ()


@dataclass
class Program:
    arity: dict
    rules: list
    edb: dict

    def idb(self):
        return sorted({r.head[0] for r in self.rules})

    def max_value(self) -> int:
        m = 0
        for a in self.edb.values():
            if a.size:
                m = max(m, int(a.max()))
        for r in self.rules:
            for atom in (r.head,) + tuple(r.body):
                for t in atom[1]:
                    if isinstance(t, int):
                        m = max(m, t)
        return m


def tc_program(edges: np.ndarray) -> Program:
    """Transitive closure (Section 2): path(x,y) <- edge(x,y);
    path(x,z) <- edge(x,y), path(y,z)."""
    return Program(
        {"edge": 2, "path": 2},
        [Rule(("path", ("x", "y")), (("edge", ("x", "y")),)),
         Rule(("path", ("x", "z")), (("edge", ("x", "y")), ("path", ("y", "z"))))],
        {"edge": edges})


def sg_program(edges: np.ndarray) -> Program:
    """Same generation as the forest workload states it: the inequality only
    in the non-recursive rule."""
    return Program(
        {"edge": 2, "sg": 2},
        [Rule(("sg", ("x", "y")), (("edge", ("p", "x")), ("edge", ("p", "y"))), (("x", "y"),)),
         Rule(("sg", ("x", "y")), (("edge", ("a", "x")), ("sg", ("a", "b")), ("edge", ("b", "y"))))],
        {"edge": edges})


def sg_paper_program(edges: np.ndarray) -> Program:
    """Same generation as printed in Section 5.2 (inequality in both rules)."""
    return Program(
        {"edge": 2, "sg": 2},
        [Rule(("sg", ("x", "y")), (("edge", ("p", "x")), ("edge", ("p", "y"))), (("x", "y"),)),
         Rule(("sg", ("x", "y")), (("edge", ("a", "x")), ("sg", ("a", "b")), ("edge", ("b", "y"))), (("x", "y"),))],
        {"edge": edges})


def points_to_program(edb: dict) -> Program:
    """Four mutually recursive points-to rules over assign / dereference."""
    return Program(
        {"assign": 2, "dereference": 2, "valueFlow": 2, "memoryAlias": 2, "valueAlias": 2},
        [Rule(("valueFlow", ("y", "x")), (("assign", ("y", "x")),)),
         Rule(("valueFlow", ("x", "y")), (("assign", ("x", "z")), ("memoryAlias", ("z", "y")))),
         Rule(("memoryAlias", ("x", "w")), (("dereference", ("y", "x")), ("valueAlias", ("y", "z")), ("dereference", ("z", "w")))),
         Rule(("valueAlias", ("x", "y")), (("valueFlow", ("z", "x")), ("valueFlow", ("z", "y"))))],
        dict(edb))


def owl_program(edb: dict, sch: OwlSchema) -> Program:
    """Rule instances per schema axiom (vertical partitioning): subclass
    closure, type inheritance, subproperty, transitivity, domain, range,
    inverse."""
    ar = {name: 2 for name in edb}
    ar["sct"] = 2
    P = lambda p: f"p{p}"
    rules = [Rule(("sct", ("c", "d")), (("sc", ("c", "d")),)),
             Rule(("sct", ("c", "e")), (("sc", ("c", "d")), ("sct", ("d", "e")))),
             Rule(("type", ("x", "d")), (("type", ("x", "c")), ("sc", ("c", "d"))))]
    for p, q in sch.sub_prop:
        rules.append(Rule((P(q), ("x", "y")), ((P(p), ("x", "y")),)))
    for p in sch.transitive:
        rules.append(Rule((P(p), ("x", "z")), ((P(p), ("x", "y")), (P(p), ("y", "z")))))
    for p, c in sch.domain:
        rules.append(Rule(("type", ("x", c)), ((P(p), ("x", "y")),)))
    for p, c in sch.range_:
        rules.append(Rule(("type", ("y", c)), ((P(p), ("x", "y")),)))
    for p, q in sch.inverse:
        rules.append(Rule((P(q), ("y", "x")), ((P(p), ("x", "y")),)))
        rules.append(Rule((P(p), ("y", "x")), ((P(q), ("x", "y")),)))
    return Program(ar, rules, dict(edb))


def batched_program(graphs: list, kinds: list) -> Program:
    """Many independent TC / SG instances as one program whose relations
    carry a leading instance column: instance i's facts are (i, u, v)."""
    tc_e = [np.concatenate([np.full((len(g), 1), i, np.uint32), g], axis=1)
            for i, (g, k) in enumerate(zip(graphs, kinds)) if k == "tc"]
    sg_e = [np.concatenate([np.full((len(g), 1), i, np.uint32), g], axis=1)
            for i, (g, k) in enumerate(zip(graphs, kinds)) if k == "sg"]
    cat = lambda xs: np.concatenate(xs) if xs else np.zeros((0, 3), np.uint32)
    return Program(
        {"tc_edge": 3, "tc_path": 3, "sg_edge": 3, "sg": 3},
        [Rule(("tc_path", ("i", "x", "y")), (("tc_edge", ("i", "x", "y")),)),
         Rule(("tc_path", ("i", "x", "z")), (("tc_edge", ("i", "x", "y")), ("tc_path", ("i", "y", "z")))),
         Rule(("sg", ("i", "x", "y")), (("sg_edge", ("i", "p", "x")), ("sg_edge", ("i", "p", "y"))), (("x", "y"),)),
         Rule(("sg", ("i", "x", "y")), (("sg_edge", ("i", "a", "x")), ("sg", ("i", "a", "b")), ("sg_edge", ("i", "b", "y"))))],
        {"tc_edge": cat(tc_e), "sg_edge": cat(sg_e)})


def random_program(seed: int, n_const: int = 5, max_facts: int = 8) -> Program:
    """A tiny random Datalog program for brute-force cross-checks: two EDB
    and two IDB relations of arity 1..3, 3-5 rules with 1-3 body atoms,
    constants, repeated variables and inequalities."""
    z = splitmix64(stream(seed, 61), np.arange(4096, dtype=np.uint64))
    k = [0]

    def r(m):
        v = int(uniform_below(z[k[0]], m)); k[0] += 1
        return v

    names = ["e0", "e1", "i0", "i1"]
    arity = {nm: 1 + r(3) for nm in names}
    arity["i0"] = 2
    edb = {}
    for nm in ("e0", "e1"):
        rows = {tuple(r(n_const) for _ in range(arity[nm])) for _ in range(1 + r(max_facts))}
        edb[nm] = np.array(sorted(rows), dtype=np.uint32).reshape(-1, arity[nm])
    rules = []
    vars_ = ["x", "y", "z", "w"]
    for _ in range(3 + r(3)):
        head_rel = names[2 + r(2)]
        nbody = 1 + r(3)
        body = []
        for _ in range(nbody):
            rel = names[r(4)]
            terms = tuple(vars_[r(4)] if r(6) else r(n_const) for _ in range(arity[rel]))
            body.append((rel, terms))
        bound = [t for _, ts in body for t in ts if isinstance(t, str)]
        if not bound:
            body[0] = (body[0][0], ("x",) + body[0][1][1:])
            bound = ["x"]
        head = tuple(bound[r(len(bound))] if r(5) else r(n_const) for _ in range(arity[head_rel]))
        neq = ()
        if r(3) == 0 and len(set(bound)) >= 2:
            a, b = sorted(set(bound))[:2]
            neq = ((a, b),)
        rules.append(Rule((head_rel, head), tuple(body), neq))
    return Program(arity, rules, edb)
