"""Pins of the CPU oracle against facts fixed outside it (CPU only).

Each check below is independent of the oracle's code: breadth-first search
and Warshall's closure for transitive closure, the closed form of
same-generation on a forest, brute-force grounding of tiny random programs,
the rule-closure and input-containment invariants, and the equality of the
semi-naive and naive rounds (Jacobi rounds make every per-round delta
canonical).  A dropped semi-naive variant, a wrong join index, a transposed
head column or a wrong round count fails at least one of them.
"""
import itertools
from collections import deque

import numpy as np
import pytest

from paper_2501_13051_gb300 import workloads as W


def as_set(rows):
    return {tuple(int(v) for v in r) for r in np.asarray(rows)}


# ---------------------------------------------------------------- TC pins

def bfs_closure(n, edges):
    """Pairs (s, t) joined by a path of >= 1 edges, with the shortest such
    length; plain BFS from every source's successors."""
    succ = [[] for _ in range(n)]
    for u, v in edges:
        succ[int(u)].append(int(v))
    dist = {}
    for s in range(n):
        seen = {}
        q = deque()
        for v in succ[s]:
            if v not in seen:
                seen[v] = 1
                q.append(v)
        while q:
            x = q.popleft()
            for y in succ[x]:
                if y not in seen:
                    seen[y] = seen[x] + 1
                    q.append(y)
        for t, d in seen.items():
            dist[(s, t)] = d
    return dist


@pytest.mark.parametrize("n,m,seed", [(30, 45, 3), (200, 300, 4), (60, 200, 5), (1000, 1500, 1)])
def test_tc_matches_bfs(oracle_lib, n, m, seed):
    e = W.er_graph(n, m, seed)
    res = oracle_lib.run_program(W.tc_program(e))
    dist = bfs_closure(n, e)
    assert as_set(res.relations["path"]) == set(dist)
    # round k derives exactly the pairs whose shortest path has k edges
    hist = np.bincount(np.fromiter(dist.values(), dtype=np.int64))
    assert res.deltas["path"][:-1] == [int(h) for h in hist[1:]]
    assert res.deltas["path"][-1] == 0
    assert res.iterations == max(dist.values())
    assert res.relations["edge"].shape[0] == m


@pytest.mark.parametrize("seed", range(6))
def test_tc_matches_warshall(oracle_lib, seed):
    n = 8 + 7 * seed
    m = min(n * (n - 1), 2 * n)
    e = W.er_graph(n, m, 100 + seed)
    a = np.zeros((n, n), dtype=bool)
    a[e[:, 0], e[:, 1]] = True
    r = a.copy()
    for k in range(n):  # Warshall's algorithm
        r |= np.outer(r[:, k], r[k, :])
    res = oracle_lib.run_program(W.tc_program(e))
    assert as_set(res.relations["path"]) == {(int(i), int(j)) for i, j in zip(*np.nonzero(r))}


# ---------------------------------------------------------------- SG pins

def forest_depths(n, edges):
    par = -np.ones(n, dtype=np.int64)
    par[edges[:, 1]] = edges[:, 0]
    depth = np.zeros(n, dtype=np.int64)
    root = np.arange(n)
    for i in range(n):  # parents precede children in a recursive forest
        if par[i] >= 0:
            depth[i] = depth[par[i]] + 1
            root[i] = root[par[i]]
    return par, depth, root


@pytest.mark.parametrize("n,seed", [(300, 7), (2000, 8), (5000, 2)])
@pytest.mark.parametrize("prog", [W.sg_program, W.sg_paper_program])
def test_sg_forest_closed_form(oracle_lib, n, seed, prog):
    f = W.random_forest(n, seed, cross_frac=0.0)
    par, depth, root = forest_depths(n, f)
    groups = {}
    for v in range(n):
        groups.setdefault((int(root[v]), int(depth[v])), []).append(v)
    res = oracle_lib.run_program(prog(f))
    got = res.relations["sg"]
    # |sg| = sum over (tree, depth) of c (c - 1)
    assert len(got) == sum(len(g) * (len(g) - 1) for g in groups.values())
    want = set()
    for g in groups.values():
        want.update((x, y) for x in g for y in g if x != y)
    assert as_set(got) == want

    # round k derives the pairs whose lowest common ancestor is k levels up
    def lca_dist(x, y):
        k = 0
        while x != y:
            x, y, k = int(par[x]), int(par[y]), k + 1
        return k
    d = np.bincount([lca_dist(x, y) for x, y in got]) if len(got) else np.zeros(1)
    assert res.deltas["sg"][:-1] == [int(c) for c in d[1:]]
    assert res.iterations == len(d) - 1


# ------------------------------------------------------- brute force pins

def brute_force(program):
    """Least fixpoint by grounding every rule over the active domain and
    iterating T to a fixpoint (no joins, no indexes, no semi-naive)."""
    dom = set()
    for rows in program.edb.values():
        dom.update(int(v) for v in np.asarray(rows).ravel())
    for r in program.rules:
        for _, ts in (r.head,) + tuple(r.body):
            dom.update(t for t in ts if isinstance(t, int))
    dom = sorted(dom)
    facts = {nm: set() for nm in program.arity}
    for nm, rows in program.edb.items():
        facts[nm] |= as_set(rows)
    rounds = []
    while True:
        derived = {nm: set() for nm in program.arity}
        for r in program.rules:
            vs = sorted({t for _, ts in r.body for t in ts if isinstance(t, str)})
            for vals in itertools.product(dom, repeat=len(vs)):
                env = dict(zip(vs, vals))
                g = lambda ts: tuple(env[t] if isinstance(t, str) else t for t in ts)
                if all(g(ts) in facts[nm] for nm, ts in r.body) and \
                        all(env[a] != env[b] for a, b in r.neq):
                    derived[r.head[0]].add(g(r.head[1]))
        new = {nm: derived[nm] - facts[nm] for nm in program.arity}
        rounds.append(sum(len(v) for v in new.values()))
        for nm in program.arity:
            facts[nm] |= new[nm]
        if rounds[-1] == 0:
            return facts, rounds


@pytest.mark.parametrize("seed", range(40))
def test_random_programs_match_brute_force(oracle_lib, seed):
    prog = W.random_program(seed)
    facts, rounds = brute_force(prog)
    for naive in (False, True):
        res = oracle_lib.run_program(prog, naive=naive)
        for nm in prog.arity:
            assert as_set(res.relations[nm]) == facts[nm], (nm, naive)
        per_round = [sum(res.deltas[nm][k] for nm in prog.arity) for k in range(res.rounds)]
        assert per_round == rounds
        assert res.iterations == len(rounds) - 1


def test_hand_program_with_constants_and_repeats(oracle_lib):
    # p(x) <- e(x, x); q(x, 7) <- e(x, y), p(y), x != y; q(y, x) <- q(x, y)
    prog = W.Program(
        {"e": 2, "p": 1, "q": 2},
        [W.Rule(("p", ("x",)), (("e", ("x", "x")),)),
         W.Rule(("q", ("x", 7)), (("e", ("x", "y")), ("p", ("y",))), (("x", "y"),)),
         W.Rule(("q", ("y", "x")), (("q", ("x", "y")),))],
        {"e": np.array([[1, 1], [2, 1], [1, 3], [3, 3], [4, 4], [3, 1]], np.uint32)})
    res = oracle_lib.run_program(prog)
    assert as_set(res.relations["p"]) == {(1,), (3,), (4,)}
    assert as_set(res.relations["q"]) == {(2, 7), (1, 7), (3, 7), (7, 2), (7, 1), (7, 3)}
    # round 1: p; round 2: q(., 7); round 3: the swapped q(7, .)
    assert res.deltas["p"] == [3, 0, 0, 0] and res.deltas["q"] == [0, 3, 3, 0]
    assert res.iterations == 3


# ------------------------------------------------ semi-naive == naive

@pytest.mark.parametrize("make", [
    lambda: W.tc_program(W.er_graph(300, 500, 9)),
    lambda: W.sg_program(W.random_forest(1500, 10)),
    lambda: W.sg_paper_program(W.random_forest(1500, 10)),
    lambda: W.points_to_program(W.points_to_edb(1 / 4096, 11)),
    lambda: W.owl_program(*W.owl_triples(20000, 12, n_entities=5000, n_classes=60)),
])
def test_seminaive_equals_naive(oracle_lib, make):
    prog = make()
    a = oracle_lib.run_program(prog)
    b = oracle_lib.run_program(prog, naive=True)
    assert a.iterations == b.iterations and a.rounds == b.rounds
    for nm in prog.arity:
        assert np.array_equal(a.relations[nm], b.relations[nm]), nm
        assert a.deltas[nm] == b.deltas[nm], nm


# ---------------------------------------------------------- invariants

def closed_and_contains_edb(program, rels):
    facts = {nm: as_set(rows) for nm, rows in rels.items()}
    for nm, rows in program.edb.items():
        assert as_set(rows) <= facts[nm]
    for r in program.rules:  # one application of T adds nothing
        envs = [{}]
        for nm, ts in r.body:
            nxt = []
            for env in envs:
                for t in facts[nm]:
                    e2 = dict(env)
                    ok = True
                    for term, v in zip(ts, t):
                        if isinstance(term, int):
                            ok &= term == v
                        elif term in e2:
                            ok &= e2[term] == v
                        else:
                            e2[term] = v
                    if ok:
                        nxt.append(e2)
            envs = nxt
        for env in envs:
            if all(env[a] != env[b] for a, b in r.neq):
                h = tuple(env[t] if isinstance(t, str) else t for t in r.head[1])
                assert h in facts[r.head[0]]


def test_invariants_small_programs(oracle_lib):
    for prog in (W.tc_program(W.er_graph(40, 80, 13)), W.sg_program(W.random_forest(120, 14)),
                 W.points_to_program(W.points_to_edb(1 / 200000, 15))):
        res = oracle_lib.run_program(prog)
        closed_and_contains_edb(prog, res.relations)
        for rows in res.relations.values():  # sorted, unique
            t = [tuple(r) for r in rows.tolist()]
            assert t == sorted(set(t))


def test_max_iters_reports_error(oracle_lib):
    with pytest.raises(RuntimeError):
        oracle_lib.run_program(W.tc_program(W.er_graph(100, 200, 1)), max_iters=2)


@pytest.mark.parametrize("n,seed", [(1, 1), (2, 3), (300, 7), (2000, 8), (5000, 2)])
def test_sg_closed_form_module_matches_oracle(oracle_lib, n, seed):
    """oracle.closed_forms.sg_forest (vectorised; the form the full-size GPU
    test uses) against the std::set evaluator and against the pairs it
    describes: every pair within a (tree, depth) group, x != y."""
    from oracle import closed_forms as C
    f = W.random_forest(n, seed, cross_frac=0.0)
    cf = C.sg_forest(n, f)
    res = oracle_lib.run_program(W.sg_program(f))
    got = res.relations["sg"]
    assert cf["size"] == len(got)
    assert cf["deltas"] == res.deltas["sg"][:-1] and res.deltas["sg"][-1] == 0
    assert cf["iterations"] == res.iterations
    g = cf["group"]
    want = {(x, y) for x in range(n) for y in range(n) if x != y and g[x] == g[y]} \
        if n <= 300 else None
    if want is not None:
        assert as_set(got) == want
    # the per-row properties the full-size GPU test checks prove the same set
    assert np.all(g[got[:, 0]] == g[got[:, 1]]) and np.all(got[:, 0] != got[:, 1])
    deg = np.bincount(got[:, 0], minlength=n) if len(got) else np.zeros(n, np.int64)
    assert np.array_equal(deg, cf["group_size"][g] - 1)


def test_sg_closed_form_rejects_non_forests():
    from oracle import closed_forms as C
    with pytest.raises(ValueError):
        C.sg_forest(3, np.array([[0, 2], [1, 2]]))
    with pytest.raises(ValueError):
        C.sg_forest(3, np.array([[2, 1]]))
