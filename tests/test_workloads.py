"""Shape checks of the seeded input generators (CPU only)."""
import numpy as np

from paper_2501_13051_gb300 import workloads as W


def test_splitmix_counter_form_matches_sequential_form():
    # sequential SplitMix64: state += gamma; output = mix(state)
    def seq(seed, k):
        m = (1 << 64) - 1
        s, out = seed, []
        for _ in range(k):
            s = (s + 0x9E3779B97F4A7C15) & m
            z = s
            z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
            z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
            out.append(z ^ (z >> 31))
        return out
    got = W.splitmix64(np.uint64(12345), np.arange(6, dtype=np.uint64))
    assert [int(v) for v in got] == seq(12345, 6)


def test_er_graph_shape():
    e = W.er_graph(1000, 1500, 1)
    assert e.shape == (1500, 2) and e.dtype == np.uint32
    assert (e[:, 0] != e[:, 1]).all()
    assert len({tuple(r) for r in e.tolist()}) == 1500
    assert np.array_equal(e, W.er_graph(1000, 1500, 1))


def test_forest_shape():
    n = 20000
    f = W.random_forest(n, 2)
    tree, cross = f[: len(f) - n // 50], f[len(f) - n // 50:]
    assert (tree[:, 0] < tree[:, 1]).all()            # parent drawn from earlier nodes
    assert len(np.unique(tree[:, 1])) == len(tree)     # one parent per child
    assert 0.97 < len(tree) / (n - 1) < 0.99
    assert len(cross) == n // 50 and (cross[:, 0] != cross[:, 1]).all()
    assert len({tuple(r) for r in f.tolist()}) == len(f)


def test_points_to_and_owl_shapes():
    edb = W.points_to_edb(1 / 1024, 3)
    assert set(edb) == {"assign", "dereference"}
    assert edb["assign"].shape[1] == 2 and len(edb["assign"]) <= 4_000_000 // 1024
    tri, sch = W.owl_triples(20000, 4, n_entities=5000, n_classes=60)
    assert len(sch.sub_prop) == 40 and len(sch.transitive) == 10
    assert len(sch.domain) == 60 and len(sch.range_) == 60 and len(sch.inverse) == 10
    assert tri["type"][:, 1].min() >= 5000
    prog = W.owl_program(tri, sch)
    assert len(prog.rules) == 3 + 40 + 10 + 60 + 60 + 20


def test_batched_sizes_log_uniform():
    s = W.batched_graph_sizes(512, 5)
    assert s.min() >= 1000 and s.max() <= 500000
    assert 0.3 < np.mean(np.log(s) < np.log(np.sqrt(1e3 * 5e5))) < 0.7


def test_zipf_rank_frequencies():
    """P(rank r) is r^-s / H(s): the frequencies of the hottest ranks
    (through the permutation) match within sampling error."""
    universe, s, count = 1000, 1.1, 400_000
    perm = np.arange(universe, dtype=np.uint64)[::-1].copy()  # rank r -> id universe - r
    ids = W.zipf_ids(count, universe, s, 9, 1, perm)
    h = np.sum(np.arange(1, universe + 1, dtype=np.float64) ** -s)
    for r in (1, 2, 10, 100):
        p = r ** -s / h
        got = np.count_nonzero(ids == universe - r) / count
        assert abs(got - p) < 5 * np.sqrt(p * (1 - p) / count), (r, got, p)


def test_forest_parents_uniform_below_the_child():
    """Node i >= 1 draws its parent uniformly from [0, i): parent / i has
    mean 1/2 and variance 1/12 over many nodes; cross edges have uniform
    endpoints."""
    n = 200_000
    f = W.random_forest(n, 3)
    tree, cross = f[: len(f) - n // 50], f[len(f) - n // 50:]
    q = tree[:, 0].astype(np.float64) / tree[:, 1]
    assert abs(q.mean() - 0.5) < 0.005 and abs(q.var() - 1 / 12) < 0.005
    m = cross.astype(np.float64).mean(axis=0) / n
    assert (abs(m - 0.5) < 0.03).all()


def test_owl_schema_is_a_layered_dag():
    """Every subclass edge goes one level up (so the subclass graph is a
    DAG of the stated depth), every non-root class has one or two
    parents, and subproperty edges go from a lower to a higher property."""
    n_classes, levels, ne = 120, 12, 5000
    _, sch = W.owl_triples(4000, 6, n_entities=ne, n_classes=n_classes, levels=levels)
    lvl = (np.arange(n_classes) * levels) // n_classes
    parents = {}
    for c, d in sch.sub_class:
        assert lvl[c - ne] == lvl[d - ne] + 1, (c, d)
        parents.setdefault(c, set()).add(d)
    for c in range(n_classes):
        if lvl[c] > 0:
            assert 1 <= len(parents.get(ne + c, ())) <= 2, c
        else:
            assert ne + c not in parents
    assert all(a < b for a, b in sch.sub_prop) and len(set(sch.sub_prop)) == 40
    assert not set(sch.transitive) & {p for pair in sch.inverse for p in pair}
