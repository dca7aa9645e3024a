"""Step (d) by Algorithm 2 (option dedup) against the CPU oracle, through
the C ABI: Full of eligible derived relations in the decomposed storage
model (rows in insertion order, a sorted index of surrogate ids and the
unique hashmap per column; or the hash-only multimap), new tuples tested by
the overlap of their id ranges, delta appended and merged into the indexes.
Whole fixpoints must be bit-exact with the oracle: tuples, iteration counts
and per-round delta sizes, as with the merge form of step (d)."""
import numpy as np
import pytest

from paper_2501_13051_gb300 import workloads as W

pytestmark = pytest.mark.gpu

MODES = pytest.mark.parametrize("dedup", [1, 2], ids=["hybrid", "hash-only"])


@pytest.fixture(scope="module")
def cdl():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a GPU"
    from paper_2501_13051_gb300 import build as B
    B.build()
    from paper_2501_13051_gb300 import cdl as C
    return C


def check(cdl, oracle_lib, prog, expect_dedup=True, **opts):
    with cdl.Engine(timing=True, **opts) as e:
        e.load_program(prog)
        st = e.run()
        got = {nm: e.export(nm) for nm in prog.arity}
        launches = {p["kernel"]: p["launches"] for p in e.kernel_profile()}
    want = oracle_lib.run_program(prog)
    for nm in prog.arity:
        assert np.array_equal(got[nm], want.relations[nm]), nm
    assert st.iterations == want.iterations and st.rounds == want.rounds
    per_round = [sum(want.deltas[nm][k] for nm in prog.idb()) for k in range(want.rounds)]
    assert st.delta_per_round == per_round
    assert st.derived_tuples == want.derived(prog)
    # Algorithm 2 ran (its probe is the "dedup" kernel class)
    assert (launches.get("dedup", 0) > 0) == expect_dedup
    return st, launches


@MODES
@pytest.mark.parametrize("dense", [0, -1], ids=["dense", "sorted"])
@pytest.mark.parametrize("n,m,seed", [(1000, 1500, 1), (50, 120, 2), (400, 380, 3)])
def test_transitive_closure(cdl, oracle_lib, n, m, seed, dense, dedup):
    check(cdl, oracle_lib, W.tc_program(W.er_graph(n, m, seed)), dense_bits=dense, dedup=dedup)


@MODES
@pytest.mark.parametrize("n,seed", [(2000, 2), (5000, 11)])
@pytest.mark.parametrize("make", [W.sg_program, W.sg_paper_program])
def test_same_generation(cdl, oracle_lib, n, seed, make, dedup):
    _, launches = check(cdl, oracle_lib, make(W.random_forest(n, seed)), dense_bits=-1,
                        dedup=dedup)
    # no difference-and-merge of sorted rows for sg: the hybrid form merges
    # only its per-column indexes, the hash-only form nothing
    if dedup == 2:
        assert launches.get("diff_merge", 0) == 0
    else:
        assert launches.get("diff_merge", 0) > 0


@MODES
def test_points_to_mixes_both_forms(cdl, oracle_lib, dedup):
    """valueFlow's Full is read (valueAlias joins it with itself), so it
    keeps the merge form; memoryAlias and valueAlias take Algorithm 2."""
    prog = W.points_to_program(W.points_to_edb(1 / 2048, 3))
    _, launches = check(cdl, oracle_lib, prog, dense_bits=-1, dedup=dedup)
    assert launches.get("diff_merge", 0) > 0


@MODES
@pytest.mark.parametrize("seed", range(0, 40, 3))
def test_random_programs(cdl, oracle_lib, seed, dedup):
    """Arity 1-3, constants, repeated variables, inequalities; relations
    read through Full keep the merge form."""
    prog = W.random_program(seed)
    with cdl.Engine(dense_bits=-1, dedup=dedup) as e:
        e.load_program(prog)
        st = e.run()
        got = {nm: e.export(nm) for nm in prog.arity}
    want = oracle_lib.run_program(prog)
    for nm in prog.arity:
        assert np.array_equal(got[nm], want.relations[nm]), nm
    assert st.iterations == want.iterations


@MODES
def test_loaded_facts_of_a_derived_relation(cdl, oracle_lib, dedup):
    """Facts loaded into the derived relation itself become the decomposed
    Full's first rows (ids 0 ..) at the first merge."""
    e = W.er_graph(300, 420, 9)
    prog = W.tc_program(e)
    prog.edb["path"] = W.er_graph(300, 200, 10)
    check(cdl, oracle_lib, prog, dense_bits=-1, dedup=dedup)


@MODES
def test_arity_three_and_skew(cdl, oracle_lib, dedup):
    """A ternary closure with a constant column (three hashmaps, the
    smallest id range walked) over a hub-heavy graph."""
    arity = {"e": 2, "t": 3}
    edges = np.concatenate([W.er_graph(200, 300, 5),
                            np.stack([np.zeros(150, np.uint32),
                                      np.arange(1, 151, dtype=np.uint32)], axis=1)])
    edges = np.unique(edges, axis=0)
    rules = [W.Rule(("t", ("x", "y", 3)), (("e", ("x", "y")),)),
             W.Rule(("t", ("x", "z", "c")), (("t", ("x", "y", "c")), ("e", ("y", "z"))))]
    check(cdl, oracle_lib, W.Program(arity, rules, {"e": edges}), dense_bits=-1, dedup=dedup)


def test_dedup_option_checked(cdl):
    with pytest.raises(cdl.CdlError):
        cdl.Engine(dedup=3)
