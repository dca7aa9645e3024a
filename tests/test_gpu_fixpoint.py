"""Whole-fixpoint parity of the GPU engine with the CPU oracle, through the
C ABI: the same sorted tuple sets, the same iteration counts and the same
per-round delta sizes on the same seeded inputs; plus the engine's error
paths (reserved value, round limit, rule shape, call order)."""
import numpy as np
import pytest

from paper_2501_13051_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cdl():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a GPU"
    from paper_2501_13051_gb300 import build as B
    B.build()
    from paper_2501_13051_gb300 import cdl as C
    return C


def check(cdl, oracle_lib, prog, **opts):
    got, st = cdl.run_program(prog, **opts)
    want = oracle_lib.run_program(prog)
    for nm in prog.arity:
        assert np.array_equal(got[nm], want.relations[nm]), nm
    assert st.iterations == want.iterations
    assert st.rounds == want.rounds
    per_round = [sum(want.deltas[nm][k] for nm in prog.idb()) for k in range(want.rounds)]
    assert st.delta_per_round == per_round
    assert st.derived_tuples == want.derived(prog)
    return st


# Every small-domain program below runs in both forms of the round's new
# tuples: bitmaps of the tuple space (dense_bits default) and sorted rows.
FORMS = pytest.mark.parametrize("dense", [0, -1], ids=["dense", "sorted"])


@FORMS
@pytest.mark.parametrize("n,m,seed", [(1000, 1500, 1), (1000, 1500, 11), (50, 120, 2), (400, 380, 3)])
def test_transitive_closure(cdl, oracle_lib, n, m, seed, dense):
    check(cdl, oracle_lib, W.tc_program(W.er_graph(n, m, seed)), dense_bits=dense)


@FORMS
@pytest.mark.parametrize("n,seed", [(2000, 2), (5000, 11)])
@pytest.mark.parametrize("make", [W.sg_program, W.sg_paper_program])
def test_same_generation(cdl, oracle_lib, n, seed, make, dense):
    check(cdl, oracle_lib, make(W.random_forest(n, seed)), dense_bits=dense)


@FORMS
def test_points_to_scaled(cdl, oracle_lib, dense):
    check(cdl, oracle_lib, W.points_to_program(W.points_to_edb(1 / 2048, 3)), dense_bits=dense)


@pytest.mark.parametrize("bits", [12, 21, 23])
def test_dense_bound_just_fits(cdl, oracle_lib, bits):
    """dense_bits below, between and above the tuple spaces of TC on 1,000
    nodes (10 + 10 bits) and of the paper's SG on 2,000 nodes (11 + 11):
    relations that fit are bitmaps, the others sorted rows."""
    prog = W.sg_paper_program(W.random_forest(2000, 7))
    check(cdl, oracle_lib, prog, dense_bits=bits)
    check(cdl, oracle_lib, W.tc_program(W.er_graph(1000, 1500, 3)), dense_bits=bits)


def test_owl_scaled(cdl, oracle_lib):
    check(cdl, oracle_lib, W.owl_program(*W.owl_triples(200_000, 4, n_entities=50_000)))


def many_relations_program(seed):
    """Six derived relations of arity 2, five of arity 1 and four of arity 3
    (independent closures over small random graphs, with a constant head
    column): a round's new tuples of each arity are sorted as one group."""
    arity, edb, rules = {}, {}, []
    for i in range(6):
        edb[f"e{i}"] = W.er_graph(300, 420, seed + i)
        arity[f"e{i}"] = arity[f"p{i}"] = 2
        rules += [W.Rule((f"p{i}", ("x", "y")), ((f"e{i}", ("x", "y")),)),
                  W.Rule((f"p{i}", ("x", "z")), ((f"p{i}", ("x", "y")), (f"e{i}", ("y", "z"))))]
    for i in range(5):
        arity[f"r{i}"] = 1
        rules += [W.Rule((f"r{i}", ("y",)), ((f"e{i}", (i, "y")),)),
                  W.Rule((f"r{i}", ("y",)), ((f"r{i}", ("x",)), (f"e{i}", ("x", "y"))))]
    for i in range(4):
        arity[f"t{i}"] = 3
        rules += [W.Rule((f"t{i}", ("x", "y", 7 + i)), ((f"e{i}", ("x", "y")),)),
                  W.Rule((f"t{i}", ("x", "z", "c")),
                         ((f"t{i}", ("x", "y", "c")), (f"e{i}", ("y", "z"))))]
    return W.Program(arity, rules, edb)


@FORMS
@pytest.mark.parametrize("seed", [1, 2])
def test_relations_sorted_as_groups(cdl, oracle_lib, seed, dense):
    check(cdl, oracle_lib, many_relations_program(seed), dense_bits=dense)


@FORMS
@pytest.mark.parametrize("seed", range(40))
def test_random_programs(cdl, oracle_lib, seed, dense):
    check(cdl, oracle_lib, W.random_program(seed), dense_bits=dense)


STAR_FORMS = pytest.mark.parametrize("star", [0, -1], ids=["star", "chain"])


@STAR_FORMS
@pytest.mark.parametrize("dense", [0, -1], ids=["dense", "sorted"])
@pytest.mark.parametrize("make", [W.sg_program, W.sg_paper_program])
def test_same_generation_star_and_chain(cdl, oracle_lib, make, dense, star):
    """The recursive rule edge(a, x), sg(a, b), edge(b, y): with star joins
    delta sg probes edge's index on a and on b and writes (x, y) for every
    pair of matches; as a chain of binary joins it writes (x, b) first."""
    st = check(cdl, oracle_lib, make(W.random_forest(3000, 7)), dense_bits=dense, star=star)
    assert (st.star_joins > 0) == (star == 0)


@STAR_FORMS
def test_points_to_star_and_chain(cdl, oracle_lib, star):
    # memoryAlias(x, w) :- dereference(y, x), valueAlias(y, z), dereference(z, w)
    st = check(cdl, oracle_lib, W.points_to_program(W.points_to_edb(1 / 2048, 5)), dense_bits=-1,
               star=star)
    assert (st.star_joins > 0) == (star == 0)


@pytest.mark.parametrize("seed", range(40))
def test_random_programs_as_chains(cdl, oracle_lib, seed):
    check(cdl, oracle_lib, W.random_program(seed), dense_bits=-1, star=-1)


def test_random_programs_take_star_joins(cdl):
    # the same programs with star joins on (their parity: test_random_programs)
    n = sum(cdl.run_program(W.random_program(s), dense_bits=-1)[1].star_joins for s in range(40))
    assert n > 0


@pytest.mark.parametrize("star", [0, -1], ids=["star", "chain"])
def test_star_join_row_past_2_32_outputs(cdl, star):
    """One probe row of q(x, y) :- e(a, x), s(a, b), e(b, y) meets 2^16
    edges on each side: 2^32 outputs, one more than a relation holds.  The
    star join's count pass flags the product, the chain's second join its
    total; both stop with CDL_E_CAPACITY."""
    kids = np.arange(1 << 16, dtype=np.uint32)
    e = np.concatenate([np.stack([np.full(1 << 16, 1, np.uint32), 100 + kids], axis=1),
                        np.stack([np.full(1 << 16, 2, np.uint32), 70000 + kids], axis=1)])
    R = W.Rule
    prog = W.Program({"e": 2, "s0": 2, "s": 2, "q": 2},
                     [R(("s", ("a", "b")), (("s0", ("a", "b")),)),
                      R(("q", ("x", "y")), (("e", ("a", "x")), ("s", ("a", "b")), ("e", ("b", "y"))))],
                     {"e": e, "s0": np.array([[1, 2]], dtype=np.uint32)})
    with cdl.Engine(dense_bits=-1, star=star) as eng:
        eng.load_program(prog)
        with pytest.raises(cdl.CdlError) as err:
            eng.run()
    assert cdl.STATUS[err.value.status] == "CDL_E_CAPACITY"


@pytest.mark.parametrize("opts", [dict(radix_bits=8), dict(radix_bits=9), dict(radix_bits=10), dict(hash_load=0.8), dict(timing=True)])
def test_engine_options_do_not_change_results(cdl, oracle_lib, opts):
    check(cdl, oracle_lib, W.sg_program(W.random_forest(1500, 5)), **opts)


def test_device_load_and_export(cdl, oracle_lib):
    import torch
    e = W.er_graph(200, 300, 7)
    prog = W.tc_program(e)
    with cdl.Engine() as eng:
        eng.relation("edge", 2)
        eng.relation("path", 2)
        cols = [torch.from_numpy(np.ascontiguousarray(e[:, k]).view(np.int32)).cuda() for k in range(2)]
        eng.load("edge", cols)
        for r in prog.rules:
            eng.rule(r.head, r.body, r.neq)
        eng.run()
        dcols = eng.export("path", device=True)
        got = np.stack([c.cpu().numpy().view(np.uint32) for c in dcols], axis=1)
    want = oracle_lib.run_program(prog)
    assert np.array_equal(got, want.relations["path"])


def test_load_deduplicates_and_merges(cdl):
    with cdl.Engine() as eng:
        eng.relation("r", 2)
        eng.load("r", np.array([[3, 1], [1, 2], [3, 1]], np.uint32))
        eng.load("r", np.array([[1, 2], [0, 9]], np.uint32))
        assert eng.export("r").tolist() == [[0, 9], [1, 2], [3, 1]]


def test_reserved_value_rejected(cdl):
    with cdl.Engine() as eng:
        eng.relation("r", 1)
        with pytest.raises(cdl.CdlError) as ei:
            eng.load("r", np.array([[5], [0xFFFFFFFF]], np.uint32))
        assert ei.value.name == "CDL_E_VALUE"
        eng.load("r", np.array([[5]], np.uint32))  # the engine stays usable
        assert eng.size("r") == 1


def test_load_many_is_all_or_nothing(cdl):
    import torch
    good = np.array([[1, 2], [3, 4], [1, 2]], np.uint32)
    bad = np.array([[5, 6], [7, 0xFFFFFFFF]], np.uint32)
    with cdl.Engine() as eng:
        for nm in ("a", "b", "c"):
            eng.relation(nm, 2)
        with pytest.raises(cdl.CdlError) as ei:
            eng.load_many({"a": good, "b": bad})
        assert ei.value.name == "CDL_E_VALUE"
        assert eng.size("a") == 0 and eng.size("b") == 0  # neither was added
        dev = [torch.from_numpy(np.ascontiguousarray(good[:, k]).view(np.int32)).cuda()
               for k in range(2)]
        eng.load_many({"a": good, "c": np.zeros((0, 2), np.uint32)})
        eng.load_many({"b": dev})
        assert eng.size("a") == 2 and eng.size("b") == 2 and eng.size("c") == 0
        with pytest.raises(ValueError):
            eng.load_many({"a": good, "b": dev})  # host and device columns in one call


def test_max_iters(cdl):
    prog = W.tc_program(W.er_graph(100, 200, 1))
    with pytest.raises(cdl.CdlError) as ei:
        cdl.run_program(prog, max_iters=2)
    assert ei.value.name == "CDL_E_MAXITER"


def test_rule_and_state_errors(cdl):
    with cdl.Engine() as eng:
        eng.relation("a", 2)
        eng.relation("b", 2)
        with pytest.raises(cdl.CdlError):  # head variable not bound in the body
            eng.rule(("b", ("x", "q")), [("a", ("x", "y"))])
        with pytest.raises(cdl.CdlError):  # arity mismatch
            eng.rule(("b", ("x",)), [("a", ("x", "y"))])
        eng.rule(("b", ("x", "y")), [("a", ("x", "y"))])
        eng.run()
        with pytest.raises(cdl.CdlError) as ei:
            eng.rule(("b", ("x", "y")), [("a", ("x", "y"))])
        assert ei.value.name == "CDL_E_STATE"
        with pytest.raises(cdl.CdlError):
            eng.run()


def test_export_capacity(cdl):
    import ctypes
    with cdl.Engine() as eng:
        eng.relation("r", 1)
        eng.load("r", np.arange(10, dtype=np.uint32).reshape(-1, 1))
        buf = np.zeros(4, np.uint32)
        got = ctypes.c_uint64()
        st = cdl.lib().cdl_relation_export(eng._h, eng.rels["r"], cdl._ptrs([buf.ctypes.data]), 4,
                                           ctypes.byref(got), 0)
        assert st == -3 and got.value == 10


def test_export_to_pinned_memory(cdl):
    # > 64 MB of columns into pinned host buffers: equal to the pageable export
    import torch
    prog = W.sg_program(W.random_forest(20000, 41))
    with cdl.Engine() as e:
        e.load_program(prog)
        e.run()
        n = e.size("sg")
        assert n * 8 > (64 << 20)
        pinned = [torch.empty(n, dtype=torch.int32, pin_memory=True) for _ in range(2)]
        e.export("sg", out=[t.data_ptr() for t in pinned])
        want = e.export("sg")
    got = np.stack([t.numpy().view(np.uint32) for t in pinned], 1)
    assert np.array_equal(got, want)


def declare(e, prog):
    for nm, ar in prog.arity.items():
        e.relation(nm, ar)
    for r in prog.rules:
        e.rule(r.head, r.body, r.neq)


@pytest.mark.parametrize("make,stop,graph", [
    (lambda: W.tc_program(W.er_graph(1000, 1500, 1)), 10, False),
    (lambda: W.sg_program(W.random_forest(2000, 51)), 4, True),
    (lambda: W.points_to_program(W.points_to_edb(1 / 2048, 52)), 3, False)])
def test_checkpoint_and_resume(cdl, oracle_lib, tmp_path, make, stop, graph):
    prog = make()
    want = oracle_lib.run_program(prog)
    path = str(tmp_path / "ckpt.bin")
    with cdl.Engine(max_iters=stop) as e:
        e.load_program(prog)
        with pytest.raises(cdl.CdlError) as ex:
            e.run()
        assert ex.value.name == "CDL_E_MAXITER"
        e.checkpoint_save(path)
    with cdl.Engine(graph=graph) as e:  # no facts loaded: the checkpoint holds them
        declare(e, prog)
        e.checkpoint_load(path)
        st = e.run()
        got = {nm: e.export(nm) for nm in prog.arity}
    for nm in prog.arity:
        assert np.array_equal(got[nm], want.relations[nm]), nm
    assert st.iterations == want.iterations and st.rounds == want.rounds
    per_round = [sum(want.deltas[nm][k] for nm in prog.idb()) for k in range(want.rounds)]
    assert st.delta_per_round == per_round


def test_checkpoint_errors(cdl, tmp_path):
    prog = W.tc_program(W.er_graph(50, 120, 2))
    path = str(tmp_path / "ckpt.bin")
    with cdl.Engine() as e:
        e.load_program(prog)
        with pytest.raises(cdl.CdlError) as ex:
            e.checkpoint_save(path)  # before run
        assert ex.value.name == "CDL_E_STATE"
        e.run()
        e.checkpoint_save(path)
    junk = tmp_path / "junk.bin"
    junk.write_bytes(b"not a checkpoint at all")
    with cdl.Engine() as e:
        declare(e, prog)
        with pytest.raises(cdl.CdlError) as ex:
            e.checkpoint_load(str(junk))
        assert ex.value.name == "CDL_E_INVALID"
    with cdl.Engine() as e:  # the same names with another arity
        e.relation("edge", 3)
        e.relation("path", 2)
        with pytest.raises(cdl.CdlError) as ex:
            e.checkpoint_load(path)
        assert ex.value.name == "CDL_E_INVALID"


@pytest.mark.parametrize("n,m,seed", [(300, 450, 4), (1000, 1500, 5)])
def test_nonlinear_closure_merges_its_index(cdl, oracle_lib, n, m, seed):
    """path(x, z) <- path(x, y), path(y, z).  The plain form builds on the
    smaller side (the delta) and probes Full.  The learned form (estimator
    on) picks the orientation that moves fewer bytes; building on Full, its
    index on the second column is, from the second round on, the previous
    round's index merged with the round's delta (no new sort of Full).  All
    stay bit-exact."""
    e = W.er_graph(n, m, seed)
    prog = W.Program({"edge": 2, "path": 2},
                     [W.Rule(("path", ("x", "y")), (("edge", ("x", "y")),)),
                      W.Rule(("path", ("x", "z")), (("path", ("x", "y")), ("path", ("y", "z"))))],
                     {"edge": e})
    st = check(cdl, oracle_lib, prog, dense_bits=-1)
    assert st.index_merges == 0
    # launches priced low: at this size the byte count alone decides
    st = check(cdl, oracle_lib, prog, dense_bits=-1, estimator=1, plan_launch_bytes=1.0)
    assert st.index_merges > 0
    st = check(cdl, oracle_lib, prog, dense_bits=-1, estimator=1)
    assert st.index_merges == 0  # at the default price the small Full is probed


def wide_program(seed):
    """Relations of arity 5 to 8 and rules of up to six body atoms (the
    shape of TGD-style rules): paths of five edges as 6-ary tuples, 8-node
    windows of walks that start at a node with a given attribute, slid one
    node per round (recursive), and an attribute relation of arity 5 joined
    on two columns with a constant and an inequality."""
    e = W.er_graph(60, 100, seed)
    rng = np.random.default_rng(seed)
    attr = np.unique(np.stack([np.arange(60), rng.integers(0, 3, 60), rng.integers(0, 3, 60),
                               rng.integers(0, 5, 60), rng.integers(0, 2, 60)],
                              axis=1).astype(np.uint32), axis=0)
    R = W.Rule
    rules = [
        R(("t6", ("a", "b", "c", "d", "f", "g")),
          (("e", ("a", "b")), ("e", ("b", "c")), ("e", ("c", "d")), ("e", ("d", "f")),
           ("e", ("f", "g")))),
        R(("w8", ("a", "b", "c", "d", "f", "g", "h", "i")),
          (("t6", ("a", "b", "c", "d", "f", "g")), ("e", ("g", "h")), ("e", ("h", "i")),
           ("attr", ("a", 0, "p", "q", "r")))),
        R(("w8", ("b", "c", "d", "f", "g", "h", "i", "j")),
          (("w8", ("a", "b", "c", "d", "f", "g", "h", "i")), ("e", ("i", "j")))),
        R(("m7", ("x", "y", "p", "q", "r", "s", 9)),
          (("e", ("x", "y")), ("attr", ("x", "p", "q", "r", "s")), ("attr", ("y", "p", "q", "u", "v")),
           ("e", ("y", "z")), ("attr", ("z", "p", "k", "l", "m")), ("e", ("z", "x2"))),
          (("x", "y"),)),
    ]
    arity = {"e": 2, "attr": 5, "t6": 6, "w8": 8, "m7": 7}
    return W.Program(arity, rules, {"e": e, "attr": attr})


@pytest.mark.parametrize("seed", [1, 2])
@pytest.mark.parametrize("dense", [0, -1], ids=["dense", "sorted"])
def test_wide_relations_and_long_bodies(cdl, oracle_lib, seed, dense):
    check(cdl, oracle_lib, wide_program(seed), dense_bits=dense)
