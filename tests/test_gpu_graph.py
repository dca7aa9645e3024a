"""Rounds captured as one CUDA graph with a device-side loop (option graph):
the same fixpoints as the oracle, bit-exact in relations, iteration counts
and per-round delta sizes; buffers that a later round outgrows (small
starting capacities) hand the round to the host and the graph is rebuilt."""
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
    return st


@pytest.mark.parametrize("graph", [True, 64, 1024])
@pytest.mark.parametrize("n,m,seed", [(1000, 1500, 1), (1000, 1500, 11), (300, 420, 4)])
def test_transitive_closure_as_graph(cdl, oracle_lib, n, m, seed, graph):
    check(cdl, oracle_lib, W.tc_program(W.er_graph(n, m, seed)), graph=graph)


@pytest.mark.parametrize("graph", [True, 64])
@pytest.mark.parametrize("make", [lambda: W.sg_program(W.random_forest(2000, 31)),
                                  lambda: W.sg_paper_program(W.random_forest(3000, 32)),
                                  lambda: W.sg_program(W.random_forest(5000, 33))])
def test_same_generation_as_graph(cdl, oracle_lib, make, graph):
    # one star join per round (delta sg probing edge twice), with and without x != y
    check(cdl, oracle_lib, make(), graph=graph)


@pytest.mark.parametrize("graph", [True, 64])
def test_same_generation_as_graph_with_binary_joins(cdl, oracle_lib, graph):
    # two captured joins per round (edge, delta sg, edge) and the table between them
    check(cdl, oracle_lib, W.sg_program(W.random_forest(3000, 34)), graph=graph, star=-1)


def test_graph_runs_the_rounds_on_the_device(cdl, oracle_lib):
    prog = W.tc_program(W.er_graph(1000, 1500, 1))
    _, plain = cdl.run_program(prog, timing=True)
    _, g = cdl.run_program(prog, graph=True)
    assert g.delta_per_round == plain.delta_per_round
    # the same kernels run (counted once per captured round)
    assert g.kernel_launches > 0


def test_batched_instances_as_graph(cdl, oracle_lib):
    graphs, kinds = W.batched_instances(10, 81, 50, 2000)
    prog = W.batched_program(graphs, kinds)
    with cdl.Engine(n_instances=10, graph=True) as e:
        e.load_program(prog)
        st = e.run()
        rel = {"tc": e.export("tc_path"), "sg": e.export("sg")}
    whole = oracle_lib.run_program(prog)
    assert np.array_equal(rel["tc"], whole.relations["tc_path"])
    assert np.array_equal(rel["sg"], whole.relations["sg"])
    for i, (g, k) in enumerate(zip(graphs, kinds)):
        single = W.tc_program(g) if k == "tc" else W.sg_program(g)
        assert st.iters_per_instance[i] == oracle_lib.run_program(single).iterations, i


@pytest.mark.parametrize("count,seed,lo,hi", [(64, 84, 50, 4000), (96, 85, 20, 1500)])
def test_batched_graph_retires_on_the_device(cdl, oracle_lib, count, seed, lo, hi):
    """Batched rounds inside the captured graph, converged instances' rows
    moved out of Full by the device (decision, segment tables and gather):
    every instance equal to its own oracle run, tuples and iteration count."""
    graphs, kinds = W.batched_instances(count, seed, lo, hi)
    prog = W.batched_program(graphs, kinds)
    with cdl.Engine(n_instances=count, graph=True) as e:
        e.load_program(prog)
        st = e.run()
        rel = {"tc": e.export("tc_path"), "sg": e.export("sg")}
    assert st.graph_rounds > 0 and st.graph_retirements > 0
    for i, (g, k) in enumerate(zip(graphs, kinds)):
        single = W.tc_program(g) if k == "tc" else W.sg_program(g)
        want = oracle_lib.run_program(single)
        rows = rel[k]
        assert np.array_equal(rows[rows[:, 0] == i][:, 1:],
                              want.relations["path" if k == "tc" else "sg"]), i
        assert st.iters_per_instance[i] == want.iterations, i
    assert max(st.iters_per_instance) == st.iterations


def test_programs_outside_the_graph_class_run_as_usual(cdl, oracle_lib):
    # mutually recursive rules joining derived relations with each other
    check(cdl, oracle_lib, W.points_to_program(W.points_to_edb(1 / 2048, 5)), graph=True)


def test_graph_honours_max_iters(cdl):
    prog = W.tc_program(W.er_graph(1000, 1500, 1))  # 37 iterations
    with pytest.raises(cdl.CdlError) as ex:
        cdl.run_program(prog, graph=True, max_iters=10)
    assert ex.value.name == "CDL_E_MAXITER"
