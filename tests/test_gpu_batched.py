"""Batched independent fixpoints (instance column leading) against the
oracle, per instance: the same tuples and the same iteration count as the
instance run alone, bit-exact."""
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


@pytest.mark.parametrize("count,seed,lo,hi,retire,star", [(12, 77, 50, 3000, True, 0),
                                                         (12, 77, 50, 3000, False, 0),
                                                         (33, 78, 20, 800, True, 0),
                                                         (33, 78, 20, 800, True, -1)])
def test_batched_equals_each_instance(cdl, oracle_lib, count, seed, lo, hi, retire, star):
    graphs, kinds = W.batched_instances(count, seed, lo, hi)
    prog = W.batched_program(graphs, kinds)
    with cdl.Engine(n_instances=count, retire=retire, timing=True, star=star) as e:
        e.load_program(prog)
        st = e.run()
        rel = {"tc": e.export("tc_path"), "sg": e.export("sg")}
        moved = {p["kernel"]: p["launches"] for p in e.kernel_profile()}.get("retire", 0)
    # converged instances left the merged relations (and came back at the end)
    assert (moved > 0) == retire
    whole = oracle_lib.run_program(prog)
    assert np.array_equal(rel["tc"], whole.relations["tc_path"])
    assert np.array_equal(rel["sg"], whole.relations["sg"])
    assert st.iterations == whole.iterations
    for i, (g, k) in enumerate(zip(graphs, kinds)):
        single = W.tc_program(g) if k == "tc" else W.sg_program(g)
        want = oracle_lib.run_program(single)
        rows = rel[k]
        mine = rows[rows[:, 0] == i][:, 1:]
        assert np.array_equal(mine, want.relations["path" if k == "tc" else "sg"]), i
        assert st.iters_per_instance[i] == want.iterations, i
    assert max(st.iters_per_instance) == st.iterations
    # sg's recursive rule keys both edge atoms on (instance, delta sg's columns)
    assert (st.star_joins > 0) == (star == 0)


def test_export_of_one_instance(cdl):
    graphs, kinds = W.batched_instances(9, 83, 50, 2000)
    prog = W.batched_program(graphs, kinds)
    with cdl.Engine(n_instances=9) as e:
        e.load_program(prog)
        e.run()
        rows = e.export("tc_path")
        for i in range(9):
            mine = e.export_instance("tc_path", i)
            assert np.array_equal(mine, rows[rows[:, 0] == i]), i
        with pytest.raises(cdl.CdlError):
            e.instance_rows("tc_path", 9)


def test_batched_with_estimator_is_exact(cdl, oracle_lib):
    graphs, kinds = W.batched_instances(10, 79, 100, 4000)
    prog = W.batched_program(graphs, kinds)
    with cdl.Engine(n_instances=10, estimator=2) as e:
        e.load_program(prog)
        e.run()
        X, y = e.estimator_log()
    with cdl.Engine() as t:
        t.estimator_train(X, y, epochs=1500)
        params = t.estimator_params()
    with cdl.Engine(n_instances=10, estimator=1, est_params=params, est_min_rows=1) as e:
        e.load_program(prog)
        st = e.run()
        got = e.export("tc_path")
    assert np.array_equal(got, oracle_lib.run_program(prog).relations["tc_path"])
    assert st.est_predictions > 0


def test_batched_contract_is_checked(cdl):
    graphs, kinds = W.batched_instances(4, 80, 20, 100)
    prog = W.batched_program(graphs, kinds)
    with cdl.Engine(n_instances=3) as e:  # instance 3 is out of range
        e.load_program(prog)
        with pytest.raises(cdl.CdlError) as ex:
            e.run()
        assert ex.value.name == "CDL_E_VALUE"
    with cdl.Engine(n_instances=4) as e:  # a rule that ignores the instance column
        e.relation("a", 3)
        e.relation("b", 3)
        e.load("a", np.array([[0, 1, 2]], dtype=np.uint32))
        e.rule(("b", ["x", "x", "y"]), [("a", ["i", "x", "y"])])
        with pytest.raises(cdl.CdlError) as ex:
            e.run()
        assert ex.value.name == "CDL_E_INVALID"
