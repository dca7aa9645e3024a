"""Out-of-core relations (option host_full) against the CPU oracle, through
the C ABI: the Full version of derived relations that only step (d) reads
lives in pinned host memory, merged in place by the GPU over the CPU-GPU
link.  Fixpoints must be bit-exact with the oracle, and a device budget
(mem_limit) too small for Full in device memory must still be enough."""
import json
import os

import numpy as np
import pytest

from paper_2501_13051_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


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
    assert st.iterations == want.iterations and st.rounds == want.rounds
    per_round = [sum(want.deltas[nm][k] for nm in prog.idb()) for k in range(want.rounds)]
    assert st.delta_per_round == per_round
    return st


@pytest.mark.parametrize("dense", [0, -1], ids=["dense", "sorted"])
@pytest.mark.parametrize("n,m,seed", [(1000, 1500, 1), (400, 380, 3)])
def test_transitive_closure(cdl, oracle_lib, n, m, seed, dense):
    check(cdl, oracle_lib, W.tc_program(W.er_graph(n, m, seed)), dense_bits=dense, host_full=1)


@pytest.mark.parametrize("make", [W.sg_program, W.sg_paper_program])
def test_same_generation(cdl, oracle_lib, make):
    check(cdl, oracle_lib, make(W.random_forest(5000, 11)), dense_bits=-1, host_full=1)


def test_points_to_mixes_both_places(cdl, oracle_lib):
    """valueFlow's Full is read by a join, so it stays in device memory;
    memoryAlias and valueAlias keep theirs in host memory."""
    check(cdl, oracle_lib, W.points_to_program(W.points_to_edb(1 / 2048, 3)), dense_bits=-1,
          host_full=1)


@pytest.mark.parametrize("seed", range(0, 40, 4))
def test_random_programs(cdl, oracle_lib, seed):
    check(cdl, oracle_lib, W.random_program(seed), dense_bits=-1, host_full=1)


def test_export_to_device_and_host(cdl):
    """Exports read host-resident Full where it is, into host or device
    buffers, with the same rows."""
    prog = W.sg_program(W.random_forest(3000, 4))
    with cdl.Engine(host_full=1) as e:
        e.load_program(prog)
        e.run()
        host = e.export("sg")
        dev = e.export("sg", device=True)
    assert np.array_equal(np.stack([c.cpu().numpy().view(np.uint32) for c in dev], axis=1), host)


def test_sg_50k_beyond_a_device_budget(cdl):
    """SG on the 50,000-node forest with cross edges (1.16e8 tuples): with
    1.2 GB of device memory allowed the device-resident form runs out
    (its Full and merged copy need about 2 GB), the host-resident form
    reaches the oracle's fixpoint (digests of the stored expected values)."""
    from oracle.golden import SPECS, make_program, relation_digest
    with open(os.path.join(GOLDEN, "fixpoint_sg-forest-50k.json")) as f:
        g = json.load(f)
    prog = make_program(SPECS["sg-forest-50k"])
    budget = 1_200_000_000
    with cdl.Engine(mem_limit=budget) as e:
        e.load_program(prog)
        with pytest.raises(cdl.CdlError) as err:
            e.run()
    assert cdl.STATUS[err.value.status] == "CDL_E_NOMEM"
    with cdl.Engine(mem_limit=budget, host_full=1) as e:
        e.load_program(prog)
        st = e.run()
        rows = {nm: e.export(nm) for nm in prog.arity}
    assert st.iterations == g["iterations"] and st.derived_tuples == g["derived"]
    for nm, want in g["relations"].items():
        assert len(rows[nm]) == want["n"] and relation_digest(rows[nm]) == want["sha256"], nm
