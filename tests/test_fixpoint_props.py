"""The sampled fixpoint checks (tests/fixpoint_props.py) that stand in for
the oracle at the benchmarked points-to size, pinned on the CPU: they
accept the oracle's fixpoint and reject planted mistakes (tuples dropped
from a relation, tuples with no derivation added, a rule's heads left
out)."""
import numpy as np
import pytest

from fixpoint_props import points_to_fixpoint_checks
from paper_2501_13051_gb300 import workloads as W


@pytest.fixture(scope="module")
def fixpoint(oracle_lib):
    edb = W.points_to_edb(1 / 1024, 7)
    prog = W.points_to_program(edb)
    res = oracle_lib.run_program(prog)
    rel = {nm: res.relations[nm] for nm in prog.idb()}
    assert all(len(r) > 100 for r in rel.values())
    return edb, rel


def test_accepts_the_oracle_fixpoint(fixpoint):
    edb, rel = fixpoint
    points_to_fixpoint_checks(edb, rel, np.random.default_rng(1), 2000)


def _with(rel, name, rows):
    out = dict(rel)
    out[name] = rows
    return out


@pytest.mark.parametrize("name", ["valueFlow", "memoryAlias", "valueAlias"])
def test_rejects_dropped_tuples(fixpoint, name):
    edb, rel = fixpoint
    kept = rel[name][np.arange(len(rel[name])) % 5 != 0]  # every fifth tuple gone
    with pytest.raises(AssertionError):
        points_to_fixpoint_checks(edb, _with(rel, name, kept), np.random.default_rng(2), 2000)


@pytest.mark.parametrize("name", ["valueFlow", "memoryAlias", "valueAlias"])
def test_rejects_tuples_without_a_derivation(fixpoint, name):
    edb, rel = fixpoint
    r = rel[name]
    rng = np.random.default_rng(3)
    hi = int(r.max()) + 1000
    bogus = rng.integers(hi - 500, hi, size=(len(r) // 4, 2)).astype(np.uint32)  # ids no rule reaches
    rows = np.unique(np.concatenate([r, bogus]), axis=0)
    with pytest.raises(AssertionError):
        points_to_fixpoint_checks(edb, _with(rel, name, rows), np.random.default_rng(4), 2000)


def test_rejects_unsorted_rows(fixpoint):
    edb, rel = fixpoint
    with pytest.raises(AssertionError):
        points_to_fixpoint_checks(edb, _with(rel, "valueAlias", rel["valueAlias"][::-1]),
                                  np.random.default_rng(5), 100)
