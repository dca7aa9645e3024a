"""The launch-parameter tuner: in tuning mode it times every candidate
(radix digit width and block size, hash load factor) and writes what it
measured to its file; in cache mode it reads that file back.  No candidate
may change a result, so every tuned run is compared with the oracle or with
the untuned run, bit-exact."""
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


def read_cache(path):
    rows = {}
    for line in open(path):
        key, cand, n, cost = line.split()
        rows.setdefault(key, {})[int(cand)] = (int(n), float(cost))
    return rows


def test_tuning_runs_cover_every_candidate(cdl, oracle_lib, tmp_path):
    cache = str(tmp_path / "tune.txt")
    prog = W.sg_program(W.random_forest(5000, 21))
    want = oracle_lib.run_program(prog)
    for _ in range(8):  # each run measures the candidates not yet tried twice
        # sorted rows (dense_bits=-1): a bitmap of this tuple space needs no sort
        got, st = cdl.run_program(prog, autotune=2, tune_cache=cache, dense_bits=-1)
        assert np.array_equal(got["sg"], want.relations["sg"])
        assert st.iterations == want.iterations
    rows = read_cache(cache)
    sorts = [k for k in rows if k.startswith("sort.")]
    assert sorts, rows
    for k in sorts:  # all four (digit width, block size) candidates timed
        assert sorted(rows[k]) == [0, 1, 2, 3], (k, rows[k])
        assert all(n >= 1 and c > 0 for n, c in rows[k].values())
    # cache mode reads the file and takes the cheapest candidates
    got, st = cdl.run_program(prog, autotune=1, tune_cache=cache, dense_bits=-1)
    assert np.array_equal(got["sg"], want.relations["sg"])


@pytest.mark.parametrize("radix_bits", [0, 8, 9, 10])
def test_every_sort_candidate_is_exact(cdl, tmp_path, radix_bits):
    # a larger forest: sorts and indexes past the tuner's size thresholds
    prog = W.sg_program(W.random_forest(40000, 22))
    base, _ = cdl.run_program(prog)
    cache = str(tmp_path / "tune.txt")
    for _ in range(5):
        got, _ = cdl.run_program(prog, autotune=2, tune_cache=cache, radix_bits=radix_bits)
        assert np.array_equal(got["sg"], base["sg"])
    rows = read_cache(cache)
    assert any(k.startswith("load.") for k in rows), rows
    for k, c in rows.items():
        if k.startswith("load."):
            assert sorted(c) == [0, 1, 2, 3], (k, c)


def test_missing_cache_file_is_not_an_error(cdl, oracle_lib, tmp_path):
    prog = W.tc_program(W.er_graph(300, 450, 5))
    got, st = cdl.run_program(prog, autotune=1, tune_cache=str(tmp_path / "absent.txt"))
    assert np.array_equal(got["path"], oracle_lib.run_program(prog).relations["path"])


def test_unwritable_cache_file_is_reported(cdl, tmp_path):
    prog = W.tc_program(W.er_graph(1000, 1500, 6))  # sorts large enough to be timed
    bad = str(tmp_path / "no-such-dir" / "tune.txt")
    with pytest.raises(cdl.CdlError) as ex:
        cdl.run_program(prog, autotune=2, tune_cache=bad, dense_bits=-1)
    assert ex.value.name == "CDL_E_INVALID"
