"""Pins of the step-by-step oracle (oracle.primitives), CPU only.

The values of the paper's worked join example (Sections 3 and 4, Algorithm
1) and independent library routines (numpy's unique / cumsum / lexsort and
Python set algebra) fix every step.
"""
import json
import os

import numpy as np
import pytest

from oracle import primitives as P

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_paper_join_example():
    g = json.load(open(os.path.join(GOLDEN, "paper_join_example.json")))
    b, p, want = g["build_sorted_keys"], g["probe_keys"], g["expected"]
    idx = P.hash_index(b)
    assert list(idx[1]) == want["hash_entry_key_1"]
    cnt = P.join_counts(p, idx)
    assert cnt.tolist() == want["range_lengths"]
    off, total = P.exclusive_scan(cnt)
    assert total == want["total"]
    assert off.tolist() == want["offsets"]
    pr, br = P.join_pairs(p, b)
    assert [int(pr[2]), int(br[2])] == want["position_2_pair"]
    assert len(pr) == want["total"]


@pytest.mark.parametrize("seed", range(5))
def test_primitives_against_library(seed):
    rng = np.random.default_rng(seed)
    keys = np.sort(rng.integers(0, 40, size=300)).astype(np.uint32)
    idx = P.hash_index(keys)
    u, first, counts = np.unique(keys, return_index=True, return_counts=True)
    assert idx == {int(k): (int(s), int(c)) for k, s, c in zip(u, first, counts)}

    probe = rng.integers(0, 50, size=120).astype(np.uint32)
    cnt = P.join_counts(probe, idx)
    assert cnt.tolist() == [int((keys == k).sum()) for k in probe]
    off, total = P.exclusive_scan(cnt)
    assert total == int(cnt.sum())
    assert np.array_equal(off, np.concatenate([[0], np.cumsum(cnt)[:-1]]).astype(np.uint64))

    pr, br = P.join_pairs(probe, keys)
    # output-partitioned order == nested-loop order (probe row, then build row)
    nested = [(j, i) for j in range(len(probe)) for i in range(len(keys)) if keys[i] == probe[j]]
    assert list(zip(pr.tolist(), br.tolist())) == nested

    rows = rng.integers(0, 6, size=(200, 3)).astype(np.uint32)
    s = P.lex_sort(rows)
    assert np.array_equal(s, rows[np.lexsort(rows.T[::-1])])
    uq = P.unique_sorted(s)
    assert np.array_equal(uq, np.unique(rows, axis=0))

    full = np.unique(rng.integers(0, 6, size=(150, 3)).astype(np.uint32), axis=0)
    d = P.difference(rows, full)
    want = sorted({tuple(r) for r in rows.tolist()} - {tuple(r) for r in full.tolist()})
    assert d.tolist() == [list(t) for t in want]
    m = P.merge(full, d)
    assert np.array_equal(m, np.unique(np.concatenate([full, rows]), axis=0))


def test_hash_index_rejects_unsorted():
    with pytest.raises(ValueError):
        P.hash_index([3, 1, 2])
