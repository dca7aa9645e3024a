"""Plain CPU statements of the steps of one semi-naive round.

TEST INFRASTRUCTURE ONLY (imported by tests, the smoke check and the bench's
CPU-baseline leg).  Shares no code with the GPU library.  Each function is
the definition of one step written out directly, with Python/numpy loops or a
single library call per step, and no blocking or fusion:

* ``hash_index``     -- Section 3, hybrid index: for each distinct value of a
                        column sorted by value, the pair (start offset in the
                        sorted order, number of occurrences).
* ``join_counts``    -- Algorithm 1, probe loop: the length of the matched
                        range of each probe value (0 when the value is absent).
* ``exclusive_scan`` -- Algorithm 1: output offset of each probe row
                        (pos_buf) and the total join size.
* ``join_pairs``     -- Algorithm 1, output-partitioned write: for output
                        position n, the probe row j with
                        pos_buf[j] <= n < pos_buf[j] + count[j] and the build
                        row start_j + (n - pos_buf[j]).
* ``lex_sort`` / ``unique_sorted`` -- the tuple order used for sets (Section
                        5 compares per-column radix sorting to row merge sort;
                        the order itself is lexicographic on unsigned values).
* ``difference`` / ``merge`` -- Section 4, "Union and Deduplication": the
                        difference operator New - Full and the union of the
                        deduplicated delta into Full.
"""
from __future__ import annotations

import bisect

import numpy as np


def hash_index(sorted_keys) -> dict:
    """key -> (start, count) over a column already sorted by value."""
    out = {}
    keys = [int(k) for k in np.asarray(sorted_keys).ravel()]
    for i, k in enumerate(keys):
        if i > 0 and keys[i - 1] > k:
            raise ValueError("column not sorted")
        if k in out:
            s, c = out[k]
            out[k] = (s, c + 1)
        else:
            out[k] = (i, 1)
    return out


def join_counts(probe_keys, index: dict) -> np.ndarray:
    return np.array([index.get(int(k), (0, 0))[1] for k in np.asarray(probe_keys).ravel()],
                    dtype=np.uint64)


def exclusive_scan(counts):
    counts = [int(c) for c in np.asarray(counts).ravel()]
    off, run = [], 0
    for c in counts:
        off.append(run)
        run += c
    return np.array(off, dtype=np.uint64), run


def join_pairs(probe_keys, sorted_build_keys):
    """Output-ordered (probe_row, build_row) pairs of an equi-join whose build
    side is sorted by its key."""
    idx = hash_index(sorted_build_keys)
    cnt = join_counts(probe_keys, idx)
    off, total = exclusive_scan(cnt)
    probe = np.asarray(probe_keys).ravel()
    pr = np.zeros(total, dtype=np.uint64)
    br = np.zeros(total, dtype=np.uint64)
    nonempty = [j for j in range(len(cnt)) if cnt[j] > 0]
    starts = [int(off[j]) for j in nonempty]
    for n in range(total):
        # the one non-empty range holding position n: the last start <= n
        j = nonempty[bisect.bisect_right(starts, n) - 1]
        start = idx[int(probe[j])][0]
        pr[n] = j
        br[n] = start + (n - int(off[j]))
    return pr, br


def lex_sort(rows) -> np.ndarray:
    rows = np.asarray(rows, dtype=np.uint32)
    if rows.ndim == 1:
        rows = rows.reshape(-1, 1)
    order = sorted(range(rows.shape[0]), key=lambda i: tuple(int(v) for v in rows[i]))
    return rows[order].reshape(rows.shape)


def unique_sorted(rows) -> np.ndarray:
    rows = np.asarray(rows, dtype=np.uint32)
    keep = [i for i in range(rows.shape[0]) if i == 0 or tuple(rows[i]) != tuple(rows[i - 1])]
    return rows[keep].reshape(-1, rows.shape[1])


def difference(new_rows, full_rows) -> np.ndarray:
    """Tuples of ``new_rows`` absent from ``full_rows``, sorted, unique."""
    full = {tuple(int(v) for v in r) for r in np.asarray(full_rows)}
    arity = np.asarray(new_rows).shape[1]
    d = sorted({tuple(int(v) for v in r) for r in np.asarray(new_rows)} - full)
    return np.array(d, dtype=np.uint32).reshape(-1, arity)


def merge(full_rows, delta_rows) -> np.ndarray:
    arity = np.asarray(full_rows).shape[1]
    s = {tuple(int(v) for v in r) for r in np.asarray(full_rows)}
    s |= {tuple(int(v) for v in r) for r in np.asarray(delta_rows)}
    return np.array(sorted(s), dtype=np.uint32).reshape(-1, arity)
