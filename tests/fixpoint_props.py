"""Sampled checks that exported relations are a fixpoint of the points-to
rules, for sizes beyond the oracle (test helper; no GPU needed).

Relations are (n, 2) uint32 arrays sorted lexicographically, as exports
are.  Pairs are looked up as uint64 keys x << 32 | y by binary search.
"""
import numpy as np


def _keys(rows):
    """Sorted uint64 keys x << 32 | y of sorted, unique pairs."""
    return (rows[:, 0].astype(np.uint64) << np.uint64(32)) | rows[:, 1].astype(np.uint64)


def _flip(rows):
    """Keys of the pairs with their columns swapped, sorted."""
    return np.sort((rows[:, 1].astype(np.uint64) << np.uint64(32)) | rows[:, 0].astype(np.uint64))


def _member(keys, q):
    q = np.atleast_1d(np.asarray(q, dtype=np.uint64))
    if len(keys) == 0:
        return np.zeros(len(q), dtype=bool)
    i = np.minimum(np.searchsorted(keys, q), len(keys) - 1)
    return keys[i] == q


def _row(keys, x):
    """Second columns of the pairs whose first column is x."""
    lo = np.searchsorted(keys, np.uint64(x) << np.uint64(32))
    hi = np.searchsorted(keys, (np.uint64(x) + np.uint64(1)) << np.uint64(32))
    return keys[lo:hi] & np.uint64(0xFFFFFFFF)


def _pair(x, ys):
    return (np.uint64(x) << np.uint64(32)) | np.asarray(ys, dtype=np.uint64)


def points_to_fixpoint_checks(edb, rel, rng, samples):
    """Asserts, on `samples` random picks each, that the derived relations
    of the points-to program (workloads.points_to_program) are sorted and
    unique, that sampled tuples have a derivation by one of the rules from
    the relations (support), and that sampled rule instances over the
    relations land in them (closure; every assign pair is checked).  The
    rules:
      valueFlow(y, x)   <- assign(y, x)
      valueFlow(x, y)   <- assign(x, z), memoryAlias(z, y)
      memoryAlias(x, w) <- dereference(y, x), valueAlias(y, z), dereference(z, w)
      valueAlias(x, y)  <- valueFlow(z, x), valueFlow(z, y)
    """
    vf, ma, va = rel["valueFlow"], rel["memoryAlias"], rel["valueAlias"]
    K = {nm: _keys(r) for nm, r in rel.items()}
    for nm, k in K.items():
        assert bool((k[1:] > k[:-1]).all()), nm  # sorted and unique
    A, D = edb["assign"], edb["dereference"]
    KA, KD, KDt, KVFt = _keys(A), _keys(D), _flip(D), _flip(vf)

    # support: each sampled tuple is derived by a rule from the relations
    for x, y in vf[rng.integers(0, len(vf), samples)] if len(vf) else ():
        zs = _row(KA, x)
        ok = bool(_member(KA, _pair(x, [y]))[0]) or bool(
            _member(K["memoryAlias"], (zs << np.uint64(32)) | np.uint64(y)).any())
        assert ok, ("valueFlow", int(x), int(y))
    for x, y in va[rng.integers(0, len(va), samples)] if len(va) else ():
        zs = _row(KVFt, x)
        assert bool(_member(K["valueFlow"], (zs << np.uint64(32)) | np.uint64(y)).any()), \
            ("valueAlias", int(x), int(y))
    for x, w in ma[rng.integers(0, len(ma), samples)] if len(ma) else ():
        ys, zs = _row(KDt, x), _row(KDt, w)
        assert any(bool(_member(K["valueAlias"], _pair(y, zs)).any()) for y in ys), \
            ("memoryAlias", int(x), int(w))

    # closure: sampled rule instances over the relations land in them
    assert bool(_member(K["valueFlow"], KA).all()), "assign"
    for x, z in A[rng.integers(0, len(A), samples)]:
        ys = _row(K["memoryAlias"], z)
        if len(ys) > 4096:
            ys = rng.choice(ys, 4096, replace=False)
        assert bool(_member(K["valueFlow"], _pair(x, ys)).all()), ("rule 2", int(x), int(z))
    for y, x in D[rng.integers(0, len(D), samples)]:
        zs = _row(K["valueAlias"], y)
        if len(zs) > 64:
            zs = rng.choice(zs, 64, replace=False)
        for z in zs:
            assert bool(_member(K["memoryAlias"], _pair(x, _row(KD, z))).all()), \
                ("rule 3", int(x), int(z))
    for z in vf[rng.integers(0, len(vf), samples), 0] if len(vf) else ():
        xs = _row(K["valueFlow"], z)
        a, b = rng.choice(xs, 64), rng.choice(xs, 64)
        assert bool(_member(K["valueAlias"], (a << np.uint64(32)) | b).all()), ("rule 4", int(z))
