"""Step-by-step parity of the sm_103a kernels with the CPU oracle
(oracle.primitives), through the C ABI, bit-exact.  Sizes span several
tiles (scan tiles of 2048, sort tiles of 4096, merge tiles of 2048) plus a
ragged tail, and the edge cases: empty, one row, all-equal keys, the largest
allowed value 0xFFFFFFFE."""
import numpy as np
import pytest

from oracle import primitives as P

pytestmark = pytest.mark.gpu

MAXV = 0xFFFFFFFE


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a GPU"
    from paper_2501_13051_gb300 import build as B
    B.build()
    return torch


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.uint32)).view(np.int32)).cuda()


def host(t):
    return t.cpu().numpy().view(np.uint32)


def rows_of(cols):
    if not cols or cols[0].numel() == 0:
        return np.zeros((0, len(cols)), np.uint32)
    return np.stack([host(c) for c in cols], axis=1)


def keys_case(rng, kind, n):
    if kind == "uniform":
        return np.sort(rng.integers(0, max(1, n // 3), size=n)).astype(np.uint32)
    if kind == "equal":
        return np.full(n, 7, np.uint32)
    if kind == "max":
        return np.sort(rng.integers(MAXV - 50, MAXV + 1, size=n, dtype=np.uint64)).astype(np.uint32)
    if kind == "zipf":
        return np.sort(np.minimum(rng.zipf(1.3, size=n), 5000)).astype(np.uint32)
    raise ValueError(kind)


@pytest.mark.parametrize("kind", ["uniform", "equal", "max", "zipf"])
@pytest.mark.parametrize("n", [0, 1, 33, 2048 * 5 + 17])
def test_hash_build_and_count(torch_cuda, kind, n):
    from paper_2501_13051_gb300 import cdl
    rng = np.random.default_rng(n + len(kind))
    keys = keys_case(rng, kind, n)
    probe = np.concatenate([keys[rng.permutation(n)][: n // 2],
                            rng.integers(0, 1 << 20, size=n // 3 + 3).astype(np.uint32),
                            np.array([MAXV, 0], np.uint32)])
    table = cdl.hash_build(dev(torch_cuda, keys))
    got = host(cdl.join_count(dev(torch_cuda, probe), table))
    want = P.join_counts(probe, P.hash_index(keys))
    assert np.array_equal(got.astype(np.uint64), want)


@pytest.mark.parametrize("n", [0, 1, 2047, 2048, 2049, 2048 * 9 + 5, 300_001])
def test_exclusive_scan(torch_cuda, n):
    from paper_2501_13051_gb300 import cdl
    rng = np.random.default_rng(n)
    c = rng.integers(0, 50, size=n).astype(np.uint32)
    if n > 10:
        c[n // 2] = 0xFFFFFFFF  # sums pass 2^32: offsets must be 64-bit
    off, total = cdl.exclusive_scan(dev(torch_cuda, c))
    woff, wtotal = P.exclusive_scan(c)
    assert total == wtotal
    assert np.array_equal(off.cpu().numpy().astype(np.uint64), woff)


@pytest.mark.parametrize("shape", ["paper", "uniform", "skew", "empty_probe", "no_match"])
def test_join_matches_algorithm_1(torch_cuda, shape):
    from paper_2501_13051_gb300 import cdl
    rng = np.random.default_rng(hash(shape) % 1000)
    if shape == "paper":
        b = np.array([1, 1, 1, 2, 3, 3, 3, 3, 4, 4, 4, 4], np.uint32)
        p = np.array([1, 2, 3, 4, 7], np.uint32)
    elif shape == "uniform":
        b = np.sort(rng.integers(0, 4000, size=9000)).astype(np.uint32)
        p = rng.integers(0, 4500, size=7000).astype(np.uint32)
    elif shape == "skew":
        b = np.sort(np.concatenate([np.full(20000, 5, np.uint32),
                                    rng.integers(0, 3000, size=3000).astype(np.uint32)]))
        p = np.concatenate([np.full(3, 5, np.uint32), rng.integers(0, 3000, size=5000).astype(np.uint32)])
    elif shape == "empty_probe":
        b = np.arange(100, dtype=np.uint32)
        p = np.zeros(0, np.uint32)
    else:
        b = np.arange(100, dtype=np.uint32)
        p = np.arange(1000, 1100, dtype=np.uint32)
    bpay = (np.arange(len(b)) * 7 + 3).astype(np.uint32)   # build payload column
    ppay = (np.arange(len(p)) * 11 + 1).astype(np.uint32)  # probe payload column
    # head = (probe payload, build payload, constant 9)
    out = cdl.join([dev(torch_cuda, p), dev(torch_cuda, ppay)], 0,
                   [dev(torch_cuda, b), dev(torch_cuda, bpay)], 0,
                   [(0, 1), (1, 1), (2, 9)])
    pr, br = P.join_pairs(p, b)
    want = np.stack([ppay[pr.astype(np.int64)], bpay[br.astype(np.int64)],
                     np.full(len(pr), 9, np.uint32)], axis=1) if len(pr) else np.zeros((0, 3), np.uint32)
    assert np.array_equal(rows_of(out), want)  # output order is Algorithm 1's


def test_join_with_inequality(torch_cuda):
    from paper_2501_13051_gb300 import cdl
    rng = np.random.default_rng(3)
    b = np.sort(rng.integers(0, 500, size=6000)).astype(np.uint32)
    bx = rng.integers(0, 40, size=6000).astype(np.uint32)
    p = rng.integers(0, 600, size=5000).astype(np.uint32)
    px = rng.integers(0, 40, size=5000).astype(np.uint32)
    out = cdl.join([dev(torch_cuda, p), dev(torch_cuda, px)], 0,
                   [dev(torch_cuda, b), dev(torch_cuda, bx)], 0,
                   [(0, 1), (1, 1)], neq=[((0, 1), (1, 1))])
    pr, br = P.join_pairs(p, b)
    a, c = px[pr.astype(np.int64)], bx[br.astype(np.int64)]
    keep = a != c
    want = P.lex_sort(np.stack([a[keep], c[keep]], axis=1))
    assert np.array_equal(P.lex_sort(rows_of(out)), want)  # packed in any order


@pytest.mark.parametrize("arity", [1, 2, 3, 4])
@pytest.mark.parametrize("n", [0, 1, 4095, 4096 * 3 + 100])
@pytest.mark.parametrize("dist", ["small", "wide", "max"])
def test_sort_unique(torch_cuda, arity, n, dist):
    from paper_2501_13051_gb300 import cdl
    rng = np.random.default_rng(arity * 1000 + n)
    if dist == "small":
        rows = rng.integers(0, 7, size=(n, arity))
    elif dist == "wide":
        rows = rng.integers(0, 1 << 32, size=(n, arity), dtype=np.uint64) & 0xFFFFFFF0
    else:
        rows = rng.integers(MAXV - 3, MAXV + 1, size=(n, arity), dtype=np.uint64)
    rows = rows.astype(np.uint32)
    out = cdl.sort_unique([dev(torch_cuda, rows[:, k]) for k in range(arity)])
    want = P.unique_sorted(P.lex_sort(rows)) if n else np.zeros((0, arity), np.uint32)
    assert np.array_equal(rows_of(out), want)


@pytest.mark.parametrize("arity", [1, 2, 3])
@pytest.mark.parametrize("nf,nu", [(0, 0), (0, 5000), (5000, 0), (20000, 7000), (7000, 20000), (1, 1)])
def test_diff_merge(torch_cuda, arity, nf, nu):
    from paper_2501_13051_gb300 import cdl
    rng = np.random.default_rng(nf * 7 + nu + arity)
    hi = 40 if arity > 1 else 30000
    full = P.unique_sorted(P.lex_sort(rng.integers(0, hi, size=(nf, arity)).astype(np.uint32))) \
        if nf else np.zeros((0, arity), np.uint32)
    fresh = P.lex_sort(rng.integers(0, hi, size=(nu, arity)).astype(np.uint32)) \
        if nu else np.zeros((0, arity), np.uint32)
    d, m = cdl.diff_merge([dev(torch_cuda, full[:, k]) for k in range(arity)],
                          [dev(torch_cuda, fresh[:, k]) for k in range(arity)])
    wd = P.difference(fresh, full)
    assert np.array_equal(rows_of(d), wd)
    assert np.array_equal(rows_of(m), P.merge(full, wd))
