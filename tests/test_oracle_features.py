"""Pins of the float64 feature statement (oracle.features), CPU only: the
published MurmurHash3 test vectors for the hash, and joins whose features
have closed forms (one repeated key, identical unique key sets, empty
sides), plus library cross-checks of entropy and cosine."""
import math

import numpy as np
import pytest

from oracle import features as F


def test_fmix32_published_vectors():
    # MurmurHash3_x86_32 of the empty key is fmix32(seed); SMHasher's
    # published values for seeds 1 and 0xFFFFFFFF
    assert int(F.fmix32(1)) == 0x514E28B7
    assert int(F.fmix32(0xFFFFFFFF)) == 0x81F16F39
    assert int(F.fmix32(0)) == 0


def test_fmix32_is_a_bijection_on_a_block():
    k = np.arange(1 << 16, dtype=np.uint64) * 65537
    assert len(np.unique(F.fmix32(k))) == len(k)


def test_stride_sample_definition():
    for n in (0, 1, 7, 2048, 2049, 5000, 10 ** 7):
        got = F.stride_sample(n)
        m = min(n, 2048)
        assert [int(x) for x in got] == [s * n // m for s in range(m)]


def test_one_repeated_key_gives_the_exact_join_size():
    probe, build = np.full(100, 5, np.uint32), np.full(40, 5, np.uint32)
    f = F.join_features(probe, build, (1000, 1, 3, 77, 9, 1))
    assert f[6] == pytest.approx(math.log2(1 + 100 * 40))  # E = 4000 = |join|
    assert f[3] == f[4] == pytest.approx(1.0)             # one distinct hash each
    assert f[5] == pytest.approx(math.log2(41))
    assert f[7] == f[8] == 1.0 and f[9] == f[10] == 0.0 and f[11] == pytest.approx(1.0)
    assert list(f[[0, 1, 2, 12, 13, 14, 15]]) == pytest.approx(
        [math.log2(101), math.log2(41), math.log2(1001), 3, math.log2(78), math.log2(10), 1])


def test_identical_unique_keys_estimate_the_join_exactly():
    rng = np.random.default_rng(1)
    keys = rng.choice(1 << 30, size=1500, replace=False).astype(np.uint32)
    f = F.join_features(keys, np.sort(keys), (1500, 1500, 1, 0, 0, 0))
    assert f[6] == pytest.approx(math.log2(1 + 1500))      # sum_b c_b^2 / c_b
    assert f[3] == f[4] == pytest.approx(math.log2(1501))
    assert f[11] == pytest.approx(1.0)
    from scipy.stats import entropy
    b = (F.key_hash(keys) >> 27).astype(np.int64)
    counts = np.bincount(b, minlength=32)
    assert f[9] == pytest.approx(entropy(counts, base=2)) and f[10] == pytest.approx(f[9])
    assert f[7] == pytest.approx(counts.max() / 1500)


def test_cosine_and_two_column_keys():
    rng = np.random.default_rng(2)
    p0, p1 = rng.integers(0, 50, 3000).astype(np.uint32), rng.integers(0, 9, 3000).astype(np.uint32)
    b0, b1 = rng.integers(0, 80, 999).astype(np.uint32), rng.integers(0, 9, 999).astype(np.uint32)
    f = F.join_features(p0, b0, (3000, 400, 2, 10, 10, 0), probe_k1=p1, build_k1=b1)
    ip = F.stride_sample(3000)
    hp = F.key_hash(p0[ip], p1[ip])
    hb = F.key_hash(b0, b1)
    cp = np.bincount((hp >> 27).astype(np.int64), minlength=32) / len(ip)
    cb = np.bincount((hb >> 27).astype(np.int64), minlength=32) / 999
    from scipy.spatial.distance import cosine
    assert f[11] == pytest.approx(1.0 - cosine(cp, cb))
    assert f[3] == pytest.approx(math.log2(1 + len(set(zip(p0[ip].tolist(), p1[ip].tolist())))))
    assert f[4] == pytest.approx(math.log2(1 + len(set(zip(b0.tolist(), b1.tolist())))))


def test_empty_probe_side():
    f = F.join_features(np.zeros(0, np.uint32), np.arange(10, dtype=np.uint32), (0, 10, 1, 0, 0, 0))
    assert f[0] == 0 and f[3] == 0 and f[6] == 0 and f[7] == 0 and f[9] == 0 and f[11] == 0
    assert f[4] == pytest.approx(math.log2(11))
