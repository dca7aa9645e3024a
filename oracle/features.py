"""Float64 statement of the join-size estimator's 16 input features.

TEST INFRASTRUCTURE ONLY (imported by tests).  Shares no code with the GPU
library.  The paper has no learned part; the features follow the reading of
"delta/full sizes, sampled distinct counts and 32-bucket key histograms"
this library takes (all sizes enter as log2(1 + x)):

  sample     -- a deterministic stride sample of at most 2048 keys per side:
                sample s of a side with n keys is key floor(s * n / m),
                m = min(n, 2048);
  key hash   -- h(k0, k1) = fmix32(k0 XOR fmix32(k1 + 0x9e3779b9)), with
                k1 = 0 for one-column keys and fmix32 the 32-bit finaliser of
                MurmurHash3 (Appleby, public domain); the value 0xFFFFFFFF
                is taken as 0xFFFFFFFE;
  bucket     -- the top 5 bits of the key hash (32 buckets);
  distinct   -- distinct key hashes among a side's sample.

   0  log2(1 + probe rows)          1  log2(1 + build rows)
   2  log2(1 + |full| of the probe relation)
   3  log2(1 + distinct sampled probe hashes)
   4  log2(1 + distinct sampled build hashes)
   5  log2(1 + build rows / max(1, distinct build keys))
   6  log2(1 + E), E = sum_b (hP[b] n_p / m_p) (hB[b] n_b / m_b)
                      / max(1, dB[b] u_b / d_b):
      hP, hB the sampled bucket counts, dB[b] the distinct sampled build
      hashes in bucket b, u_b the build side's distinct keys, d_b the
      distinct sampled build hashes (the scale is 0 when d_b = 0)
   7, 8   largest bucket share of the probe / build sample
   9, 10  entropy (bits) of the probe / build bucket shares
   11     cosine of the two share vectors (0 when either is empty)
   12     the semi-naive round
   13     log2(1 + exact output of the same rule step in the previous round)
   14     log2(1 + the head relation's previous delta)
   15     1 when the step filters (inequalities or equalities), else 0
Entries 2, 5 (its u_b), 12-15 come from the host (``host``: probe_full,
build_distinct, round, prev_output, prev_delta, filtered).
"""
from __future__ import annotations

import math

import numpy as np

SAMPLE = 2048
BUCKETS = 32


def fmix32(k):
    """MurmurHash3's 32-bit finaliser on uint32 numpy values."""
    k = np.asarray(k, dtype=np.uint64) & 0xFFFFFFFF
    k ^= k >> 16
    k = (k * 0x85EBCA6B) & 0xFFFFFFFF
    k ^= k >> 13
    k = (k * 0xC2B2AE35) & 0xFFFFFFFF
    k ^= k >> 16
    return k


def key_hash(k0, k1=None):
    k0 = np.asarray(k0, dtype=np.uint64)
    k1 = np.zeros_like(k0) if k1 is None else np.asarray(k1, dtype=np.uint64)
    h = fmix32(k0 ^ fmix32((k1 + 0x9E3779B9) & 0xFFFFFFFF))
    return np.where(h == 0xFFFFFFFF, 0xFFFFFFFE, h).astype(np.uint64)


def stride_sample(n: int) -> np.ndarray:
    m = min(n, SAMPLE)
    return (np.arange(m, dtype=np.uint64) * np.uint64(n)) // np.uint64(max(m, 1))


def side_stats(k0, k1=None):
    """(sample size, bucket counts, distinct hashes, distinct hashes per bucket)."""
    n = len(k0)
    idx = stride_sample(n)
    h = key_hash(np.asarray(k0)[idx], None if k1 is None else np.asarray(k1)[idx])
    b = (h >> 27).astype(np.int64)
    counts = np.bincount(b, minlength=BUCKETS).astype(np.float64)
    uh = np.unique(h)
    dist_b = np.bincount((uh >> 27).astype(np.int64), minlength=BUCKETS).astype(np.float64)
    return len(idx), counts, len(uh), dist_b


def join_features(probe_k0, build_k0, host, probe_k1=None, build_k1=None) -> np.ndarray:
    """The 16 features of one join, in float64."""
    probe_full, build_distinct, rnd, prev_out, prev_delta, filtered = [float(x) for x in host]
    n_p, n_b = len(probe_k0), len(build_k0)
    m_p, hP, d_p, _ = side_stats(probe_k0, probe_k1)
    m_b, hB, d_b, dB = side_stats(build_k0, build_k1)
    f_p = n_p / m_p if m_p else 0.0
    f_b = n_b / m_b if m_b else 0.0
    u_scale = build_distinct / d_b if d_b else 0.0
    est = float(np.sum((hP * f_p) * (hB * f_b) / np.maximum(1.0, dB * u_scale)))
    qP = hP / m_p if m_p else np.zeros(BUCKETS)
    qB = hB / m_b if m_b else np.zeros(BUCKETS)

    def entropy(q):
        q = q[q > 0]
        return float(-np.sum(q * np.log2(q)))

    nP, nB = float(np.dot(qP, qP)), float(np.dot(qB, qB))
    cos = float(np.dot(qP, qB)) / math.sqrt(nP * nB) if nP > 0 and nB > 0 else 0.0
    lg = lambda x: math.log2(1.0 + x)
    return np.array([lg(n_p), lg(n_b), lg(probe_full), lg(d_p), lg(d_b),
                     lg(n_b / max(1.0, build_distinct)), lg(est),
                     float(qP.max()) if m_p else 0.0, float(qB.max()) if m_b else 0.0,
                     entropy(qP), entropy(qB), cos, rnd, lg(prev_out), lg(prev_delta),
                     filtered], dtype=np.float64)
