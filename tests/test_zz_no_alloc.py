"""The allocation-free scan (cdl_exclusive_scan_noalloc) through the C ABI,
against the oracle's exclusive scan and the workspace scan
(cdl_exclusive_scan).

cdl_exclusive_scan_noalloc serves callers that cannot allocate device
memory and so cannot hand the library a workspace; it keeps its scratch in a
fixed array inside the library.  Its offsets and total must equal the
oracle's, bit for bit (integer results), on calls in a row: the second call
scans fewer tiles than the first through the multi-tile passes, so the
array still holds the first call's tile sums past the second call's last
tile; the third is a single-tile scan.  This file is collected last so that
a run stopping at the first failure has run every other test."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

MAX_N = 65536 * 2048


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a GPU"
    from paper_2501_13051_gb300 import build as B
    B.build()
    from paper_2501_13051_gb300 import cdl
    return torch, cdl


def noalloc_scan(torch, cdl, counts):
    n = counts.numel()
    out = torch.empty(max(1, n), dtype=torch.int64, device="cuda")
    total = ctypes.c_uint64(12345)
    st = cdl.lib().cdl_exclusive_scan_noalloc(counts.data_ptr(), n, out.data_ptr(),
                                             ctypes.byref(total),
                                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, cdl.STATUS.get(st, st)
    return out[:n], int(total.value)


def test_noalloc_scan_matches_oracle_in_a_row(env):
    torch, cdl = env
    from oracle import primitives as P
    rng = np.random.default_rng(7)
    # 1st call: 301 tiles with a ragged tail and sums past 2^32;
    # 2nd call: 41 tiles (above the single-block cutoff of 65,536 counts), run
    #           while the array still holds the 1st call's 301 tile sums;
    # 3rd call: one block, which reads no tile sums at all.
    for n in (2048 * 300 + 77, 2048 * 40 + 5, 2048 * 3 + 5):
        c = rng.integers(0, 1 << 20, size=n).astype(np.uint32)
        c[n // 3] = 0xFFFFFFFF
        counts = torch.from_numpy(c.view(np.int32)).cuda()
        want_off, want_total = P.exclusive_scan(c)
        got_off, got_total = noalloc_scan(torch, cdl, counts)
        assert got_total == want_total
        assert np.array_equal(got_off.cpu().numpy().view(np.uint64), want_off)
        # and the workspace scan gives the same offsets
        ws_off, ws_total = cdl.exclusive_scan(counts)
        assert ws_total == want_total and torch.equal(got_off, ws_off)


def test_noalloc_scan_edges(env):
    torch, cdl = env
    off, total = noalloc_scan(torch, cdl, torch.zeros(1, dtype=torch.int32, device="cuda")[:0])
    assert total == 0 and off.numel() == 0
    one = torch.tensor([9], dtype=torch.int32, device="cuda")
    off, total = noalloc_scan(torch, cdl, one)
    assert total == 9 and off.tolist() == [0]
    # past the fixed scratch: refused before anything runs
    big = ctypes.c_uint64()
    st = cdl.lib().cdl_exclusive_scan_noalloc(one.data_ptr(), MAX_N + 1, one.data_ptr(),
                                             ctypes.byref(big), None)
    assert cdl.STATUS[st] == "CDL_E_CAPACITY"
