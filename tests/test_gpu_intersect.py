"""GPU parity of decoding fused into a consumer (Sec. 7): membership of a
sorted query list in a compressed sorted list (bp128_intersect), and the
same consumer over a decoded list (sorted_intersect), both compared bit for
bit, and by count, with the oracle's merge of the two sorted lists."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1209_2137_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1209_2137_gb300 as icx  # noqa: E402

DELTAS = [icx.DELTA_NONE, icx.DELTA_1, icx.DELTA_4]
FMTS = [icx.FMT_PAPER, icx.FMT_W32]
# lengths across block, metablock and tile edges, several tiles, ragged tails
LENGTHS = [1, 5, 127, 128, 129, 2047, 2048, 2049, 4095, 16384 * 8 + 5, 16384 * 9 + 2048 * 3 + 130]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def want(a, b):
    bits, cnt = oracle.member_bits(a, b)
    return bits, cnt


def fused(x, b, delta, fmt, with_index=True):
    enc = oracle.bp128_encode(x, delta, fmt)
    a = oracle.bp128_decode(enc, x.size, delta, fmt)  # the list the stream decodes to
    idx = dev(oracle.bp128_index(enc, x.size, fmt)) if with_index else None
    ws = icx.Workspace(max(1, x.size))
    bits, cnt = icx.bp128_intersect(dev(enc), x.size, dev(b), delta, fmt, index=idx, workspace=ws)
    assert ws.status() == icx.OK
    return a, bits.cpu().numpy().view(np.uint32), int(cnt.cpu().view(torch.int64)[0])


def unfused(a, b):
    bits, cnt = icx.sorted_intersect(dev(a), dev(b))
    return bits.cpu().numpy().view(np.uint32), int(cnt.cpu().view(torch.int64)[0])


@pytest.mark.parametrize("delta", DELTAS)
@pytest.mark.parametrize("fmt", FMTS)
def test_fused_matches_oracle(delta, fmt):
    for i, n in enumerate(LENGTHS):
        x = W.uniform_sorted(n, 24, 700 + i)
        for hit in (0.0, 0.5, 1.0):
            b = W.query_list(x, max(1, n // 3), 24, 900 + i, hit_frac=hit)
            a, bits, cnt = fused(x, b, delta, fmt, with_index=n >= 17 * 128 or i % 2 == 0)
            wb, wc = want(a, b)
            assert cnt == wc, (n, hit)
            assert np.array_equal(bits, wb), (n, hit)


def test_unfused_matches_oracle():
    for i, n in enumerate(LENGTHS):
        x = W.uniform_sorted(n, 24, 710 + i)
        for hit in (0.0, 0.5, 1.0):
            b = W.query_list(x, max(1, 2 * n), 24, 910 + i, hit_frac=hit)
            bits, cnt = unfused(x, b)
            wb, wc = want(x, b)
            assert cnt == wc and np.array_equal(bits, wb), (n, hit)


def test_duplicates_and_extremes():
    # repeats in both lists (equal values across metablock boundaries count
    # once), the query list longer than the list, values at 0 and 2^32 - 1
    rng = np.random.default_rng(3)
    x = np.sort(rng.integers(0, 3000, 2048 * 5 + 77)).astype(np.uint32)
    x[-40:] = 0xFFFFFFFF
    x[:40] = 0
    b = np.sort(np.concatenate([rng.integers(0, 3100, 20000).astype(np.uint32),
                                np.array([0, 0, 0xFFFFFFFF, 0xFFFFFFFE], np.uint32)]))
    for delta in (icx.DELTA_NONE, icx.DELTA_1, icx.DELTA_4):
        for fmt in FMTS:
            a, bits, cnt = fused(x, b, delta, fmt)
            wb, wc = want(a, b)
            assert cnt == wc and np.array_equal(bits, wb), (delta, fmt)
    bits, cnt = unfused(x, b)
    wb, wc = want(x, b)
    assert cnt == wc and np.array_equal(bits, wb)


def test_degenerate_inputs():
    x = W.uniform_sorted(5000, 20, 5)
    enc = dev(oracle.bp128_encode(x, icx.DELTA_1, icx.FMT_PAPER))
    idx = dev(oracle.bp128_index(oracle.bp128_encode(x, icx.DELTA_1, icx.FMT_PAPER), x.size, icx.FMT_PAPER))
    # empty query list: count 0, nothing written
    bits, cnt = icx.bp128_intersect(enc, x.size, dev(np.zeros(0, np.uint32)), icx.DELTA_1, index=idx)
    assert bits.numel() == 0 and int(cnt.cpu().view(torch.int64)[0]) == 0
    # empty list: every bit cleared, even in a reused bitmap
    b = dev(np.arange(0, 1000, 7, dtype=np.uint32))
    stale = torch.full(((b.numel() + 31) // 32,), -1, dtype=torch.int32, device="cuda").view(torch.uint32)
    bits, cnt = icx.bp128_intersect(enc[:0], 0, b, icx.DELTA_1, bits=stale)
    assert int(cnt.cpu().view(torch.int64)[0]) == 0 and not bits.cpu().numpy().any()
    # queries all below / all above the list
    for q in (np.arange(10, dtype=np.uint32) + 0, np.arange(10, dtype=np.uint32) + (1 << 21)):
        if q[0] == 0:
            q = q[~np.isin(q, x)]
        bits, cnt = icx.bp128_intersect(enc, x.size, dev(q), icx.DELTA_1, index=idx)
        wb, wc = want(x, q)
        assert int(cnt.cpu().view(torch.int64)[0]) == wc
        assert np.array_equal(bits.cpu().numpy().view(np.uint32), wb)
    # the query list equal to the list: every bit set
    bits, cnt = icx.bp128_intersect(enc, x.size, dev(x), icx.DELTA_1, index=idx)
    assert int(cnt.cpu().view(torch.int64)[0]) == x.size


def test_full_size_uniform_against_oracle():
    # the benchmark's workload: 2^26 sorted integers in [0, 2^29) and a
    # query list of ~2^22, stride 4 and stride 1, paper layout
    x, b = W.workload_intersect()
    for delta in (icx.DELTA_4, icx.DELTA_1):
        e = icx.bp128_encode(dev(x), delta, icx.FMT_PAPER)
        bits, cnt = icx.bp128_intersect(e.data, x.size, dev(b), delta, icx.FMT_PAPER, index=e.index)
        wb, wc = want(x, b)
        assert int(cnt.cpu().view(torch.int64)[0]) == wc
        assert np.array_equal(bits.cpu().numpy().view(np.uint32), wb)
        out = icx.bp128_decode(e.data, x.size, delta, icx.FMT_PAPER, index=e.index)
        bits2, cnt2 = icx.sorted_intersect(out, dev(b))
        assert int(cnt2.cpu().view(torch.int64)[0]) == wc
        assert np.array_equal(bits2.cpu().numpy().view(np.uint32), wb)
