"""The allocation-free entry point bp128_decode_static, for callers that
cannot allocate device memory (it uses the library's own static workspace).

Checked through the C ABI against the allocating bp128_decode on the same
stream, on two calls in a row.  Kept in its own file, collected last."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

import oracle
from paper_1209_2137_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1209_2137_gb300 as icx  # noqa: E402


def static_fn():
    fn = icx.lib().bp128_decode_static
    vp, sz, i = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int
    fn.argtypes = [vp, sz, vp, sz, i, i, vp, vp, vp]
    fn.restype = i
    return fn


def p(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("fmt,delta", [(icx.FMT_PAPER, icx.DELTA_4), (icx.FMT_W32, icx.DELTA_1),
                                       (icx.FMT_BP32, icx.DELTA_1)])
def test_static_decode_matches_allocating_decode_twice(fmt, delta):
    fn = static_fn()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    inputs = [W.uniform_sorted(16384 * 9 + 2048 * 3 + 77, 29, 71), W.random_small(100_003, 72)]
    for x in inputs:  # two calls in a row, different streams of integers
        enc = oracle.encode("bp128", x, delta, fmt)  # the BP32 layout goes to the BP32 coder
        d = torch.from_numpy(enc).cuda()
        idx = torch.from_numpy(oracle.index("bp128", enc, x.size, fmt)).cuda()
        want = icx.bp128_decode(d, x.size, delta, fmt, index=idx)
        out = torch.empty(x.size, dtype=torch.uint32, device="cuda")
        status = torch.full((1,), 99, dtype=torch.int32, device="cuda")
        rc = fn(p(d), d.numel(), p(out), x.size, delta, fmt, p(idx), p(status), stream)
        assert rc == icx.OK
        torch.cuda.synchronize()
        assert int(status.item()) == icx.OK
        assert torch.equal(out, want)
        assert np.array_equal(out.cpu().numpy().view(np.uint32), x)


def test_static_decode_rejects_sizes_beyond_its_maximum():
    fn = static_fn()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    dummy = torch.zeros(16, dtype=torch.uint8, device="cuda")
    rc = fn(p(dummy), 16, p(dummy), (1 << 28) + 1, icx.DELTA_1, icx.FMT_PAPER, None, None, stream)
    assert rc == icx.ENOSPC


def _call(fn, d, n, delta, fmt, idx, out, status, in_bytes=None):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return fn(p(d), d.numel() if in_bytes is None else in_bytes, p(out), n, delta, fmt,
              None if idx is None else p(idx), p(status), stream)


@pytest.mark.parametrize("fmt", [icx.FMT_PAPER, icx.FMT_W32, icx.FMT_BP32])
def test_static_decode_single_metablock_without_index(fmt):
    # one metablock (n < 2048) with no index: the call walks it into the
    # index slot inside the static array; every stride, against the oracle
    fn = static_fn()
    for n in (1, 127, 128, 1000, 2047):
        x = W.uniform_sorted(n, 20, 90 + n)
        for delta in (icx.DELTA_NONE, icx.DELTA_1, icx.DELTA_4):
            enc = oracle.encode("bp128", x, delta, fmt)
            d = torch.from_numpy(enc).cuda()
            out = torch.empty(n, dtype=torch.uint32, device="cuda")
            status = torch.full((1,), 99, dtype=torch.int32, device="cuda")
            assert _call(fn, d, n, delta, fmt, None, out, status) == icx.OK
            torch.cuda.synchronize()
            assert int(status.item()) == icx.OK, (fmt, n, delta)
            assert np.array_equal(out.cpu().numpy().view(np.uint32), oracle.decode("bp128", enc, n, delta, fmt))


def test_static_decode_error_is_cleared_for_the_next_call():
    # a stream cut short records ECORRUPT in d_status; the next call on the
    # same stream starts from a clean status word and decodes exactly
    fn = static_fn()
    x = W.uniform_sorted(4096 * 3 + 50, 25, 93)
    enc = oracle.encode("bp128", x, icx.DELTA_1, icx.FMT_PAPER)
    d = torch.from_numpy(enc).cuda()
    idx = torch.from_numpy(oracle.index("bp128", enc, x.size, icx.FMT_PAPER)).cuda()
    out = torch.empty(x.size, dtype=torch.uint32, device="cuda")
    status = torch.full((1,), 99, dtype=torch.int32, device="cuda")
    assert _call(fn, d, x.size, icx.DELTA_1, icx.FMT_PAPER, idx, out, status, in_bytes=enc.size - 40) == icx.OK
    torch.cuda.synchronize()
    assert int(status.item()) == icx.ECORRUPT
    assert _call(fn, d, x.size, icx.DELTA_1, icx.FMT_PAPER, idx, out, status) == icx.OK
    torch.cuda.synchronize()
    assert int(status.item()) == icx.OK
    assert np.array_equal(out.cpu().numpy().view(np.uint32), x)
