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
