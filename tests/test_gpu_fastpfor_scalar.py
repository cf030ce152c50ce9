"""GPU parity of the scalar FastPFOR (Sec. 5, the non-vectorised variant:
one-lane packing of a block's low parts and of each exception array, padded
to 32 values): page walk, decoding and the GPU encoder through the
SIMD-FastPFOR calls with layout ICX_FMT_SCALAR, bit for bit against the
oracle on the same seeded inputs."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1209_2137_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1209_2137_gb300 as icx  # noqa: E402

SC = icx.FMT_SCALAR
PAGE = 65536
LENGTHS = [1, 127, 128, 129, 2048, 2049, PAGE - 1, PAGE, PAGE + 1, 2 * PAGE + 16384 * 3 + 77]
CASES = {
    "exceptions": W.exception_heavy(2 * PAGE + 16384 * 3 + 77, 71),
    "sorted": W.uniform_sorted(2 * PAGE + 16384 * 3 + 77, 29, 72),
    "widths": W.random_small(2 * PAGE + 16384 * 3 + 77, 73),
}


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("delta", [icx.DELTA_NONE, icx.DELTA_1, icx.DELTA_4])
@pytest.mark.parametrize("case", sorted(CASES))
def test_scalar_decode_matches_oracle(case, delta):
    for n in LENGTHS:
        x = CASES[case][:n]
        enc = oracle.fastpfor_encode(x, delta, oracle.SCALAR)
        idx = oracle.fastpfor_index(enc, n, oracle.SCALAR)
        ws = icx.Workspace(n)
        y = icx.fastpfor_decode(dev(enc), n, delta, index=dev(idx), workspace=ws, fmt=SC)
        assert ws.status() == icx.OK, (case, delta, n)
        want = oracle.fastpfor_decode(enc, n, delta, oracle.SCALAR)
        got = host(y)
        assert np.array_equal(got, want), (case, delta, n, int(np.argmax(got != want)))


def test_scalar_every_exception_width():
    # b = 0 blocks whose few values have bit length d: exceptions of width d
    # in every array, counts across the 32-value padding unit
    for d in range(1, 33):
        x = np.zeros(128 * 8, np.uint32)
        for e in range(70):
            x[128 * (e % 8) + 3 * (e // 8) + 1] = np.uint32((1 << (d - 1)) | (e & ((1 << (d - 1)) - 1)))
        enc = oracle.fastpfor_encode(x, 0, oracle.SCALAR)
        y = icx.fastpfor_decode(dev(enc), x.size, 0, fmt=SC)
        assert np.array_equal(host(y), x), d


def test_scalar_index_walk_and_gpu_encoder():
    for case, xs in CASES.items():
        for n in LENGTHS:
            x = xs[:n]
            for delta in (icx.DELTA_NONE, icx.DELTA_1, icx.DELTA_4):
                ref = oracle.fastpfor_encode(x, delta, oracle.SCALAR)
                e = icx.fastpfor_encode(dev(x), delta, fmt=SC)
                assert np.array_equal(e.data.cpu().numpy(), ref), (case, delta, n)
                want_idx = oracle.fastpfor_index(ref, n, oracle.SCALAR)
                assert np.array_equal(e.index.cpu().numpy().view(np.uint64), want_idx), (case, delta, n)
                gi = icx.fastpfor_index(dev(ref), n, fmt=SC)
                assert np.array_equal(gi.cpu().numpy().view(np.uint64), want_idx), (case, delta, n)


def test_scalar_corrupt_stream_reports_error():
    x = CASES["exceptions"][: PAGE + 2048]
    enc = oracle.fastpfor_encode(x, 0, oracle.SCALAR)
    idx = oracle.fastpfor_index(enc, x.size, oracle.SCALAR)
    bad = enc.copy()
    bad[0:4] = 0xFF  # the first page's byte-array offset far past the page
    ws = icx.Workspace(x.size)
    icx.fastpfor_decode(dev(bad), x.size, 0, index=dev(idx), workspace=ws, fmt=SC)
    assert ws.status() == icx.ECORRUPT
    y = icx.fastpfor_decode(dev(enc), x.size, 0, index=dev(idx), workspace=ws, fmt=SC)
    assert ws.status() == icx.OK and np.array_equal(host(y), x)


def test_scalar_full_size_uniform():
    # 2^26 sorted integers in [0, 2^29), stride 1: GPU bytes = oracle bytes,
    # and the decode returns the input
    x = W.workload_uniform_long()
    d = dev(x)
    e = icx.fastpfor_encode(d, icx.DELTA_1, fmt=SC)
    ref = oracle.fastpfor_encode(x, icx.DELTA_1, oracle.SCALAR)
    assert np.array_equal(e.data.cpu().numpy(), ref)
    y = icx.fastpfor_decode(e.data, x.size, icx.DELTA_1, index=e.index, fmt=SC)
    assert torch.equal(y, d)
