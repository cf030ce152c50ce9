"""GPU parity of SimplePFOR (Sec. 5: the scalar FastPFOR page whose
exception high parts form one Simple-8b stream per page, Table 2): page
walk, decoding and the GPU encoder through the SIMD-FastPFOR calls with
layout ICX_FMT_SIMPLE8B, bit for bit against the oracle on the same seeded
inputs."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1209_2137_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1209_2137_gb300 as icx  # noqa: E402

S8 = icx.FMT_SIMPLE8B
PAGE = 65536
LENGTHS = [1, 127, 128, 129, 2048, 2049, PAGE - 1, PAGE, PAGE + 1, 2 * PAGE + 16384 * 3 + 77]
CASES = {
    "exceptions": W.exception_heavy(2 * PAGE + 16384 * 3 + 77, 91),
    "sorted": W.uniform_sorted(2 * PAGE + 16384 * 3 + 77, 29, 92),
    "widths": W.random_small(2 * PAGE + 16384 * 3 + 77, 93),
}


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("delta", [icx.DELTA_NONE, icx.DELTA_1, icx.DELTA_4])
@pytest.mark.parametrize("case", sorted(CASES))
def test_simplepfor_decode_matches_oracle(case, delta):
    for n in LENGTHS:
        x = CASES[case][:n]
        enc = oracle.simplepfor_encode(x, delta)
        idx = oracle.simplepfor_index(enc, n)
        ws = icx.Workspace(n)
        y = icx.fastpfor_decode(dev(enc), n, delta, index=dev(idx), workspace=ws, fmt=S8)
        assert ws.status() == icx.OK, (case, delta, n)
        want = oracle.simplepfor_decode(enc, n, delta)
        got = host(y)
        assert np.array_equal(got, want), (case, delta, n, int(np.argmax(got != want)))


def test_simplepfor_every_selector_and_long_streams():
    # pages whose high parts take every Simple-8b selector: runs of zeros
    # (b = 0 blocks with maxbits above 0 give high parts of 1), small and
    # 30-bit high parts, and pages with one exception per position
    rng = np.random.default_rng(5)
    for bits in (1, 2, 3, 5, 8, 12, 20, 30, 31):
        x = np.zeros(128 * 40, np.uint32)
        sel = rng.random(x.size) < 0.3
        x[sel] = (rng.integers(0, 1 << bits, int(sel.sum())) | 1).astype(np.uint32)
        enc = oracle.simplepfor_encode(x, 0)
        y = icx.fastpfor_decode(dev(enc), x.size, 0, fmt=S8)
        assert np.array_equal(host(y), x), bits
    x = np.full(128 * 600, 0xFFFFFFFF, np.uint32)
    x[::2] = 0  # b = 0: every other value an exception of 32 bits (one per word)
    enc = oracle.simplepfor_encode(x, 0)  # two pages: the index is needed
    idx = dev(oracle.simplepfor_index(enc, x.size))
    assert np.array_equal(host(icx.fastpfor_decode(dev(enc), x.size, 0, index=idx, fmt=S8)), x)


def test_simplepfor_index_walk_and_gpu_encoder():
    for case, xs in CASES.items():
        for n in LENGTHS:
            x = xs[:n]
            for delta in (icx.DELTA_NONE, icx.DELTA_1, icx.DELTA_4):
                ref = oracle.simplepfor_encode(x, delta)
                e = icx.fastpfor_encode(dev(x), delta, fmt=S8)
                assert np.array_equal(e.data.cpu().numpy(), ref), (case, delta, n)
                want_idx = oracle.simplepfor_index(ref, n)
                assert np.array_equal(e.index.cpu().numpy().view(np.uint64), want_idx), (case, delta, n)
                gi = icx.fastpfor_index(dev(ref), n, fmt=S8)
                assert np.array_equal(gi.cpu().numpy().view(np.uint64), want_idx), (case, delta, n)


def test_simplepfor_corrupt_stream_reports_error():
    x = CASES["exceptions"][: PAGE + 2048]
    enc = oracle.simplepfor_encode(x, 0)
    idx = oracle.simplepfor_index(enc, x.size)
    ws = icx.Workspace(x.size)
    bad = enc.copy()
    bad[0:4] = 0xFF  # the first page's byte-array offset far past the page
    icx.fastpfor_decode(dev(bad), x.size, 0, index=dev(idx), workspace=ws, fmt=S8)
    assert ws.status() == icx.ECORRUPT
    # N one too large: the words no longer hold the page's high parts
    len_at = 4 * int(enc[0:4].view(np.uint32)[0])
    L = int(enc[len_at:len_at + 4].view(np.uint32)[0])
    q = len_at + 4 + (L + 3) // 4 * 4
    bad = enc.copy()
    bad[q:q + 4] = (np.array([int(enc[q:q + 4].view(np.uint32)[0]) + 1], np.uint32)).view(np.uint8)
    icx.fastpfor_decode(dev(bad), x.size, 0, index=dev(idx), workspace=ws, fmt=S8)
    assert ws.status() == icx.ECORRUPT
    y = icx.fastpfor_decode(dev(enc), x.size, 0, index=dev(idx), workspace=ws, fmt=S8)
    assert ws.status() == icx.OK and np.array_equal(host(y), x)


def test_simplepfor_full_size_uniform():
    x = W.workload_uniform_long()
    d = dev(x)
    e = icx.fastpfor_encode(d, icx.DELTA_1, fmt=S8)
    ref = oracle.simplepfor_encode(x, icx.DELTA_1)
    assert np.array_equal(e.data.cpu().numpy(), ref)
    y = icx.fastpfor_decode(e.data, x.size, icx.DELTA_1, index=e.index, fmt=S8)
    assert torch.equal(y, d)
