"""GPU parity of BP32 (Sec. 6.2, the paper's scalar binary packing of
32-integer blocks, four per metablock): decoding, the index walk and the
GPU encoder, through the SIMD-BP128 calls with layout ICX_FMT_BP32, bit for
bit against the oracle on the same seeded inputs."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1209_2137_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1209_2137_gb300 as icx  # noqa: E402

BP32 = icx.FMT_BP32
# lengths across block (32), metablock (128), unit (2048) and tile edges,
# several tiles, ragged tails
LENGTHS = [1, 31, 32, 127, 128, 129, 2047, 2048, 2049, 2175, 4095, 16384 * 8 + 5, 16384 * 9 + 2048 * 3 + 130]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.cpu().numpy().view(np.uint32)


CASES = {
    "sorted": W.uniform_sorted(16384 * 9 + 2048 * 3 + 130, 29, 51),
    "widths": W.random_small(16384 * 9 + 2048 * 3 + 130, 52),
}


@pytest.mark.parametrize("delta", [icx.DELTA_NONE, icx.DELTA_1, icx.DELTA_4])
@pytest.mark.parametrize("case", sorted(CASES))
def test_bp32_decode_matches_oracle(delta, case):
    for n in LENGTHS:
        x = CASES[case][:n]
        enc = oracle.bp32_encode(x, delta)
        idx = oracle.bp32_index(enc, n)
        ws = icx.Workspace(n)
        # the stream in a buffer cut to its exact length: nothing past it is read
        y = icx.bp128_decode(dev(enc), n, delta, BP32, index=dev(idx), workspace=ws)
        assert ws.status() == icx.OK, (case, delta, n)
        assert np.array_equal(host(y), oracle.bp32_decode(enc, n, delta)), (case, delta, n)


def test_bp32_index_walk_and_single_unit_without_index():
    for n in LENGTHS:
        x = CASES["sorted"][:n]
        enc = oracle.bp32_encode(x, icx.DELTA_1)
        gi = icx.bp128_index(dev(enc), n, BP32)
        assert np.array_equal(gi.cpu().numpy().view(np.uint64), oracle.bp32_index(enc, n)), n
        if n < 17 * 128:
            y = icx.bp128_decode(dev(enc), n, icx.DELTA_1, BP32)
            assert np.array_equal(host(y), x), n


@pytest.mark.parametrize("delta", [icx.DELTA_NONE, icx.DELTA_1, icx.DELTA_4])
def test_bp32_gpu_encoder_writes_the_oracle_bytes(delta):
    for case, xs in CASES.items():
        for n in LENGTHS:
            x = xs[:n]
            e = icx.bp128_encode(dev(x), delta, BP32)
            assert np.array_equal(e.data.cpu().numpy(), oracle.bp32_encode(x, delta)), (case, delta, n)
            assert np.array_equal(e.index.cpu().numpy().view(np.uint64), oracle.bp32_index(oracle.bp32_encode(x, delta), n))


def test_bp32_corrupt_width_reports_error():
    x = CASES["sorted"][: 2048 * 3 + 77]
    enc = oracle.bp32_encode(x, icx.DELTA_1)
    idx = oracle.bp32_index(enc, x.size)
    bad = enc.copy()
    bad[int(idx[1]) + 2] = 40  # a width byte of the second unit
    ws = icx.Workspace(x.size)
    icx.bp128_decode(dev(bad), x.size, icx.DELTA_1, BP32, index=dev(idx), workspace=ws)
    assert ws.status() == icx.ECORRUPT
    y = icx.bp128_decode(dev(enc), x.size, icx.DELTA_1, BP32, index=dev(idx), workspace=ws)
    assert ws.status() == icx.OK and np.array_equal(host(y), x)


def test_bp32_full_size_uniform():
    # 2^26 sorted integers in [0, 2^29), stride 1: the GPU encoder writes the
    # oracle's bytes and index, and the decode gives the input back
    x = W.workload_uniform_long()
    d = dev(x)
    e = icx.bp128_encode(d, icx.DELTA_1, BP32)
    ref = oracle.bp32_encode(x, icx.DELTA_1)
    assert np.array_equal(e.data.cpu().numpy(), ref)
    assert np.array_equal(e.index.cpu().numpy().view(np.uint64), oracle.bp32_index(ref, x.size))
    y = icx.bp128_decode(e.data, x.size, icx.DELTA_1, BP32, index=e.index)
    assert torch.equal(y, d)
