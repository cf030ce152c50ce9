"""GPU parity: SIMD-BP128 / W32 decoding, index walk, GPU encoders and the
standalone differential decoder, all through the C ABI, compared bit for bit
with the CPU oracle on the same seeded inputs."""
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
# lengths spanning empty, single partial blocks, metablock edges, several CTA
# tiles (8 metablocks each) and ragged tails
LENGTHS = [1, 3, 127, 128, 129, 2047, 2048, 2049, 2175, 2176, 4095, 16384 * 8 + 5,
           16384 * 9 + 2048 * 3 + 130]


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.cuda()


def host_u32(t):
    return t.cpu().numpy().view(np.uint32)


def cases():
    return {
        "widths": W.random_small(16384 * 9 + 2048 * 3 + 130, 31),
        "exceptions": W.exception_heavy(16384 * 9 + 2048 * 3 + 130, 32),
        "sorted": W.uniform_sorted(16384 * 9 + 2048 * 3 + 130, 29, 33),
    }


CASES = cases()


def gpu_decode(enc_bytes, n, delta, fmt, with_index=True, ws=None):
    d = dev(enc_bytes)
    idx = None
    if with_index:
        idx = dev(oracle.bp128_index(enc_bytes, n, fmt))
    ws = ws or icx.Workspace(n)
    out = icx.bp128_decode(d, n, delta, fmt, index=idx, workspace=ws)
    st = ws.status()
    return host_u32(out), st


def test_config1_sorted_65536_d1_paper():
    x = W.workload_sorted_small()
    enc = oracle.bp128_encode(x, icx.DELTA_1, icx.FMT_PAPER)
    y, st = gpu_decode(enc, x.size, icx.DELTA_1, icx.FMT_PAPER)
    assert st == icx.OK
    assert np.array_equal(y, oracle.bp128_decode(enc, x.size, 1, 0))
    assert np.array_equal(y, x)


@pytest.mark.parametrize("fmt", FMTS)
@pytest.mark.parametrize("delta", DELTAS)
@pytest.mark.parametrize("case", list(CASES))
def test_bp128_decode_matches_oracle(case, delta, fmt):
    x_all = CASES[case]
    for n in LENGTHS:
        x = x_all[:n]
        enc = oracle.bp128_encode(x, delta, fmt)
        y, st = gpu_decode(enc, n, delta, fmt)
        assert st == icx.OK, n
        want = oracle.bp128_decode(enc, n, delta, fmt)
        assert np.array_equal(y, want), (n, int(np.argmax(y != want)))


@pytest.mark.parametrize("fmt", FMTS)
def test_bp128_index_matches_oracle(fmt):
    for case in CASES.values():
        for n in [129, 2048, 16384 * 8 + 5, case.size]:
            enc = oracle.bp128_encode(case[:n], 1, fmt)
            ws = icx.Workspace(n)
            idx = icx.bp128_index(dev(enc), n, fmt, workspace=ws)
            assert ws.status() == icx.OK
            assert np.array_equal(idx.cpu().numpy().view(np.uint64), oracle.bp128_index(enc, n, fmt))


@pytest.mark.parametrize("fmt", FMTS)
def test_bp128_null_index_single_metablock(fmt):
    x = W.random_small(2175, 40)
    for n in [1, 100, 128, 2048, 2175]:
        enc = oracle.bp128_encode(x[:n], 4, fmt)
        y, st = gpu_decode(enc, n, 4, fmt, with_index=False)
        assert st == icx.OK
        assert np.array_equal(y, x[:n])


@pytest.mark.parametrize("fmt", FMTS)
@pytest.mark.parametrize("delta", DELTAS)
def test_gpu_encoder_bytes_match_oracle(delta, fmt):
    for case in CASES.values():
        for n in [0, 5, 128, 2049, 16384 * 8 + 5, case.size]:
            x = case[:n]
            enc = icx.bp128_encode(dev(x) if n else torch.empty(0, dtype=torch.uint32, device="cuda"), delta, fmt)
            want = oracle.bp128_encode(x, delta, fmt)
            got = enc.data.cpu().numpy()
            assert got.size == want.size, (n, got.size, want.size)
            assert np.array_equal(got, want), n
            assert np.array_equal(enc.index.cpu().numpy().view(np.uint64), oracle.bp128_index(want, n, fmt))


@pytest.mark.parametrize("delta", [icx.DELTA_NONE, icx.DELTA_1, icx.DELTA_4])
def test_delta_decode_matches_oracle(delta):
    d = W.uniform_u32(16384 * 11 + 37, 51, 32)
    for n in [1, 3, 4, 5, 2048, 16384 + 1, d.size]:
        ws = icx.Workspace(n)
        got = host_u32(icx.delta_decode(dev(d[:n]), delta, workspace=ws))
        assert ws.status() == icx.OK
        assert np.array_equal(got, oracle.delta_decode(d[:n], delta))
    # in place
    t = dev(d)
    icx.delta_decode(t, delta, out=t)
    assert np.array_equal(host_u32(t), oracle.delta_decode(d, delta))


@pytest.mark.parametrize("delta", [icx.DELTA_NONE, icx.DELTA_1, icx.DELTA_4])
def test_delta_encode_matches_oracle(delta):
    x = W.uniform_u32(100_003, 52, 32)
    got = host_u32(icx.delta_encode(dev(x), delta))
    assert np.array_equal(got, oracle.delta_encode(x, delta))


def test_workspace_reuse_many_launches():
    x = CASES["sorted"]
    enc = oracle.bp128_encode(x, 4, 0)
    d, idx = dev(enc), dev(oracle.bp128_index(enc, x.size, 0))
    ws = icx.Workspace(x.size)
    out = torch.empty(x.size, dtype=torch.uint32, device="cuda")
    for _ in range(40):
        out.zero_()
        icx.bp128_decode(d, x.size, 4, 0, index=idx, out=out, workspace=ws)
        assert np.array_equal(host_u32(out), x)
    assert ws.status() == icx.OK


def test_corrupt_streams_report_error_and_workspace_recovers():
    x = CASES["widths"][:16384 * 2 + 77]
    n = x.size
    good = oracle.bp128_encode(x, 1, 0)
    idx = oracle.bp128_index(good, n, 0)
    ws = icx.Workspace(n)
    # a width byte above 32 (keeps the metablock size consistent otherwise)
    bad = good.copy()
    bad[int(idx[3])] = 40
    icx.bp128_decode(dev(bad), n, 1, 0, index=dev(idx), workspace=ws)
    assert ws.status() == icx.ECORRUPT
    # an index entry past the end of the stream
    bidx = idx.copy()
    bidx[5] = good.size + 4096
    icx.bp128_decode(dev(good), n, 1, 0, index=dev(bidx), workspace=ws)
    assert ws.status() == icx.ECORRUPT
    # truncated Variable Byte tail
    icx.bp128_decode(dev(good[:-1]), n, 1, 0, index=dev(idx), workspace=ws)
    assert ws.status() == icx.ECORRUPT
    # the same workspace still decodes a good stream
    y = host_u32(icx.bp128_decode(dev(good), n, 1, 0, index=dev(idx), workspace=ws))
    assert ws.status() == icx.OK
    assert np.array_equal(y, x)


def test_argument_errors_are_synchronous():
    x = dev(W.random_small(4096, 3))
    ws = icx.Workspace(4096)
    data = torch.zeros(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(icx.IcxError) as e:
        icx.bp128_decode(data, 4096, 3, 0, workspace=ws)  # bad delta
    assert e.value.code == icx.EINVAL
    with pytest.raises(icx.IcxError) as e:
        icx.bp128_decode(data[1:], 100, 1, 0, workspace=ws)  # misaligned
    assert e.value.code == icx.EALIGN
    with pytest.raises(icx.IcxError) as e:
        icx.bp128_decode(data, 1 << 20, 1, 0, workspace=ws)  # workspace too small
    assert e.value.code == icx.ENOSPC
    with pytest.raises(icx.IcxError) as e:
        icx.bp128_decode(data, 4096 * 4, 1, 0, workspace=icx.Workspace(4096 * 4))  # needs an index
    assert e.value.code == icx.EINVAL
    del x


@pytest.mark.parametrize("fmt", FMTS)
@pytest.mark.parametrize("delta", [icx.DELTA_1, icx.DELTA_4])
def test_full_size_uniform_2pow26(delta, fmt):
    x = W.workload_uniform_long()
    enc = icx.bp128_encode(dev(x), delta, fmt)
    want = oracle.bp128_encode(x, delta, fmt)
    assert enc.nbytes == want.size
    ws = icx.Workspace(x.size)
    y = host_u32(icx.decode(enc, workspace=ws))
    assert ws.status() == icx.OK
    assert np.array_equal(y, x)


def test_full_size_clustered_d4():
    x = W.workload_clustered_long()
    enc_o = oracle.bp128_encode(x, 4, 0)
    y, st = gpu_decode(enc_o, x.size, 4, 0)
    assert st == icx.OK
    assert np.array_equal(y, x)
