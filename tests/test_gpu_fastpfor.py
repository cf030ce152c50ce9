"""GPU parity: SIMD-FastPFOR page walk, decoding (unpack + exception patch +
differential decoding) and the GPU encoder, through the C ABI, bit for bit
against the CPU oracle on the same seeded inputs."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1209_2137_gb300 import workloads as W
from tests import fmt_reader as F

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1209_2137_gb300 as icx  # noqa: E402

DELTAS = [icx.DELTA_NONE, icx.DELTA_1, icx.DELTA_4]
PAGE = 65536
LENGTHS = [1, 127, 128, 129, 2048, 2049, PAGE - 1, PAGE, PAGE + 1, PAGE + 128, 2 * PAGE + 16384 * 3 + 77,
           4 * PAGE + 2048 * 5 + 130]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host_u32(t):
    return t.cpu().numpy().view(np.uint32)


CASES = {
    "exceptions": W.exception_heavy(4 * PAGE + 2048 * 5 + 130, 61),
    "sorted": W.uniform_sorted(4 * PAGE + 2048 * 5 + 130, 29, 62),
    "widths": W.random_small(4 * PAGE + 2048 * 5 + 130, 63),
}


def gpu_decode(enc, n, delta, with_index=True, ws=None):
    d = dev(enc)
    idx = dev(oracle.fastpfor_index(enc, n)) if with_index else None
    ws = ws or icx.Workspace(n)
    out = icx.fastpfor_decode(d, n, delta, index=idx, workspace=ws)
    return host_u32(out), ws.status()


@pytest.mark.parametrize("delta", DELTAS)
@pytest.mark.parametrize("case", list(CASES))
def test_fastpfor_decode_matches_oracle(case, delta):
    x_all = CASES[case]
    for n in LENGTHS:
        x = x_all[:n]
        enc = oracle.fastpfor_encode(x, delta)
        y, st = gpu_decode(enc, n, delta)
        assert st == icx.OK, n
        want = oracle.fastpfor_decode(enc, n, delta)
        assert np.array_equal(y, want), (n, int(np.argmax(y != want)))


def test_fastpfor_every_exception_width():
    # blocks of zeros with a few values of bit length d: b = 0, exceptions of
    # width d, counts 1, 127, 128, 129 per page (Sec. 5)
    _every_exception_width(0)


@pytest.mark.parametrize("delta", [icx.DELTA_1, icx.DELTA_4])
def test_fastpfor_every_exception_width_with_deltas(delta):
    # the same values as differences: high parts of every width 1..32 through
    # entries (up to 24 bits) and through blocks decoded whole (wider)
    _every_exception_width(delta)


def _every_exception_width(delta):
    for d in range(1, 33):
        for total in (1, 127, 128, 129):
            nblocks = (total + 4) // 5
            x = np.zeros(128 * nblocks + 3, dtype=np.uint32)
            left = total
            for k in range(nblocks):
                for e in range(min(5, left)):
                    x[128 * k + 3 + 17 * e] = (1 << (d - 1)) | ((k * 7 + e) & ((1 << (d - 1)) - 1))
                left -= min(5, left)
            xs = oracle.delta_decode(x, 4 if delta == icx.DELTA_4 else 1) if delta else x
            enc = oracle.fastpfor_encode(xs, delta)
            y, st = gpu_decode(enc, x.size, delta)
            assert st == icx.OK and np.array_equal(y, xs), (d, total)


def test_fastpfor_index_matches_oracle():
    for case in CASES.values():
        for n in [129, PAGE + 1, case.size]:
            enc = oracle.fastpfor_encode(case[:n], 1)
            ws = icx.Workspace(n)
            idx = icx.fastpfor_index(dev(enc), n, workspace=ws)
            assert ws.status() == icx.OK
            assert np.array_equal(idx.cpu().numpy().view(np.uint64), oracle.fastpfor_index(enc, n))


def test_fastpfor_null_index_single_page():
    x = CASES["exceptions"]
    for n in [5, 128, 4000, PAGE, PAGE + 127]:
        enc = oracle.fastpfor_encode(x[:n], 4)
        y, st = gpu_decode(enc, n, 4, with_index=False)
        assert st == icx.OK and np.array_equal(y, x[:n])


@pytest.mark.parametrize("delta", DELTAS)
def test_gpu_fastpfor_encoder_bytes_match_oracle(delta):
    for case in CASES.values():
        for n in [0, 5, 128, 2049, PAGE + 1, case.size]:
            x = case[:n]
            enc = icx.fastpfor_encode(dev(x) if n else torch.empty(0, dtype=torch.uint32, device="cuda"), delta)
            want = oracle.fastpfor_encode(x, delta)
            got = enc.data.cpu().numpy()
            assert got.size == want.size, (n, got.size, want.size)
            assert np.array_equal(got, want), (n, int(np.argmax(got != want)))
            assert np.array_equal(enc.index.cpu().numpy().view(np.uint64), oracle.fastpfor_index(want, n))


def test_fastpfor_corrupt_streams_report_error():
    x = CASES["exceptions"][: 2 * PAGE + 300]
    n = x.size
    good = oracle.fastpfor_encode(x, 1)
    idx = oracle.fastpfor_index(good, n)
    ws = icx.Workspace(n)
    bad = good.copy()
    bad[int(idx[1]):int(idx[1]) + 4] = 0xFF  # header word of page 1 points far away
    icx.fastpfor_decode(dev(bad), n, 1, index=dev(idx), workspace=ws)
    assert ws.status() == icx.ECORRUPT
    bad = good.copy()
    len_at = int(idx[0]) + 4 * int(good[0:4].view("<u4")[0])
    bad[len_at + 4 + 1] = 40  # maxbits of block 0 above 32
    icx.fastpfor_decode(dev(bad), n, 1, index=dev(idx), workspace=ws)
    assert ws.status() == icx.ECORRUPT
    icx.fastpfor_decode(dev(good[:-1]), n, 1, index=dev(idx), workspace=ws)
    assert ws.status() == icx.ECORRUPT
    y = host_u32(icx.fastpfor_decode(dev(good), n, 1, index=dev(idx), workspace=ws))
    assert ws.status() == icx.OK and np.array_equal(y, x)


@pytest.mark.parametrize("delta", [icx.DELTA_NONE, icx.DELTA_1])
def test_fastpfor_full_size_exception_heavy(delta):
    x = W.workload_exceptions()
    enc = icx.fastpfor_encode(dev(x), delta)
    want = oracle.fastpfor_encode(x, delta)
    assert enc.nbytes == want.size
    ws = icx.Workspace(x.size)
    y = host_u32(icx.decode(enc, workspace=ws))
    assert ws.status() == icx.OK and np.array_equal(y, x)


@pytest.mark.parametrize("delta", [icx.DELTA_1, icx.DELTA_4])
def test_fastpfor_full_size_sorted(delta):
    x = W.workload_uniform_long()
    enc = icx.fastpfor_encode(dev(x), delta)
    ws = icx.Workspace(x.size)
    y = host_u32(icx.decode(enc, workspace=ws))
    assert ws.status() == icx.OK and np.array_equal(y, x)


def _blocks_with_exceptions(enc, n, at_least):
    """(block index, stream offset of its positions, count) of every block
    with at least `at_least` exceptions."""
    pages, _ = F.fastpfor_walk(enc, n)
    out = []
    for p, pg in enumerate(pages):
        for k, ((b, mb, pos), at) in enumerate(zip(pg["records"], pg["pos_at"])):
            if at is not None and len(pos) >= at_least:
                out.append((512 * p + k, at, len(pos)))
    return out


@pytest.mark.parametrize("delta", [icx.DELTA_1, icx.DELTA_4])
def test_fastpfor_positions_out_of_order(delta):
    # The format stores a block's exception positions as a list; the encoder
    # writes them in increasing order, but any order (and a repeated
    # position, whose high parts are OR-ed) decodes by the same patch rule
    # (Sec. 5).  Blocks with reversed, swapped and repeated positions, alone
    # in their warp's pair and filling a whole pair, against the oracle.
    n = 2 * PAGE + 4096 * 3 + 77
    x = W.uniform_sorted(n, 29, 64)
    enc = oracle.fastpfor_encode(x, delta).copy()
    blocks = _blocks_with_exceptions(enc, n, 3)
    assert len(blocks) > 200
    chosen = {}
    for blk, at, c in blocks:
        chosen.setdefault(blk // 32, []).append((blk, at, c))
    pairs = sorted(chosen)
    edits = 0
    # one edited block in each of a few pairs, a different edit each time
    for i, pr in enumerate(pairs[1:40:6]):
        blk, at, c = chosen[pr][0]
        seg = enc[at:at + c].copy()
        if i % 4 == 0:
            enc[at:at + c] = seg[::-1]  # reversed
        elif i % 4 == 1:
            enc[at + 1] = seg[0]  # a repeated position next to the first
        elif i % 4 == 2:
            enc[at + c - 1] = seg[0]  # the last equals the first
        else:
            enc[at], enc[at + 1] = seg[1], seg[0]  # first two swapped
        edits += 1
    # every block of one pair reversed
    for blk, at, c in chosen[pairs[-2]]:
        enc[at:at + c] = enc[at:at + c][::-1].copy()
        edits += 1
    assert edits > 8
    want = oracle.fastpfor_decode(enc, n, delta)
    assert want.size == n
    y, st = gpu_decode(enc, n, delta)
    assert st == icx.OK
    assert np.array_equal(y, want), int(np.argmax(y != want))
    # and the same stream through both decoders
    for mode in (2, 1, 0):
        icx.set_tuning("fastpfor.blocklane", mode)
        try:
            y0, st0 = gpu_decode(enc, n, delta)
        finally:
            icx.set_tuning("fastpfor.blocklane", -1)
        assert st0 == icx.OK and np.array_equal(y0, want), mode


@pytest.mark.parametrize("delta", [icx.DELTA_1, icx.DELTA_4])
def test_fastpfor_position_past_the_block_is_corrupt(delta):
    n = PAGE + 4096 + 5
    x = W.uniform_sorted(n, 29, 65)
    enc = oracle.fastpfor_encode(x, delta).copy()
    idx = oracle.fastpfor_index(enc, n)  # the page sizes do not change
    blk, at, c = _blocks_with_exceptions(enc, n, 2)[40]
    enc[at + 1] = 200
    with pytest.raises(oracle.CorruptStream):  # the oracle refuses the stream
        oracle.fastpfor_decode(enc, n, delta)
    ws = icx.Workspace(n)
    icx.fastpfor_decode(dev(enc), n, delta, index=dev(idx), workspace=ws)
    assert ws.status() == icx.ECORRUPT
