"""GPU parity of every launch variant the tuning keys select: the same
streams decode bit for bit to the oracle's decode with SIMD-BP128 / W32 at 4,
8 and 16 warps per CTA, with and without the L2 prefetch ahead, and with
SIMD-FastPFOR at 4 and 8 warps per CTA."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1209_2137_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1209_2137_gb300 as icx  # noqa: E402

N = 3 * 65536 + 2048 * 7 + 77  # several tiles of every width, a partial metablock and a tail


@pytest.fixture(scope="module")
def streams():
    x = W.uniform_sorted(N, 27, 91)
    out = []
    for codec, delta, fmt in [("bp128", 1, 0), ("bp128", 4, 0), ("bp128", 1, 1), ("bp128", 4, 1), ("fastpfor", 1, 0),
                              ("fastpfor", 4, 0)]:
        enc = oracle.encode(codec, x, delta, fmt)
        out.append((codec, delta, fmt, enc, oracle.index(codec, enc, N, fmt), oracle.decode(codec, enc, N, delta, fmt)))
    return out


def decode(codec, delta, fmt, enc, idx):
    d = torch.from_numpy(enc).cuda()
    ix = torch.from_numpy(idx.view(np.int64)).cuda()
    ws = icx.Workspace(N)
    if codec == "bp128":
        y = icx.bp128_decode(d, N, delta, fmt, ix.view(torch.uint64), workspace=ws)
    else:
        y = icx.fastpfor_decode(d, N, delta, ix.view(torch.uint64), workspace=ws)
    assert ws.status() == icx.OK
    return y.cpu().numpy().view(np.uint32)


def test_every_launch_variant_matches_oracle(streams):
    try:
        for warps in (4, 8, 16):
            for l2 in (0, 1):
                icx.set_tuning("bp128.warps_per_cta", warps)
                icx.set_tuning("bp128.l2_prefetch", l2)
                for codec, delta, fmt, enc, idx, want in streams:
                    if codec == "bp128":
                        assert np.array_equal(decode(codec, delta, fmt, enc, idx), want), (warps, l2, delta, fmt)
        for warps in (4, 8):
            icx.set_tuning("fastpfor.warps_per_cta", warps)
            for codec, delta, fmt, enc, idx, want in streams:
                if codec == "fastpfor":
                    assert np.array_equal(decode(codec, delta, fmt, enc, idx), want), (warps, delta)
    finally:
        icx.set_tuning("bp128.warps_per_cta", 0)
        icx.set_tuning("bp128.l2_prefetch", 1)
        icx.set_tuning("fastpfor.warps_per_cta", 0)


def test_blocklane_variants_match_oracle(streams):
    """The two-phase block-per-lane decoders (SIMD-BP128 and SIMD-FastPFOR,
    strides 1 and 4): every output store path, grids of 1, 2 and 5 CTAs (a
    few warps take all the tasks, group scans and the tail), the shortest and
    the longest lead of sums before decodes, and the single-pass decoders
    they replace."""
    try:
        for w in (4, 5, 6):  # warps per CTA of the SIMD-FastPFOR stream kernel
            icx.set_tuning("fastpfor.stream_warps", w)
            for codec, delta, fmt, enc, idx, want in streams:
                if codec == "fastpfor":
                    assert np.array_equal(decode(codec, delta, fmt, enc, idx), want), ("stream warps", w, delta)
        icx.set_tuning("fastpfor.stream_warps", 0)
        for overlap in (0, 1, 2, 4, 6, 7):  # the prepare / scan / stream chain: stream order, each boundary, all
            icx.set_tuning("fastpfor.chain_overlap", overlap)
            for codec, delta, fmt, enc, idx, want in streams:
                if codec == "fastpfor":
                    assert np.array_equal(decode(codec, delta, fmt, enc, idx), want), ("chain overlap", overlap, delta)
        for fp_mode in (2, 1):  # the two SIMD-FastPFOR decoders that take these settings
            icx.set_tuning("fastpfor.blocklane", fp_mode)
            for store in (0, 1, 2):
                icx.set_tuning("bp128.blocklane_store", store)
                for ctas in (0, 1, 5):
                    icx.set_tuning("bp128.blocklane_ctas", ctas)
                    for codec, delta, fmt, enc, idx, want in streams:
                        if codec == "fastpfor":
                            assert np.array_equal(decode(codec, delta, fmt, enc, idx), want), (fp_mode, store, ctas)
            icx.set_tuning("bp128.blocklane_ctas", 0)
            icx.set_tuning("bp128.blocklane_store", -1)
        icx.set_tuning("fastpfor.blocklane", 1)
        for store in (0, 1, 2):
            icx.set_tuning("bp128.blocklane_store", store)
            for ctas in (0, 1, 2, 5):
                icx.set_tuning("bp128.blocklane_ctas", ctas)
                for codec, delta, fmt, enc, idx, want in streams:
                    if fmt == icx.FMT_PAPER:
                        assert np.array_equal(decode(codec, delta, fmt, enc, idx), want), (codec, store, ctas, delta)
        icx.set_tuning("bp128.blocklane_ctas", 0)
        icx.set_tuning("bp128.blocklane_store", -1)
        for lead in (128, 1 << 30):  # the shortest lead, and every sum before the first decode
            icx.set_tuning("bp128.blocklane_lead", lead)
            for codec, delta, fmt, enc, idx, want in streams:
                if fmt == icx.FMT_PAPER:
                    assert np.array_equal(decode(codec, delta, fmt, enc, idx), want), (codec, "lead", lead, delta)
        icx.set_tuning("bp128.blocklane_lead", 0)
        for sumw in (1, 2, 5):  # warps specialised for summing and decoding
            icx.set_tuning("bp128.blocklane_sum_warps", sumw)
            for ctas in (0, 1):
                icx.set_tuning("bp128.blocklane_ctas", ctas)
                for codec, delta, fmt, enc, idx, want in streams:
                    if fmt == icx.FMT_PAPER:
                        assert np.array_equal(decode(codec, delta, fmt, enc, idx), want), (codec, "sum warps", sumw,
                                                                                           ctas)
        icx.set_tuning("bp128.blocklane_sum_warps", 0)
        icx.set_tuning("bp128.blocklane_ctas", 0)
        icx.set_tuning("bp128.blocklane", 0)
        icx.set_tuning("fastpfor.blocklane", 0)
        for codec, delta, fmt, enc, idx, want in streams:
            if fmt == icx.FMT_PAPER:
                assert np.array_equal(decode(codec, delta, fmt, enc, idx), want), (codec, "single pass", delta)
    finally:
        icx.set_tuning("bp128.blocklane_sum_warps", 0)
        icx.set_tuning("bp128.blocklane", 1)
        icx.set_tuning("fastpfor.blocklane", -1)
        icx.set_tuning("fastpfor.stream_warps", 0)
        icx.set_tuning("fastpfor.chain_overlap", -1)
        icx.set_tuning("bp128.blocklane_store", -1)
        icx.set_tuning("bp128.blocklane_ctas", 0)
        icx.set_tuning("bp128.blocklane_lead", 0)


def test_workspace_shared_by_decoders_of_different_lengths():
    # one workspace serves SIMD-FastPFOR and SIMD-BP128* decodes of different
    # lengths in turn (as the batched plan's one-call-per-list baseline does):
    # the regions one decoder writes must not disturb the other's next launch
    xs = [W.uniform_sorted(n, 28, 300 + n % 89) for n in (70_000, 300_000 + 77, 9_000, 150_000)]
    ws = icx.Workspace(max(x.size for x in xs))
    for _ in range(2):
        for i, x in enumerate(xs):
            for codec, delta in (("fastpfor", 1), ("bp128", 4), ("bp128", 1)):
                enc = oracle.encode(codec, x, delta, 0)
                d = torch.from_numpy(enc).cuda()
                ix = torch.from_numpy(oracle.index(codec, enc, x.size, 0).view(np.int64)).cuda().view(torch.uint64)
                if codec == "bp128":
                    y = icx.bp128_decode(d, x.size, delta, 0, ix, workspace=ws)
                else:
                    y = icx.fastpfor_decode(d, x.size, delta, ix, workspace=ws)
                assert ws.status() == icx.OK, (i, codec, delta)
                assert np.array_equal(y.cpu().numpy().view(np.uint32), x), (i, codec, delta)
