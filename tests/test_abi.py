"""Host-side checks of the C ABI library: it builds for sm_103a, loads, and
exports every function declared in include/icx.h; the pure size helpers agree
with the format definitions.  No GPU needed."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1209_2137_gb300 import builder as b
    b.build()
    import paper_1209_2137_gb300 as icx
    return icx.lib()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "icx.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b([a-z][a-z0-9_]*)\s*\(", text)) - {"defined"})


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 17
    raw = ctypes.CDLL(os.path.join(ROOT, "paper_1209_2137_gb300", "libicx.so"))
    for name in names:
        assert hasattr(raw, name), name
    import paper_1209_2137_gb300 as icx
    assert set(icx.EXPORTED) <= set(names)


def test_size_helpers_match_format(lib):
    import paper_1209_2137_gb300 as icx
    for n in [0, 1, 127, 128, 2047, 2048, 2049, 2176, 65536, 65537, 1 << 26, 56273636]:
        assert icx.bp128_index_len(n) == oracle._load().orc_bp128_index_len(n)
        assert icx.fastpfor_index_len(n) == oracle._load().orc_fastpfor_index_len(n)
        assert icx.bp128_max_bytes(n, 0) >= oracle._load().orc_bp128_max_bytes(n) - 128 * ((n // 128 + 15) // 16)
        assert icx.workspace_bytes(n) >= 256 + 32 * ((n // 128 + 15) // 16 + 2) // 8
    assert icx.version().startswith("icx")


def test_worst_case_streams_fit_max_bytes(lib):
    import numpy as np
    import paper_1209_2137_gb300 as icx
    x = np.full(2048 * 3 + 100, 0xFFFFFFFF, dtype=np.uint32)
    for fmt in (0, 1):
        assert oracle.bp128_encode(x, 0, fmt).size <= icx.bp128_max_bytes(x.size, fmt)
    assert oracle.bp32_encode(x, 0).size <= icx.bp128_max_bytes(x.size, icx.FMT_BP32)
    assert oracle.fastpfor_encode(x, 0).size <= icx.fastpfor_max_bytes(x.size)


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    import paper_1209_2137_gb300 as icx
    monkeypatch.setattr(icx, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(icx, "_lib", None)
    with pytest.raises(icx.IcxError):
        icx.lib()


def test_plan_create_rejects_bad_lists(lib):
    # argument checks run on the host before any device call
    import paper_1209_2137_gb300 as icx
    tune = {"warps_per_cta": 8, "order": 0, "l2_prefetch": 0}
    empty = icx.ListDesc(None, 0, None, 0, None, icx.CODEC_BP128, icx.DELTA_1, icx.FMT_PAPER)
    cases = [
        (icx.ListDesc(16, 64, 32, 128, 48, 7, 1, 0), icx.EINVAL),            # unknown codec
        (icx.ListDesc(16, 64, 32, 128, 48, icx.CODEC_BP128, 2, 0), icx.EINVAL),   # stride 2
        (icx.ListDesc(16, 64, 32, 128, 48, icx.CODEC_BP128, 1, icx.FMT_BP32), icx.EINVAL),  # BP32 not batched
        (icx.ListDesc(16, 64, 32, 128, 48, icx.CODEC_BP128, 1, 5), icx.EINVAL),   # layout
        (icx.ListDesc(20, 64, 32, 128, 48, icx.CODEC_BP128, 1, 0), icx.EALIGN),   # stream not 16-byte aligned
        (icx.ListDesc(16, 64, 36, 128, 48, icx.CODEC_FASTPFOR, 1, 0), icx.EALIGN),  # output
        (icx.ListDesc(16, 64, 32, 5000, None, icx.CODEC_BP128, 1, 0), icx.EINVAL),  # 3 metablocks, no index
        (icx.ListDesc(16, 64, 32, 70000, None, icx.CODEC_FASTPFOR, 1, 0), icx.EINVAL),  # 2 pages, no index
        (icx.ListDesc(None, 64, 32, 128, 48, icx.CODEC_BP128, 1, 0), icx.EINVAL),  # no stream
    ]
    for desc, code in cases:
        with pytest.raises(icx.IcxError) as e:
            icx.Plan([empty, empty, desc], tune)
        assert e.value.code == code and "(list 2)" in str(e.value), (desc.codec, str(e.value))
    with pytest.raises(icx.IcxError) as e:
        icx.Plan([empty], {"warps_per_cta": 6, "order": 0, "l2_prefetch": 0})
    assert e.value.code == icx.EINVAL


def test_tuning_keys(lib):
    # host-side settings: known keys accepted, unknown refused
    import paper_1209_2137_gb300 as icx
    for key, value in [("bp128.warps_per_cta", 0), ("bp128.l2_prefetch", 1), ("fastpfor.warps_per_cta", 0),
                       ("bp128.blocklane", 1), ("fastpfor.blocklane", -1), ("bp128.blocklane_store", -1),
                       ("bp128.blocklane_ctas", 0), ("bp128.blocklane_lead", 0), ("bp128.blocklane_sum_warps", 0),
                       ("fastpfor.stream_warps", 0), ("fastpfor.chain_overlap", 1)]:
        icx.set_tuning(key, value)
    with pytest.raises(icx.IcxError) as e:
        icx.set_tuning("no.such.key", 1)
    assert e.value.code == icx.EINVAL


def test_layout_and_consumer_argument_checks(lib):
    # host-side refusals that return before any device call
    import ctypes

    import paper_1209_2137_gb300 as icx
    L = icx.lib()
    vp = ctypes.c_void_p
    a16, a4 = vp(4096), vp(4100)  # a 16-byte aligned and a 4-byte aligned fake device address
    # SIMD-FastPFOR calls: W32 is not a FastPFOR layout; SCALAR and SIMPLE8B are
    assert L.fastpfor_decode(a16, 64, a16, 128, icx.DELTA_1, icx.FMT_W32, None, a16, 1 << 20, None) == icx.EINVAL
    assert L.fastpfor_index(a16, 64, 128, 7, a16, a16, 1 << 20, None) == icx.EINVAL
    assert L.fastpfor_encode(a16, 128, icx.DELTA_1, icx.FMT_W32, a16, 1 << 20, a16, a16, a16, 1 << 20,
                             None) == icx.EINVAL
    for fmt in (icx.FMT_PAPER, icx.FMT_SCALAR, icx.FMT_SIMPLE8B):  # accepted, then refused for alignment
        assert L.fastpfor_decode(a4, 64, a16, 128, icx.DELTA_1, fmt, None, a16, 1 << 20, None) == icx.EALIGN
    # SIMD-BP128 calls accept BP32; a bad layout value is refused
    assert L.bp128_decode(a4, 64, a16, 128, icx.DELTA_1, icx.FMT_BP32, None, a16, 1 << 20, None) == icx.EALIGN
    assert L.bp128_decode(a16, 64, a16, 128, icx.DELTA_1, 9, None, a16, 1 << 20, None) == icx.EINVAL
    # the fused consumer: BP32 refused, a count pointer required, alignment checked
    b = (a16, 64, 128, icx.DELTA_1)
    assert L.bp128_intersect(*b, icx.FMT_BP32, None, a16, 10, a16, a16, a16, 1 << 20, None) == icx.EINVAL
    assert L.bp128_intersect(*b, icx.FMT_PAPER, None, a16, 10, a16, None, a16, 1 << 20, None) == icx.EINVAL
    assert L.bp128_intersect(*b, icx.FMT_PAPER, None, vp(4098), 10, a16, a16, a16, 1 << 20, None) == icx.EALIGN
    assert L.bp128_intersect(*b, icx.FMT_PAPER, None, a16, 10, a16, vp(4100), a16, 1 << 20, None) == icx.EALIGN
    assert L.sorted_intersect(a16, 128, a16, 10, a16, None, None) == icx.EINVAL
    assert L.sorted_intersect(a4, 128, a16, 10, a16, a16, None) == icx.EALIGN
    # size helpers of the new layouts
    assert icx.bp128_max_bytes(1 << 20, icx.FMT_BP32) >= (1 << 20) // 128 * 516
    assert L.icx_fastpfor_max_bytes(1 << 20) >= (1 << 20) // 128 * (512 + 131 + 1024)


def test_static_decode_refusals_before_any_device_call(lib):
    # the allocation-free entry point checks its arguments on the host and
    # returns before touching the device or its static workspace
    import paper_1209_2137_gb300 as icx
    fn = icx.lib().bp128_decode_static
    vp, sz, i = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int
    fn.argtypes = [vp, sz, vp, sz, i, i, vp, vp, vp]
    fn.restype = i
    a16, a4 = vp(4096), vp(4100)
    assert fn(a16, 64, a16, 128, icx.DELTA_1, icx.FMT_SIMPLE8B, None, None, None) == icx.EINVAL  # not a BP128 layout
    assert fn(a16, 64, a16, 128, 2, icx.FMT_PAPER, None, None, None) == icx.EINVAL  # no stride 2
    assert fn(a4, 64, a16, 128, icx.DELTA_1, icx.FMT_PAPER, None, None, None) == icx.EALIGN
    assert fn(a16, 64, a4, 128, icx.DELTA_1, icx.FMT_W32, None, None, None) == icx.EALIGN
    assert fn(a16, 64, a16, 128, icx.DELTA_1, icx.FMT_BP32, vp(4104), None, None) == icx.EALIGN
    assert fn(a16, 1 << 20, a16, 2049 * 16, icx.DELTA_4, icx.FMT_PAPER, None, None, None) == icx.EINVAL  # M > 1, no index
    assert fn(a16, 64, a16, (1 << 28) + 1, icx.DELTA_1, icx.FMT_PAPER, a16, None, None) == icx.ENOSPC
    assert fn(None, 0, None, 0, icx.DELTA_1, icx.FMT_PAPER, None, None, None) == icx.OK  # nothing to decode


def test_workspace_layout_keeps_tagged_and_plain_regions_apart(lib):
    # decodes of different lengths share a workspace: the look-back states and
    # the block-per-lane scratch (epoch-tagged words) of every length it serves
    # never overlap the plain records of any other length
    import paper_1209_2137_gb300 as icx
    L = icx.lib()
    out = (ctypes.c_size_t * 6)()
    for cap in (128, 4096 + 77, 65536 * 3 + 5, 1 << 26, 56273636):
        ws = icx.workspace_bytes(cap)
        assert L.icx_workspace_layout(cap, ws - 1, out) == icx.EINVAL
        lens = sorted(m for m in {1, 129, 2048, 4096 * 5 + 3, 65537, cap // 3, cap // 2 + 1, cap} if m <= cap)
        regs = {}
        for n in lens:
            assert L.icx_workspace_layout(n, ws, out) == icx.OK
            N, states_end, plain, fp2, plain_end, scratch = list(out)
            assert N >= cap and states_end <= plain <= fp2 <= plain_end <= scratch <= ws
            regs[n] = (states_end, plain, plain_end, scratch)
        for n, (se, _, _, sc) in regs.items():
            for m, (_, pl, pe, _) in regs.items():
                assert se <= pl and pe <= sc, (n, m)  # n's tagged regions vs m's plain ones
