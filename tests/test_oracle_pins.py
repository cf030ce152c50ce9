"""Pins of the CPU oracle to facts fixed outside it (worked examples printed in
the paper, printed listings, closed forms, invariants and brute force).

These run without a GPU.  Each test names the passage it follows."""
from __future__ import annotations

import itertools
import math
import os

import numpy as np
import pytest

import oracle
from paper_1209_2137_gb300 import workloads as W
from tests import fmt_reader as F

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split(":", 1)
            out[k.strip()] = v.strip()
    return out


# --------------------------------------------------------------- Sec. 2 ----

def test_bitlen_is_binary_digit_count():
    # Sec. 2: binary notation needs ceil(log2(x+1)) bits: 1->1, 2->2, 3->2.
    assert oracle.bitlen(0) == 0
    assert oracle.bitlen(1) == 1 and oracle.bitlen(2) == 2 and oracle.bitlen(3) == 2
    for x in [4, 5, 127, 128, 255, 256, 2**31 - 1, 2**31, 2**32 - 1]:
        assert oracle.bitlen(x) == int(x).bit_length() == math.ceil(math.log2(x + 1))


# -------------------------------------------------------- Figs. 5 and 7 ----

def _listing_words(spec, values):
    """Build packed words from a printed shift/mask recipe (Fig. 5)."""
    words = [0, 0]
    for v, part in zip(values, spec.split()):
        segs = part.split("|")
        w, sh, bits = map(int, segs[0].split(":"))
        words[w] |= (v & ((1 << bits) - 1)) << sh
        if len(segs) > 1:
            w2, sh2, bits2, left = map(int, segs[1].split(":"))
            words[w2] |= ((v >> left) & ((1 << bits2) - 1)) << sh2
    return [x & 0xFFFFFFFF for x in words]


@pytest.mark.parametrize("b", [4, 5])
def test_fig5_scalar_unpack_listing(b):
    g = read_golden("unpack_listings.txt")
    rng = np.random.default_rng(b)
    for _ in range(50):
        vals = [int(x) for x in rng.integers(0, 1 << b, 8)]
        words = _listing_words(g[f"b{b}"], vals)
        nwords = 1 if b == 4 else 2
        raw = np.array(words[:nwords], dtype="<u4").view(np.uint8)
        assert list(oracle.unpack(raw, 8, 1, b)) == vals
        assert list(oracle.pack(vals, 1, b)) == list(raw)  # unused bits zero (R11)


def test_fig7_vertical_b5_listing():
    # Fig. 7: SIMDunpack5_8 applies the unpack5_8 recipe to each of 4 lanes;
    # integers 4r+l (0-based) are field r of lane l.  Row 0 / row 1 are the
    # first and second 128-bit words.
    g = read_golden("unpack_listings.txt")
    lanes = int(g["vertical_lanes"])
    rng = np.random.default_rng(7)
    for _ in range(50):
        vals = [int(x) for x in rng.integers(0, 32, 32)]
        rows = [[0] * lanes, [0] * lanes]
        for l in range(lanes):
            w = _listing_words(g["b5"], [vals[4 * r + l] for r in range(8)])
            rows[0][l], rows[1][l] = w
        raw = np.array(rows[0] + rows[1], dtype="<u4").view(np.uint8)
        assert list(oracle.unpack(raw, 32, 4, 5)) == vals
        assert list(oracle.pack(vals, 4, 5)) == list(raw)
    # Fig. 6 caption: integers 25-28 (1-based) straddle the two rows.
    vals = [0] * 32
    vals[24:28] = [31, 30, 29, 28]
    packed = oracle.pack(vals, 4, 5).view("<u4")
    for l in range(4):
        assert (packed[l] >> 30) == (vals[24 + l] & 3)
        assert (packed[4 + l] & 7) == (vals[24 + l] >> 2)


# --------------------------------------------------------------- Sec. 2.4 --

def test_vbyte_example_200():
    g = read_golden("vbyte_example.txt")
    enc = oracle.vbyte_encode([int(g["value"])])
    assert [f"{x:02x}" for x in enc] == g["stored_bytes_hex"].split()
    assert list(oracle.vbyte_decode(enc, 1)) == [200]
    one = oracle.vbyte_encode([int(g["single_byte_max"])])
    assert list(one) == [0x80 | 127]
    two = oracle.vbyte_encode([int(g["two_byte_min"])])
    assert list(two) == [0x00, 0x81]


def test_vbyte_roundtrip_and_lengths():
    vals = [0, 1, 127, 128, 2**14 - 1, 2**14, 2**21, 2**28 - 1, 2**28, 2**32 - 1]
    enc = oracle.vbyte_encode(vals)
    lengths = [1, 1, 1, 2, 2, 3, 4, 4, 5, 5]
    assert enc.size == sum(lengths)
    assert sum(int(x >> 7) for x in enc) == len(vals)  # one flagged byte each
    assert list(oracle.vbyte_decode(enc, len(vals))) == vals


def test_vbyte_rejects_truncated_and_overlong():
    with pytest.raises(oracle.CorruptStream):
        oracle.vbyte_decode(np.array([0x00, 0x00], dtype=np.uint8), 1)
    with pytest.raises(oracle.CorruptStream):
        oracle.vbyte_decode(np.array([0, 0, 0, 0, 0x90], dtype=np.uint8), 1)  # > 32 bits


# ----------------------------------------------------------------- Sec. 3 --

def test_delta_examples():
    g = read_golden("delta_examples.txt")
    v1 = [int(x) for x in g["d1_values"].split()]
    d1 = [int(x) for x in g["d1_deltas"].split()]
    assert list(oracle.delta_encode(v1, 1)) == d1
    assert list(oracle.delta_decode(d1, 1)) == v1
    v4 = [int(x) for x in g["d4_values"].split()]
    d4 = [int(x) for x in g["d4_deltas"].split()]
    assert list(oracle.delta_encode(v4, 4)) == d4
    assert list(oracle.delta_decode(d4, 4)) == v4


@pytest.mark.parametrize("n", [0, 1, 3, 4, 5, 1000, 4099])
def test_delta_closed_forms(n):
    d = W.uniform_u32(n, 11, 32)
    # D1: the prefix sum modulo 2^32 (numpy cumsum in uint64, reduced).
    want1 = (np.cumsum(d.astype(np.uint64)) % (1 << 32)).astype(np.uint32)
    assert np.array_equal(oracle.delta_decode(d, 1), want1)
    # D4: four independent prefix sums over the residues mod 4.
    want4 = np.zeros(n, dtype=np.uint32)
    for r in range(4):
        want4[r::4] = (np.cumsum(d[r::4].astype(np.uint64)) % (1 << 32)).astype(np.uint32)
    assert np.array_equal(oracle.delta_decode(d, 4), want4)
    assert np.array_equal(oracle.delta_decode(d, 0), d)
    for s in (0, 1, 4):
        assert np.array_equal(oracle.delta_encode(oracle.delta_decode(d, s), s), d)


# ----------------------------------------------------------------- Sec. 5 --

def test_fastpfor_worked_example():
    g = read_golden("fastpfor_worked_example.txt")
    vals = [int(x, 2) for x in g["values_binary"].split()]
    b, mb, c, costs = oracle.fastpfor_choose(vals)
    assert mb == int(g["maxbits"])
    for kv in g["costs_for_b"].split():
        bb, cost = map(int, kv.split(":"))
        assert costs[bb] == cost
    assert b == int(g["chosen_b"])
    for kv in g["exceptions_for_b"].split():
        bb, cnt = map(int, kv.split(":"))
        assert sum(1 for v in vals if v >= (1 << bb)) == cnt
    assert c == 3
    rec, high = oracle.fastpfor_block_record(vals)
    assert list(rec) == [int(x) for x in g["byte_array"].split()]
    assert list(high) == [int(x, 2) for x in g["high_bits"].split()]
    exc = [int(x, 2) for x in g["exceptions"].split()]
    assert [vals[p] for p in rec[3:]] == exc
    trunc = [int(x, 2) for x in g["truncated_binary"].split()]
    packed = oracle.pack([v & ((1 << b) - 1) for v in vals], 1, b)
    assert list(oracle.unpack(packed, 16, 1, b)) == trunc
    total = 8 * packed.size + 8 * rec.size + (mb - b) * len(high)
    assert total == int(g["total_bits"])
    assert total / 16 == float(g["bits_per_int"])


def _cost_table(vals, length):
    mb = max(int(v).bit_length() for v in vals) if len(vals) else 0
    out = {}
    for b in range(mb + 1):
        c = sum(1 for v in vals if int(v) >= (1 << b))
        out[b] = length * b + c * (8 + mb - b)
    return mb, out


def test_fastpfor_choice_brute_force_small_blocks():
    # every block of length 1..5 over {0..7}: the chosen b is the largest
    # minimiser of the printed cost (R10), and scalar packing round-trips.
    for length in range(1, 6):
        for vals in itertools.product(range(8), repeat=length):
            b, mb, c, _ = oracle.fastpfor_choose(vals)
            tmb, table = _cost_table(vals, length)
            best = min(table.values())
            assert mb == tmb
            assert b == max(bb for bb, cost in table.items() if cost == best)
            assert c == sum(1 for v in vals if v >= (1 << b))
            if length == 5:
                continue
            w = tmb
            assert list(oracle.unpack(oracle.pack(vals, 1, w), length, 1, w)) == list(vals)


@pytest.mark.parametrize("lanes", [1, 4, 32])
def test_pack_every_width_single_fields(lanes):
    count = 128
    for b in range(0, 33):
        cases = [np.zeros(count, np.uint32), np.full(count, (1 << b) - 1 if b else 0, np.uint32)]
        for bit in range(b):
            z = np.zeros(count, np.uint32)
            z[(bit * 7) % count] = 1 << bit
            cases.append(z)
        for v in cases:
            raw = oracle.pack(v, lanes, b)
            assert raw.size == 4 * lanes * ((count // lanes * b + 31) // 32)
            assert np.array_equal(oracle.unpack(raw, count, lanes, b), v)
            # total set bits equal total bits of the values: nothing leaks
            assert int(np.unpackbits(raw).sum()) == int(sum(int(x).bit_count() for x in v))


# --------------------------------------------------------------- Sec. 6.2 --

def _bp128_invariants(x, delta, layout):
    n = x.size
    enc = oracle.bp128_encode(x, delta, layout)
    d = np.asarray(oracle.delta_encode(x, delta))
    metas, tail = F.bp128_walk(enc, n, layout)
    for m, (off, widths, size, k) in enumerate(metas):
        for kk in range(k):
            blk = d[128 * (16 * m + kk):128 * (16 * m + kk + 1)]
            assert widths[kk] == max(int(v).bit_length() for v in blk)  # R12
        assert all(w == 0 for w in widths[k:])  # R1
    # closed-form size: metablocks then the Variable Byte tail
    tail_vals = d[128 * (n // 128):]
    tail_len = sum(max(1, math.ceil(int(v).bit_length() / 7)) for v in tail_vals)
    assert enc.size == tail + tail_len
    idx = oracle.bp128_index(enc, n, layout)
    assert list(idx[:-1]) == [m[0] for m in metas] and idx[-1] == tail
    return enc


@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("delta", [0, 1, 4])
def test_bp128_roundtrip_generated(delta, layout):
    cases = [W.workload_sorted_small(), W.uniform_sorted(100_003, 29, 5),
             W.random_small(20_000, 3), W.exception_heavy(9_000, 4)]
    for x in cases:
        enc = _bp128_invariants(x, delta, layout)
        y = oracle.bp128_decode(enc, x.size, delta, layout)
        assert np.array_equal(x, y)


def test_bp128_sorted_output_nondecreasing():
    x = W.workload_sorted_small()
    for delta in (1, 4):
        y = oracle.bp128_decode(oracle.bp128_encode(x, delta), x.size, delta)
        assert np.all(np.diff(y.astype(np.int64)) >= 0)


@pytest.mark.parametrize("layout", [0, 1])
def test_bp128_every_length_up_to_4200(layout):
    x = W.uniform_sorted(4200, 20, 99)
    for n in range(0, 4201):
        if n > 300 and n % 7 and n not in (2047, 2048, 2049, 4095, 4096, 4097):
            continue  # every length up to 300, then a stride plus the edges
        enc = oracle.bp128_encode(x[:n], 1, layout)
        assert np.array_equal(oracle.bp128_decode(enc, n, 1, layout), x[:n])


def test_bp128_all_lengths_exhaustive_paper_layout():
    x = W.uniform_sorted(4200, 20, 98)
    for n in range(0, 4201):
        enc = oracle.bp128_encode(x[:n], 4, 0)
        assert np.array_equal(oracle.bp128_decode(enc, n, 4, 0), x[:n])


def test_bp128_appendix_bound():
    # Appendix A: sorted distinct arrays coded with D1 and blocks of B = 128
    # cost at most 8/B + 1 + log2(B) + log2(2^32/n) bits per integer.
    for n, bits in [(2048 * 32, 22), (2048 * 16, 29), (2048 * 8, 32)]:
        x = W.uniform_sorted(n, bits, n)
        enc = oracle.bp128_encode(x, 1, 0)
        per_int = 8 * enc.size / n
        assert per_int <= 8 / 128 + 1 + 7 + math.log2(2**32 / n)


def test_w32_payload_is_paper_payload_reshuffled():
    # R16: a W32 lane holds the same fields as the paper layout, so the bit
    # count per metablock is the same up to padding to whole 128-byte rows.
    x = W.random_small(2048 * 3 + 128 * 5, 17)
    p = oracle.bp128_encode(x, 0, 0)
    w = oracle.bp128_encode(x, 0, 1)
    mp, _ = F.bp128_walk(p, x.size, 0)
    mw, _ = F.bp128_walk(w, x.size, 1)
    for (_, wid_p, size_p, k), (_, wid_w, size_w, _) in zip(mp, mw):
        assert wid_p == wid_w
        assert size_w - 16 == 128 * math.ceil((size_p - 16) / 128)


def test_w32_lane_assignment():
    # R16: lane j = 4g + l holds integers 16g + 4m + l of each block.
    x = np.arange(128, dtype=np.uint32)
    x[0] = 0
    enc = oracle.bp128_encode(x, 0, 1)
    b = int(enc[0])
    assert b == 7
    payload = enc[16:]
    for j in range(32):
        g, l = divmod(j, 4)
        lane_words = payload.view("<u4")[j::32]
        bits = 0
        for i, w in enumerate(lane_words):
            bits |= int(w) << (32 * i)
        got = [(bits >> (m * b)) & ((1 << b) - 1) for m in range(4)]
        assert got == [16 * g + 4 * m + l for m in range(4)]


def test_bp128_corrupt_width_rejected():
    x = W.random_small(4096, 5)
    enc = oracle.bp128_encode(x, 0, 0).copy()
    enc[0] = 33
    with pytest.raises(oracle.CorruptStream):
        oracle.bp128_decode(enc, x.size, 0, 0)
    with pytest.raises(oracle.CorruptStream):
        oracle.bp128_decode(oracle.bp128_encode(x, 0, 0)[:-5], x.size, 0, 0)


# ----------------------------------------------------- Sec. 5, SIMD variant --

def _fastpfor_invariants(x, delta):
    n = x.size
    enc = oracle.fastpfor_encode(x, delta)
    d = np.asarray(oracle.delta_encode(x, delta))
    pages, tail = F.fastpfor_walk(enc, n)
    for p, pg in enumerate(pages):
        counts = {}
        packed = 16
        for k, (b, mb, pos) in enumerate(pg["records"]):
            blk = d[128 * (512 * p + k):128 * (512 * p + k + 1)]
            tmb, table = _cost_table(blk, 128)
            assert mb == tmb
            best = min(table.values())
            assert b == max(bb for bb, c in table.items() if c == best)  # R10
            exc = [i for i in range(128) if int(blk[i]) >= (1 << b)]
            assert pos == exc  # ascending positions, count = #{v >= 2^b}
            if exc:
                counts[mb - b] = counts.get(mb - b, 0) + len(exc)
            packed += 16 * b
        assert pg["len_at"] == packed  # R5
        assert {d_: c for d_, (c, _) in pg["arrays"].items()} == counts  # R7, R8
        for d_, (c, off) in pg["arrays"].items():
            assert off % 16 == 0  # R9
        assert pg["offset"] % 16 == 0 and pg["size"] % 16 == 0  # R14
        # closed-form page size
        L = pg["byte_len"]
        size = 4 + 12 + packed - 16 + 4 + F.pad(L, 4) + 4
        for d_ in sorted(counts):
            size = F.pad(size + 4, 16) + 16 * d_ * ((counts[d_] + 127) // 128)
        assert pg["size"] == F.pad(size, 16)
    idx = oracle.fastpfor_index(enc, n)
    assert list(idx[:-1]) == [pg["offset"] for pg in pages] and idx[-1] == tail
    return enc


@pytest.mark.parametrize("delta", [0, 1, 4])
def test_fastpfor_roundtrip_generated(delta):
    cases = [W.workload_sorted_small(), W.exception_heavy(70_001, 8),
             W.uniform_sorted(140_000, 29, 6), W.random_small(5000, 9)]
    for x in cases:
        enc = _fastpfor_invariants(x, delta)
        assert np.array_equal(oracle.fastpfor_decode(enc, x.size, delta), x)


def test_fastpfor_every_exception_width_and_count():
    # d in [1, 32] with 1, 127, 128 and 129 exceptions of width d in a page:
    # blocks of zeros with a few values of bitlen d choose b = 0 (Sec. 5 cost).
    for d in range(1, 33):
        for total in (1, 127, 128, 129):
            per_block = 5
            nblocks = (total + per_block - 1) // per_block
            x = np.zeros(128 * nblocks, dtype=np.uint32)
            left = total
            for k in range(nblocks):
                for e in range(min(per_block, left)):
                    x[128 * k + 3 + 17 * e] = (1 << (d - 1)) | ((k * 7 + e) & ((1 << (d - 1)) - 1))
                left -= min(per_block, left)
            enc = oracle.fastpfor_encode(x, 0)
            pages, _ = F.fastpfor_walk(enc, x.size)
            assert pages[0]["arrays"][d][0] == total
            assert np.array_equal(oracle.fastpfor_decode(enc, x.size, 0), x)
            # the values read back independently: array d in chunks of 128
            # vertically packed values (element q: chunk q // 128, lane q % 4,
            # field (q % 128) // 4)
            _, vals, end = F.fastpfor_simd_read(enc, x.size)
            assert vals == [int(v) for v in x] and end == enc.size, (d, total)


def _diffs(x, delta):
    # closed-form differences (Sec. 3): x_i - x_{i-s} mod 2^32, x_i for i < s
    s = delta if delta else 1
    xi = [int(v) for v in x]
    return [(xi[i] - (xi[i - s] if (delta and i >= s) else 0)) % (1 << 32) for i in range(len(xi))]


@pytest.mark.parametrize("layout", [oracle.PAPER, oracle.W32])
def test_bp128_values_read_back_independently(layout):
    # Sec. 4 (Figs. 6-7) and Sec. 6.2: every coded delta, rebuilt from the
    # bytes with Python integers (word w of lane l at byte 16w + 4l, value i
    # = field i // 4 of lane i % 4; W32 per R16), equals the closed-form
    # difference of the input, for strides 0, 1 and 4, partial metablocks
    # and Variable Byte tails; random widths 0..32 cover every field width
    cases = [(n, W.uniform_sorted(n, 26, 700 + n % 91)) for n in
             (1, 127, 128, 129, 2047, 2048, 2049, 4096 + 77, 16 * 128 * 3 + 5, 65536 + 130)]
    cases.append((16 * 128 * 2 + 40, W.random_small(16 * 128 * 2 + 40, 77)))
    for n, x in cases:
        for delta in (0, 1, 4):
            if delta and np.any(x[1:] < x[:-1]):
                continue
            enc = oracle.bp128_encode(x, delta, layout)
            vals, end = F.bp128_read(enc, n, layout)
            assert vals == _diffs(x, delta), (n, delta, layout)
            assert end == enc.size


def test_fastpfor_simd_values_read_back_independently():
    # Sec. 5 (SIMD variant): every coded value of multi-page streams (the
    # vertical low parts, the exception arrays in vertical chunks of 128, the
    # positions) rebuilt from the bytes equals the closed-form difference of
    # the input, for strides 0, 1 and 4
    cases = [W.uniform_sorted(65536 * 2 + 128 * 7 + 99, 27, 61), W.exception_heavy(65536 + 128 * 3 + 5, 62),
             W.random_small(65536 + 2048 + 17, 63)]
    for x in cases:
        for delta in (0, 1, 4):
            if delta and np.any(x[1:] < x[:-1]):
                continue
            enc = oracle.fastpfor_encode(x, delta)
            pages, vals, end = F.fastpfor_simd_read(enc, x.size)
            assert vals == _diffs(x, delta), delta
            assert end == enc.size
            assert len(pages) == (x.size // 128 + 511) // 512


def test_fastpfor_lengths_and_pages():
    x = W.exception_heavy(65536 * 2 + 128 * 3 + 77, 12)
    for n in [0, 1, 127, 128, 129, 65535, 65536, 65537, 65536 + 128, x.size]:
        enc = _fastpfor_invariants(x[:n], 0)
        assert np.array_equal(oracle.fastpfor_decode(enc, n, 0), x[:n])


def test_fastpfor_corrupt_rejected():
    x = W.exception_heavy(4096, 13)
    enc = oracle.fastpfor_encode(x, 0).copy()
    bad = enc.copy()
    bad[0:4] = 0xFF  # byte-array offset far past the page
    with pytest.raises(oracle.CorruptStream):
        oracle.fastpfor_decode(bad, x.size, 0)
    with pytest.raises(oracle.CorruptStream):
        oracle.fastpfor_decode(enc[:-20], x.size, 0)


def test_fastpfor_padding_overhead_range():
    # Sec. 5: SIMD-FastPFOR's padding costs roughly 0.3-0.4 bit/int on the
    # paper's data; on a long sorted array the total stays within a few
    # tenths of a bit of the unpadded sum of its parts.
    x = W.uniform_sorted(1 << 18, 29, 21)
    enc = oracle.fastpfor_encode(x, 1)
    pages, _ = F.fastpfor_walk(enc, x.size)
    unpadded = 0
    for pg in pages:
        unpadded += 8 * (pg["len_at"] - 16) + 8 * pg["byte_len"]
        unpadded += sum(d * c for d, (c, _) in pg["arrays"].items())
    overhead = (8 * enc.size - unpadded) / x.size
    assert 0.0 <= overhead < 1.0


# -- Sec. 7: sorted-list membership (the consumer fused with decoding) -------

def _member_brute(a, b):
    s = set(int(v) for v in a)
    flags = [int(v) in s for v in b]
    bits = np.zeros(max(1, (len(b) + 31) // 32), dtype=np.uint32)
    for j, f in enumerate(flags):
        if f:
            bits[j // 32] |= np.uint32(1 << (j % 32))
    return bits[: (len(b) + 31) // 32], sum(flags)


def test_member_bits_brute_force_with_duplicates():
    # tiny sorted lists with repeated values on both sides, values drawn from
    # a small range so that hits, misses and runs all occur
    rng = np.random.default_rng(5)
    for t in range(300):
        na, nb = int(rng.integers(0, 40)), int(rng.integers(0, 70))
        hi = int(rng.integers(1, 60))
        a = np.sort(rng.integers(0, hi, na)).astype(np.uint32)
        b = np.sort(rng.integers(0, hi + 5, nb)).astype(np.uint32)
        bits, cnt = oracle.member_bits(a, b)
        want_bits, want_cnt = _member_brute(a, b)
        assert cnt == want_cnt, t
        assert np.array_equal(bits, want_bits), t


def test_member_bits_special_cases():
    a = np.arange(0, 1000, 3, dtype=np.uint32)
    bits, cnt = oracle.member_bits(a, np.zeros(0, np.uint32))
    assert bits.size == 0 and cnt == 0
    b = np.arange(0, 100, dtype=np.uint32)
    bits, cnt = oracle.member_bits(np.zeros(0, np.uint32), b)
    assert cnt == 0 and not bits.any()
    bits, cnt = oracle.member_bits(a, a)  # b a subset of a: every bit set
    assert cnt == a.size and int(sum(bin(int(w)).count("1") for w in bits)) == a.size
    bits, cnt = oracle.member_bits(a, a + 1)  # disjoint
    assert cnt == 0 and not bits.any()
    # bits past nb stay zero; the extremes of the value range
    b = np.array([0, 5, 0xFFFFFFFE, 0xFFFFFFFF], dtype=np.uint32)
    bits, cnt = oracle.member_bits(np.array([0, 0xFFFFFFFF], np.uint32), b)
    assert cnt == 2 and bits.tolist() == [0b1001]


def test_member_bits_matches_isin():
    # a special case that reduces to a library routine: numpy's isin
    x = W.uniform_sorted(200000, 24, 33)
    rng = np.random.default_rng(9)
    b = np.sort(np.concatenate([rng.choice(x, 5000), rng.integers(0, 1 << 24, 5000).astype(np.uint32)]))
    bits, cnt = oracle.member_bits(x, b)
    flags = np.isin(b, x)
    got = np.unpackbits(bits.view(np.uint8), bitorder="little")[: b.size].astype(bool)
    assert np.array_equal(got, flags) and cnt == int(flags.sum())


# -- Sec. 6.2: BP32 (scalar binary packing, NEXT-3) --------------------------

def _vbyte_len(v):
    return max(1, (int(v).bit_length() + 6) // 7)


def test_bp32_bytes_read_back_independently():
    # the bytes, read with Python integers from the format definition, give
    # the deltas whose closed-form prefix sums are the input; every width
    # byte is the largest bit length of its 32 deltas; sizes are closed form
    for n in [0, 1, 127, 128, 129, 255, 256, 2047, 2048, 2049, 4096 + 77, 16 * 128 * 3 + 5]:
        x = W.uniform_sorted(n, 26, 400 + n % 97) if n else np.zeros(0, np.uint32)
        for delta in (0, 1, 4):
            enc = oracle.bp32_encode(x, delta)
            metas, deltas, tail = F.bp32_read(enc, n)
            s = delta if delta else 1
            xi = [int(v) for v in x]
            want = [xi[i] - (xi[i - s] if (delta and i >= s) else 0) for i in range(n)]
            want = [w % (1 << 32) for w in want]
            assert deltas == want[: 128 * (n // 128)], (n, delta)
            for m, (off, widths) in enumerate(metas):
                for j, b in enumerate(widths):
                    blk = want[128 * m + 32 * j: 128 * m + 32 * j + 32]
                    assert b == max(v.bit_length() for v in blk), (n, delta, m, j)
            size = sum(4 + 4 * sum(w) for _, w in metas) + sum(_vbyte_len(v) for v in want[128 * (n // 128):])
            assert enc.size == size == tail + sum(_vbyte_len(v) for v in want[128 * (n // 128):])
            assert np.array_equal(oracle.bp32_decode(enc, n, delta), x)
            idx = oracle.bp32_index(enc, n)
            assert list(idx[:-1]) == [metas[16 * u][0] for u in range((n // 128 + 15) // 16)]
            assert int(idx[-1]) == tail


def test_bp32_every_width_single_bit_fields():
    # brute force: each width 0..32, a single set bit in each of the 32
    # positions of block 2 of a metablock
    for b in range(33):
        for i in range(32):
            d = np.zeros(128, np.uint32)
            if b:
                d[64 + i] = np.uint32(1 << (b - 1))
            enc = oracle.bp32_encode(d, 0)
            assert list(enc[:4]) == [0, 0, b, 0]
            assert np.array_equal(oracle.bp32_decode(enc, 128, 0), d)
            if b:
                bitpos = 8 * (4 + 0) + i * b + (b - 1)  # block 2 starts right after the descriptor
                assert (int.from_bytes(enc.tobytes(), "little") >> bitpos) & 1 == 1


def test_bp32_corrupt_rejected():
    x = W.uniform_sorted(1000, 20, 6)
    enc = oracle.bp32_encode(x, 1)
    bad = enc.copy()
    bad[0] = 33
    with pytest.raises(oracle.CorruptStream):
        oracle.bp32_decode(bad, x.size, 1)
    with pytest.raises(oracle.CorruptStream):
        oracle.bp32_decode(enc[:100], x.size, 1)


# -- Sec. 5: the scalar FastPFOR (one-lane packing, NEXT-3) ------------------

def test_fastpfor_scalar_bytes_read_back_independently():
    # the page bytes, read with Python integers, give back the coded values
    # (the closed-form differences of the input); arrays padded to 32
    for x in (W.uniform_sorted(65536 * 2 + 128 * 7 + 99, 27, 61), W.exception_heavy(65536 + 128 * 3 + 5, 62)):
        for delta in (0, 1, 4):
            if delta and x[1] < x[0]:
                continue
            enc = oracle.fastpfor_encode(x, delta, oracle.SCALAR)
            pages, vals, tail = F.fastpfor_scalar_read(enc, x.size)
            s = delta if delta else 1
            xi = [int(v) for v in x]
            want = [(xi[i] - (xi[i - s] if (delta and i >= s) else 0)) % (1 << 32) for i in range(x.size)]
            assert vals == want[: 128 * (x.size // 128)], delta
            for pg in pages:
                for d, (cnt, off) in pg["arrays"].items():
                    assert off % 16 == 0 and cnt > 0
            assert np.array_equal(oracle.fastpfor_decode(enc, x.size, delta, oracle.SCALAR), x)
            idx = oracle.fastpfor_index(enc, x.size, oracle.SCALAR)
            assert [int(v) for v in idx[:-1]] == [pg["offset"] for pg in pages] and int(idx[-1]) == tail
            # the same records as SIMD-FastPFOR: only the bit-packed sections differ
            simd_pages, _ = F.fastpfor_walk(oracle.fastpfor_encode(x, delta), x.size)
            assert [pg["records"] for pg in pages] == [pg["records"] for pg in simd_pages]


def test_fastpfor_scalar_every_exception_width():
    # one block per width d = 1..32 with exceptions of exactly d high bits,
    # counts across the 32-value padding unit
    for d in range(1, 33):
        for count in (1, 31, 32, 33):
            x = np.zeros(128 * 4, np.uint32)
            for e in range(count):
                blk, pos = divmod(e, 16)
                x[128 * blk + 5 * pos + 1] = np.uint32(((1 << (d - 1)) | (e & ((1 << (d - 1)) - 1))) << 0)
            # widths: the block's low width b = 0 makes every nonzero value an exception of width d
            enc = oracle.fastpfor_encode(x, 0, oracle.SCALAR)
            pages, vals, _ = F.fastpfor_scalar_read(enc, x.size)
            assert vals == [int(v) for v in x]
            assert np.array_equal(oracle.fastpfor_decode(enc, x.size, 0, oracle.SCALAR), x)


# -- Sec. 2 / Sec. 5: Simple-8b and SimplePFOR (NEXT-4) ----------------------

S8 = F.simple8b_table(os.path.join(os.path.dirname(__file__), "golden", "simple8b_table.txt"))


def _greedy_ok(values, sels):
    # every word took the smallest selector whose whole count of next values
    # exists and fits (the paper's greedy rule, R23)
    p = 0
    for s in sels:
        for t in range(s):
            cnt, bits = S8[t]
            feasible = p + cnt <= len(values) and all(v < (1 << bits) for v in values[p:p + cnt])
            assert not feasible, (p, s, t)
        p += S8[s][0]
    assert p == len(values)


def test_simple8b_table_modes():
    # for each selector, a run that fits it and no smaller selector is coded
    # with that selector in one word (32-bit values reach selector 15 only
    # above 2^30, which the 30-bit selector 14 cannot hold)
    for s, (cnt, bits) in S8.items():
        if s == 0:
            vals = [0] * 240
        elif s == 1:
            vals = [0] * 120  # 240 zeros do not exist
        elif s == 15:
            vals = [0xFFFFFFFF]
        else:
            vals = [(1 << bits) - 1] * cnt
        words = oracle.simple8b_encode(np.array(vals, np.uint32))
        got, sels = F.simple8b_read(words, S8)
        assert got == vals and sels == [s], (s, sels)
        assert list(oracle.simple8b_decode(words, len(vals))) == vals


def test_simple8b_random_streams_greedy_and_exact():
    rng = np.random.default_rng(17)
    for t in range(200):
        n = int(rng.integers(0, 700))
        kind = t % 4
        if kind == 0:
            v = rng.integers(0, 2, n)
        elif kind == 1:
            v = (rng.random(n) < 0.05) * rng.integers(0, 1 << 20, n)
        elif kind == 2:
            v = rng.integers(0, 1 << int(rng.integers(1, 33)), n, dtype=np.uint64)
        else:
            v = np.where(rng.random(n) < 0.5, 0, rng.integers(0, 16, n))
        v = v.astype(np.uint32)
        words = oracle.simple8b_encode(v)
        got, sels = F.simple8b_read(words, S8)
        assert got == [int(a) for a in v], t
        _greedy_ok([int(a) for a in v], sels)
        assert np.array_equal(oracle.simple8b_decode(words, n), v)
        if words.size:
            with pytest.raises(oracle.CorruptStream):
                oracle.simple8b_decode(words, n + 1)


def test_simplepfor_bytes_read_back_independently():
    for x in (W.uniform_sorted(65536 * 2 + 128 * 7 + 99, 27, 81), W.exception_heavy(65536 + 128 * 3 + 5, 82)):
        for delta in (0, 1, 4):
            if delta and x[1] < x[0]:
                continue
            enc = oracle.simplepfor_encode(x, delta)
            pages, vals, tail = F.simplepfor_read(enc, x.size, S8)
            s = delta if delta else 1
            xi = [int(v) for v in x]
            want = [(xi[i] - (xi[i - s] if (delta and i >= s) else 0)) % (1 << 32) for i in range(x.size)]
            assert vals == want[: 128 * (x.size // 128)], delta
            for pg in pages:
                _greedy_ok(pg["high"], pg["sels"])
            assert np.array_equal(oracle.simplepfor_decode(enc, x.size, delta), x)
            idx = oracle.simplepfor_index(enc, x.size)
            assert [int(v) for v in idx[:-1]] == [pg["offset"] for pg in pages] and int(idx[-1]) == tail
            # as many exception high parts as the scalar FastPFOR of the same input has exceptions
            sc, _ = F.fastpfor_walk(oracle.fastpfor_encode(x, delta, oracle.SCALAR), x.size, chunk=32)
            assert sum(pg["N"] for pg in pages) == sum(len(r[2]) for p in sc for r in p["records"])


def test_simplepfor_corrupt_rejected():
    x = W.exception_heavy(4096, 83)
    enc = oracle.simplepfor_encode(x, 0)
    bad = enc.copy()
    bad[0:4] = 0xFF
    with pytest.raises(oracle.CorruptStream):
        oracle.simplepfor_decode(bad, x.size, 0)
    with pytest.raises(oracle.CorruptStream):
        oracle.simplepfor_decode(enc[:-20], x.size, 0)
