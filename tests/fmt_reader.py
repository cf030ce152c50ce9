"""A second, independent reader of the stream layouts, used by the tests.

It walks the byte layout with Python integers -- the structure (widths,
records, counts and sizes) and the coded values themselves -- so that the
oracle's encoder can be checked against the format definitions without
trusting the oracle's own parser.  Layouts: SIMD-BP128 metablocks (Sec. 6.2)
and the W32 variant, SIMD-FastPFOR pages (Sec. 5), BP32, the scalar FastPFOR
and SimplePFOR; readings R1-R23 are listed in the oracle's header.
"""
from __future__ import annotations

import struct


def le32(buf, off):
    return struct.unpack_from("<I", bytes(buf[off:off + 4]))[0]


def pad(x, a):
    return (x + a - 1) // a * a


def bp128_walk(buf, n, layout):
    """Yields (offset, widths, size) per metablock; returns tail offset."""
    buf = bytes(memoryview(buf))
    nb = n // 128
    metas = []
    pos = 0
    for m in range((nb + 15) // 16):
        k = min(16, nb - 16 * m)
        widths = list(buf[pos:pos + 16])
        sb = sum(widths[:k])
        size = 16 + 16 * sb if layout == 0 else 16 + 128 * ((4 * sb + 31) // 32)
        metas.append((pos, widths, size, k))
        pos += size
    return metas, pos


def fastpfor_walk(buf, n, chunk=128):
    """Parses every page; returns (pages, tail offset).  A page is a dict with
    the per-block records and the exception arrays' counts and offsets.
    chunk: the padding unit of an exception array (128 values for
    SIMD-FastPFOR, 32 for the scalar FastPFOR)."""
    buf = bytes(memoryview(buf))
    nb = n // 128
    pages = []
    pos = 0
    for p in range((nb + 511) // 512):
        k = min(512, nb - 512 * p)
        base = pos
        len_at = 4 * le32(buf, base)
        L = le32(buf, base + len_at)
        rec_at = base + len_at + 4
        records = []
        pos_at = []  # stream offset of each block's first position (None: no exceptions)
        r = 0
        for _ in range(k):
            b, mb = buf[rec_at + r], buf[rec_at + r + 1]
            r += 2
            pos_list = []
            at = None
            if mb > b:
                c = buf[rec_at + r]
                r += 1
                at = rec_at + r
                pos_list = list(buf[rec_at + r:rec_at + r + c])
                r += c
            records.append((b, mb, pos_list))
            pos_at.append(at)
        assert r == L, (r, L)
        q = rec_at + pad(L, 4)
        bitset = le32(buf, q)
        q += 4
        arrays = {}
        for d in range(1, 33):
            if (bitset >> (d - 1)) & 1:
                cnt = le32(buf, q)
                q = base + pad(q + 4 - base, 16)
                arrays[d] = (cnt, q)
                q += chunk // 8 * d * ((cnt + chunk - 1) // chunk)
        end = base + pad(q - base, 16)
        pages.append(dict(offset=base, blocks=k, len_at=len_at, byte_len=L, records=records,
                          bitset=bitset, arrays=arrays, size=end - base, pos_at=pos_at))
        pos = end
    return pages, pos


def bp32_read(buf, n):
    """BP32 (Sec. 6.2): per 128-integer metablock a little-endian descriptor
    word (byte j = width of 32-integer block j) and four blocks of b_j words,
    integer i of a block at bits [i*b, (i+1)*b) of the block's words taken as
    one little-endian bit string.  Returns (metablocks as (offset, widths),
    the n//128*128 coded deltas, tail offset), read with Python integers."""
    buf = bytes(memoryview(buf))
    metas, deltas, pos = [], [], 0
    for _ in range(n // 128):
        widths = list(buf[pos:pos + 4])
        metas.append((pos, widths))
        off = pos + 4
        for b in widths:
            bits = int.from_bytes(buf[off:off + 4 * b], "little")
            deltas.extend((bits >> (i * b)) & ((1 << b) - 1) for i in range(32))
            off += 4 * b
        pos = off
    return metas, deltas, pos


def fastpfor_scalar_read(buf, n):
    """The scalar FastPFOR (Sec. 5, one-lane packing): rebuilds the coded
    values of every full block from the bytes with Python integers: the low
    parts as fields i*b of the block's bit string, each exception's high
    part as field q*d of its array's bit string, OR-ed in at its position."""
    buf = bytes(memoryview(buf))
    pages, tail = fastpfor_walk(buf, n, chunk=32)
    out = []
    for pg in pages:
        base = pg["offset"]
        arrays = {d: int.from_bytes(buf[off:off + 4 * d * ((cnt + 31) // 32)], "little")
                  for d, (cnt, off) in pg["arrays"].items()}
        cursor = {d: 0 for d in arrays}
        packed = base + 16
        for b, mb, pos_list in pg["records"]:
            bits = int.from_bytes(buf[packed:packed + 16 * b], "little")
            vals = [(bits >> (i * b)) & ((1 << b) - 1) for i in range(128)]
            packed += 16 * b
            if mb > b:
                d = mb - b
                for p in pos_list:
                    vals[p] |= ((arrays[d] >> (cursor[d] * d)) & ((1 << d) - 1)) << b
                    cursor[d] += 1
            out.extend(vals)
    return pages, out, tail


def simple8b_table(path):
    """(count, bits) per selector from the golden copy of the paper's table."""
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    return {int(r[0]): (int(r[1]), int(r[2])) for r in rows}


def simple8b_read(words, table):
    """Integers of a list of Simple-8b words, selector in bits 60..63."""
    out, sels = [], []
    for w in words:
        w = int(w)
        sel = w >> 60
        count, bits = table[sel]
        sels.append(sel)
        out.extend(0 if bits == 0 else (w >> (i * bits)) & ((1 << bits) - 1) for i in range(count))
    return out, sels


def simplepfor_read(buf, n, table):
    """SimplePFOR pages (scalar low parts, one Simple-8b stream of exception
    high parts per page): rebuilds every full block's coded values."""
    buf = bytes(memoryview(buf))
    nb = n // 128
    out, pages, pos = [], [], 0
    for p in range((nb + 511) // 512):
        k = min(512, nb - 512 * p)
        base = pos
        len_at = 4 * le32(buf, base)
        L = le32(buf, base + len_at)
        rec_at = base + len_at + 4
        q = rec_at + pad(L, 4)
        N, W = le32(buf, q), le32(buf, q + 4)
        woff = base + pad(q + 8 - base, 16)
        words = [int.from_bytes(buf[woff + 8 * i:woff + 8 * i + 8], "little") for i in range(W)]
        high, sels = simple8b_read(words, table)
        assert len(high) == N
        r, packed, e = 0, base + 16, 0
        for _ in range(k):
            b, mb = buf[rec_at + r], buf[rec_at + r + 1]
            r += 2
            bits = int.from_bytes(buf[packed:packed + 16 * b], "little")
            vals = [(bits >> (i * b)) & ((1 << b) - 1) for i in range(128)]
            packed += 16 * b
            if mb > b:
                c = buf[rec_at + r]
                for j in range(c):
                    vals[buf[rec_at + r + 1 + j]] |= high[e] << b
                    e += 1
                r += 1 + c
            out.extend(vals)
        end = base + pad(woff + 8 * W - base, 16)
        pages.append(dict(offset=base, N=N, W=W, words=words, sels=sels, high=high, size=end - base))
        pos = end
    return pages, out, pos


# -- values of the SIMD layouts, rebuilt from the bytes --------------------

def lane_bits(buf, off, words, lanes, lane):
    """The bit string of one lane of an interleaved block: word w of the lane
    sits at byte off + 4 * (lanes * w + lane), little endian; word w holds
    bits [32w, 32w + 32) of the lane's string."""
    out = 0
    for w in range(words):
        out |= le32(buf, off + 4 * (lanes * w + lane)) << (32 * w)
    return out


def vertical_values(buf, off, b, count=128):
    """Values 0..count-1 of a 4-lane vertical block of width b at `off`
    (Sec. 4, Figs. 6-7): value i is field i // 4 of lane i % 4."""
    if b == 0:
        return [0] * count
    words = (count // 4 * b + 31) // 32
    lanes = [lane_bits(buf, off, words, 4, l) for l in range(4)]
    mask = (1 << b) - 1
    return [(lanes[i % 4] >> ((i // 4) * b)) & mask for i in range(count)]


def vbyte_read(buf, pos, count):
    """Variable Byte (Sec. 2.4): 7 data bits per byte, low group first, high
    bit set on the last byte of each integer."""
    out = []
    for _ in range(count):
        v, shift = 0, 0
        while True:
            byte = buf[pos]
            pos += 1
            v |= (byte & 0x7F) << shift
            shift += 7
            if byte & 0x80:
                break
        out.append(v)
    return out, pos


def bp128_read(buf, n, layout):
    """SIMD-BP128 (layout 0, Sec. 6.2) or W32 (layout 1, R16): every coded
    delta of the stream, the n // 128 full blocks from the packed bits and the
    n % 128 last ones from the Variable Byte tail."""
    buf = bytes(memoryview(buf))
    metas, tail = bp128_walk(buf, n, layout)
    out = []
    for off, widths, size, k in metas:
        if layout == 0:
            q = off + 16
            for b in widths[:k]:
                out.extend(vertical_values(buf, q, b))
                q += 16 * b
        else:
            # lane j = 4g + l: block after block, the integers 16g + 4m + l
            # (m = 0..3) at width b_k, fields packed on from the previous block
            words = (size - 16) // 128
            lanes = [lane_bits(buf, off + 16, words, 32, j) for j in range(32)]
            bit = 0
            for b in widths[:k]:
                blk = [0] * 128
                mask = (1 << b) - 1
                for j in range(32):
                    g, l = divmod(j, 4)
                    for m in range(4):
                        blk[16 * g + 4 * m + l] = (lanes[j] >> (bit + m * b)) & mask
                out.extend(blk)
                bit += 4 * b
    rest, end = vbyte_read(buf, tail, n - 128 * (n // 128))
    return out + rest, end


def fastpfor_simd_read(buf, n):
    """SIMD-FastPFOR (Sec. 5, SIMD variant): every full block's coded values
    from the page bytes: the low parts in the vertical layout, the exception
    arrays as vertical blocks of 128 values (element q of array d is value
    q % 128 of the chunk q // 128, each chunk 16 * d bytes), OR-ed in at their
    positions in block order; the Variable Byte tail after the last page."""
    buf = bytes(memoryview(buf))
    pages, tail = fastpfor_walk(buf, n, chunk=128)
    out = []
    for pg in pages:
        base = pg["offset"]
        arrays = {}
        for d, (cnt, off) in pg["arrays"].items():
            vals = []
            for c in range((cnt + 127) // 128):
                vals.extend(vertical_values(buf, off + 16 * d * c, d))
            arrays[d] = vals[:cnt]
        cursor = {d: 0 for d in arrays}
        packed = base + 16
        for b, mb, pos_list in pg["records"]:
            vals = vertical_values(buf, packed, b)
            packed += 16 * b
            if mb > b:
                d = mb - b
                for p in pos_list:
                    vals[p] |= arrays[d][cursor[d]] << b
                    cursor[d] += 1
            out.extend(vals)
        for d in arrays:
            assert cursor[d] == len(arrays[d]), (d, cursor[d], len(arrays[d]))
    rest, end = vbyte_read(buf, tail, n - 128 * (n // 128))
    return pages, out + rest, end
