// SIMD-BP128 / W32 device building blocks shared by the single-array and the
// batched decoders: vertical unpacking of one block (Sec. 4, Fig. 7
// generalised to every width) and the checked unpack of one metablock
// (Sec. 6.2).
#pragma once

#include "icx_tile.cuh"

namespace icx {

constexpr int kMetaMax = 16 + 16 * 16 * 32;  // 8208: every width 32
constexpr int kBuf = kMetaMax + 128;         // slack for reading one row past
constexpr int kBp32UnitMax = 16 * (4 + 4 * 4 * 32);  // 8256: 16 BP32 metablocks at width 32
static_assert(kBp32UnitMax + 15 + 32 <= kBuf, "a BP32 unit, its 16-byte alignment and the read-past slack fit");

template <int FMT>
__device__ __forceinline__ uint4 unpack_block(const uint8_t* buf, uint32_t base_bytes, uint32_t bitbase,
                                              uint32_t b, int lane) {
    const uint32_t mask = width_mask(b);
    if (FMT == ICX_FMT_PAPER) {
        // Fig. 7 generalised: lane t extracts field t of each of the 4 lanes
        // (integers 4t..4t+3) from rows (t*b)/32 and the next one.
        const uint32_t bit = (uint32_t)lane * b;
        const uint4* rows = reinterpret_cast<const uint4*>(buf + base_bytes);
        const uint4 r0 = rows[bit >> 5], r1 = rows[(bit >> 5) + 1];
        const uint32_t s = bit & 31;
        return make_uint4(__funnelshift_r(r0.x, r1.x, s) & mask, __funnelshift_r(r0.y, r1.y, s) & mask,
                          __funnelshift_r(r0.z, r1.z, s) & mask, __funnelshift_r(r0.w, r1.w, s) & mask);
    } else {
        // W32: lane j's own column; fields m = 0..3 at bits bitbase + m*b.
        const uint32_t* col = reinterpret_cast<const uint32_t*>(buf + 16) + lane;
        uint32_t r[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const uint32_t bit = bitbase + (uint32_t)m * b;
            const uint32_t w = bit >> 5;
            r[m] = __funnelshift_r(col[32 * w], col[32 * (w + 1)], bit & 31) & mask;
        }
        return make_uint4(r[0], r[1], r[2], r[3]);
    }
}

// Width of block k from a metablock descriptor (byte k).
__device__ __forceinline__ uint32_t desc_width(const uint4& desc, int k) {
    return (comp(desc, k >> 2) >> (8 * (k & 3))) & 255u;
}

// Checks the metablock staged in `buf` (its `size` bytes, K blocks: every
// width <= 32 and the size the widths imply) and unpacks it into v (paper
// layout: row ownership; W32: residue ownership).  Returns false, with
// ECORRUPT recorded, if the check fails.
template <int FMT>
__device__ __forceinline__ bool bp128_unpack_unit(const uint8_t* buf, uint32_t size, uint32_t K, uint4 (&v)[16],
                                                  WsHeader* h, int lane) {
    const uint4 desc = *reinterpret_cast<const uint4*>(buf);
    uint32_t sum = 0, maxw = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const uint32_t b = ((uint32_t)k < K) ? desc_width(desc, k) : 0u;
        sum += b;
        maxw = max(maxw, b);
    }
    const uint32_t want = FMT == ICX_FMT_PAPER ? 16 + 16 * sum : 16 + 128 * ((4 * sum + 31) / 32);
    if (maxw > 32 || want != size) {
        if (lane == 0) set_error(h, ICX_ECORRUPT);
        return false;
    }
    uint32_t base = 16, bitbase = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        if ((uint32_t)k < K) {
            const uint32_t b = desc_width(desc, k);
            v[k] = unpack_block<FMT>(buf, base, bitbase, b, lane);
            base += 16 * b;
            bitbase += 4 * b;
        }
    }
    return true;
}

// BP32 (Sec. 6.2; R20): checks and unpacks the K metablocks of 128
// integers staged at `p` (4-byte aligned, `size` bytes).  Metablock k is a
// descriptor word (byte j = width of 32-integer block j) and blocks of b_j
// words packed LSB-first in one lane.  Lane t takes integers 4(t%8)..+3 of
// block t/8, which are integers 4t..4t+3 of the metablock: row ownership,
// as for the paper layout.  Returns false, with ECORRUPT recorded, if a
// width exceeds 32 or the widths do not add up to `size`.
__device__ __forceinline__ bool bp32_unpack_unit(const uint8_t* p, uint32_t size, uint32_t K, uint4 (&v)[16],
                                                 WsHeader* h, int lane) {
    const uint32_t* w32 = reinterpret_cast<const uint32_t*>(p);
    const uint32_t j = (uint32_t)lane >> 3, i0 = 4 * ((uint32_t)lane & 7);
    uint32_t off = 0;  // words
    bool bad = false;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        if ((uint32_t)k < K) {
            const uint32_t desc = off < size / 4 ? w32[off] : 0xFFFFFFFFu;
            const uint32_t b0 = desc & 255u, b1 = (desc >> 8) & 255u, b2 = (desc >> 16) & 255u, b3 = desc >> 24;
            bad = bad || b0 > 32 || b1 > 32 || b2 > 32 || b3 > 32;
            const uint32_t b = bad ? 0u : j == 0 ? b0 : j == 1 ? b1 : j == 2 ? b2 : b3;
            const uint32_t start = off + 1 + (j > 0 ? b0 : 0u) + (j > 1 ? b1 : 0u) + (j > 2 ? b2 : 0u);
            const uint32_t mask = width_mask(b);
            uint32_t r[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const uint32_t bit = (i0 + c) * b, w = start + (bit >> 5);
                r[c] = w + 1 < size / 4 + 8 ? __funnelshift_r(w32[w], w32[w + 1], bit & 31) & mask : 0u;
            }
            v[k] = make_uint4(r[0], r[1], r[2], r[3]);
            off += bad ? 0u : 1 + b0 + b1 + b2 + b3;
        }
    }
    if (bad || 4 * off != size) {
        if (lane == 0) set_error(h, ICX_ECORRUPT);
        return false;
    }
    return true;
}

}  // namespace icx
