// The tile epilogue shared by the decoders: a CTA of kWarps warps decodes
// kWarps consecutive units of up to 16 blocks (2048 integers, 64 per lane in
// registers), then
//   1. each warp scans its unit locally (differential decoding, Sec. 3),
//   2. warp 0 scans the kWarps unit aggregates and runs one decoupled
//      look-back for the whole tile to get the carry-in,
//   3. every warp adds its prefix and stores with 128-bit stores.
#pragma once

#include "icx_device.cuh"

namespace icx {

constexpr int kWarps = 8;     // default warps per CTA
constexpr int kMaxWarps = 16;

// Shared state of a CTA tile (sized for the largest CTA).
struct TileShared {
    uint4 agg[kMaxWarps];
    uint4 pref[kMaxWarps];
    uint32_t tile;
    uint32_t next;
    uint32_t nx[2];  // next tile id, double-buffered by iteration parity
};

// Local scan of a unit held in row ownership (lane t: integers 128k + 4t..+3
// of block k in v[k]); `residue` means the values arrive in W32 residue
// ownership and are moved to row ownership here.  Returns the unit aggregate
// (stride 1: .x; stride 4: one per residue).
constexpr int kScanGroup = 8;  // blocks whose stride-1 scans are interleaved (8 or 16 measure the same)

template <int DELTA>
__device__ __forceinline__ uint4 unit_local_scan(uint4 (&v)[16], uint32_t K, bool residue, int lane) {
    // The 16 blocks' scans are independent except for the carry between
    // blocks, so every step runs across all blocks before the next step
    // (16 independent shuffles in flight instead of one dependent chain).
    uint4 agg = make_uint4(0, 0, 0, 0);
    if (DELTA == ICX_DELTA_4 && residue) {
        // W32 residue ownership: serial over m, then a 3-step scan over the
        // 8 groups, then the block carries, then back to row ownership.
        uint32_t incl[16], tot[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            v[k].y += v[k].x;
            v[k].z += v[k].y;
            v[k].w += v[k].z;
            incl[k] = v[k].w;
        }
#pragma unroll
        for (int off = 4; off < 32; off <<= 1) {
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const uint32_t y = __shfl_up_sync(FULL, incl[k], off);
                if (lane >= off) incl[k] += y;
            }
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) tot[k] = __shfl_sync(FULL, incl[k], 28 + (lane & 3));
        uint32_t carry = 0;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const uint32_t add = carry + incl[k] - v[k].w;
            v[k] = make_uint4(v[k].x + add, v[k].y + add, v[k].z + add, v[k].w + add);
            if ((uint32_t)k < K) carry += tot[k];
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = residue_to_row(v[k], lane);
        agg.x = __shfl_sync(FULL, carry, 0);
        agg.y = __shfl_sync(FULL, carry, 1);
        agg.z = __shfl_sync(FULL, carry, 2);
        agg.w = __shfl_sync(FULL, carry, 3);
        return agg;
    }
    if (residue) {
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = residue_to_row(v[k], lane);
    }
    if (DELTA == ICX_DELTA_1) {
        // two groups of 8 blocks, each with its 8 scans interleaved step by
        // step: enough independent shuffles in flight, half the temporaries
        uint32_t carry = 0;
#pragma unroll
        for (int g = 0; g < 16; g += kScanGroup) {
            uint32_t incl[kScanGroup];
#pragma unroll
            for (int i = 0; i < kScanGroup; ++i) {
                uint4& x = v[g + i];
                x.y += x.x;
                x.z += x.y;
                x.w += x.z;
                incl[i] = x.w;
            }
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
#pragma unroll
                for (int i = 0; i < kScanGroup; ++i) {
                    const uint32_t y = __shfl_up_sync(FULL, incl[i], off);
                    if (lane >= off) incl[i] += y;
                }
            }
#pragma unroll
            for (int i = 0; i < kScanGroup; ++i) {
                const uint32_t tot = __shfl_sync(FULL, incl[i], 31);
                uint4& x = v[g + i];
                const uint32_t add = carry + incl[i] - x.w;
                x = make_uint4(x.x + add, x.y + add, x.z + add, x.w + add);
                carry += tot;
            }
        }
        agg.x = carry;
    } else if (DELTA == ICX_DELTA_4) {
        uint4 carry = make_uint4(0, 0, 0, 0);
#pragma unroll
        for (int k = 0; k < 16; ++k)
            if ((uint32_t)k < K) v[k] = row_scan_d4(v[k], carry, lane);
        agg = carry;
    }
    return agg;
}

// Aggregate of a unit straight after unpacking (before its local scan):
// stride 1: the sum of all its deltas in .x; stride 4: one sum per residue
// mod 4.  In row ownership (lane t: integers 4t..4t+3 of every block)
// component c is residue c; in W32 residue ownership lane j holds residue
// j & 3 in all four components.
template <int DELTA>
__device__ __forceinline__ uint4 unit_sum(const uint4 (&v)[16], bool residue) {
    if constexpr (DELTA == ICX_DELTA_NONE) {
        return make_uint4(0, 0, 0, 0);
    } else {
        uint4 s = v[0];
#pragma unroll
        for (int k = 1; k < 16; ++k) s = add4(s, v[k]);
        uint32_t t = s.x + s.y + s.z + s.w;
        if constexpr (DELTA == ICX_DELTA_1) {
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) t += __shfl_xor_sync(FULL, t, off);
            return make_uint4(t, 0, 0, 0);
        } else {
            if (residue) {
#pragma unroll
                for (int off = 16; off >= 4; off >>= 1) t += __shfl_xor_sync(FULL, t, off);
                return make_uint4(__shfl_sync(FULL, t, 0), __shfl_sync(FULL, t, 1), __shfl_sync(FULL, t, 2),
                                  __shfl_sync(FULL, t, 3));
            }
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) {
                s.x += __shfl_xor_sync(FULL, s.x, off);
                s.y += __shfl_xor_sync(FULL, s.y, off);
                s.z += __shfl_xor_sync(FULL, s.z, off);
                s.w += __shfl_xor_sync(FULL, s.w, off);
            }
            return s;
        }
    }
}

// Warp 0 of a tile: inclusive scan of the W unit aggregates in S.agg (lane i
// < W gets unit i), returning the lane's own aggregate in `mine`.
template <int W>
__device__ __forceinline__ uint4 tile_agg_scan(const TileShared& S, uint4& mine, int lane) {
    mine = lane < W ? S.agg[lane] : make_uint4(0, 0, 0, 0);
    uint4 incl = mine;
#pragma unroll
    for (int off = 1; off < W; off <<= 1) {
        const uint4 y = make_uint4(__shfl_up_sync(FULL, incl.x, off), __shfl_up_sync(FULL, incl.y, off),
                                   __shfl_up_sync(FULL, incl.z, off), __shfl_up_sync(FULL, incl.w, off));
        if (lane >= off) incl = add4(incl, y);
    }
    return incl;
}

// Stride-4 scan of a whole unit in row ownership through an 8 KB shared
// scratch (the warp's staging buffer, free after unpacking): the 16 x 32 x 4
// values are written in position order, each lane then owns two columns
// (block k = lane/2, residues 2*(lane&1) and +1): one pass down the 32 rows
// sums them, one shuffle scan over the blocks gives the column carries, a
// second pass writes the running sums back in place, and the values are read
// back in row ownership.  Word (k, t, c) lives at
// 128k + 4(t ^ (k & 7)) + c, which keeps both the 128-bit row accesses and
// the 64-bit column accesses free of bank conflicts.  Returns the unit's
// four residue aggregates.
__device__ __forceinline__ uint4 unit_scan_d4_smem(uint4 (&v)[16], uint32_t* scratch, int lane) {
#pragma unroll
    for (int k = 0; k < 16; ++k)
        *reinterpret_cast<uint4*>(scratch + 128 * k + 4 * (lane ^ (k & 7))) = v[k];
    __syncwarp();
    const int k = lane >> 1, c0 = 2 * (lane & 1);
    uint32_t* col = scratch + 128 * k + c0;
    // pass 1: the two column totals
    uint32_t sx = 0, sy = 0;
#pragma unroll
    for (int t = 0; t < 32; ++t) {
        const uint2 e = *reinterpret_cast<const uint2*>(col + 4 * (t ^ (k & 7)));
        sx += e.x;
        sy += e.y;
    }
    // carries of the earlier blocks: exclusive scan over k (lanes of one parity)
    uint32_t ix = sx, iy = sy;
#pragma unroll
    for (int off = 2; off < 32; off <<= 1) {
        const uint32_t a = __shfl_up_sync(FULL, ix, off), b = __shfl_up_sync(FULL, iy, off);
        if (lane >= off) {
            ix += a;
            iy += b;
        }
    }
    // pass 2: running sums written back in place (no register copy of the columns)
    uint32_t rx = ix - sx, ry = iy - sy;
#pragma unroll
    for (int t = 0; t < 32; ++t) {
        uint2* p = reinterpret_cast<uint2*>(col + 4 * (t ^ (k & 7)));
        const uint2 e = *p;
        rx += e.x;
        ry += e.y;
        *p = make_uint2(rx, ry);
    }
    __syncwarp();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk)
        v[kk] = *reinterpret_cast<const uint4*>(scratch + 128 * kk + 4 * (lane ^ (kk & 7)));
    const uint4 agg = make_uint4(__shfl_sync(FULL, ix, 30), __shfl_sync(FULL, iy, 30), __shfl_sync(FULL, ix, 31),
                                 __shfl_sync(FULL, iy, 31));
    __syncwarp();
    return agg;
}

// CTA-wide: exclusive prefix of this warp's unit (tile carry-in from the
// look-back plus the aggregates of the tile's earlier units).  Contains two
// __syncthreads; every thread of the CTA must call it.
template <int DELTA, int W = kWarps>
__device__ __forceinline__ uint4 tile_prefix(TileShared& S, uint4 agg, uint32_t tile, uint32_t epoch, WsHeader* h,
                                             int warp, int lane) {
    if (DELTA == ICX_DELTA_NONE) return make_uint4(0, 0, 0, 0);
    if (lane == 0) S.agg[warp] = agg;
    __syncthreads();
    if (warp == 0) {
        const uint4 mine = lane < W ? S.agg[lane] : make_uint4(0, 0, 0, 0);
        uint4 incl = mine;
#pragma unroll
        for (int off = 1; off < W; off <<= 1) {
            uint4 y = make_uint4(__shfl_up_sync(FULL, incl.x, off), __shfl_up_sync(FULL, incl.y, off),
                                 __shfl_up_sync(FULL, incl.z, off), __shfl_up_sync(FULL, incl.w, off));
            if (lane >= off) incl = add4(incl, y);
        }
        const uint4 total = shfl4(incl, W - 1);
        const uint4 base = DELTA == ICX_DELTA_1 ? lookback<1>(h, epoch, tile, total)
                                                : lookback<4>(h, epoch, tile, total);
        if (lane < W) S.pref[lane] = add4(base, sub4(incl, mine));
    }
    __syncthreads();
    uint4 pref = S.pref[warp];
    if (DELTA == ICX_DELTA_1) pref = make_uint4(pref.x, pref.x, pref.x, pref.x);
    return pref;
}

// Stores blocks 0..K-1 of a unit whose first integer is `first`; integers at
// or beyond n are dropped (the Variable Byte tail unit).
__device__ __forceinline__ void store_unit(uint32_t* __restrict__ out, size_t first, size_t n, const uint4 (&v)[16],
                                           uint32_t K, uint4 pref, int lane) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        if ((uint32_t)k < K) {
            const size_t p = first + 128 * (size_t)k + 4 * (size_t)lane;
            const uint4 r = add4(v[k], pref);
            if (p + 4 <= n) {
                // streaming (evict-first): the output passes through L2 without
                // pushing out the input prefetched there one grid ahead
                __stcs(reinterpret_cast<uint4*>(out + p), r);
            } else {
                for (int c = 0; c < 4; ++c)
                    if (p + c < n) out[p + c] = comp(r, c);
            }
        }
    }
}

// Grabs the next tile id for the CTA (thread 0), broadcast through S.tile.
__device__ __forceinline__ uint32_t next_tile(TileShared& S, WsHeader* h) {
    if (threadIdx.x == 0) S.tile = atomicAdd(&h->tile_counter, 1u);
    __syncthreads();
    return S.tile;
}

// ----------------------------------------------------------- tail (VByte)

// Warp-parallel Variable Byte decoder (Sec. 2.4): 32 bytes per step; a
// ballot of the terminating bytes gives every byte its integer and its group
// position.  Decodes `count` (<= 127) integers starting at in[start] into
// vals[0..127] (zero-filled).  Returns false (and records ECORRUPT) on a
// truncated stream or an integer above 32 bits / 5 bytes.
__device__ __forceinline__ bool vbyte_decode_warp(const uint8_t* __restrict__ in, size_t start, size_t in_bytes,
                                  uint32_t count, uint32_t* vals, WsHeader* h) {
    const int lane = threadIdx.x & 31;
    for (int i = lane; i < 128; i += 32) vals[i] = 0;
    __syncwarp();
    uint32_t k0 = 0, carry = 0;
    size_t pos = start;
    bool bad = false;
    while (k0 < count) {
        const size_t p = pos + lane;
        const bool have = p < in_bytes;
        const uint32_t byte = have ? in[p] : 0u;
        const unsigned have_mask = __ballot_sync(FULL, have);
        const unsigned term = __ballot_sync(FULL, have && (byte & 0x80u));
        const unsigned before = term & ((1u << lane) - 1u);
        const uint32_t idx = k0 + __popc(before);
        const uint32_t posin = before ? (uint32_t)(lane - (31 - __clz(before)) - 1) : carry + lane;
        if (have && idx < count) {
            if (posin > 4 || (posin == 4 && (byte & 0x70u)))
                bad = true;
            else
                atomicOr(&vals[idx], (byte & 0x7Fu) << (7 * posin));
        }
        k0 += __popc(term);
        carry = term ? (uint32_t)(__clz(term)) : carry + 32;
        pos += 32;
        if (have_mask != FULL) {
            if (k0 < count) bad = true;
            break;
        }
    }
    bad = __any_sync(FULL, bad);
    if (bad && lane == 0) set_error(h, ICX_ECORRUPT);
    __syncwarp();
    return !bad;
}


// Decodes the Variable Byte tail (count <= 127 integers at in[start]) into
// row ownership of block 0 (scratch: 128 words of shared memory).
__device__ __forceinline__ void tail_unit(const uint8_t* __restrict__ in, size_t in_bytes, uint64_t start,
                                          uint32_t count, uint32_t* scratch, uint4 (&v)[16], WsHeader* h, int lane) {
    if (start <= in_bytes && vbyte_decode_warp(in, start, in_bytes, count, scratch, h))
        v[0] = *reinterpret_cast<const uint4*>(scratch + 4 * lane);
    else if (start > in_bytes && lane == 0)
        set_error(h, ICX_ECORRUPT);
    __syncwarp();
}

}  // namespace icx
