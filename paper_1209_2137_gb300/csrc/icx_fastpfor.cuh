// SIMD-FastPFOR device building blocks shared by the single-array and the
// batched decoders: the page parse (byte array records -> fixed block
// records) and the unpack + exception patch of one unit of 16 blocks
// (Sec. 5).
#pragma once

#include "icx_tile.cuh"

namespace icx {

constexpr uint32_t kBlocksPerPage = 512;
constexpr uint32_t kUnitsPerPage = kBlocksPerPage / 16;
constexpr int kUnitMax = 16 * 16 * 32;  // packed bytes of 16 blocks at width 32
constexpr int kExScratch = 16 * 128;    // owner block of each exception of a unit (bytes)
constexpr int kExScratchBytes = kExScratch + 32;  // then 16 x uint16 exceptions-before-block
constexpr int kFBuf = kUnitMax + 128;

__device__ __forceinline__ uint32_t ld32(const uint8_t* p) { return __ldg(reinterpret_cast<const uint32_t*>(p)); }
__host__ __device__ __forceinline__ size_t pad_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// ------------------------------------------------------------ page parse
//
// One CTA per page.  The page's byte array holds one record per block: b,
// maxbits and, when maxbits > b, the exception count c followed by c
// positions (Sec. 5).  A record's length follows from its own first three
// bytes only, so the record starts form a chain.  For a window of the array
// the CTA tabulates, at every byte position, the length of a record starting
// there (J1) and, by doubling, the bytes spanned by 2, 4 and 8 consecutive
// records (J8); one thread follows the chain 8 records per step, then every
// thread expands the starts of the 8 records of one step.  Offsets of the
// packed low bits, exception cursors and all checks are then scans over the
// blocks.

constexpr int kMetaThreads = 128;
constexpr uint32_t kMetaWin = 4096;             // chain positions per window
constexpr uint32_t kMetaSpan = kMetaWin + 1024;  // bytes held per window
constexpr uint32_t kRecMax = 132;  // longest record the chain follows (c > 128 is corrupt anyway)
constexpr uint32_t kGroups = kBlocksPerPage / 8;

// 30 KB, so that 7 CTAs fit an SM and a 2^26-integer stream's 1,024 pages
// are parsed at once on 152 SMs.
struct MetaSmem {
    uint32_t bytes[kMetaSpan / 4 + 4];  // window of the byte array (zero past its end)
    uint16_t ja[kMetaSpan];             // J2, then J8
    uint16_t jb[kMetaSpan];             // J4
    uint32_t grp[kGroups];              // start of records 8g .. 8g+7
    uint32_t start[kBlocksPerPage];     // record starts
    uint32_t bmc[kBlocksPerPage];       // b | maxbits << 8 | c << 16
    uint2 urng[kUnitsPerPage];          // per unit: packed offset of its first block, end of its last
    uint32_t wcnt[kMetaThreads / 32][32];  // per warp, exceptions per width
    uint32_t wpk[kMetaThreads / 32];       // per warp, sum of b
    uint32_t ctl[4];                       // window start, next group, chain state
    uint32_t uexc[kUnitsPerPage];          // SimplePFOR: per unit, page index of its first exception
    uint32_t s8[4];                        // SimplePFOR: words offset, word count, chunk carry
};

// SimplePFOR (Sec. 5): a page's exception high parts form one Simple-8b
// stream (Table 2: per selector, integers per 64-bit word and their width;
// the selector in bits 60..63, integer i at bits [i*b, (i+1)*b)).
constexpr int kSimple = ICX_FMT_SIMPLE8B;  // LAYOUT value of SimplePFOR in these templates
__device__ __forceinline__ uint32_t s8_count(uint32_t sel) {
    // 240 120 60 30 20 15 12 10 8 7 6 5 4 3 2 1
    return sel < 2 ? 240u >> sel : sel < 4 ? 60u >> (sel - 2) : sel < 6 ? 20u - 5u * (sel - 4) :
           sel < 8 ? 12u - 2u * (sel - 6) : sel <= 15 ? 16u - sel : 0u;
}
__device__ __forceinline__ uint32_t s8_bits(uint32_t sel) {
    // 0 0 1 2 3 4 5 6 7 8 10 12 15 20 30 60
    return sel < 2 ? 0u : sel < 10 ? sel - 1 : sel == 10 ? 10u : sel == 11 ? 12u : sel == 12 ? 15u :
           sel == 13 ? 20u : sel == 14 ? 30u : 60u;
}

__device__ __forceinline__ uint32_t rec_len(uint32_t b, uint32_t mb, uint32_t c) {
    return mb > b ? 3u + min(c, 129u) : 2u;
}

// Length of the record that would start at byte i of the staged window.
__device__ __forceinline__ uint32_t rec_len_at(const uint32_t* bytes, uint32_t i) {
    const uint32_t x = __funnelshift_r(bytes[i >> 2], bytes[(i >> 2) + 1], 8 * (i & 3));
    return rec_len(x & 0xFF, (x >> 8) & 0xFF, (x >> 16) & 0xFF);
}

// Bytes of an exception array of nd values of width d: SIMD-FastPFOR packs
// chunks of 128 in 4 lanes (16d bytes each), the scalar FastPFOR groups of
// 32 in one lane (4d bytes each).
template <int LAYOUT>
__device__ __forceinline__ uint64_t array_bytes(uint32_t d, uint32_t nd) {
    return LAYOUT == ICX_FMT_SCALAR ? 4 * (uint64_t)d * ((nd + 31) / 32) : 16 * (uint64_t)d * ((nd + 127) / 128);
}

// Whole warp: the exception arrays after a page's byte array.  Their offsets
// follow from the page's per-width counts (lane d-1 holds cnt_total of
// width d): after the bitset, each present width d has its stored count and
// then, from the next 16-byte boundary, its array of s_d bytes; the next
// count follows the array directly.  So array starts advance by
// pad16(s_d + 4) from the first (one warp scan), and a count sits s bytes
// past the previous present width's array (the first right after the
// bitset).  Lane d-1 checks the stored count of array d against its total,
// and the arrays must end exactly at the page end.  Writes the page record
// pg (array offsets, then the flag word) and returns the warp-uniform `bad`.
template <int LAYOUT>
__device__ __forceinline__ bool page_arrays(const uint8_t* page, uint32_t psize, uint32_t bytes_at, uint32_t Lpad,
                                            uint32_t cnt_total, bool bad, uint32_t* __restrict__ pg, WsHeader* h,
                                            int lane) {
    uint32_t my_off = 0, my_cnt_at = 0;
    bool present = false;
    if (!bad) {
        const uint32_t bitset = ld32(page + bytes_at + Lpad);
        present = (bitset >> lane) & 1u;
        if (!present && cnt_total) bad = true;
        const uint32_t sz = present ? (uint32_t)array_bytes<LAYOUT>(lane + 1, cnt_total) : 0u;
        const uint32_t step = present ? (uint32_t)pad_up(sz + 4, 16) : 0u;
        const uint32_t incl = warp_incl_scan(step, lane);
        const uint32_t q0 = bytes_at + Lpad + 4;           // the first stored count
        const uint32_t a0 = (uint32_t)pad_up(q0 + 4, 16);  // the first array
        my_off = a0 + incl - step;
        // the present width before this lane's: its array's end is this count
        const unsigned below = __ballot_sync(FULL, present) & ((1u << lane) - 1u);
        const int prev = below ? 31 - __clz(below) : 0;
        const uint32_t prev_end = __shfl_sync(FULL, my_off + sz, prev);
        my_cnt_at = below ? prev_end : q0;
        const unsigned all = __ballot_sync(FULL, present);
        const uint64_t q_end = all ? (uint64_t)__shfl_sync(FULL, my_off + sz, 31 - __clz(all)) : (uint64_t)q0;
        if (q_end > psize || pad_up(q_end, 16) != psize) bad = true;
    }
    bad = __any_sync(FULL, bad);
    if (!bad && present && ld32(page + my_cnt_at) != cnt_total) bad = true;
    bad = __any_sync(FULL, bad);
    pg[lane] = bad || !present ? 0u : my_off;
    if (lane == 0) pg[32] = bad ? 1u : 0u;
    if (bad && lane == 0) set_error(h, ICX_ECORRUPT);
    return bad;
}

// Whole warp, SimplePFOR: after the byte array a word N (high parts) and a
// word W (Simple-8b words), then the words from the next 16-byte boundary to
// the page end.  Checks N against the records' total (lane 0's cnt_total),
// the sizes against the page, and writes pg[32] (flag), pg[33] (page offset
// of the words), pg[34] (W); pg[0..31] (each unit's first word) are filled
// by the caller.  Returns the warp-uniform `bad`.
__device__ __forceinline__ bool simple_stream(const uint8_t* page, uint32_t psize, uint32_t bytes_at, uint32_t Lpad,
                                              uint32_t cnt_total, bool bad, uint32_t* __restrict__ pg,
                                              uint32_t& woff, uint32_t& W, WsHeader* h, int lane) {
    woff = 0;
    W = 0;
    if (!bad) {
        const uint64_t q = (uint64_t)bytes_at + Lpad;
        if (q + 8 > psize) {
            bad = true;
        } else {
            const uint32_t N = ld32(page + q);
            W = ld32(page + q + 4);
            woff = (uint32_t)pad_up(q + 8, 16);
            const uint64_t wend = (uint64_t)woff + 8 * (uint64_t)W;
            bad = N != __shfl_sync(FULL, cnt_total, 0) || wend > psize || pad_up(wend, 16) != psize;
        }
    }
    bad = __any_sync(FULL, bad);
    pg[lane] = 0xFFFFFFFFu;
    if (lane == 0) {
        pg[32] = bad ? 1u : 0u;
        pg[33] = bad ? 0u : woff;
        pg[34] = bad ? 0u : W;
        if (bad) set_error(h, ICX_ECORRUPT);
    }
    return bad;
}

// Exclusive count, per block, of the earlier exceptions of the same width d
// within one warp round (lane = block; d = 0: no exceptions), added to
// `base` = the lane-(d-1) running count before the round; lane d-1 of `cnt`
// then advances by the round's total of width d.  Width by width (the
// distinct widths of a round are few).
__device__ __forceinline__ uint32_t round_cursor(uint32_t d, uint32_t c, uint32_t& cnt, int lane) {
    uint32_t within = __shfl_sync(FULL, cnt, d ? (d - 1) & 31 : 0);
    uint32_t pend = __ballot_sync(FULL, d != 0 && d <= 32);
    while (pend) {
        const uint32_t dl = __shfl_sync(FULL, d, __ffs(pend) - 1);
        const bool mine = d == dl;
        const uint32_t x = mine ? c : 0u;
        const uint32_t sc = warp_incl_scan(x, lane);
        if (mine) within += sc - x;
        const uint32_t tot = __shfl_sync(FULL, sc, 31);
        if ((uint32_t)lane == dl - 1) cnt += tot;
        pend &= ~__ballot_sync(FULL, mine);
    }
    return within;
}

// Parses one page, CTA-wide (kMetaThreads threads): the page occupies
// in[base, end) and holds K blocks; writes the K block records to pm, the
// exception-array offsets and the page flag to pg, and per unit of 16
// blocks its packed range to um.  Returns true (in every thread) when the
// page is corrupt.
template <int LAYOUT = ICX_FMT_PAPER>
__device__ __forceinline__ bool parse_page(MetaSmem& S, const uint8_t* __restrict__ in, size_t in_bytes,
                                           uint64_t base, uint64_t end, uint32_t K, BlockMeta* __restrict__ pm,
                                           uint32_t* __restrict__ pg, uint2* __restrict__ um, WsHeader* h,
                                           ulonglong2* __restrict__ rng = nullptr) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint8_t* sb = reinterpret_cast<const uint8_t*>(S.bytes);
    const uint32_t G = (K + 7) / 8;

    bool bad = !(base <= end && end <= in_bytes && (base & 15) == 0 && end - base >= 16);
    const uint8_t* page = in + base;
    const uint32_t psize = bad ? 0u : (uint32_t)min(end - base, (uint64_t)0xFFFFFFF0u);
    uint32_t len_at = 0, L = 0, bytes_at = 0;
    if (!bad) {
        len_at = 4 * ld32(page);
        bad = len_at < 16 || (len_at & 15) || (uint64_t)len_at + 4 > psize;
    }
    if (!bad) {
        L = ld32(page + len_at);
        bytes_at = len_at + 4;
        bad = (uint64_t)bytes_at + pad_up(L, 4) + 4 > psize;
    }
    const uint32_t Lpad = bad ? 0u : (uint32_t)pad_up(L, 4);
    const uint32_t* arr = reinterpret_cast<const uint32_t*>(page + bytes_at);  // 4-byte aligned
    // what follows the byte array (bitset, counts, exception arrays) is read
    // only at the end of the parse: start pulling it into L2 now
    if (!bad && tid == 0) {
        const uint32_t a0 = (bytes_at + Lpad) & ~15u;
        const uint32_t nbytes = min(psize - a0, 65536u) & ~15u;
        if (nbytes) prefetch_l2(page + a0, nbytes);
    }

    // ---- record starts, one window of the byte array at a time
    if (LAYOUT == kSimple && tid < (int)kUnitsPerPage) S.uexc[tid] = 0xFFFFFFFFu;
    if (tid == 0) {
        S.ctl[0] = 0;  // window start
        S.ctl[1] = 0;  // next group
        S.ctl[2] = 0;  // next record start
        S.ctl[3] = 0;  // chain left the array
    }
    __syncthreads();
    uint32_t g0 = 0;
    while (!bad) {
        const uint32_t ws = S.ctl[0];
        g0 = S.ctl[1];
        if (g0 >= G || S.ctl[3]) break;
        const uint32_t Lw = L - ws;  // > 0: the chain only continues at starts < L
        const uint32_t lim8 = min(kMetaWin, Lw), lim4 = lim8 + 4 * kRecMax, lim2 = lim4 + 2 * kRecMax;
        const uint32_t nw = ws < Lpad ? min(kMetaSpan / 4, (Lpad - ws) / 4) : 0u;
#pragma unroll 4
        for (uint32_t i = tid; i < kMetaSpan / 4 + 4; i += kMetaThreads) S.bytes[i] = i < nw ? __ldg(arr + ws / 4 + i) : 0u;
        __syncthreads();
        // J2 straight from the bytes (i + a + 3 <= lim2 + kRecMax + 2 stays
        // inside the window's words)
#pragma unroll 4
        for (uint32_t i = tid; i < lim2; i += kMetaThreads) {
            const uint32_t a = rec_len_at(S.bytes, i);
            S.ja[i] = (uint16_t)(a + rec_len_at(S.bytes, i + a));
        }
        __syncthreads();
#pragma unroll 4
        for (uint32_t i = tid; i < lim4; i += kMetaThreads) {
            const uint32_t a = S.ja[i];
            S.jb[i] = (uint16_t)(a + S.ja[i + a]);
        }
        __syncthreads();
#pragma unroll 4
        for (uint32_t i = tid; i < lim8; i += kMetaThreads) {
            const uint32_t a = S.jb[i];
            S.ja[i] = (uint16_t)(a + S.jb[i + a]);
        }
        __syncthreads();
        if (tid == 0) {
            uint32_t g = g0, r = S.ctl[2];
            bool off = false;
            while (g < G) {
                if (r >= L) {  // a record would start past the array
                    off = true;
                    break;
                }
                if (r - ws >= kMetaWin) break;  // continue in the next window
                S.grp[g] = r;
                ++g;
                if (g < G) r += S.ja[r - ws];
            }
            S.ctl[0] = r & ~3u;
            S.ctl[1] = g;
            S.ctl[2] = r;
            S.ctl[3] = off;
        }
        __syncthreads();
        // expand the groups found in this window
        for (uint32_t g = g0 + tid; g < S.ctl[1]; g += kMetaThreads) {
            uint32_t q = S.grp[g] - ws;
            const uint32_t k1 = min(K, 8 * g + 8);
            for (uint32_t k = 8 * g; k < k1; ++k) {
                const uint32_t b = sb[q], mb = sb[q + 1], c = sb[q + 2];
                S.start[k] = ws + q;
                S.bmc[k] = b | mb << 8 | c << 16;
                q += rec_len(b, mb, c);
            }
        }
        __syncthreads();
    }
    bad = bad || S.ctl[1] < G || S.ctl[3];

    // ---- per block: checks, packed offsets, exception cursors
    // warp w takes blocks 128w .. 128w+127 in four rounds of 32
    uint32_t cnt = 0;  // lane l: this warp's exceptions of width l+1 so far
    uint32_t b_[4], d_[4], c_[4], cur[4], pk[4];
    uint32_t run = 0;  // this warp's sum of b so far
    bool rbad = false;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint32_t k = 128 * warp + 32 * i + lane;
        const bool valid = !bad && k < K;
        uint32_t b = 0, mb = 0, c = 0, st = 0;
        if (valid) {
            const uint32_t x = S.bmc[k];
            b = x & 0xFF;
            mb = (x >> 8) & 0xFF;
            c = x >> 16;
            st = S.start[k];
        }
        const uint32_t d = mb > b ? mb - b : 0u;
        if (!d) c = 0;
        if (valid && (b > 32 || mb > 32 || mb < b || c > 128 || (uint64_t)st + (d ? 3 + c : 2) > L)) rbad = true;
        const uint32_t bb = b <= 32 ? b : 0u;
        const uint32_t incl = warp_incl_scan(bb, lane);
        pk[i] = run + incl - bb;
        run += __shfl_sync(FULL, incl, 31);
        // SimplePFOR: one stream for all widths, so one running count
        const uint32_t within = round_cursor(LAYOUT == kSimple ? (d ? 1u : 0u) : d, c, cnt, lane);
        b_[i] = bb;
        d_[i] = d;
        c_[i] = c;
        cur[i] = within;
    }
    S.wcnt[warp][lane] = cnt;
    if (lane == 0) S.wpk[warp] = run;
    bad = __syncthreads_or(bad || rbad) != 0;
    uint32_t pk_base = 0, cnt_total = 0;
    for (int w = 0; w < kMetaThreads / 32; ++w) {
        if (w < warp) pk_base += S.wpk[w];
        cnt_total += S.wcnt[w][lane];
    }
    uint32_t packed_total = 0;
    for (int w = 0; w < kMetaThreads / 32; ++w) packed_total += S.wpk[w];
    if (!bad && 16 + 16 * packed_total != len_at) bad = true;  // b <= 32, K <= 512: no overflow
    if (!bad) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint32_t k = 128 * warp + 32 * i + lane;
            if (k < K) {
                const uint32_t d = d_[i];
                uint32_t cbase = 0;
                const int cls = LAYOUT == kSimple ? 0 : (d ? (int)d - 1 : 0);
                for (int w = 0; w < warp; ++w) cbase += S.wcnt[w][cls];
                BlockMeta m;
                m.packed_off = 16 + 16 * (pk_base + pk[i]);
                m.pos_off = d ? bytes_at + S.start[k] + 3 : 0u;
                m.cursor = d ? cbase + cur[i] : 0u;
                m.b = (uint8_t)b_[i];
                m.d = (uint8_t)d;
                m.c = (uint8_t)c_[i];
                m.flags = 0;
                pm[k] = m;
                if (LAYOUT == kSimple && c_[i]) atomicMin(&S.uexc[k / 16], m.cursor);
                if (k % 16 == 0) S.urng[k / 16].x = m.packed_off;
                if (k % 16 == 15 || k == K - 1) S.urng[k / 16].y = m.packed_off + 16 * b_[i];
            }
        }
    }
    // ---- exception arrays (warp 0)
    if (LAYOUT == kSimple) {
        if (warp == 0) {
            uint32_t woff, W;
            bad = simple_stream(page, psize, bytes_at, Lpad, cnt_total, bad, pg, woff, W, h, lane);
            if (lane == 0) {
                S.s8[0] = woff;
                S.s8[1] = bad ? 0u : W;
                S.s8[2] = 0;
            }
        }
        __syncthreads();
        bad = pg[32] != 0;
        // each unit's first word: the word whose values cover the unit's
        // first exception (chunks of kMetaThreads words, a CTA scan of their
        // counts); its offset in that word goes to the first block's flags
        const uint32_t woff = S.s8[0], W = S.s8[1];
        const uint32_t nunits_s = (K + 15) / 16;
        for (uint32_t cb = 0; cb < W; cb += kMetaThreads) {
            const uint32_t w = cb + tid;
            uint32_t cnt_w = 0;
            if (w < W) {
                const uint64_t word = *reinterpret_cast<const uint64_t*>(page + woff + 8 * (size_t)w);
                cnt_w = s8_count((uint32_t)(word >> 60));
            }
            const uint32_t incl = warp_incl_scan(cnt_w, lane);
            if (lane == 31) S.wpk[warp] = incl;
            __syncthreads();
            uint32_t start = S.s8[2] + incl - cnt_w;
            for (int ww = 0; ww < warp; ++ww) start += S.wpk[ww];
            if (cnt_w) {
                for (uint32_t u = 0; u < nunits_s; ++u) {
                    const uint32_t e = S.uexc[u];
                    if (e >= start && e < start + cnt_w) {
                        pg[u] = w;
                        pm[16 * u].flags = (uint8_t)(e - start);
                    }
                }
            }
            __syncthreads();
            if (tid == kMetaThreads - 1) {
                uint32_t tot = 0;
                for (int ww = 0; ww < kMetaThreads / 32; ++ww) tot += S.wpk[ww];
                S.s8[2] += tot;
            }
            __syncthreads();
        }
        if (!bad && tid == 0 && S.s8[2] != cnt_total) {  // the words hold exactly N values
            pg[32] = 1u;
            set_error(h, ICX_ECORRUPT);
        }
        __syncthreads();
        bad = pg[32] != 0;
    } else {
        if (warp == 0) bad = page_arrays<LAYOUT>(page, psize, bytes_at, Lpad, cnt_total, bad, pg, h, lane);
        __syncthreads();
        bad = *reinterpret_cast<volatile const uint32_t*>(pg + 32) != 0;
    }
    // per unit of 16 blocks: where its packed low bits start and how long they are
    const uint32_t nunits = (K + 15) / 16;
    if ((uint32_t)tid < nunits) {
        uint2 x = make_uint2(0, ~0u);
        if (!bad) {
            const uint2 r = S.urng[tid];
            x = make_uint2(r.x, r.y - r.x);
            um[tid] = x;
        }
        if (rng) rng[tid] = make_ulonglong2(bad ? 0ull : reinterpret_cast<uint64_t>(page + x.x), x.y);
    }
    return bad;
}


// ------------------------------------------------------ small-page parse
//
// One warp per page of at most kSmallK blocks (short lists): the byte array
// prefix that K records can occupy is staged in shared memory, lane 0 walks
// the K record starts there, then one lane per block does what one round of
// the CTA parse does.

constexpr uint32_t kSmallK = 32;
constexpr uint32_t kSmallWin = kSmallK * kRecMax + 16;  // every record of <= 32 blocks

struct SmallPageSmem {
    uint32_t bytes[kSmallWin / 4 + 4];
    uint32_t start[kSmallK];
};

__device__ __forceinline__ void parse_small_page(SmallPageSmem& S, const uint8_t* __restrict__ in, size_t in_bytes,
                                                 uint64_t base, uint64_t end, uint32_t K,
                                                 BlockMeta* __restrict__ pm, uint32_t* __restrict__ pg,
                                                 uint2* __restrict__ um, WsHeader* h,
                                                 ulonglong2* __restrict__ rng = nullptr) {
    const int lane = threadIdx.x & 31;
    const uint8_t* sb = reinterpret_cast<const uint8_t*>(S.bytes);
    bool bad = !(base <= end && end <= in_bytes && (base & 15) == 0 && end - base >= 16);
    const uint8_t* page = in + base;
    const uint32_t psize = bad ? 0u : (uint32_t)min(end - base, (uint64_t)0xFFFFFFF0u);
    uint32_t len_at = 0, L = 0, bytes_at = 0;
    if (!bad) {
        len_at = 4 * ld32(page);
        bad = len_at < 16 || (len_at & 15) || (uint64_t)len_at + 4 > psize;
    }
    if (!bad) {
        L = ld32(page + len_at);
        bytes_at = len_at + 4;
        bad = (uint64_t)bytes_at + pad_up(L, 4) + 4 > psize;
    }
    const uint32_t Lpad = bad ? 0u : (uint32_t)pad_up(L, 4);
    const uint32_t* arr = reinterpret_cast<const uint32_t*>(page + bytes_at);
    const uint32_t nw = min(kSmallWin, Lpad) / 4;
    for (uint32_t i = lane; i < kSmallWin / 4 + 4; i += 32) S.bytes[i] = i < nw ? __ldg(arr + i) : 0u;
    __syncwarp();
    if (lane == 0 && !bad) {
        // K <= 32 records of <= kRecMax bytes: every start stays in the window
        uint32_t r = 0;
        for (uint32_t k = 0; k < K; ++k) {
            if (r + 2 > L) {
                bad = true;
                break;
            }
            S.start[k] = r;
            r += rec_len(sb[r], sb[r + 1], sb[r + 2]);
        }
    }
    bad = __shfl_sync(FULL, bad, 0);
    __syncwarp();
    const bool valid = !bad && (uint32_t)lane < K;
    uint32_t b = 0, mb = 0, c = 0, st = 0;
    if (valid) {
        st = S.start[lane];
        b = sb[st];
        mb = sb[st + 1];
        c = sb[st + 2];
    }
    const uint32_t d = mb > b ? mb - b : 0u;
    if (!d) c = 0;
    bool rbad = valid && (b > 32 || mb > 32 || mb < b || c > 128 || (uint64_t)st + (d ? 3 + c : 2) > L);
    const uint32_t bb = b <= 32 ? b : 0u;
    const uint32_t incl = warp_incl_scan(bb, lane);
    const uint32_t packed_total = __shfl_sync(FULL, incl, 31);
    uint32_t cnt = 0;
    const uint32_t cursor = round_cursor(d, c, cnt, lane);
    bad = __any_sync(FULL, bad || rbad) || (!bad && 16 + 16 * packed_total != len_at);
    const uint32_t poff = 16 + 16 * (incl - bb);
    if (!bad && valid) {
        BlockMeta m;
        m.packed_off = poff;
        m.pos_off = d ? bytes_at + st + 3 : 0u;
        m.cursor = d ? cursor : 0u;
        m.b = (uint8_t)bb;
        m.d = (uint8_t)d;
        m.c = (uint8_t)c;
        m.flags = 0;
        pm[lane] = m;
    }
    bad = page_arrays<ICX_FMT_PAPER>(page, psize, bytes_at, Lpad, cnt, bad, pg, h, lane);
    // per unit of 16 blocks (at most two): its packed range
    const uint32_t k0 = 16 * (uint32_t)(lane & 1), k1 = min(K, k0 + 16) - 1;
    const uint32_t f0 = __shfl_sync(FULL, poff, (int)k0), f1 = __shfl_sync(FULL, poff, (int)(k1 & 31)),
                   b1 = __shfl_sync(FULL, bb, (int)(k1 & 31));
    if (lane < 2 && k0 < K) {
        const uint2 x = bad ? make_uint2(0, ~0u) : make_uint2(f0, f1 + 16 * b1 - f0);
        if (!bad) um[lane] = x;
        if (rng) rng[lane] = make_ulonglong2(bad ? 0ull : reinterpret_cast<uint64_t>(page + x.x), x.y);
    }
}

// ---------------------------------------------------------- unit decode

// Unpacks the K blocks of a SIMD-FastPFOR unit whose packed low bits were
// copied to `buf` (block k at buf + m[k].packed_off - m[0].packed_off; its
// records in m) and ORs in every exception as high << b (Sec. 5): exception
// j of block k is element cursor + j of exception array d = maxbits - b of
// the page (at pbase + pg[d - 1], vertical layout: chunk e/128, lane e%4,
// field (e%128)/4; scalar FastPFOR: one lane, field e), its position the
// j-th byte after pos_off.  The scalar layout packs a block's low parts in
// one lane, 4 groups of 32 integers of b words each.  The patch rows reuse
// `buf` once unpacked; blk_of is a kExScratchBytes scratch.
//
// SimplePFOR (LAYOUT kSimple): scalar low parts; the high parts come from the
// page's Simple-8b words.  pg[0] is the unit's first word, pg[1] the page
// offset of the words, pg[2] their count, m[0].flags the offset of the
// unit's first exception in its first word.  Windows of 32 words (one per
// lane) are staged in s8 (32 words, then 32 value starts) with a warp scan
// of their counts; each exception finds its word by a 5-step search.
constexpr int kS8Scratch = 32 * 8 + 32 * 4;

template <int LAYOUT = ICX_FMT_PAPER>
__device__ __forceinline__ void fp_unit_unpack_patch(const uint8_t* __restrict__ in, uint64_t pbase,
                                                     const uint32_t* __restrict__ pg, const BlockMeta* m,
                                                     uint32_t K, uint8_t* buf, uint8_t* blk_of, uint4 (&v)[16],
                                                     WsHeader* h, int lane, uint8_t* s8 = nullptr) {
    uint32_t* buf32 = reinterpret_cast<uint32_t*>(buf);
    const uint32_t first = m[0].packed_off;
    uint32_t C = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        if ((uint32_t)k < K) {
            const uint32_t b = m[k].b, mask = width_mask(b);
            if (LAYOUT == ICX_FMT_SCALAR || LAYOUT == kSimple) {
                // lane t: fields 4(t%8)..+3 of group t/8 (integers 4t..4t+3)
                const uint32_t* words = reinterpret_cast<const uint32_t*>(buf + (m[k].packed_off - first));
                const uint32_t g = (uint32_t)lane >> 3, i0 = 4 * ((uint32_t)lane & 7);
                uint32_t r[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const uint32_t bit = (i0 + c) * b, w = b * g + (bit >> 5);
                    r[c] = __funnelshift_r(words[w], words[w + 1], bit & 31) & mask;
                }
                v[k] = make_uint4(r[0], r[1], r[2], r[3]);
            } else {
                const uint32_t bit = (uint32_t)lane * b;
                const uint4* rows = reinterpret_cast<const uint4*>(buf + (m[k].packed_off - first));
                const uint4 r0 = rows[bit >> 5], r1 = rows[(bit >> 5) + 1];
                const uint32_t s = bit & 31;
                v[k] = make_uint4(__funnelshift_r(r0.x, r1.x, s) & mask, __funnelshift_r(r0.y, r1.y, s) & mask,
                                  __funnelshift_r(r0.z, r1.z, s) & mask, __funnelshift_r(r0.w, r1.w, s) & mask);
            }
            C += m[k].c;
        }
    }
    if (C) {
        // patch: high << b of every exception of the unit (Sec. 5)
        __syncwarp();
        // pre[k]: the unit's exceptions before block k (kept in the scratch
        // after blk_of, so the gathers below hold no table in registers)
        uint16_t* pre = reinterpret_cast<uint16_t*>(blk_of + kExScratch);
        uint32_t run = 0;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            if (lane == 0) pre[k] = (uint16_t)run;
            const uint32_t c = (uint32_t)k < K ? m[k].c : 0u;
            for (uint32_t j = lane; j < c; j += 32) blk_of[run + j] = (uint8_t)k;
            if (c) reinterpret_cast<uint4*>(buf + 512 * k)[lane] = make_uint4(0, 0, 0, 0);
            run += c;
        }
        __syncwarp();
        bool badpos = false;
        if (LAYOUT == kSimple) {
            uint64_t* sw = reinterpret_cast<uint64_t*>(s8);
            int32_t* ss = reinterpret_cast<int32_t*>(s8 + 32 * 8);
            const uint64_t* words = reinterpret_cast<const uint64_t*>(in + pbase + pg[1]);
            const uint32_t W = pg[2];
            uint32_t wbase = pg[0], q0 = 0;
            int32_t vbase = -(int32_t)m[0].flags;  // value index of the window's first value
            bool bad8 = wbase == 0xFFFFFFFFu;
            while (q0 < C && !bad8) {
                const uint32_t w = wbase + lane;
                const bool valid = w < W;
                const uint64_t word = valid ? words[w] : 0ull;
                const uint32_t cnt = valid ? s8_count((uint32_t)(word >> 60)) : 0u;
                const uint32_t incl = warp_incl_scan(cnt, lane);
                const uint32_t total = __shfl_sync(FULL, incl, 31);
                __syncwarp();
                sw[lane] = word;
                ss[lane] = vbase + (int32_t)(incl - cnt);  // past the last word: the window's end
                __syncwarp();
                if (total == 0) {
                    bad8 = true;
                    break;
                }
                const int32_t wend = vbase + (int32_t)total;
                const uint32_t qend = wend <= 0 ? 0u : min(C, (uint32_t)wend);
                for (uint32_t qq = q0; qq < qend; qq += 128) {
                    uint32_t kk[4], pos[4], hv[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const uint32_t q = qq + 32 * i + lane;
                        kk[i] = 0xFFu;
                        if (q < qend) {
                            uint32_t j = 0;
#pragma unroll
                            for (uint32_t st = 16; st; st >>= 1)
                                if (ss[j + st] <= (int32_t)q) j += st;
                            const uint64_t wj = sw[j];
                            const uint32_t sel = (uint32_t)(wj >> 60), b8 = s8_bits(sel);
                            const uint32_t idx = q - (uint32_t)ss[j];
                            hv[i] = sel < 2 ? 0u : (uint32_t)((wj >> (idx * b8)) & ((1ull << b8) - 1));
                            const uint32_t k = blk_of[q];
                            kk[i] = k;
                            pos[i] = in[pbase + m[k].pos_off + (q - pre[k])];
                        }
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        if (kk[i] != 0xFFu) {
                            if (pos[i] < 128)
                                atomicOr(&buf32[128 * kk[i] + pos[i]], hv[i] << m[kk[i]].b);
                            else
                                badpos = true;
                        }
                    }
                }
                q0 = qend;
                wbase += 32;
                vbase = wend;
                if (q0 < C && wbase >= W) bad8 = true;  // the words ran out
                __syncwarp();
            }
            if (bad8) badpos = true;
        }
        // four independent exceptions per lane per round, so their
        // loads are in flight together
        for (uint32_t q0 = 0; q0 < (LAYOUT == kSimple ? 0u : C); q0 += 128) {
            uint32_t kk[4], pos[4], lo[4], hi[4], sh[4], dw[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const uint32_t q = q0 + 32 * i + lane;
                kk[i] = 0xFFu;
                if (q < C) {
                    const uint32_t k = blk_of[q];
                    const BlockMeta mk = m[k];
                    const uint32_t jj = q - pre[k];
                    const uint32_t d = mk.d, e = mk.cursor + jj;
                    const uint8_t* wp;
                    uint32_t bit, next;  // next: bytes from a word to the same lane's next word
                    if (LAYOUT == ICX_FMT_SCALAR) {
                        bit = e * d;
                        wp = in + pbase + pg[d - 1] + 4 * (size_t)(bit >> 5);
                        next = 4;
                    } else {
                        const uint8_t* arr = in + pbase + pg[d - 1] + 16 * (size_t)d * (e >> 7);
                        const uint32_t ii = e & 127;
                        bit = (ii >> 2) * d;
                        wp = arr + 16 * (bit >> 5) + 4 * (ii & 3);
                        next = 16;
                    }
                    kk[i] = k;
                    sh[i] = bit & 31;
                    dw[i] = d;
                    pos[i] = in[pbase + mk.pos_off + jj];
                    lo[i] = ld32(wp);
                    hi[i] = (bit & 31) + d > 32 ? ld32(wp + next) : 0u;
                }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (kk[i] != 0xFFu) {
                    const uint32_t high = __funnelshift_r(lo[i], hi[i], sh[i]) & width_mask(dw[i]);
                    if (pos[i] < 128)
                        atomicOr(&buf32[128 * kk[i] + pos[i]], high << m[kk[i]].b);
                    else
                        badpos = true;
                }
            }
        }
        if (__any_sync(FULL, badpos) && lane == 0) set_error(h, ICX_ECORRUPT);
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            if ((uint32_t)k < K && m[k].c) {
                const uint4 pv = reinterpret_cast<const uint4*>(buf + 512 * k)[lane];
                v[k].x |= pv.x;
                v[k].y |= pv.y;
                v[k].z |= pv.z;
                v[k].w |= pv.w;
            }
        }
    }
}

}  // namespace icx
