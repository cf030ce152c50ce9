// SIMD-FastPFOR decoding (Sec. 5, SIMD variant): page walk, page parse and
// the fused unpack + exception patch + differential decoding.
//
// The byte array of a page (per block b, maxbits and, for blocks with
// exceptions, the count c and c positions) has variable-length records, so
// finding block k's record needs the records before it.  The decode is
// therefore two launches:
//  1. fastpfor_meta_kernel -- one CTA per page finds the record starts of
//     its byte array (jump tables + an 8-record chain, see below) and writes
//     a fixed 16-byte record per block (packed offset, positions offset,
//     exception cursor, b, d, c) plus the page-relative offsets of the 32
//     exception arrays;
//  2. fastpfor_decode_kernel -- units of 16 blocks exactly like the
//     SIMD-BP128 decoder: one bulk copy of the unit's packed low bits into
//     shared memory, vertical unpacking, then every exception of the unit is
//     fetched by random access into its vertically packed array (element q:
//     chunk q/128, lane q%4, field (q%128)/4) and OR-ed in as high << b
//     (Sec. 5 "patching"), then the tile epilogue (scan, look-back, stores).
#include "icx_kernels.cuh"
#include "icx_tile.cuh"

namespace icx {

constexpr uint32_t kBlocksPerPage = 512;
constexpr uint32_t kUnitsPerPage = kBlocksPerPage / 16;

__device__ __forceinline__ uint32_t ld32(const uint8_t* p) { return __ldg(reinterpret_cast<const uint32_t*>(p)); }
__host__ __device__ __forceinline__ size_t pad_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// ------------------------------------------------------------- page walk

// Sequential walk over the pages: each page's size follows from its header
// word, byte-array length, bitset and exception counts.
__global__ void fastpfor_index_kernel(const uint8_t* __restrict__ in, size_t in_bytes, size_t n,
                                      uint64_t* __restrict__ index, WsHeader* h) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const size_t nb = n / 128, P = (nb + kBlocksPerPage - 1) / kBlocksPerPage;
    size_t pos = 0;
    bool bad = false;
    for (size_t p = 0; p < P; ++p) {
        index[p] = pos;
        if (bad) continue;
        if (pos + 16 > in_bytes) {
            bad = true;
            continue;
        }
        const size_t len_at = 4 * (size_t)ld32(in + pos);
        if (len_at < 16 || (len_at & 15) || pos + len_at + 4 > in_bytes) {
            bad = true;
            continue;
        }
        const size_t L = ld32(in + pos + len_at);
        size_t q = pos + len_at + 4 + pad_up(L, 4);
        if (q + 4 > in_bytes) {
            bad = true;
            continue;
        }
        const uint32_t bitset = ld32(in + q);
        q += 4;
        for (int d = 1; d <= 32 && !bad; ++d) {
            if (!((bitset >> (d - 1)) & 1u)) continue;
            if (q + 4 > in_bytes) {
                bad = true;
                break;
            }
            const size_t cnt = ld32(in + q);
            q = pos + pad_up(q + 4 - pos, 16) + 16 * (size_t)d * ((cnt + 127) / 128);
            if (q > in_bytes) bad = true;
        }
        const size_t end = pos + pad_up(q - pos, 16);
        if (end > in_bytes) bad = true;
        pos = end;
    }
    index[P] = bad ? in_bytes : pos;
    if (bad) set_error(h, ICX_ECORRUPT);
}

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

struct MetaSmem {
    uint32_t bytes[kMetaSpan / 4 + 4];  // window of the byte array (zero past its end)
    uint32_t j1[kMetaSpan / 4];         // record length at each position, one byte each
    uint16_t ja[kMetaSpan];             // J2, then J8
    uint16_t jb[kMetaSpan];             // J4
    uint32_t grp[kGroups];              // start of records 8g .. 8g+7
    uint32_t start[kBlocksPerPage];     // record starts
    uint32_t bmc[kBlocksPerPage];       // b | maxbits << 8 | c << 16
    uint32_t poff[kBlocksPerPage];      // page-relative offset of the packed low bits
    uint32_t wcnt[kMetaThreads / 32][32];  // per warp, exceptions per width
    uint32_t wpk[kMetaThreads / 32];       // per warp, sum of b
    uint32_t ctl[4];                       // window start, next group, chain state
};

__device__ __forceinline__ uint32_t rec_len(uint32_t b, uint32_t mb, uint32_t c) {
    return mb > b ? 3u + min(c, 129u) : 2u;
}

__global__ void __launch_bounds__(kMetaThreads)
    fastpfor_meta_kernel(const uint8_t* __restrict__ in, size_t in_bytes, size_t n, const uint64_t* __restrict__ index,
                         BlockMeta* __restrict__ meta, uint32_t* __restrict__ pmeta, uint2* __restrict__ umeta,
                         WsHeader* h) {
    __shared__ MetaSmem S;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint8_t* sb = reinterpret_cast<const uint8_t*>(S.bytes);
    const uint8_t* s1 = reinterpret_cast<const uint8_t*>(S.j1);
    const size_t nb = n / 128;
    const size_t p = blockIdx.x;
    const uint32_t K = (uint32_t)min((size_t)kBlocksPerPage, nb - kBlocksPerPage * p);
    const uint32_t G = (K + 7) / 8;
    BlockMeta* pm = meta + kBlocksPerPage * p;
    uint32_t* pg = pmeta + kPageMetaWords * p;

    const uint64_t base = index[p], end = index[p + 1];
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

    // ---- record starts, one window of the byte array at a time
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
        const uint32_t lim8 = min(kMetaWin, Lw), lim4 = lim8 + 4 * kRecMax, lim2 = lim4 + 2 * kRecMax,
                       lim1 = lim2 + kRecMax;
        const uint32_t nw = ws < Lpad ? min(kMetaSpan / 4, (Lpad - ws) / 4) : 0u;
        for (uint32_t i = tid; i < kMetaSpan / 4 + 4; i += kMetaThreads) S.bytes[i] = i < nw ? __ldg(arr + ws / 4 + i) : 0u;
        __syncthreads();
        for (uint32_t w = tid; w < (lim1 + 3) / 4; w += kMetaThreads) {
            const uint32_t lo = S.bytes[w], hi = S.bytes[w + 1];
            uint32_t packed = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t x = __funnelshift_r(lo, hi, 8 * j);
                packed |= rec_len(x & 0xFF, (x >> 8) & 0xFF, (x >> 16) & 0xFF) << (8 * j);
            }
            S.j1[w] = packed;
        }
        __syncthreads();
        for (uint32_t i = tid; i < lim2; i += kMetaThreads) {
            const uint32_t a = s1[i];
            S.ja[i] = (uint16_t)(a + s1[i + a]);
        }
        __syncthreads();
        for (uint32_t i = tid; i < lim4; i += kMetaThreads) {
            const uint32_t a = S.ja[i];
            S.jb[i] = (uint16_t)(a + S.ja[i + a]);
        }
        __syncthreads();
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
                S.start[k] = ws + q;
                S.bmc[k] = sb[q] | (uint32_t)sb[q + 1] << 8 | (uint32_t)sb[q + 2] << 16;
                q += s1[q];
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
        // exclusive count of earlier exceptions of the same width, one width at a time
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
                for (int w = 0; w < warp; ++w) cbase += S.wcnt[w][d ? d - 1 : 0];
                BlockMeta m;
                m.packed_off = 16 + 16 * (pk_base + pk[i]);
                m.pos_off = d ? bytes_at + S.start[k] + 3 : 0u;
                m.cursor = d ? cbase + cur[i] : 0u;
                m.b = (uint8_t)b_[i];
                m.d = (uint8_t)d;
                m.c = (uint8_t)c_[i];
                m.flags = 0;
                pm[k] = m;
                S.poff[k] = m.packed_off;
            }
        }
    }
    // ---- exception arrays (warp 0): offsets follow from the page's counts;
    // lane d-1 checks the stored count of array d against the records
    if (warp == 0) {
        uint32_t my_off = 0, my_cnt_at = 0;
        if (!bad) {
            const uint32_t bitset = ld32(page + bytes_at + Lpad);
            uint64_t q = (uint64_t)bytes_at + Lpad + 4;
            for (int d = 1; d <= 32; ++d) {
                const uint32_t nd = __shfl_sync(FULL, cnt_total, d - 1);
                if (!((bitset >> (d - 1)) & 1u)) {
                    if (nd) bad = true;
                    continue;
                }
                if (lane == d - 1) {
                    my_cnt_at = (uint32_t)q;
                    my_off = (uint32_t)pad_up(q + 4, 16);
                }
                q = pad_up(q + 4, 16) + 16 * (uint64_t)d * ((nd + 127) / 128);
                if (q > psize) {
                    bad = true;
                    break;
                }
            }
            if (pad_up(q, 16) != psize) bad = true;
            if (!bad && ((bitset >> lane) & 1u) && ld32(page + my_cnt_at) != cnt_total) bad = true;
            bad = __any_sync(FULL, bad);
        }
        pg[lane] = bad ? 0u : my_off;
        if (lane == 0) pg[32] = bad ? 1u : 0u;
        if (bad && lane == 0) set_error(h, ICX_ECORRUPT);
    }
    __syncthreads();
    // per unit of 16 blocks: where its packed low bits start and how long they are
    const uint32_t nunits = (K + 15) / 16;
    if (!bad && (uint32_t)tid < nunits) {
        const uint32_t k0 = 16 * tid, k1 = min(K, k0 + 16) - 1;
        const uint32_t first = S.poff[k0];
        umeta[kUnitsPerPage * p + tid] = make_uint2(first, S.poff[k1] + 16 * (S.bmc[k1] & 0xFF) - first);
    }
}

// ---------------------------------------------------------------- decode

constexpr int kUnitMax = 16 * 16 * 32;  // packed bytes of 16 blocks at width 32
constexpr int kFBuf = kUnitMax + 128;

struct FpSmem {
    TileShared t;
    uint64_t bar[kWarps];
    BlockMeta m[kWarps][16];
    uint8_t blk_of[kWarps][16 * 128];  // block of the unit's q-th exception
};

// A CTA of kWarps warps takes tiles of kWarps consecutive units of 16 blocks
// (then the Variable Byte tail), one look-back per tile, exactly like the
// SIMD-BP128 decoder: per warp its unit's block records, one bulk copy of
// its packed low bits, unpack, exception patch, local scan.
template <int DELTA>
__global__ void __launch_bounds__(kWarps * 32, 2)
    fastpfor_decode_kernel(const uint8_t* __restrict__ in, size_t in_bytes, uint32_t* __restrict__ out, size_t n,
                           const uint64_t* __restrict__ index, const BlockMeta* __restrict__ meta,
                           const uint32_t* __restrict__ pmeta, const uint2* __restrict__ umeta, WsHeader* h) {
    extern __shared__ __align__(128) uint8_t smem_raw[];
    FpSmem& S = *reinterpret_cast<FpSmem*>(smem_raw);
    uint8_t* bufs = smem_raw + ((sizeof(FpSmem) + 127) / 128) * 128;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t* buf = bufs + (size_t)warp * kFBuf;
    uint32_t* buf32 = reinterpret_cast<uint32_t*>(buf);
    uint64_t* bar = &S.bar[warp];
    BlockMeta* m = S.m[warp];
    uint8_t* blk_of = S.blk_of[warp];
    const size_t nb = n / 128;
    const uint32_t U = (uint32_t)((nb + 15) / 16);  // units of 16 blocks
    const uint32_t P = (uint32_t)((nb + kBlocksPerPage - 1) / kBlocksPerPage);
    const uint32_t ntiles = (U + 1 + kWarps - 1) / kWarps;  // then the Variable Byte tail
    const uint32_t epoch = launch_epoch(h);
    if (lane == 0) mbar_init(bar, 1);
    fence_mbar_init();
    __syncthreads();
    uint32_t phase = 0;

    // records of a unit: lane 0 its page base, page flag and packed region,
    // lanes 0..15 its block records
    struct Rec {
        uint64_t pbase;
        uint2 um;
        uint32_t bad;
        uint4 mrec;
    };
    auto prefetch = [&](uint32_t t, Rec& r) {
        const uint32_t uu = t * kWarps + warp;
        if (t < ntiles && uu < U) {
            const uint32_t p = uu / kUnitsPerPage;
            const uint32_t K = (uint32_t)min((size_t)16, nb - 16 * (size_t)uu);
            if (lane == 0) {
                r.pbase = index[p];
                r.um = umeta[uu];
                r.bad = pmeta[kPageMetaWords * p + 32];
            }
            if ((uint32_t)lane < K) r.mrec = reinterpret_cast<const uint4*>(meta + 16 * (size_t)uu)[lane];
        }
    };
    // publishes the records and starts the bulk copy; returns 0 = nothing to
    // wait for, 1 = copy in flight, 2 = bad page
    auto issue = [&](uint32_t t, const Rec& r) -> uint32_t {
        uint32_t res = 0;
        const uint32_t uu = t * kWarps + warp;
        if (t < ntiles && uu < U) {
            if (lane < 16) reinterpret_cast<uint4*>(m)[lane] = r.mrec;
            __syncwarp();
            if (lane == 0) {
                if (r.bad) {
                    res = 2;
                } else if (r.um.y) {
                    fence_proxy_async();
                    mbar_expect_tx(bar, r.um.y);
                    bulk_load(buf, in + r.pbase + r.um.x, r.um.y, bar);
                    res = 1;
                }
            }
        }
        return __shfl_sync(FULL, res, 0);
    };

    for (;;) {
        const uint32_t tile = next_tile(S.t, h);
        if (tile >= ntiles) break;
        const uint32_t u = tile * kWarps + warp;
        uint4 v[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = make_uint4(0, 0, 0, 0);
        uint32_t K = 0;
        if (u < U) {
            K = (uint32_t)min((size_t)16, nb - 16 * (size_t)u);
            const uint32_t* pg = pmeta + kPageMetaWords * (u / kUnitsPerPage);
            Rec r{};
            prefetch(tile, r);
            const uint64_t pbase = __shfl_sync(FULL, r.pbase, 0);
            const uint32_t st = issue(tile, r);
            bool ok = st != 2;
            if (!ok) {
                if (lane == 0) set_error(h, ICX_ECORRUPT);
            } else if (st == 1) {
                ok = __all_sync(FULL, mbar_wait(bar, phase));
                phase ^= 1;
                if (!ok && lane == 0) set_error(h, ICX_ETIMEOUT);
            }
            if (ok) {
                const uint32_t first = m[0].packed_off;
                uint32_t C = 0;
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    if ((uint32_t)k < K) {
                        const uint32_t b = m[k].b;
                        const uint32_t bit = (uint32_t)lane * b;
                        const uint4* rows = reinterpret_cast<const uint4*>(buf + (m[k].packed_off - first));
                        const uint4 r0 = rows[bit >> 5], r1 = rows[(bit >> 5) + 1];
                        const uint32_t s = bit & 31, mask = width_mask(b);
                        v[k] = make_uint4(__funnelshift_r(r0.x, r1.x, s) & mask, __funnelshift_r(r0.y, r1.y, s) & mask,
                                          __funnelshift_r(r0.z, r1.z, s) & mask,
                                          __funnelshift_r(r0.w, r1.w, s) & mask);
                        C += m[k].c;
                    }
                }
                if (C) {
                    // patch: high << b of every exception of the unit (Sec. 5)
                    __syncwarp();
                    uint32_t pre[16];
                    uint32_t run = 0;
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        pre[k] = run;
                        const uint32_t c = (uint32_t)k < K ? m[k].c : 0u;
                        for (uint32_t j = lane; j < c; j += 32) blk_of[run + j] = (uint8_t)k;
                        if (c) reinterpret_cast<uint4*>(buf + 512 * k)[lane] = make_uint4(0, 0, 0, 0);
                        run += c;
                    }
                    __syncwarp();
                    bool badpos = false;
                    // four independent exceptions per lane per round, so their
                    // loads are in flight together
                    for (uint32_t q0 = 0; q0 < C; q0 += 128) {
                        uint32_t kk[4], pos[4], lo[4], hi[4], sh[4], dw[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const uint32_t q = q0 + 32 * i + lane;
                            kk[i] = 0xFFu;
                            if (q < C) {
                                const uint32_t k = blk_of[q];
                                const BlockMeta mk = m[k];
                                uint32_t pk = 0;
#pragma unroll
                                for (int j = 0; j < 16; ++j)
                                    if ((uint32_t)j == k) pk = pre[j];
                                const uint32_t jj = q - pk;
                                const uint32_t d = mk.d, e = mk.cursor + jj;
                                const uint8_t* arr = in + pbase + pg[d - 1] + 16 * (size_t)d * (e >> 7);
                                const uint32_t ii = e & 127, bit = (ii >> 2) * d;
                                const uint8_t* wp = arr + 16 * (bit >> 5) + 4 * (ii & 3);
                                kk[i] = k;
                                sh[i] = bit & 31;
                                dw[i] = d;
                                pos[i] = in[pbase + mk.pos_off + jj];
                                lo[i] = ld32(wp);
                                hi[i] = (bit & 31) + d > 32 ? ld32(wp + 16) : 0u;
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
        } else if (u == U) {
            const uint32_t count = (uint32_t)(n - 128 * nb);
            if (count) {
                tail_unit(in, in_bytes, index[P], count, buf32, v, h, lane);
                K = 1;
            }
        }
        __syncwarp();
        uint4 agg;
        if (DELTA == ICX_DELTA_4)
            agg = unit_scan_d4_smem(v, buf32, lane);
        else
            agg = unit_local_scan<DELTA>(v, K, false, lane);
        const uint4 pref = tile_prefix<DELTA>(S.t, agg, tile, epoch, h, warp, lane);
        if (u <= U) store_unit(out, u < U ? 2048 * (size_t)u : 128 * nb, n, v, K, pref, lane);
        if (DELTA == ICX_DELTA_NONE) __syncthreads();
    }
    finish_launch(h, epoch);
}

// ------------------------------------------------------------ launchers

cudaError_t launch_fastpfor_index(const uint8_t* in, size_t in_bytes, size_t n, uint64_t* index, WsHeader* h,
                                  cudaStream_t s) {
    fastpfor_index_kernel<<<1, 32, 0, s>>>(in, in_bytes, n, index, h);
    return cudaGetLastError();
}

template <int DELTA>
static cudaError_t launch_fp(const uint8_t* in, size_t in_bytes, uint32_t* out, size_t n, const uint64_t* index,
                             WsHeader* h, cudaStream_t s) {
    auto kern = fastpfor_decode_kernel<DELTA>;
    const int smem = (int)(((sizeof(FpSmem) + 127) / 128) * 128 + (size_t)kWarps * kFBuf);
    static int blocks_per_sm = -1;
    static int sms = 0;
    if (blocks_per_sm < 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, kWarps * 32, smem);
        if (e != cudaSuccess) return e;
        if (blocks_per_sm < 1) blocks_per_sm = 1;
    }
    char* ws = reinterpret_cast<char*>(h);
    BlockMeta* meta = reinterpret_cast<BlockMeta*>(ws + ws_blockmeta_off(n));
    uint32_t* pmeta = reinterpret_cast<uint32_t*>(ws + ws_pagemeta_off(n));
    uint2* umeta = reinterpret_cast<uint2*>(ws + ws_unitmeta_off(n));
    const size_t nb = n / 128, P = (nb + kBlocksPerPage - 1) / kBlocksPerPage, U = (nb + 15) / 16;
    if (P > 0) {
        fastpfor_meta_kernel<<<(unsigned)P, kMetaThreads, 0, s>>>(in, in_bytes, n, index, meta, pmeta, umeta, h);
    }
    const size_t ntiles = (U + 1 + kWarps - 1) / kWarps;
    const int grid = (int)min((size_t)blocks_per_sm * sms, ntiles);
    kern<<<grid, kWarps * 32, smem, s>>>(in, in_bytes, out, n, index, meta, pmeta, umeta, h);
    return cudaGetLastError();
}

cudaError_t launch_fastpfor_decode(int delta, const uint8_t* in, size_t in_bytes, uint32_t* out, size_t n,
                                   const uint64_t* index, WsHeader* h, cudaStream_t s) {
    if (delta == ICX_DELTA_1) return launch_fp<ICX_DELTA_1>(in, in_bytes, out, n, index, h, s);
    if (delta == ICX_DELTA_4) return launch_fp<ICX_DELTA_4>(in, in_bytes, out, n, index, h, s);
    return launch_fp<ICX_DELTA_NONE>(in, in_bytes, out, n, index, h, s);
}

}  // namespace icx
