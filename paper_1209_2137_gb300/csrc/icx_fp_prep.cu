// SIMD-FastPFOR decoding fused with differential decoding (Sec. 5, Sec. 6.2):
// the kernels that follow the page parse (fastpfor_meta_kernel, which writes
// one record per block: packed offset, positions offset, exception cursor,
// b, d, c).
//
//  1. fastpfor_prep_kernel, one CTA per tile of 256 blocks (half a page), one
//     thread per block: sums the block's integers -- the low parts by walking
//     its packed rows, plus high << b for each exception -- and leaves the
//     block's exceptions for the stream kernel in its pair's own output
//     region: one 32-bit entry (position | high << 8) per exception, in
//     position order.  A block whose exceptions cannot be written so (high
//     parts wider than 24 bits, positions out of order or repeated) is
//     written there whole instead, as its 128 differences (every exception
//     OR-ed in as high << b, in stream order); a pair whose packed bits and
//     entries would not fit the stream kernel's staging slot is left as
//     differences in its own output.  A CTA scan gives each block its carry
//     inside the tile (written with its packed offset and entry offset) and
//     the tile's sum.
//  2. fastpfor_tile_scan_kernel, one CTA: turns the tile sums into tile
//     prefixes (Sec. 3) and decodes the Variable Byte tail (Sec. 2.4).
//  3. fastpfor_stream_kernel, persistent warps, one pair of 32 blocks per
//     step: one bulk copy of the pair's packed low bits and one of its
//     entries (or complete blocks) from its output region into shared
//     memory; then lane L walks block L's fields from its carry plus the
//     tile prefix as the SIMD-BP128 decoder does, ORs each entry into its
//     field just before that field is emitted, and the fields are written
//     through the restaging buffer.  A pair's output region is read before
//     it is written, and by the warp that writes it.
//
// No kernel waits on another CTA.  The scan and stream kernels are launched
// as programmatic dependents of the kernel before them: they may be
// scheduled while it drains and wait for it (grid_dependency_wait) before
// their first memory access.
#include <cstddef>

#include "icx_blocklane.cuh"
#include "icx_fastpfor.cuh"
#include "icx_kernels.cuh"

namespace icx {

namespace fp2 {

constexpr uint32_t kPairsPerPage = kBlocksPerPage / 32;
constexpr uint32_t kHighMax = 24;    // widest high part an entry holds
constexpr uint32_t kRaw = 1u << 31;  // record: the block's area holds its 128 differences
constexpr uint32_t kDirect = 1u << 30;  // record: the block is decoded by the prepare kernel
constexpr uint32_t kBad = 1u << 16;  // record: the block's page is corrupt

// One thread's block in the prepare kernel: high part j of its exceptions
// (element cur + j of the page's array of width d at arr).
__device__ __forceinline__ uint32_t high_part(const uint8_t* arr, uint32_t e, uint32_t d) {
    const uint32_t i = e & 127, bit = (i >> 2) * d;
    const uint8_t* w = arr + 16 * (size_t)d * (e >> 7) + 16 * (bit >> 5) + 4 * (i & 3);
    const uint32_t s = bit & 31;
    const uint32_t lo = ld32(w), hi = s + d > 32 ? ld32(w + 16) : 0u;
    return __funnelshift_r(lo, hi, s) & width_mask(d);
}

// Rows of the stream read with predicated loads, so that threads of one warp
// whose windows move at different fields do not diverge; a row past `avail`
// reads as zeros.
struct PredRows {
    const uint8_t* base;
    uint64_t avail;
    __device__ __forceinline__ uint4 operator()(uint32_t off) const {
        return (uint64_t)off + 16 <= avail ? __ldg(reinterpret_cast<const uint4*>(base + off)) : make_uint4(0, 0, 0, 0);
    }
    __device__ __forceinline__ uint32_t cursor(uint32_t off) const { return off; }
    __device__ __forceinline__ void advance(uint4& r0, uint4& r1, uint32_t& sh, uint32_t& nxt) const {
        const bool p = sh >= 32;
        uint4 r2 = r1;
        if (p && (uint64_t)nxt + 16 <= avail) r2 = __ldg(reinterpret_cast<const uint4*>(base + nxt));
        else if (p) r2 = make_uint4(0, 0, 0, 0);
        r0 = p ? r1 : r0;
        r1 = r2;
        nxt += p ? 16u : 0u;
        sh &= 31;
    }
};

struct NoMid {
    __device__ __forceinline__ void operator()() {}
};

}  // namespace fp2

// ------------------------------------------------------------------ kernel 1

namespace fp2 {
constexpr int kPrepThreads = 256;  // blocks per tile of the prepare kernel (half a page)
constexpr uint32_t kCoopMax = 2048;  // exceptions of a pair handled by the whole warp
}

template <int DELTA>
__global__ void __launch_bounds__(fp2::kPrepThreads, 4)
    fastpfor_prep_kernel(const uint8_t* __restrict__ in, size_t in_bytes, uint32_t* __restrict__ out, size_t n,
                         const uint64_t* __restrict__ index, const BlockMeta* __restrict__ meta,
                         const uint32_t* __restrict__ pmeta, uint4* __restrict__ rec, uint4* __restrict__ tile_sum,
                         WsHeader* h) {
    using namespace fp2;
    using namespace bl;
    constexpr int NWARP = kPrepThreads / 32;
    __shared__ uint4 wtot[NWARP];
    // per warp: the owner lane of each of the pair's exceptions, each lane's
    // exception parameters, area offset and exception sums
    __shared__ uint8_t own_s[NWARP][kCoopMax];
    __shared__ uint4 par_s[NWARP][32];
    __shared__ uint4 xsum_s[NWARP][32];
    __shared__ uint32_t ent_s[NWARP][32];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const size_t nb = n / 128;
    const uint32_t t = blockIdx.x;  // tile: blocks 256 t .. 256 t + 255
    grid_dependency_wait();         // the page parse's records
    allow_dependents();
    {
        const size_t k = (size_t)kPrepThreads * t + tid;  // this thread's block
        const size_t pgi = k / kBlocksPerPage;           // a tile lies in one page
        const uint64_t base = __ldg(index + pgi);
        const uint32_t* pg = pmeta + kPageMetaWords * pgi;
        const bool bad = __ldg(pg + 32) != 0 || base >= in_bytes;
        const bool valid = !bad && k < nb;
        uint32_t b = 0, d = 0, c = 0, pk = 0, po = 0, cur = 0;
        if (valid) {
            const uint4 m = __ldg(reinterpret_cast<const uint4*>(meta + k));
            pk = m.x;
            po = m.y;
            cur = m.z;
            b = m.w & 0xFF;
            d = (m.w >> 8) & 0xFF;
            c = d ? (m.w >> 16) & 0xFF : 0u;
        }
        const uint8_t* page = in + (bad ? 0 : base);
        const uint8_t* arr = page + (d ? __ldg(pg + d - 1) : 0u);
        // The pair's exceptions (block after block) are taken by the whole
        // warp, 32 at a time, when there are at most kCoopMax of them (each
        // lane finds its exception's block in own_s); otherwise each lane
        // takes its own block's.  First pass: positions strictly increasing
        // inside each block and below 128, else the block is raw (as is a
        // block whose high parts are wider than an entry holds).
        const uint32_t cincl = warp_incl_scan(c, lane), ctot = __shfl_sync(FULL, cincl, 31);
        const uint32_t cex = cincl - c;
        const bool coop = ctot <= kCoopMax;
        bool raw = d > kHighMax, corrupt = false;
        if (coop) {
            for (uint32_t j = 0; j < c; ++j) own_s[warp][cex + j] = (uint8_t)lane;
            par_s[warp][lane] = make_uint4(po, cur, d ? __ldg(pg + d - 1) : 0u, b | d << 8 | cex << 16);
            xsum_s[warp][lane] = make_uint4(0, 0, 0, 0);
            __syncwarp();
            uint32_t marked = 0, carry_p = 0, carry_o = 0xFFu;
            for (uint32_t q0 = 0; q0 < ctot; q0 += 32) {
                const uint32_t q = q0 + lane;
                const bool v = q < ctot;
                const uint32_t o = v ? own_s[warp][q] : 0xFFu;
                uint32_t pos = 0;
                if (v) {
                    const uint4 pr = par_s[warp][o];
                    pos = __ldg(page + pr.x + (q - (pr.w >> 16)));
                }
                uint32_t pp = __shfl_up_sync(FULL, pos, 1), po_ = __shfl_up_sync(FULL, o, 1);
                if (lane == 0) {
                    pp = carry_p;
                    po_ = carry_o;
                }
                carry_p = __shfl_sync(FULL, pos, 31);
                carry_o = __shfl_sync(FULL, o, 31);
                const bool out_of_order = v && (pos >= 128 || (po_ == o && pos <= pp));
                corrupt |= v && pos >= 128;
                marked |= __reduce_or_sync(FULL, out_of_order ? 1u << o : 0u);
            }
            raw |= (marked >> lane) & 1u;
        } else {
            uint32_t prev = 0;
            for (uint32_t j0 = 0; j0 < c; j0 += 4) {
                uint32_t q[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) q[i] = j0 + i < c ? __ldg(page + po + j0 + i) : 0u;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    if (j0 + i < c) {
                        corrupt |= q[i] >= 128;
                        if (q[i] >= 128 || (j0 + i && q[i] <= prev)) raw = true;
                        prev = q[i];
                    }
                }
            }
        }
        if (__any_sync(FULL, corrupt) && lane == 0) set_error(h, ICX_ECORRUPT);
        // a pair (this warp's 32 blocks) whose packed bits and area do not
        // fit the decoder's staging slot is decoded here, every block in its
        // own output
        uint32_t E = !valid ? 0u : raw ? 128u : c;
        const uint32_t Sp = __reduce_add_sync(FULL, 16 * b);
        const bool direct = Sp + ((4 * __reduce_add_sync(FULL, E) + 15) & ~15u) > kRing;
        if (direct) E = 0;
        const uint32_t ent = warp_incl_scan(E, lane) - E;
        uint32_t* area = direct ? out + 128 * k : out + 4096 * (k / 32) + ent;
        // the low parts' sum: the block's fields, walked like the decoder
        Walk w;
        w.b = b;
        w.mask = width_mask(b);
        const PredRows rows{page, bad ? 0 : in_bytes - base};
        w.r0 = valid ? rows(pk) : make_uint4(0, 0, 0, 0);
        w.r1 = valid ? rows(pk + 16) : make_uint4(0, 0, 0, 0);
        w.nxt = pk + 32;
        w.sh = 0;
        w.acc = make_uint4(0, 0, 0, 0);
        const uint32_t maxb = __reduce_max_sync(FULL, valid && !raw && !direct ? b : 0u);
        NoPatch np;
        NoMid nm;
        if (maxb) {
            if (maxb <= 8)
                walk_block<DELTA, false, 0, 4, true>(rows, w, nm, np);
            else if (maxb <= 16)
                walk_block<DELTA, false, 0, 2>(rows, w, nm, np);
            else
                walk_block<DELTA, false, 0, 1>(rows, w, nm, np);
        }
        uint4 s = w.acc;
        if (coop && !direct) {
            // second pass: the entries of the blocks that are not raw, and
            // the exceptions' share of each block sum
            ent_s[warp][lane] = ent;
            const unsigned rawmask = __ballot_sync(FULL, raw);
            __syncwarp();
            uint32_t* region = out + 4096 * (k / 32);
            for (uint32_t q0 = 0; q0 < ctot; q0 += 32) {
                const uint32_t q = q0 + lane;
                if (q < ctot) {
                    const uint32_t o = own_s[warp][q];
                    if (!((rawmask >> o) & 1u)) {
                        const uint4 pr = par_s[warp][o];
                        const uint32_t j = q - (pr.w >> 16), od = (pr.w >> 8) & 0xFF, ob = pr.w & 0xFF;
                        const uint32_t pos = __ldg(page + pr.x + j);
                        const uint32_t hv = high_part(page + pr.z, pr.y + j, od);
                        region[ent_s[warp][o] + j] = pos | hv << 8;
                        atomicAdd(reinterpret_cast<uint32_t*>(&xsum_s[warp][o]) + (pos & 3), hv << ob);
                    }
                }
            }
            __syncwarp();
            if (valid && !raw) s = add4(s, xsum_s[warp][lane]);
        } else if (valid && !raw && !direct) {
            for (uint32_t j0 = 0; j0 < c; j0 += 4) {
                uint32_t q[4], hv[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const bool in_range = j0 + i < c;
                    q[i] = in_range ? __ldg(page + po + j0 + i) : 0u;
                    hv[i] = in_range ? high_part(arr, cur + j0 + i, d) : 0u;
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    if (j0 + i < c) {
                        area[j0 + i] = q[i] | hv[i] << 8;
                        const uint32_t x = hv[i] << b;
                        s.x += (q[i] & 3) == 0 ? x : 0u;
                        s.y += (q[i] & 3) == 1 ? x : 0u;
                        s.z += (q[i] & 3) == 2 ? x : 0u;
                        s.w += (q[i] & 3) == 3 ? x : 0u;
                    }
                }
            }
        }
        if (valid && (raw || direct)) {
            // the 128 differences: low parts, then every exception OR-ed in
            const uint32_t mask = width_mask(b);
            for (uint32_t r = 0; r < 32; ++r) {
                const uint32_t bit = r * b, wo = 16 * (bit >> 5), sh = bit & 31;
                uint4 lo = make_uint4(0, 0, 0, 0), hi = lo;
                if (b) {
                    lo = rows(pk + wo);
                    if (sh + b > 32) hi = rows(pk + wo + 16);
                }
                *reinterpret_cast<uint4*>(area + 4 * r) =
                    make_uint4(__funnelshift_r(lo.x, hi.x, sh) & mask, __funnelshift_r(lo.y, hi.y, sh) & mask,
                               __funnelshift_r(lo.z, hi.z, sh) & mask, __funnelshift_r(lo.w, hi.w, sh) & mask);
            }
            for (uint32_t j = 0; j < c; ++j) {
                const uint32_t q = __ldg(page + po + j);
                if (q < 128) area[q] |= high_part(arr, cur + j, d) << b;
            }
            s = make_uint4(0, 0, 0, 0);
            for (uint32_t r = 0; r < 32; ++r) s = add4(s, *reinterpret_cast<const uint4*>(area + 4 * r));
        }
        if (DELTA == ICX_DELTA_1) s = make_uint4(s.x + s.y + s.z + s.w, 0, 0, 0);
        // ---- the tile's scan: each block's carry within the tile, and the
        // tile's total (the scan over tiles adds the tiles before it)
        const uint4 ti = warp_scan_carry<DELTA>(s, lane);
        if (lane == 31) wtot[warp] = ti;
        __syncthreads();
        uint4 woff = make_uint4(0, 0, 0, 0), tot = woff;
#pragma unroll
        for (int ww = 0; ww < NWARP; ++ww) {
            if (ww < warp) woff = add4(woff, wtot[ww]);
            tot = add4(tot, wtot[ww]);
        }
        if (tid == 0) tile_sum[t] = tot;
        if (k < nb) {
            uint4 info = make_uint4(0, 0, kBad, 0);
            if (!bad) info = make_uint4(pk, ent | (raw ? kRaw : 0u) | (direct ? kDirect : 0u), b | c << 8, 0);
            rec[2 * k] = add4(woff, sub4(ti, s));
            rec[2 * k + 1] = info;
        }
    }
}

// The scan over tiles (one CTA): each tile's exclusive prefix replaces its
// total; warp 0 then decodes the Variable Byte tail (Sec. 2.4) with the sum
// of every block as its carry.
constexpr int kScanThreads = 1024;

template <int DELTA>
__global__ void __launch_bounds__(kScanThreads)
    fastpfor_tile_scan_kernel(const uint8_t* __restrict__ in, size_t in_bytes, uint32_t* __restrict__ out, size_t n,
                              const uint64_t* __restrict__ index, uint4* __restrict__ tile_sum, WsHeader* h,
                              uint32_t tail) {
    __shared__ uint4 wtot[kScanThreads / 32];
    __shared__ __align__(16) uint32_t scratch[128];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const size_t nb = n / 128, T = (nb + fp2::kPrepThreads - 1) / fp2::kPrepThreads;
    const size_t per = (T + kScanThreads - 1) / kScanThreads, t0 = per * tid, t1 = min(T, t0 + per);
    grid_dependency_wait();  // the prepare kernel's tile sums
    allow_dependents();
    uint4 run = make_uint4(0, 0, 0, 0);
    for (size_t t = t0; t < t1; ++t) run = add4(run, tile_sum[t]);
    const uint4 ti = bl::warp_scan_carry<DELTA>(run, lane);
    if (lane == 31) wtot[warp] = ti;
    __syncthreads();
    uint4 off = make_uint4(0, 0, 0, 0), total = off;
    for (int w = 0; w < kScanThreads / 32; ++w) {
        if (w < warp) off = add4(off, wtot[w]);
        total = add4(total, wtot[w]);
    }
    uint4 acc = add4(off, sub4(ti, run));
    for (size_t t = t0; t < t1; ++t) {
        const uint4 v = tile_sum[t];
        tile_sum[t] = acc;
        acc = add4(acc, v);
    }
    if (tail && warp == 0) {
        uint4 carry = total;
        const uint64_t tstart = __ldg(index + (nb + kBlocksPerPage - 1) / kBlocksPerPage);
        uint4 v = make_uint4(0, 0, 0, 0);
        if (tstart <= in_bytes && vbyte_decode_warp(in, tstart, in_bytes, tail, scratch, h))
            v = *reinterpret_cast<const uint4*>(scratch + 4 * lane);
        else if (tstart > in_bytes && lane == 0)
            set_error(h, ICX_ECORRUPT);
        __syncwarp();
        uint4 o;
        if (DELTA == ICX_DELTA_4) {
            o = row_scan_d4(v, carry, lane);
        } else {
            v.y += v.x;
            v.z += v.y;
            v.w += v.z;
            const uint32_t incl = warp_incl_scan(v.w, lane);
            const uint32_t q = carry.x + incl - v.w;
            o = make_uint4(v.x + q, v.y + q, v.z + q, v.w + q);
        }
        const size_t q0 = 128 * nb + 4 * (size_t)lane;
        for (int cc = 0; cc < 4; ++cc)
            if (q0 + cc < n) out[q0 + cc] = comp(o, cc);
    }
}

// ------------------------------------------------------------------ kernel 2

namespace fp2 {

// The records of pair p (loaded a step ahead): lane L's block record
// (carry, then packed offset, area offset | raw, b | c << 8 | bad) and, in
// lane 0, the page's offset in the stream.
struct Pre {
    uint4 carry, info;
    uint32_t tpre;  // lane j < 4: component j of the tile's prefix
    uint64_t page;
};

// Pair p as the warp decodes it: its staged copy (space bytes) holds the
// packed low bits (Sp bytes from the page offset `first`) and then the area
// of its output region (`area` bytes); this lane's rows and entries are at
// pk_at and ent_at in it.  A pair of a corrupt page is not ok; a pair the
// prepare kernel left as differences in its output is `direct`.
struct Desc {
    uint64_t page;
    uint32_t first, Sp, area, space, K;
    uint32_t b, c, pk_at, ent_at;
    bool ok, direct;
    uint4 carry;
};

// Entries (position | high << 8, in position order) of the lane's block: the
// next one n and the one after it q sit in registers, so applying one never
// waits for the load of the next; 0xFF marks the end.
template <class Src>
struct EntryHook {
    Src src;
    uint32_t n, q, at, end, b;
    __device__ __forceinline__ uint32_t fetch() {
        uint32_t v = 0xFFu;
        if (at < end) {
            v = src(at);
            at += 4;
        }
        return v;
    }
    __device__ __forceinline__ void operator()(uint4& f, int r) {
        const uint32_t e = 4 * (uint32_t)r + 4;
        while ((n & 0xFFu) < e) {
            const uint32_t k = n & 3, v = (n >> 8) << b;
            f.x |= k == 0 ? v : 0u;
            f.y |= k == 1 ? v : 0u;
            f.z |= k == 2 ? v : 0u;
            f.w |= k == 3 ? v : 0u;
            n = q;
            q = fetch();
        }
    }
};

struct SmemWords {
    uint32_t sb;
    __device__ __forceinline__ uint32_t operator()(uint32_t off) const {
        uint32_t v;
        asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(sb + off) : "memory");
        return v;
    }
};

// Decodes and stores the lane's block of pair `pair_first / 4096`: the walk
// from `carry` with the entries OR-ed into their fields.
template <int DELTA, int STORE, class Rows, class Words, class Mid>
__device__ __forceinline__ void stream_blocks(const Rows& rows, Words words, const Desc& d, uint32_t* __restrict__ out,
                                              size_t pair_first, uint8_t* rest, int lane, Mid& mid) {
    using namespace bl;
    const bool live = (uint32_t)lane < d.K;
    Walk w;
    w.b = d.b;
    w.mask = width_mask(d.b);
    w.r0 = rows(d.pk_at);
    w.r1 = rows(d.pk_at + 16);
    w.nxt = rows.cursor(d.pk_at + 32);
    w.sh = 0;
    w.acc = d.carry;
    w.prev = make_uint4(0, 0, 0, 0);
    w.live = live;
    w.dst = out + pair_first + 128 * (size_t)lane;
    const uint32_t q = lane >> 3, i7 = lane & 7;
    w.wsb = smem_u32(rest) + 128 * lane + 16 * (lane & 7);
    const uint32_t rsb = smem_u32(rest) + 128 * q;
    w.ro0 = rsb + 16 * (i7 ^ q);
    w.ro1 = rsb + 16 * (i7 ^ (q + 4));
    w.ob = out + pair_first + 128 * q + 4 * i7;
    w.actq = __ballot_sync(FULL, w.live) >> q;
    const uint32_t maxb = __reduce_max_sync(FULL, d.b);
    EntryHook<Words> pt{words, 0xFFu, 0xFFu, d.ent_at, d.ent_at + 4 * d.c, d.b};
    pt.n = pt.fetch();
    pt.q = pt.fetch();
    if (maxb <= 8)
        walk_block<DELTA, true, STORE, 4>(rows, w, mid, pt);
    else if (maxb <= 16)
        walk_block<DELTA, true, STORE, 2>(rows, w, mid, pt);
    else
        walk_block<DELTA, true, STORE, 1>(rows, w, mid, pt);
}

}  // namespace fp2

// W warps per CTA: 6 (three CTAs of 96 registers a thread per SM) or 4 / 5
// (128 registers a thread).
template <int DELTA, int STORE, int W>
__global__ void __maxnreg__(W == 6 ? 96 : 128)
    fastpfor_stream_kernel(const uint8_t* __restrict__ in, size_t in_bytes, uint32_t* __restrict__ out, size_t n,
                           const uint64_t* __restrict__ index, const uint4* __restrict__ rec,
                           const uint4* __restrict__ tile_pre, WsHeader* h) {
    using namespace bl;
    using fp2::Desc;
    using fp2::Pre;
    extern __shared__ __align__(128) uint8_t smem[];
    Hdr& S = *reinterpret_cast<Hdr*>(smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t* ring = smem + kHdr + (size_t)warp * kWarpSmem;
    uint8_t* rest = ring + kRing + kSlack;
    uint64_t* bar = reinterpret_cast<uint64_t*>(&S.bar[2 * warp]);
    const size_t nb = n / 128;
    const uint32_t P = (uint32_t)((nb + 31) / 32);
    static_assert(W >= 1 && W <= kW, "the header holds barriers for kW warps");
    const uint32_t NW = gridDim.x * W;
    if (lane == 0) {
        mbar_init(bar, 1);
        mbar_init(bar + 1, 1);
    }
    fence_mbar_init();
    __syncwarp();
    grid_dependency_wait();  // block records and tile prefixes

    auto load = [&](uint32_t p) -> Pre {
        Pre e;
        const size_t blk = 32 * (size_t)p + lane;
        e.carry = make_uint4(0, 0, 0, 0);
        e.info = make_uint4(0, 0, fp2::kBad, 0);
        if (p < P && blk < nb) {
            e.carry = __ldcs(rec + 2 * blk);
            e.info = __ldcs(rec + 2 * blk + 1);
        }
        e.tpre = p < P && lane < 4
                     ? __ldg(reinterpret_cast<const uint32_t*>(tile_pre + (32 * (size_t)p) / fp2::kPrepThreads) + lane)
                     : 0u;
        e.page = lane == 0 && p < P ? __ldg(index + p / fp2::kPairsPerPage) : 0ull;
        return e;
    };
    auto describe = [&](uint32_t p, const Pre& e) -> Desc {
        Desc d;
        d.page = __shfl_sync(FULL, e.page, 0);
        d.K = (uint32_t)min((size_t)32, nb - 32 * (size_t)p);
        const bool active = (uint32_t)lane < d.K;
        const bool good = !__any_sync(FULL, active && (e.info.z & fp2::kBad)) && d.page < in_bytes;
        d.direct = good && __any_sync(FULL, active && (e.info.y & fp2::kDirect));
        d.ok = good && !d.direct;
        const bool live = active && d.ok;
        const bool raw = live && (e.info.y & fp2::kRaw);
        const uint32_t b = live ? e.info.z & 0xFF : 0u;
        d.c = live && !raw ? (e.info.z >> 8) & 0xFF : 0u;
        const uint32_t ent = e.info.y & 0x3FFFu;
        const uint32_t E = !live ? 0u : raw ? 128u : d.c;
        d.first = __shfl_sync(FULL, e.info.x, 0);
        const uint32_t last_end = __shfl_sync(FULL, e.info.x + 16 * b, (int)max(d.K, 1u) - 1);
        d.Sp = d.ok ? last_end - d.first : 0u;
        d.area = (4 * __reduce_add_sync(FULL, E) + 15) & ~15u;
        d.space = d.ok ? d.Sp + d.area : 0u;
        if (d.space > kRing) {  // the prepare kernel sends no such pair
            if (lane == 0) set_error(h, ICX_ECORRUPT);
            d.ok = false;
            d.space = 0;
        }
        d.b = raw ? 32u : b;
        d.pk_at = !live ? 0u : raw ? d.Sp + 4 * ent : e.info.x - d.first;
        d.ent_at = live ? d.Sp + 4 * ent : 0u;
        const uint4 tp = make_uint4(__shfl_sync(FULL, e.tpre, 0), __shfl_sync(FULL, e.tpre, 1),
                                    __shfl_sync(FULL, e.tpre, 2), __shfl_sync(FULL, e.tpre, 3));
        d.carry = add4(e.carry, tp);
        return d;
    };
    // two-slot staging ring, as in the block-per-lane decoder
    uint32_t s_iss = 0, s_wt = 0;
    bool broken = false;
    auto slot = [&](uint32_t s, const Desc& d) -> uint32_t { return (s & 1) ? kRing - d.space : 0u; };
    const uint64_t drop = l2_policy_evict_first();
    auto issue = [&](uint32_t p, const Desc& d) -> uint32_t {
        const uint32_t s = s_iss;
        if (!broken) {
            if (lane == 0) {
                fence_proxy_async();
                mbar_expect_tx(bar + (s & 1), d.space);
            }
            if (d.space) {
                __syncwarp();
                uint8_t* dst = ring + slot(s, d);
                if (lane == 0 && d.Sp) bulk_load_hint(dst, in + d.page + d.first, d.Sp, bar + (s & 1), drop);
                if (lane == 1 && d.area) {
                    fence_proxy_async();
                    bulk_load_hint(dst + d.Sp, out + 4096 * (size_t)p, d.area, bar + (s & 1), drop);
                }
            }
            ++s_iss;
        }
        return s;
    };
    auto wait = [&]() -> bool {
        if (broken) return false;
        const bool ok = __all_sync(FULL, mbar_wait(bar + (s_wt & 1), (s_wt >> 1) & 1u));
        if (ok) {
            ++s_wt;
        } else {
            broken = true;
            if (lane == 0) set_error(h, ICX_ETIMEOUT);
        }
        return ok;
    };
    auto fits = [&](const Desc& a, const Desc& b) { return a.space + b.space <= kRing; };

    uint32_t pc = blockIdx.x * W + warp;
    if (pc < P) {
        Desc dc = describe(pc, load(pc));
        uint32_t s_cur = issue(pc, dc);
        uint32_t pn = pc + NW;
        Pre en = load(pn);
        while (pc < P) {
            const uint32_t pk = pn + NW;
            Pre ek{};
            bool mid_done = false;
            auto mid = [&]() {
                ek = load(pk);
                mid_done = true;
            };
            Desc dn;
            uint32_t s_nx = 0;
            bool nx_issued = false;
            if (pn < P) {
                dn = describe(pn, en);
                if (fits(dc, dn)) {
                    s_nx = issue(pn, dn);
                    nx_issued = true;
                }
            }
            if (wait() && dc.ok) {
                uint8_t* base = ring + slot(s_cur, dc);
                fp2::stream_blocks<DELTA, STORE>(SmemRows{base, smem_u32(base)}, fp2::SmemWords{smem_u32(base)}, dc,
                                                 out, 4096 * (size_t)pc, rest, lane, mid);
            } else if (dc.direct && (uint32_t)lane < dc.K) {
                // the block's differences (in its own output) become its
                // integers
                uint4* o = reinterpret_cast<uint4*>(out + 4096 * (size_t)pc + 128 * lane);
                uint4 acc = dc.carry;
                for (int r = 0; r < 32; ++r) {
                    const uint4 f = __ldcg(o + r);
                    uint4 y;
                    if (DELTA == ICX_DELTA_4) {
                        acc = add4(acc, f);
                        y = acc;
                    } else {
                        y.x = acc.x + f.x;
                        y.y = y.x + f.y;
                        y.z = y.y + f.z;
                        y.w = y.z + f.w;
                        acc.x = y.w;
                    }
                    __stcs(o + r, y);
                }
            }
            __syncwarp();
            if (!mid_done) mid();
            if (pn < P && !nx_issued) s_nx = issue(pn, dn);
            pc = pn;
            pn = pk;
            en = ek;
            dc = dn;
            s_cur = s_nx;
        }
    }
    // a copy that never landed must not outlive the CTA's shared memory
    if (broken)
        for (uint32_t s = s_wt; s < s_iss; ++s) mbar_wait(bar + (s & 1), (s >> 1) & 1u);
}

// ------------------------------------------------------------------ launcher

// Programmatic dependent launch of the prepare, scan and stream kernels:
// bit 0, 1, 2 of the setting lets the prepare, scan, stream kernel be
// scheduled while the kernel before it is still running (it waits for it in
// grid_dependency_wait before it touches memory).  0 = plain stream order.
// Measured on the 2^26 sorted arrays, ms for SIMD-FastPFOR / SIMD-FastPFOR*
// uniform and clustered: 0: 0.1249 / 0.1400 / 0.1093 / 0.1377; 7: 0.1244 /
// 0.1444 / 0.1042 / 0.1346; 6: 0.1208 / 0.1352 / 0.1044 / 0.1321.  Prepare
// CTAs resident during the page parse (bit 0) cost more than they save.
static int g_fp_chain_overlap = 6;

void set_fastpfor_chain_overlap(int v) { g_fp_chain_overlap = v < 0 ? 6 : (v & 7); }

template <typename... KArgs, typename... Args>
static cudaError_t launch_chained(int bit, void (*kern)(KArgs...), unsigned grid, unsigned block, size_t smem,
                                  cudaStream_t s, Args... args) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = (g_fp_chain_overlap >> bit) & 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

static int g_fp_stream_warps = 0;  // warps per CTA of the stream kernel (0: by stride)

void set_fastpfor_stream_warps(int w) { g_fp_stream_warps = (w >= 4 && w <= 6) ? w : 0; }

template <int DELTA, int STORE, int W>
static cudaError_t launch_stream_w(const uint8_t* in, size_t in_bytes, uint32_t* out, size_t n,
                                   const uint64_t* index, const uint4* rec, const uint4* tiles, WsHeader* h,
                                   cudaStream_t s) {
    auto kern = fastpfor_stream_kernel<DELTA, STORE, W>;
    const int smem = (int)(bl::kHdr + (size_t)W * bl::kWarpSmem);
    static int blocks_per_sm = -1;
    static int sms = 0;
    if (blocks_per_sm < 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, W * 32, smem);
        if (e != cudaSuccess) return e;
        if (blocks_per_sm < 1) blocks_per_sm = 1;
    }
    const size_t Q = (n / 128 + 31) / 32;
    const BlocklaneTuning t = blocklane_tuning();
    size_t G = max((size_t)1, min((size_t)blocks_per_sm * sms, (Q + W - 1) / W));
    if (t.ctas > 0 && (size_t)t.ctas < G) G = (size_t)t.ctas;
    return launch_chained(2, kern, (unsigned)G, W * 32, (size_t)smem, s, in, in_bytes, out, n, index, rec, tiles, h);
}

template <int DELTA, int STORE>
static cudaError_t launch_fp2_t(const uint8_t* in, size_t in_bytes, uint32_t* out, size_t n, const uint64_t* index,
                                BlockMeta* meta, uint32_t* pmeta, uint2* umeta, WsHeader* h, size_t ws_bytes,
                                cudaStream_t s) {
    const size_t nb = n / 128, P = (nb + kBlocksPerPage - 1) / kBlocksPerPage, Q = (nb + 31) / 32;
    const size_t T = (nb + fp2::kPrepThreads - 1) / fp2::kPrepThreads;
    // plain data (no tagged words): its own workspace region after the page
    // parse's records
    char* fp2 = reinterpret_cast<char*>(h) + ws_plain_base(ws_bytes) + ws_meta_bytes(n);
    uint4* rec = reinterpret_cast<uint4*>(fp2);                           // 32 bytes per block
    uint4* tiles = reinterpret_cast<uint4*>(fp2 + ws_fp2_tiles_rel(n));  // 16 bytes per tile (8 pairs)
    if (P > 0) {
        const cudaError_t em = launch_fastpfor_meta(in, in_bytes, n, index, meta, pmeta, umeta, h, s);
        if (em != cudaSuccess) return em;
        const cudaError_t ep = launch_chained(0, fastpfor_prep_kernel<DELTA>, (unsigned)T, fp2::kPrepThreads, 0, s, in,
                                              in_bytes, out, n, index, (const BlockMeta*)meta,
                                              (const uint32_t*)pmeta, rec, tiles, h);
        if (ep != cudaSuccess) return ep;
    }
    const cudaError_t e = launch_chained(1, fastpfor_tile_scan_kernel<DELTA>, 1, kScanThreads, 0, s, in, in_bytes, out,
                                         n, index, tiles, h, (uint32_t)(n - 128 * nb));
    if (e != cudaSuccess || Q == 0) return e;
    // measured on the 2^26 sorted arrays: stride 1 is fastest with 4 warps a
    // CTA (0.1254 vs 0.1295 ms with 6), stride 4 with 6 (0.1418 vs 0.1510)
    const int w = g_fp_stream_warps ? g_fp_stream_warps : (DELTA == ICX_DELTA_1 ? 4 : 6);
    if constexpr (STORE == bl::kStoreRestage) {
        if (w == 4)
            return launch_stream_w<DELTA, STORE, 4>(in, in_bytes, out, n, index, rec, tiles, h, s);
        if (w == 5)
            return launch_stream_w<DELTA, STORE, 5>(in, in_bytes, out, n, index, rec, tiles, h, s);
    }
    return launch_stream_w<DELTA, STORE, 6>(in, in_bytes, out, n, index, rec, tiles, h, s);
}

cudaError_t launch_fastpfor_two_kernel(int delta, const uint8_t* in, size_t in_bytes, uint32_t* out, size_t n,
                                       const uint64_t* index, BlockMeta* meta, uint32_t* pmeta, uint2* umeta,
                                       WsHeader* h, size_t ws_bytes, cudaStream_t s) {
    int st = blocklane_tuning().store;
    if (st == bl::kStoreV8 && (reinterpret_cast<uintptr_t>(out) & 31u) != 0) st = bl::kStoreV4;
#define ICX_FP2(D)                                                                                                  \
    if (delta == D) {                                                                                               \
        if (st == bl::kStoreRestage)                                                                                \
            return launch_fp2_t<D, bl::kStoreRestage>(in, in_bytes, out, n, index, meta, pmeta, umeta, h, ws_bytes, s); \
        if (st == bl::kStoreV8)                                                                                     \
            return launch_fp2_t<D, bl::kStoreV8>(in, in_bytes, out, n, index, meta, pmeta, umeta, h, ws_bytes, s);  \
        return launch_fp2_t<D, bl::kStoreV4>(in, in_bytes, out, n, index, meta, pmeta, umeta, h, ws_bytes, s);      \
    }
    ICX_FP2(ICX_DELTA_4)
    ICX_FP2(ICX_DELTA_1)
#undef ICX_FP2
    return cudaErrorInvalidValue;
}

}  // namespace icx
