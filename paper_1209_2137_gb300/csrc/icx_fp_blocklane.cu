// SIMD-FastPFOR decoding fused with differential decoding (Sec. 5, Sec. 6.2)
// in two passes with one block per lane, on the task loop of the SIMD-BP128
// block-per-lane decoder.
//
// The page parse (fastpfor_meta_kernel) has already written a fixed record
// per block: where its packed low bits start, its width b, the width d =
// maxbits - b of its exceptions' high parts, its exception count c, where its
// c positions are in the page's byte array, and the index of its first
// exception in the page's array of width d.  A pair is 32 consecutive blocks
// of one page (a page holds 512 blocks, 16 pairs).  Its staged copy holds:
//   - the packed low bits of its 32 blocks (one range),
//   - the byte-array range that holds every position of the pair's
//     exceptions (from a 16-byte boundary),
//   - per distinct d, the 128-element chunks of exception array d that hold
//     the pair's high parts (vertical layout: element e in chunk e/128, lane
//     e%4, field (e%128)/4).
// Lane L walks block L's fields in order like SIMD-BP128.  Its exceptions
// come in position order (the encoder writes them so); before a field is
// emitted, the high parts of the exceptions that fall in it are OR-ed in as
// high << b (Sec. 5 "patching").  Pass A adds the exceptions to the block
// sum separately.  A lane whose positions are not strictly increasing takes a
// slower exact path (per field, every exception is looked at; in the sum, a
// repeated position counts once with its high parts OR-ed).
#include <cstddef>

#include "icx_blocklane.cuh"
#include "icx_fastpfor.cuh"
#include "icx_kernels.cuh"

namespace icx {

namespace bl {

constexpr uint32_t kPairsPerPage = kBlocksPerPage / 32;

// The loads that describe pair p (issued a task ahead): the page's offset in
// the stream and parse flag (lane 0), the offset of exception array lane+1,
// and this lane's block record.
struct FpPre {
    uint64_t page;
    uint32_t flag, arr;
    uint4 bm;
};

// Pair p as the warp works on it.  Offsets are relative to the staged copy
// when it is staged (space > 0), else to the page.  A staged pair whose high
// parts are all at most 8 bits wide also gets an entry area after its
// copies: one 16-bit entry (position << 8 | high part) per exception, lane
// after lane, written before pass B's walk.
struct FpDesc {
    uint64_t page;
    uint32_t space, tx, K;  // ring bytes, copied bytes, blocks
    uint32_t bdc;           // b | d << 8 | c << 16 of this lane's block
    uint32_t pk_at, pos_at, arr_at;  // its packed rows, first position, array-d chunk base
    uint32_t cur;           // index of its first exception in array d
    uint32_t ent_at;        // its first entry (0xFFFFFFFF: no entry area)
    uint32_t cp_src;        // the copy this lane issues: page offset,
    uint32_t cp_lendst;     // and (bytes / 16) << 16 | slot offset / 16
    bool ok;
};

// High part j of the lane's exceptions: element cur + j of the array of
// width d whose chunk 0 would sit at arr_at.
template <class Rows>
__device__ __forceinline__ uint32_t fp_high(const Rows& rows, uint32_t arr_at, uint32_t e, uint32_t d) {
    const uint32_t i = e & 127, bit = (i >> 2) * d;
    const uint32_t w = arr_at + 16 * d * (e >> 7) + 16 * (bit >> 5) + 4 * (i & 3);
    const uint32_t s = bit & 31;
    const uint32_t lo = rows.u32(w), hi = s + d > 32 ? rows.u32(w + 16) : 0u;
    return __funnelshift_r(lo, hi, s) & width_mask(d);
}

__device__ __forceinline__ void or_comp(uint4& f, uint32_t k, uint32_t v) {
    f.x |= k == 0 ? v : 0u;
    f.y |= k == 1 ? v : 0u;
    f.z |= k == 2 ? v : 0u;
    f.w |= k == 3 ? v : 0u;
}

// Exceptions j of a lane's block: position at byte pos_at + j, high part
// element cur + j of the width-d array placed at arr_at.
struct FpExc {
    uint32_t pos_at, arr_at, cur, c, b, d;
};

// The exceptions' share of the sum of a block whose positions are not
// strictly increasing (or not all below 128): each distinct position once,
// with the high parts of all its exceptions OR-ed; positions >= 128 are
// corrupt (reported by the caller) and skipped.
template <int DELTA, class Rows>
__device__ __forceinline__ uint4 fp_exact_sum(const Rows& rows, const FpExc& x) {
    uint4 es = make_uint4(0, 0, 0, 0);
    for (uint32_t j = 0; j < x.c; ++j) {
        const uint32_t p = rows.u8(x.pos_at + j);
        if (p >= 128) continue;
        bool seen = false;
        for (uint32_t k = 0; k < j; ++k) seen |= rows.u8(x.pos_at + k) == p;
        if (seen) continue;
        uint32_t v = fp_high(rows, x.arr_at, x.cur + j, x.d);
        for (uint32_t k = j + 1; k < x.c; ++k)
            if (rows.u8(x.pos_at + k) == p) v |= fp_high(rows, x.arr_at, x.cur + k, x.d);
        const uint32_t y = v << x.b;
        if (DELTA == ICX_DELTA_4) {
            es.x += (p & 3) == 0 ? y : 0u;
            es.y += (p & 3) == 1 ? y : 0u;
            es.z += (p & 3) == 2 ? y : 0u;
            es.w += (p & 3) == 3 ? y : 0u;
        } else {
            es.x += y;
        }
    }
    return es;
}

// Pass B's field hook.  The lane's next exception (position in the low half
// of pq, 0xFFFF when none is left; value nv = high << b) and the one after it
// (position in the high half of pq, value qv) are held in registers, so
// applying one and moving on never waits for a load.  e is the element index
// of the exception after those two (its position at byte e + pdelta), e_end
// the end of the lane's elements.
template <class Rows>
struct FpPatch {
    const Rows& rows;
    uint32_t pq, nv, qv, e, e_end, pdelta, arr_at, bd;
    __device__ __forceinline__ uint32_t fetch(uint32_t& v) {
        if (e < e_end) {
            const uint32_t p = rows.u8(e + pdelta);
            v = fp_high(rows, arr_at, e, bd >> 8) << (bd & 0xFF);
            ++e;
            return p;
        }
        return 0xFFFFu;
    }
    __device__ __forceinline__ void init(const FpExc& x) {
        e = x.cur;
        e_end = x.cur + x.c;
        pdelta = x.pos_at - x.cur;
        arr_at = x.arr_at;
        bd = x.b | x.d << 8;
        nv = qv = 0;
        const uint32_t p0 = fetch(nv);
        const uint32_t p1 = fetch(qv);
        pq = p0 | p1 << 16;
    }
    __device__ __forceinline__ void operator()(uint4& f, int r) {
        const uint32_t end = 4 * (uint32_t)r + 4;
        while ((pq & 0xFFFFu) < end) {
            or_comp(f, pq & 3, nv);
            nv = qv;
            pq = (pq >> 16) | fetch(qv) << 16;
        }
    }
};

// Pass B's field hook over the lane's entries (position << 8 | high part,
// 0xFF00 past the last): the next entry n and the one after it q sit in
// registers, the entry after those at shared address ea (entries end at ee).
struct EntryPatch {
    uint32_t n, q, ea, ee, b;
    __device__ __forceinline__ uint32_t fetch() {
        uint32_t v = 0xFF00u;
        if (ea < ee) {
            asm volatile("ld.shared.u16 %0, [%1];" : "=r"(v) : "r"(ea) : "memory");
            ea += 2;
        }
        return v;
    }
    __device__ __forceinline__ void operator()(uint4& f, int r) {
        const uint32_t end = (4 * (uint32_t)r + 4) << 8;
        while (n < end) {
            or_comp(f, (n >> 8) & 3, (n & 0xFFu) << b);
            n = q;
            q = fetch();
        }
    }
};

// The field hook of a warp that holds a block whose positions are out of
// order: every field looks at every exception of its lane's block (repeated
// positions OR-ed, positions >= 128 never match).
template <class Rows>
struct FpExactPatch {
    const Rows& rows;
    FpExc x;
    __device__ __forceinline__ void operator()(uint4& f, int r) {
        for (uint32_t j = 0; j < x.c; ++j) {
            const uint32_t p = rows.u8(x.pos_at + j);
            if (p >> 2 == (uint32_t)r) or_comp(f, p & 3, fp_high(rows, x.arr_at, x.cur + j, x.d) << x.b);
        }
    }
};

// SIMD-FastPFOR as a block-per-lane codec.
struct FpCodec {
    const uint64_t* index;  // page offsets, then the Variable Byte tail
    const uint4* meta;      // block records (BlockMeta)
    const uint32_t* pmeta;  // page records: exception-array offsets, flag
    const uint2* umeta;     // per 16 blocks: packed offset and size
    const uint8_t* in;
    size_t in_bytes, nb, npages;

    using Pre = FpPre;
    using Desc = FpDesc;
    struct Ahead {
        uint64_t page;
        uint2 u0, u1;
    };

    __device__ __forceinline__ Pre load(uint32_t p, int lane) const {
        const size_t pg = p / kPairsPerPage, blk = 32 * (size_t)p + lane;
        Pre e;
        e.page = lane == 0 ? __ldg(index + pg) : 0ull;
        e.flag = lane == 0 ? __ldg(pmeta + kPageMetaWords * pg + 32) : 0u;
        e.arr = __ldg(pmeta + kPageMetaWords * pg + lane);
        e.bm = blk < nb ? __ldg(meta + blk) : make_uint4(0, 0, 0, 0);
        return e;
    }

    __device__ __forceinline__ Desc describe(uint32_t p, const Pre& e, int lane) const {
        Desc d;
        d.page = __shfl_sync(FULL, e.page, 0);
        d.ok = __shfl_sync(FULL, e.flag, 0) == 0 && d.page < in_bytes;
        d.K = (uint32_t)min((size_t)32, nb - 32 * (size_t)p);
        const bool active = d.ok && (uint32_t)lane < d.K;
        const uint4 bm = e.bm;
        const uint32_t b = active ? bm.w & 0xFFu : 0u;
        const uint32_t dd = active ? (bm.w >> 8) & 0xFFu : 0u;
        const uint32_t c = active && dd ? (bm.w >> 16) & 0xFFu : 0u;
        d.bdc = b | dd << 8 | c << 16;
        d.cur = bm.z;
        // packed low bits: block 0's offset to the end of block K-1
        const uint32_t first = __shfl_sync(FULL, bm.x, 0);
        const uint32_t last_end = __shfl_sync(FULL, bm.x + 16 * b, (int)max(d.K, 1u) - 1);
        const uint32_t Sp = last_end - first;
        // positions: from the first to the last exception of the pair
        const bool hasx = c != 0;
        const uint32_t qmin = __reduce_min_sync(FULL, hasx ? bm.y : 0xFFFFFFFFu);
        const uint32_t qmax = __reduce_max_sync(FULL, hasx ? bm.y + c : 0u);
        const uint32_t qlo = qmax ? qmin & ~15u : 0u;
        const uint32_t Sq = qmax ? ((qmax + 15) & ~15u) - qlo : 0u;
        // high parts: per distinct d, the chunks that hold the pair's elements
        uint32_t pend = __ballot_sync(FULL, hasx);
        uint32_t aoff = 0, rank = 0, slice = 0;
        uint32_t cp_len = 0, cp_dst = 0;
        d.cp_src = 0;
        while (pend) {
            const uint32_t kd = __shfl_sync(FULL, dd, __ffs(pend) - 1);
            const bool mine = hasx && dd == kd;
            const uint32_t emin = __reduce_min_sync(FULL, mine ? bm.z : 0xFFFFFFFFu);
            const uint32_t emax = __reduce_max_sync(FULL, mine ? bm.z + c : 0u);
            const uint32_t clo = emin >> 7, chi = (emax - 1) >> 7;
            const uint32_t bytes = 16 * kd * (chi - clo + 1);
            const uint32_t src = __shfl_sync(FULL, e.arr, (int)kd - 1) + 16 * kd * clo;
            if (mine) slice = aoff - 16 * kd * clo;
            if ((uint32_t)lane == 2 + rank) {
                d.cp_src = src;
                cp_len = bytes;
                cp_dst = aoff;
            }
            aoff += bytes;
            ++rank;
            pend &= ~__ballot_sync(FULL, mine);
        }
        const uint32_t tx = Sp + Sq + aoff;
        // the entry area: every exception's position and high part
        const uint32_t cincl = warp_incl_scan(c, lane);
        const uint32_t ctot = __shfl_sync(FULL, cincl, 31);
        const bool entries = __reduce_max_sync(FULL, dd) <= 8;
        const uint32_t E = entries ? (2 * ctot + 15) & ~15u : 0u;
        const bool staged = d.ok && rank <= 30 && tx + E <= kRing;
        d.space = staged ? tx + E : 0u;
        d.tx = staged ? tx : 0u;
        d.ent_at = staged && entries ? tx + 2 * (cincl - c) : 0xFFFFFFFFu;
        const uint32_t arr_page = __shfl_sync(FULL, e.arr, (int)((dd ? dd : 1u) - 1));
        if (staged) {
            d.pk_at = bm.x - first;
            d.pos_at = Sp + bm.y - qlo;
            d.arr_at = Sp + Sq + slice;
            if (lane == 0) {
                d.cp_src = first;
                cp_len = Sp;
                cp_dst = 0;
            } else if (lane == 1) {
                d.cp_src = qlo;
                cp_len = Sq;
                cp_dst = Sp;
            } else {
                cp_dst += Sp + Sq;
            }
        } else {
            d.pk_at = bm.x;
            d.pos_at = bm.y;
            d.arr_at = arr_page;
            cp_len = 0;
        }
        d.cp_lendst = (cp_len / 16) << 16 | cp_dst / 16;
        if (!active) d.pk_at = d.pos_at = d.arr_at = 0;
        return d;
    }

    __device__ __forceinline__ uint32_t space(const Desc& d) const { return d.space; }

    __device__ __forceinline__ void issue(const Desc& d, uint8_t* dst, uint64_t* bar, uint64_t policy,
                                          int lane) const {
        if (lane == 0) {
            fence_proxy_async();
            mbar_expect_tx(bar, d.tx);
        }
        if (d.tx) {
            __syncwarp();
            const uint32_t len = (d.cp_lendst >> 16) * 16;
            if (len) {
                fence_proxy_async();
                bulk_load_hint(dst + 16 * (d.cp_lendst & 0xFFFFu), in + d.page + d.cp_src, len, bar, policy);
            }
        }
    }

    __device__ __forceinline__ GlobalRows global_rows(const Desc& d) const {
        return GlobalRows{in + d.page, in_bytes - d.page};
    }

    __device__ __forceinline__ Ahead ahead(uint32_t p, int lane) const {
        Ahead a{0, make_uint2(0, 0), make_uint2(0, 0)};
        if (lane == 0) {
            a.page = __ldg(index + p / kPairsPerPage);
            a.u0 = __ldg(umeta + 2 * (size_t)p);
            if (32 * (size_t)p + 16 < nb) a.u1 = __ldg(umeta + 2 * (size_t)p + 1);
        }
        return a;
    }

    __device__ __forceinline__ void prefetch(const Ahead& a, uint64_t policy, int lane) const {
        if (lane != 0) return;
        const uint64_t lo = a.page + a.u0.x;
        const uint64_t hi = a.u1.y ? a.page + a.u1.x + a.u1.y : lo + a.u0.y;
        if (lo < hi && hi <= in_bytes && hi - lo <= 2 * (uint64_t)kUnitMax && ((lo | hi) & 15) == 0)
            prefetch_l2_hint(in + lo, (uint32_t)(hi - lo), policy);
    }

    __device__ __forceinline__ uint64_t tail_start() const { return __ldg(index + npages); }

    // Pass A: the lane's block sum, low bits by the walk, exceptions added
    // here.  Pass B: the walk with the exceptions OR-ed into their fields.
    template <int DELTA, bool DECODE, int STORE, class Rows, class Mid>
    __device__ __forceinline__ uint4 blocks(const Rows& rows, const Desc& d, uint4 carry, uint32_t& flag,
                                            uint32_t* __restrict__ out, size_t pair_first, uint8_t* rest,
                                            WsHeader* h, int lane, Mid& mid) const {
        const bool active = (uint32_t)lane < d.K;
        const uint32_t b = d.bdc & 0xFFu, dd = (d.bdc >> 8) & 0xFFu, c = d.bdc >> 16;
        Walk w;
        w.b = b;
        w.mask = width_mask(b);
        w.r0 = rows(d.pk_at);
        w.r1 = rows(d.pk_at + 16);
        w.nxt = rows.cursor(d.pk_at + 32);
        w.sh = 0;
        w.acc = DECODE ? carry : make_uint4(0, 0, 0, 0);
        w.prev = make_uint4(0, 0, 0, 0);
        w.live = active;
        w.dst = out + pair_first + 128 * (size_t)lane;
        const uint32_t q = lane >> 3, i7 = lane & 7;
        w.wsb = smem_u32(rest) + 128 * lane + 16 * (lane & 7);
        const uint32_t rsb = smem_u32(rest) + 128 * q;
        w.ro0 = rsb + 16 * (i7 ^ q);
        w.ro1 = rsb + 16 * (i7 ^ (q + 4));
        w.ob = out + pair_first + 128 * q + 4 * i7;
        w.actq = __ballot_sync(FULL, w.live) >> q;
        const uint32_t maxb = __reduce_max_sync(FULL, b);
        const FpExc x{d.pos_at, d.arr_at, d.cur, c, b, dd};
        if constexpr (!DECODE) {
            NoPatch np;
            if (maxb <= 8)
                walk_block<DELTA, false, 0, 4>(rows, w, mid, np);
            else if (maxb <= 16)
                walk_block<DELTA, false, 0, 2>(rows, w, mid, np);
            else
                walk_block<DELTA, false, 0, 1>(rows, w, mid, np);
            // the exceptions' share of the block sum (high << b each), four
            // at a time with their loads in flight together, checking that
            // the positions increase strictly and stay below 128
            uint4 es = make_uint4(0, 0, 0, 0);
            uint32_t prev = 0;
            bool slow = false, badpos = false;
            for (uint32_t j0 = 0; j0 < c; j0 += 4) {
                uint32_t p[4], v[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint32_t j = j0 + k;
                    p[k] = j < c ? rows.u8(x.pos_at + j) : 0u;
                    v[k] = j < c ? fp_high(rows, x.arr_at, x.cur + j, dd) : 0u;
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (j0 + k < c) {
                        badpos |= p[k] >= 128;
                        if (p[k] >= 128 || (j0 + k > 0 && p[k] <= prev)) slow = true;
                        prev = p[k];
                        const uint32_t y = v[k] << b;
                        if (DELTA == ICX_DELTA_4)
                            or_add(es, p[k] & 3, y);
                        else
                            es.x += y;
                    }
                }
            }
            if (__any_sync(FULL, slow) && slow) es = fp_exact_sum<DELTA>(rows, x);
            if (__any_sync(FULL, badpos) && lane == 0) set_error(h, ICX_ECORRUPT);
            flag = slow ? kSumFlag : 0u;
            w.acc = add4(w.acc, es);
            if (DELTA == ICX_DELTA_1) w.acc = make_uint4(w.acc.x + w.acc.y + w.acc.z + w.acc.w, 0, 0, 0);
            return w.acc;
        } else {
            if (!__any_sync(FULL, (flag & kSumFlag) != 0) && d.ent_at != 0xFFFFFFFFu) {
                // entries: every exception's position and high part, four at
                // a time with their loads in flight together
                for (uint32_t j0 = 0; j0 < c; j0 += 4) {
                    uint32_t p[4], v[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const uint32_t j = j0 + k;
                        p[k] = j < c ? rows.u8(x.pos_at + j) : 0u;
                        v[k] = j < c ? fp_high(rows, x.arr_at, x.cur + j, dd) : 0u;
                    }
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (j0 + k < c) rows.st16(d.ent_at + 2 * (j0 + k), p[k] << 8 | v[k]);
                }
                EntryPatch pt{0xFF00u, 0xFF00u, rows.cursor(d.ent_at), rows.cursor(d.ent_at + 2 * c), b};
                pt.n = pt.fetch();
                pt.q = pt.fetch();
                if (maxb <= 8)
                    walk_block<DELTA, true, STORE, 4>(rows, w, mid, pt);
                else if (maxb <= 16)
                    walk_block<DELTA, true, STORE, 2>(rows, w, mid, pt);
                else
                    walk_block<DELTA, true, STORE, 1>(rows, w, mid, pt);
            } else if (!__any_sync(FULL, (flag & kSumFlag) != 0)) {
                FpPatch<Rows> pt{rows, 0, 0, 0, 0, 0, 0, 0, 0};
                pt.init(x);
                if (maxb <= 8)
                    walk_block<DELTA, true, STORE, 4>(rows, w, mid, pt);
                else if (maxb <= 16)
                    walk_block<DELTA, true, STORE, 2>(rows, w, mid, pt);
                else
                    walk_block<DELTA, true, STORE, 1>(rows, w, mid, pt);
            } else {
                FpExactPatch<Rows> pt{rows, x};
                walk_block<DELTA, true, STORE, 1>(rows, w, mid, pt);
            }
            return make_uint4(0, 0, 0, 0);
        }
    }

    __device__ __forceinline__ static void or_add(uint4& s, uint32_t k, uint32_t v) {
        s.x += k == 0 ? v : 0u;
        s.y += k == 1 ? v : 0u;
        s.z += k == 2 ? v : 0u;
        s.w += k == 3 ? v : 0u;
    }
};

}  // namespace bl

template <int DELTA, int STORE>
__global__ void __maxnreg__(96)
    fastpfor_blocklane_kernel(const uint8_t* __restrict__ in, size_t in_bytes, uint32_t* __restrict__ out, size_t n,
                              const uint64_t* __restrict__ index, const BlockMeta* __restrict__ meta,
                              const uint32_t* __restrict__ pmeta, const uint2* __restrict__ umeta, WsHeader* h,
                              bl::Scratch sc, uint32_t tail, uint32_t lead, uint32_t sumw) {
    const size_t nb = n / 128;
    const bl::FpCodec codec{index,
                            reinterpret_cast<const uint4*>(meta),
                            pmeta,
                            umeta,
                            in,
                            in_bytes,
                            nb,
                            (nb + kBlocksPerPage - 1) / kBlocksPerPage};
    bl::run<bl::FpCodec, DELTA, STORE>(codec, in, in_bytes, out, n, h, sc, tail, lead, sumw);
}

template <int DELTA, int STORE>
static cudaError_t launch_fpbl_t(const uint8_t* in, size_t in_bytes, uint32_t* out, size_t n, const uint64_t* index,
                                 const BlockMeta* meta, const uint32_t* pmeta, const uint2* umeta, WsHeader* h,
                                 size_t ws_bytes, cudaStream_t s) {
    auto kern = fastpfor_blocklane_kernel<DELTA, STORE>;
    const int smem = (int)(bl::kHdr + (size_t)bl::kW * bl::kWarpSmem);
    static int blocks_per_sm = -1;
    static int sms = 0;
    if (blocks_per_sm < 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, bl::kW * 32, smem);
        if (e != cudaSuccess) return e;
        if (blocks_per_sm < 1) blocks_per_sm = 1;
    }
    const BlocklaneTuning t = blocklane_tuning();
    const size_t nb = n / 128, P = (nb + 31) / 32;
    const size_t resident = (size_t)blocks_per_sm * sms;
    size_t G = max((size_t)1, min(resident, (P + bl::kW - 1) / bl::kW));
    if (t.ctas > 0 && (size_t)t.ctas < G) G = (size_t)t.ctas;
    const size_t lead = max((size_t)128, t.lead > 0 ? (size_t)t.lead : 2 * G * bl::kW);
    kern<<<(int)G, bl::kW * 32, smem, s>>>(in, in_bytes, out, n, index, meta, pmeta, umeta, h,
                                            blocklane_scratch(h, n, ws_bytes), (uint32_t)(n - 128 * nb),
                                            (uint32_t)min(lead, (size_t)0xFFFFFFFFu), (uint32_t)t.sumw);
    return cudaGetLastError();
}

template <int DELTA>
static cudaError_t launch_fpbl_d(const uint8_t* in, size_t in_bytes, uint32_t* out, size_t n, const uint64_t* index,
                                 const BlockMeta* meta, const uint32_t* pmeta, const uint2* umeta, WsHeader* h,
                                 size_t ws_bytes, cudaStream_t s) {
    int st = blocklane_tuning().store;
    if (st == bl::kStoreV8 && (reinterpret_cast<uintptr_t>(out) & 31u) != 0) st = bl::kStoreV4;
    if (st == bl::kStoreRestage)
        return launch_fpbl_t<DELTA, bl::kStoreRestage>(in, in_bytes, out, n, index, meta, pmeta, umeta, h, ws_bytes, s);
    if (st == bl::kStoreV8)
        return launch_fpbl_t<DELTA, bl::kStoreV8>(in, in_bytes, out, n, index, meta, pmeta, umeta, h, ws_bytes, s);
    return launch_fpbl_t<DELTA, bl::kStoreV4>(in, in_bytes, out, n, index, meta, pmeta, umeta, h, ws_bytes, s);
}

cudaError_t launch_fastpfor_blocklane(int delta, const uint8_t* in, size_t in_bytes, uint32_t* out, size_t n,
                                      const uint64_t* index, const BlockMeta* meta, const uint32_t* pmeta,
                                      const uint2* umeta, WsHeader* h, size_t ws_bytes, cudaStream_t s) {
    if (delta == ICX_DELTA_4)
        return launch_fpbl_d<ICX_DELTA_4>(in, in_bytes, out, n, index, meta, pmeta, umeta, h, ws_bytes, s);
    if (delta == ICX_DELTA_1)
        return launch_fpbl_d<ICX_DELTA_1>(in, in_bytes, out, n, index, meta, pmeta, umeta, h, ws_bytes, s);
    return cudaErrorInvalidValue;
}

}  // namespace icx
