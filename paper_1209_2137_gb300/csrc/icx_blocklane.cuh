// Block-per-lane decoding (one 128-integer block per GPU lane, two passes
// over a pair of 16-block groups per warp): the pieces every codec shares.
// The codec-specific parts (where a pair's bytes are, how a lane finds its
// block, the per-lane walk of a block) come in as a codec class; the task
// loop, the staging ring, the tagged sums, the group scans and the
// Variable Byte tail are here.
#pragma once

#include <cstddef>
#include <type_traits>

#include "icx_device.cuh"
#include "icx_tile.cuh"

namespace icx {

namespace bl {

constexpr int kW = 6;                  // warps per CTA
constexpr uint32_t kGroup = 64;        // pairs per group (two per lane of the warp that scans it)
constexpr uint32_t kRing = 8192;       // staging bytes per warp: two pairs in flight when they fit
constexpr uint32_t kSlack = 128;       // the window reads up to two rows past a block (keeps 128-byte alignment)
constexpr uint32_t kRestage = 4096;    // output staging: 32 blocks x 8 fields x 16 bytes
constexpr uint32_t kWarpSmem = kRing + kSlack + kRestage;
static_assert(kWarpSmem % 128 == 0 && (kRing + kSlack) % 128 == 0, "restage buffers stay 128-byte aligned");
constexpr uint32_t kHdr = 256;

struct Hdr {
    unsigned long long bar[2 * kW];  // two staging barriers per warp (left and right end of its ring)
    unsigned long long wait_limit;   // limit of the waits on published values (ns), read once
    uint32_t last;                   // this CTA finished the launch last
};
static_assert(sizeof(Hdr) <= kHdr, "header");

// Workspace region of the decoder, at the end of the caller's workspace
// (above every region the other decoders write for any length the workspace
// is sized for): tagged block sums (four 64-bit words per block), pair totals
// and pair prefixes (four words per pair each), group look-back states (four
// words per group), and a counter per group.  A word holds
// (epoch << 2 | flag) in its high half, so nothing tagged needs clearing; the
// counters are zeroed at the start of every launch by the first CTA to run.
struct Scratch {
    unsigned long long* bst;
    unsigned long long* ptot;
    unsigned long long* pre;
    unsigned long long* gst;
    unsigned int* gcnt;
};

// NL tagged words (one per chain) written by one thread.
template <int NL>
__device__ __forceinline__ void st_tagged(unsigned long long* p, uint32_t tag, uint4 v) {
    const unsigned long long t = (unsigned long long)tag << 32;
    if (NL == 1) {
        st_relaxed(p, t | v.x);
    } else {
        asm volatile("st.relaxed.gpu.global.v2.b64 [%0], {%1, %2};" ::"l"(p), "l"(t | v.x), "l"(t | v.y) : "memory");
        asm volatile("st.relaxed.gpu.global.v2.b64 [%0], {%1, %2};" ::"l"(p + 2), "l"(t | v.z), "l"(t | v.w)
                     : "memory");
    }
}

// Reads NL tagged words; true if every word carries `tag` (tag bits in IGN
// are not compared; *t0 gets the first word's tag).
template <int NL, uint32_t IGN = 0>
__device__ __forceinline__ bool ld_tagged(const unsigned long long* p, uint32_t tag, uint4& v, uint32_t* t0 = nullptr) {
    if (NL == 1) {
        const unsigned long long w = ld_relaxed(p);
        v = make_uint4((uint32_t)w, 0, 0, 0);
        if (t0) *t0 = (uint32_t)(w >> 32);
        return ((uint32_t)(w >> 32) & ~IGN) == tag;
    }
    unsigned long long w0, w1, w2, w3;
    ld_relaxed_v2(p, w0, w1);
    ld_relaxed_v2(p + 2, w2, w3);
    v = make_uint4((uint32_t)w0, (uint32_t)w1, (uint32_t)w2, (uint32_t)w3);
    if (t0) *t0 = (uint32_t)(w0 >> 32);
    return ((uint32_t)(w0 >> 32) & ~IGN) == tag && ((uint32_t)(w1 >> 32) & ~IGN) == tag &&
           ((uint32_t)(w2 >> 32) & ~IGN) == tag && ((uint32_t)(w3 >> 32) & ~IGN) == tag;
}

// Waits (bounded) until the NL words at p carry `tag`; returns their values.
template <int NL, uint32_t IGN = 0>
__device__ __forceinline__ uint4 wait_tagged(const unsigned long long* p, uint32_t tag, WsHeader* h,
                                             const unsigned long long* limit, uint32_t* t0 = nullptr) {
    uint4 v;
    if (ld_tagged<NL, IGN>(p, tag, v, t0)) return v;
    const unsigned long long ts = globaltimer();
    while (!ld_tagged<NL, IGN>(p, tag, v, t0)) {
        if (globaltimer() - ts > *limit) {
            set_error(h, ICX_ETIMEOUT);
            break;
        }
        __nanosleep(32);
    }
    return v;
}

// NL tagged words loaded without looking at them yet, so the load is in
// flight while the warp works; check_tagged reads them later.
struct RawTagged {
    unsigned long long w0, w1, w2, w3;
};

template <int NL>
__device__ __forceinline__ void ld_raw(const unsigned long long* p, RawTagged& t) {
    if (NL == 1) {
        t.w0 = ld_relaxed(p);
        t.w1 = t.w2 = t.w3 = 0;
    } else {
        ld_relaxed_v2(p, t.w0, t.w1);
        ld_relaxed_v2(p + 2, t.w2, t.w3);
    }
}

template <int NL, uint32_t IGN = 0>
__device__ __forceinline__ bool check_tagged(const RawTagged& t, uint32_t tag, uint4& v) {
    v = make_uint4((uint32_t)t.w0, (uint32_t)t.w1, (uint32_t)t.w2, (uint32_t)t.w3);
    return ((uint32_t)(t.w0 >> 32) & ~IGN) == tag &&
           (NL == 1 || (((uint32_t)(t.w1 >> 32) & ~IGN) == tag && ((uint32_t)(t.w2 >> 32) & ~IGN) == tag &&
                        ((uint32_t)(t.w3 >> 32) & ~IGN) == tag));
}

// A block sum's tag is tagA, or tagA | kSumFlag when the codec marked the
// block (SIMD-FastPFOR: exception positions out of order).
constexpr uint32_t kSumFlag = 2;

// Output store paths of pass 2.
constexpr int kStoreRestage = 0;  // 8 fields of every block through shared memory, then coalesced 16-byte stores
constexpr int kStoreV8 = 1;       // each lane stores its own 32-byte field pairs (output 32-byte aligned)
constexpr int kStoreV4 = 2;       // each lane stores its own 16-byte fields

// A pair's bytes staged in the warp's ring.  Offsets are relative to the
// staged copy; u8/u32 read the codec's other staged data (exception
// positions and high parts of SIMD-FastPFOR).
struct SmemRows {
    const uint8_t* base;
    uint32_t sb;  // shared-window address of base
    __device__ __forceinline__ uint4 operator()(uint32_t off) const {
        return *reinterpret_cast<const uint4*>(base + off);
    }
    __device__ __forceinline__ uint32_t u8(uint32_t off) const { return base[off]; }
    __device__ __forceinline__ uint32_t u32(uint32_t off) const {
        return *reinterpret_cast<const uint32_t*>(base + off);
    }
    __device__ __forceinline__ void st16(uint32_t off, uint32_t v) const {
        asm volatile("st.shared.u16 [%0], %1;" ::"r"(sb + off), "h"((unsigned short)v) : "memory");
    }
    __device__ __forceinline__ uint32_t cursor(uint32_t off) const { return sb + off; }
    // After sh += b (sh < 64): when the next field starts in the second row,
    // slide the window by one row and load the row at `nxt`; keep sh < 32.
    // Predicated, so lanes of different widths never diverge.
    __device__ __forceinline__ void advance(uint4& r0, uint4& r1, uint32_t& sh, uint32_t& nxt) const {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ge.u32 p, %8, 32;\n\t"
            "@p mov.b32 %0, %4;\n\t"
            "@p mov.b32 %1, %5;\n\t"
            "@p mov.b32 %2, %6;\n\t"
            "@p mov.b32 %3, %7;\n\t"
            "@p ld.shared.v4.u32 {%4, %5, %6, %7}, [%9];\n\t"
            "@p add.u32 %9, %9, 16;\n\t"
            "and.b32 %8, %8, 31;\n\t}"
            : "+r"(r0.x), "+r"(r0.y), "+r"(r0.z), "+r"(r0.w), "+r"(r1.x), "+r"(r1.y), "+r"(r1.z), "+r"(r1.w),
              "+r"(sh), "+r"(nxt));
    }
};

// Rows read straight from the stream (a pair too large for the ring); a read
// past the end of the stream returns zeros.
struct GlobalRows {
    const uint8_t* base;
    uint64_t avail;
    __device__ __forceinline__ uint4 operator()(uint32_t off) const {
        return (uint64_t)off + 16 <= avail ? __ldg(reinterpret_cast<const uint4*>(base + off)) : make_uint4(0, 0, 0, 0);
    }
    __device__ __forceinline__ uint32_t u8(uint32_t off) const { return off < avail ? (uint32_t)__ldg(base + off) : 0u; }
    __device__ __forceinline__ uint32_t u32(uint32_t off) const {
        return (uint64_t)off + 4 <= avail ? __ldg(reinterpret_cast<const uint32_t*>(base + off)) : 0u;
    }
    __device__ __forceinline__ void st16(uint32_t, uint32_t) const {}  // nothing is staged
    __device__ __forceinline__ uint32_t cursor(uint32_t off) const { return off; }
    __device__ __forceinline__ void advance(uint4& r0, uint4& r1, uint32_t& sh, uint32_t& nxt) const {
        if (sh >= 32) {
            sh -= 32;
            r0 = r1;
            r1 = (*this)(nxt);
            nxt += 16;
        }
    }
};

__device__ __forceinline__ void st_v8_cs(uint32_t* p, uint4 a, uint4 b) {
    asm volatile("st.global.cs.v8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "r"(a.x), "r"(a.y), "r"(a.z),
                 "r"(a.w), "r"(b.x), "r"(b.y), "r"(b.z), "r"(b.w)
                 : "memory");
}

template <int DELTA>
__device__ __forceinline__ uint4 warp_scan_carry(uint4 v, int lane) {
    if constexpr (DELTA == ICX_DELTA_4) {
        return warp_incl_scan4(v, lane);
    } else {
        return make_uint4(warp_incl_scan(v.x, lane), 0, 0, 0);
    }
}

// One lane's block while it is walked: width, two-row window, bit offset,
// running sums, and (pass B) where its decoded fields go.
struct Walk {
    uint32_t b, mask, sh, nxt;
    uint4 r0, r1, acc, prev;
    // restaged stores: write base (field i at wsb ^ 16 i), read bases for
    // blocks 4u + q (q = lane >> 3) and their output, active-block bits
    uint32_t wsb, ro0, ro1;
    uint32_t* ob;
    unsigned actq;
    // lane stores: this lane's block
    uint32_t* dst;
    bool live;
};

// Emits field r of the lane's block (pass A: adds it to the block sum; pass
// B: its decoded integers, stored through the chosen path).
template <int DELTA, bool DECODE, int STORE>
__device__ __forceinline__ void emit_field(Walk& w, uint4 f, int r, int i) {
    uint4 o;
    if (!DECODE) {
        w.acc = add4(w.acc, f);
        return;
    } else if (DELTA == ICX_DELTA_4) {
        w.acc = add4(w.acc, f);
        o = w.acc;
    } else {
        // the prefixes inside the field do not wait for the running sum, so
        // the sum's chain is one add per field
        const uint32_t p1 = f.x + f.y, p2 = p1 + f.z, p3 = p2 + f.w;
        o = make_uint4(w.acc.x + f.x, w.acc.x + p1, w.acc.x + p2, w.acc.x + p3);
        w.acc.x = o.w;
    }
    if constexpr (STORE == kStoreRestage) {
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(w.wsb ^ (16u * i)), "r"(o.x), "r"(o.y), "r"(o.z),
                     "r"(o.w)
                     : "memory");
    } else if constexpr (STORE == kStoreV8) {
        if (r & 1) {
            if (w.live) st_v8_cs(w.dst + 4 * (r - 1), w.prev, o);
        } else {
            w.prev = o;
        }
    } else {
        if (w.live) __stcs(reinterpret_cast<uint4*>(w.dst + 4 * r), o);
    }
}

// Field hook of walks that change nothing.
struct NoPatch {
    __device__ __forceinline__ void operator()(uint4&, int) {}
};

// Pass-A block sums that add several fields per operation (every width of
// the warp at most 8; b = 0 for lanes without a block).  Per residue and
// window step x holds the next fields at bits 0, b, 2b, ...:
//   MODE 4 (widths 4..8, four fields a step): one masked add folds fields
//     0 + 1 into bits [0, b + 1) and 2 + 3 into [2b, 3b + 1); the eight
//     steps add these words up.  Each half then holds at most
//     16 (2^b - 1) < 2^(b + 4) <= 2^(2b), so the low half never carries into
//     the high one, and the high half ends below bit 3b + 4 <= 28; the two
//     halves are added once at the end;
//   MODE 5 (widths 0..8, four fields a step): the same fold, its two halves
//     added at every step (b + 1 <= 2b bits each);
//   MODE 8 (widths 0..4, eight fields a step): pairs fold into bits 0, 2b,
//     4b, 6b (b + 1 bits each), the pairs into quads at 0 and 4b (b + 2 <= 4b
//     bits each), and the quads are added at every step.
// The same integers as adding the 32 fields one by one (mod 2^32 like
// them), with 5, 8 and 10 operations per residue and step instead of 11,
// 11 and 23.
template <int MODE, class Rows, class Mid>
__device__ __forceinline__ void sum_block_swar(const Rows& rows, Walk& w, Mid& mid) {
    constexpr int FPS = MODE == 8 ? 8 : 4;
    const uint32_t b = w.b, step = FPS * b, b2 = 2 * b, b4 = 4 * b;
    const uint32_t m2 = w.mask | (w.mask << b2), lo = w.mask | (w.mask << b);  // lo: the low 2b bits
    // (b <= 4 in MODE 8, so these shifts stay below 32)
    const uint32_t mE = MODE == 8 ? m2 | (m2 << b4) : 0u, mQ = MODE == 8 ? lo | (lo << b4) : 0u,
                   m4 = MODE == 8 ? lo | (lo << b2) : 0u;
    auto fold = [&](uint32_t x) -> uint32_t {
        if constexpr (MODE == 8) {
            const uint32_t s1 = (x & mE) + ((x >> b) & mE);
            const uint32_t s2 = (s1 & mQ) + ((s1 >> b2) & mQ);
            return (s2 & m4) + (s2 >> b4);
        } else {
            const uint32_t t = (x & m2) + ((x >> b) & m2);
            return MODE == 4 ? t : (t & lo) + (t >> b2);
        }
    };
    uint4 s = make_uint4(0, 0, 0, 0);
#pragma unroll 1
    for (int c = 0; c < 4; ++c) {
#pragma unroll
        for (int i = 0; i < 8; i += FPS) {
            uint4 x;
            x.x = __funnelshift_r(w.r0.x, w.r1.x, w.sh);
            x.y = __funnelshift_r(w.r0.y, w.r1.y, w.sh);
            x.z = __funnelshift_r(w.r0.z, w.r1.z, w.sh);
            x.w = __funnelshift_r(w.r0.w, w.r1.w, w.sh);
            w.sh += step;
            rows.advance(w.r0, w.r1, w.sh, w.nxt);
            s.x += fold(x.x);
            s.y += fold(x.y);
            s.z += fold(x.z);
            s.w += fold(x.w);
        }
        if (c == 0) mid();
    }
    if constexpr (MODE == 4)
        s = make_uint4((s.x & lo) + (s.x >> b2), (s.y & lo) + (s.y >> b2), (s.z & lo) + (s.z >> b2),
                       (s.w & lo) + (s.w >> b2));
    w.acc = add4(w.acc, s);
}

// The 32 fields of the lane's block, FPS fields per window step: with every
// width of the pair at most 32 / FPS, the FPS fields from the current bit
// offset all lie in one 32-bit funnel shift of the window, so the window
// moves once per FPS fields.  `patch(f, r)` may change field r before it is
// emitted.
//
// Pass A without a patch takes sum_block_swar when the widths allow: MODE 4
// always, MODES 8 and 5 only with SMALL.  (With all three the SIMD-BP128
// stride-1 decoder spills registers and measured 0.0819 against 0.0778 ms
// on 2^26 integers; the SIMD-FastPFOR prepare kernel, whose widths are
// smaller, gained 0.1126 -> 0.1090 ms on the clustered array.)
template <int DELTA, bool DECODE, int STORE, int FPS, bool SMALL = false, class Rows, class Mid, class Patch>
__device__ __forceinline__ void walk_block(const Rows& rows, Walk& w, Mid& mid, Patch& patch) {
    if constexpr (!DECODE && FPS == 4 && std::is_same<Patch, NoPatch>::value) {
        const uint32_t mx = __reduce_max_sync(FULL, w.b);
        if (SMALL && mx <= 4u) {
            sum_block_swar<8>(rows, w, mid);
            return;
        }
        if (mx <= 8u) {
            if (__reduce_min_sync(FULL, w.b ? w.b : 32u) >= 4u) {
                sum_block_swar<4>(rows, w, mid);
                return;
            }
            if (SMALL) {
                sum_block_swar<5>(rows, w, mid);
                return;
            }
        }
    }
    const uint32_t b2 = 2 * w.b, b3 = 3 * w.b, step = FPS * w.b;
#pragma unroll 1
    for (int c = 0; c < 4; ++c) {
#pragma unroll
        for (int i = 0; i < 8; i += FPS) {
            uint4 x;
            x.x = __funnelshift_r(w.r0.x, w.r1.x, w.sh);
            x.y = __funnelshift_r(w.r0.y, w.r1.y, w.sh);
            x.z = __funnelshift_r(w.r0.z, w.r1.z, w.sh);
            x.w = __funnelshift_r(w.r0.w, w.r1.w, w.sh);
            w.sh += step;
            rows.advance(w.r0, w.r1, w.sh, w.nxt);
#pragma unroll
            for (int j = 0; j < FPS; ++j) {
                const uint32_t s = j == 0 ? 0u : j == 1 ? w.b : j == 2 ? b2 : b3;
                uint4 f = make_uint4((x.x >> s) & w.mask, (x.y >> s) & w.mask, (x.z >> s) & w.mask,
                                     (x.w >> s) & w.mask);
                patch(f, 8 * c + i + j);
                emit_field<DELTA, DECODE, STORE>(w, f, 8 * c + i + j, i + j);
            }
        }
        if constexpr (DECODE && STORE == kStoreRestage) {
            __syncwarp();
            uint32_t* const oc = w.ob + 32 * c;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                uint4 v;
                asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
                             : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                             : "r"((u & 1 ? w.ro1 : w.ro0) + 512u * u)
                             : "memory");
                if (w.actq & (1u << (4 * u))) __stcs(reinterpret_cast<uint4*>(oc + 512 * u), v);
            }
            __syncwarp();
        }
        if (c == 0) mid();
    }
}

// Loads a value another CTA wrote in this launch (bypassing L1).
__device__ __forceinline__ uint4 ld_cg4(const uint4* p) { return __ldcg(p); }

__device__ __forceinline__ uint32_t ld_acquire_u32(const unsigned int* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <int NL>
__device__ __forceinline__ uint4 warp_sum(uint4 v) {
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        v.x += __shfl_xor_sync(FULL, v.x, off);
        if (NL == 4) {
            v.y += __shfl_xor_sync(FULL, v.y, off);
            v.z += __shfl_xor_sync(FULL, v.z, off);
            v.w += __shfl_xor_sync(FULL, v.w, off);
        }
    }
    return v;
}


// The task loop.  A persistent grid; task u (from the workspace's tile
// counter) maps to:
//   u < L0:                              A task of pair u
//   v = u - L0 < 2 (P - L0), v even:     A task of pair L0 + v/2
//   v = u - L0 < 2 (P - L0), v odd:      B task of pair v/2
//   otherwise:                           B task of pair v - (P - L0)
// with B index P the Variable Byte tail (`tail` = n % 128 integers,
// Sec. 2.4).  With L0 >= 128 the A tasks of every pair in the group of a B
// task's pair (and of every earlier group) come before it, so a task only
// waits for tasks taken before it.  The last CTA to finish resets the
// counters and advances the epoch.
//
// The codec C supplies, for pair p: `load(p, lane)` (the loads that describe
// it, issued a task ahead and looked at later), `describe(p, pre, lane)`
// (its Desc, with `ok`), `space(d)` (bytes it takes in the ring, 0: read it
// from the stream), `issue(d, dst, bar, policy, lane)` (arm the barrier with
// the bytes it copies and start the copies), `global_rows(d)`, `blocks<..>`
// (pass A: the lane's block sum, and in `flag` a mark kept with it; pass B:
// decode and store the block, given that mark), `ahead` /
// `prefetch` (pull a pair about one round ahead into L2) and `tail_start()`.
template <class C, int DELTA, int STORE>
__device__ __forceinline__ void run(const C& codec, const uint8_t* __restrict__ in, size_t in_bytes,
                                    uint32_t* __restrict__ out, size_t n, WsHeader* h, Scratch sc, uint32_t tail,
                                    uint32_t lead, uint32_t sumw) {
    constexpr int NL = DELTA == ICX_DELTA_4 ? 4 : 1;
    extern __shared__ __align__(128) uint8_t smem[];
    Hdr& S = *reinterpret_cast<Hdr*>(smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t* ring = smem + kHdr + (size_t)warp * kWarpSmem;
    uint8_t* rest = ring + kRing + kSlack;
    uint64_t* bar = reinterpret_cast<uint64_t*>(&S.bar[2 * warp]);
    const uint32_t epoch = launch_epoch(h);
    const uint32_t tagA = (epoch << 2) | 1u, tagI = (epoch << 2) | 2u;
    const size_t nb = n / 128;
    const uint32_t P = (uint32_t)((nb + 31) / 32);
    const uint32_t Gn = (P + kGroup - 1) / kGroup;
    const uint32_t L0 = min(P, lead), RA = P - L0;
    const uint32_t ntasks = 2 * P + (tail ? 1u : 0u);
    const uint32_t nwarps = gridDim.x * kW;
    if (lane == 0) {
        mbar_init(bar, 1);
        mbar_init(bar + 1, 1);
    }
    fence_mbar_init();
    // the first CTA to start zeroes the group counters, then raises aux[3]
    if (threadIdx.x == 0) {
        S.last = atomicAdd(&h->aux[4], 1u) == 0 ? 1u : 0u;
        S.wait_limit = wait_limit_ns(h);
    }
    __syncthreads();
    if (S.last) {
        for (uint32_t i = threadIdx.x; i < Gn; i += blockDim.x) sc.gcnt[i] = 0;
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) atomicExch(&h->aux[3], epoch + 1u);
    }
    bool counters_ready = false;

    // Task ids come from one counter; the atomic for a task is issued an
    // iteration before its value is used (take_async, then task_of).
    // Task kinds: 0 = A (sum), 1 = B (decode), 2 = tail, 3 = none left.
    // With sumw > 0 the first sumw warps of every CTA take only A tasks (pairs
    // in order, from the tile counter) and the others only B tasks (pairs in
    // order, then the tail, from aux[0]).
    const int role = sumw == 0 ? 0 : (warp < (int)sumw ? 1 : 2);
    unsigned int* const ctr = role == 2 ? &h->aux[0] : &h->tile_counter;
    auto take_async = [&]() -> uint32_t {
        uint32_t u = 0;
        if (lane == 0) u = atomicAdd(ctr, 1u);
        return u;
    };
    auto task_of = [&](uint32_t raw, uint32_t& kind, uint32_t& p) {
        const uint32_t u = __shfl_sync(FULL, raw, 0);
        if (role != 0) {
            p = u;
            kind = role == 1 ? (u < P ? 0u : 3u) : (u < P ? 1u : (u == P && tail) ? 2u : 3u);
        } else if (u >= ntasks) {
            kind = 3;
            p = 0;
        } else if (u < L0) {
            kind = 0;
            p = u;
        } else {
            const uint32_t v = u - L0;
            uint32_t b;
            if (v < 2 * RA) {
                if (!(v & 1)) {
                    kind = 0;
                    p = L0 + v / 2;
                    return;
                }
                b = v / 2;
            } else {
                b = v - RA;
            }
            kind = b < P ? 1u : 2u;
            p = b;
        }
    };

    // Staging ring: copy number s sits at the left end of the ring when s is
    // even, at the right end when odd, so two consecutive copies share the
    // ring when their sizes add up to at most kRing.  Every copy arms its
    // barrier once (with the copy's bytes, or none for a pair read straight
    // from the stream), so the barrier phases stay in step.
    using Desc = typename C::Desc;
    using Pre = typename C::Pre;
    uint32_t s_iss = 0, s_wt = 0;
    bool broken = false;
    auto slot = [&](uint32_t s, const Desc& d) -> uint32_t { return (s & 1) ? kRing - codec.space(d) : 0u; };
    auto issue = [&](const Desc& d, uint64_t policy) -> uint32_t {
        const uint32_t s = s_iss;
        if (!broken) {
            codec.issue(d, ring + slot(s, d), bar + (s & 1), policy, lane);
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
    auto fits = [&](const Desc& a, const Desc& b) { return codec.space(a) + codec.space(b) <= kRing; };
    const uint64_t keep = l2_policy_evict_last(), drop = l2_policy_evict_first();

    // The group scan, run by the A task that completes group g: the group
    // total (lane l adds pairs 2l and 2l+1, both loads in flight at once), a
    // decoupled look-back over the groups, and every pair's exclusive prefix.
    auto scan_group = [&](uint32_t g) {
        const uint32_t p0 = g * kGroup + 2 * lane;
        uint4 v0 = make_uint4(0, 0, 0, 0), v1 = v0;
        bool ok0 = true, ok1 = true;
        if (p0 < P) ok0 = ld_tagged<NL>(sc.ptot + 4 * (size_t)p0, tagA, v0);
        if (p0 + 1 < P) ok1 = ld_tagged<NL>(sc.ptot + 4 * (size_t)(p0 + 1), tagA, v1);
        if (!ok0) v0 = wait_tagged<NL>(sc.ptot + 4 * (size_t)p0, tagA, h, &S.wait_limit);
        if (!ok1) v1 = wait_tagged<NL>(sc.ptot + 4 * (size_t)(p0 + 1), tagA, h, &S.wait_limit);
        const uint4 ls = add4(v0, v1);
        const uint4 li = warp_scan_carry<DELTA>(ls, lane);
        const uint4 agg = shfl4(li, 31);
        if (lane < NL)
            st_relaxed(sc.gst + 4 * (size_t)g + lane, ((unsigned long long)(g ? tagA : tagI) << 32) | comp(agg, lane));
        const uint4 ex = lookback_resolve_at<NL>(sc.gst, h, epoch, g, agg, true, &S.wait_limit);
        const uint4 e0 = add4(ex, sub4(li, ls));
        if (p0 < P) st_tagged<NL>(sc.pre + 4 * (size_t)p0, tagI, e0);
        if (p0 + 1 < P) st_tagged<NL>(sc.pre + 4 * (size_t)(p0 + 1), tagI, add4(e0, v0));
    };
    // prefix and block sums of a B task: loaded one task ahead, looked at
    // when the task starts (and waited for only if they were not yet
    // published)
    RawTagged pr, br;
    auto load_b = [&](uint32_t p) {
        ld_raw<NL>(sc.pre + 4 * (size_t)p, pr);
        const size_t blk = 32 * (size_t)p + lane;
        if (blk < nb) ld_raw<NL>(sc.bst + 4 * blk, br);
    };
    auto load = [&](uint32_t kind, uint32_t p) -> Pre { return kind <= 1 ? codec.load(p, lane) : Pre{}; };

    uint32_t kc, pc, kn, pn;
    task_of(take_async(), kc, pc);
    Desc dc;
    uint32_t s_cur = 0;
    if (kc <= 1) {
        dc = codec.describe(pc, codec.load(pc, lane), lane);
        s_cur = issue(dc, kc == 0 ? keep : drop);
        if (kc == 1) load_b(pc);
    }
    task_of(take_async(), kn, pn);
    Pre en = load(kn, pn);
    while (kc != 3) {
        // the current B task's prefix and block sum, loaded an iteration ago
        uint4 pre_c = make_uint4(0, 0, 0, 0), bs_c = pre_c;
        bool pre_ok = true, bs_ok = true;
        uint32_t bflag = 0;  // the codec's mark on this lane's block (pass A sets it, pass B reads it)
        if (kc == 1) {
            pre_ok = check_tagged<NL>(pr, tagI, pre_c);
            if (32 * (size_t)pc + lane < nb) {
                bs_ok = check_tagged<NL, kSumFlag>(br, tagA, bs_c);
                bflag = (uint32_t)(br.w0 >> 32) & kSumFlag;
            }
        }
        // the task after next: its id is taken now and read, with its
        // describing loads requested, a quarter of the way through the
        // current task
        const uint32_t raw2 = take_async();
        uint32_t kk = 3, pk = 0;
        Pre ek{};
        bool mid_done = false;
        auto mid = [&]() {
            task_of(raw2, kk, pk);
            ek = load(kk, pk);
            mid_done = true;
        };
        Desc dn;
        uint32_t s_nx = 0;
        bool nx_issued = false;
        if (kn <= 1) {
            dn = codec.describe(pn, en, lane);
            if (kc > 1 || fits(dc, dn)) {
                s_nx = issue(dn, kn == 0 ? keep : drop);
                nx_issued = true;
            }
            if (kn == 1) load_b(pn);
        }
        if (kc == 0) {
            // ------------------------------------------------------ A task
            // the pair some warp sums about one round from now goes into L2
            // (its location is read now, the prefetch is issued after the
            // sums)
            typename C::Ahead ahead{};
            if (pc + nwarps < P) ahead = codec.ahead(pc + nwarps, lane);
            uint4 bs = make_uint4(0, 0, 0, 0);
            if (wait()) {
                if (!dc.ok) {
                    if (lane == 0) set_error(h, ICX_ECORRUPT);
                } else if (codec.space(dc)) {
                    bs = codec.template blocks<DELTA, false, 0>(
                        SmemRows{ring + slot(s_cur, dc), smem_u32(ring + slot(s_cur, dc))}, dc, bs, bflag, out, 0,
                        rest, h, lane, mid);
                } else {
                    bs = codec.template blocks<DELTA, false, 0>(codec.global_rows(dc), dc, bs, bflag, out, 0, rest, h,
                                                                lane, mid);
                }
            }
            __syncwarp();
            if (pc + nwarps < P) codec.prefetch(ahead, keep, lane);
            const size_t blk = 32 * (size_t)pc + lane;
            if (blk < nb) st_tagged<NL>(sc.bst + 4 * blk, tagA | (bflag & kSumFlag), bs);
            const uint4 tot = warp_sum<NL>(bs);
            // the group's counter (zeroed by the first CTA of this launch,
            // which raises aux[3] to epoch + 1 when done)
            if (!counters_ready) {
                if (lane == 0) {
                    const unsigned long long t0 = globaltimer();
                    while (ld_acquire_u32(&h->aux[3]) != epoch + 1u) {
                        if (globaltimer() - t0 > S.wait_limit) {
                            set_error(h, ICX_ETIMEOUT);
                            break;
                        }
                        __nanosleep(32);
                    }
                }
                __syncwarp();
                counters_ready = true;
            }
            const uint32_t g = pc / kGroup;
            uint32_t last = 0;
            if (lane == 0) {
                st_tagged<NL>(sc.ptot + 4 * (size_t)pc, tagA, tot);
                last = atomicAdd(&sc.gcnt[g], 1u) == min(kGroup, P - g * kGroup) - 1 ? 1u : 0u;
            }
            if (__shfl_sync(FULL, last, 0)) scan_group(g);
        } else if (kc == 1) {
            // ------------------------------------------------------ B task
            if (!__all_sync(FULL, pre_ok)) pre_c = wait_tagged<NL>(sc.pre + 4 * (size_t)pc, tagI, h, &S.wait_limit);
            if (!bs_ok) {
                uint32_t t0 = 0;
                bs_c = wait_tagged<NL, kSumFlag>(sc.bst + 4 * (32 * (size_t)pc + lane), tagA, h, &S.wait_limit, &t0);
                bflag = t0 & kSumFlag;
            }
            const uint4 bi = warp_scan_carry<DELTA>(bs_c, lane);
            const uint4 carry = add4(pre_c, sub4(bi, bs_c));
            if (wait() && dc.ok) {
                const size_t first = 4096 * (size_t)pc;
                if (codec.space(dc))
                    codec.template blocks<DELTA, true, STORE>(
                        SmemRows{ring + slot(s_cur, dc), smem_u32(ring + slot(s_cur, dc))}, dc, carry, bflag, out,
                        first, rest, h, lane, mid);
                else
                    codec.template blocks<DELTA, true, STORE>(codec.global_rows(dc), dc, carry, bflag, out, first,
                                                              rest, h, lane, mid);
            }
            __syncwarp();
        } else {
            // ---------------------------------------- the Variable Byte tail
            // its carry is the inclusive prefix of the last group
            uint4 carry = make_uint4(0, 0, 0, 0);
            if (P > 0) carry = wait_tagged<NL>(sc.gst + 4 * (size_t)(Gn - 1), tagI, h, &S.wait_limit);
            uint32_t* scratch = reinterpret_cast<uint32_t*>(rest);
            const uint64_t tstart = codec.tail_start();
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
            for (int c = 0; c < 4; ++c)
                if (q0 + c < n) out[q0 + c] = comp(o, c);
            __syncwarp();
        }
        if (!mid_done) mid();  // the task had no fields to walk
        if (kn <= 1 && !nx_issued) s_nx = issue(dn, kn == 0 ? keep : drop);
        kc = kn;
        pc = pn;
        kn = kk;
        pn = pk;
        en = ek;
        dc = dn;
        s_cur = s_nx;
    }
    // a copy that never landed must not outlive the CTA's shared memory
    if (broken)
        for (uint32_t s = s_wt; s < s_iss; ++s) mbar_wait(bar + (s & 1), (s >> 1) & 1u);

    // the last CTA resets the counters and advances the epoch
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        S.last = atomicAdd(&h->done_counter, 1u) == gridDim.x - 1 ? 1u : 0u;
    }
    __syncthreads();
    if (S.last) {
        __threadfence();
        if (threadIdx.x == 0) {
            h->tile_counter = 0;
            h->aux[0] = 0;
            h->aux[4] = 0;
            h->done_counter = 0;
            atomicExch(&h->epoch, (epoch + 1u) & 0x3FFFFFFFu);
        }
        __threadfence();
    }
}

}  // namespace bl

// Scratch layout of a decode of n integers inside a workspace of ws_bytes
// bytes at h: the last ws_blocklane_bytes(n) bytes (from a 256-byte
// boundary).  Every plain region any decoder writes for a length m the
// workspace serves ends below ws_bytes - ws_blocklane_bytes(capacity) (the
// layout in icx_device.cuh), and this region grows with the length, so only
// tagged words of these decoders are ever written here.
inline bl::Scratch blocklane_scratch(WsHeader* h, size_t n, size_t ws_bytes) {
    const size_t nb = n / 128, P = (nb + 31) / 32, Gn = (P + bl::kGroup - 1) / bl::kGroup;
    const size_t at = (ws_bytes - ws_blocklane_bytes(n)) / 256 * 256;
    unsigned long long* base = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(h) + at);
    bl::Scratch sc;
    sc.bst = base;
    sc.ptot = sc.bst + 4 * (nb + 1);
    sc.pre = sc.ptot + 4 * (P + 1);
    sc.gst = sc.pre + 4 * (P + 1);
    sc.gcnt = reinterpret_cast<unsigned int*>(sc.gst + 4 * (Gn + 1));
    return sc;
}

// Tuning of the block-per-lane decoders (host settings, shared by codecs).
struct BlocklaneTuning {
    int store, ctas, lead, sumw;
};
BlocklaneTuning blocklane_tuning();

}  // namespace icx
