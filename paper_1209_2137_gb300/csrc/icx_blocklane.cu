// SIMD-BP128 decoding fused with differential decoding (Sec. 3, Sec. 4,
// Sec. 6.2) in two passes with one block per lane.
//
// The paper decodes a block with a 4-lane SIMD register: step r unpacks field
// r of the four lanes, integers 4r..4r+3 of the block, and the stride-4
// prefix sum is one vector add per step (Sec. 3, Fig. 7).  Here each GPU
// lane plays that register for one block: it walks the block's 32 fields in
// order through a two-row window over the block's 16-byte rows, so both the
// stride-4 chains and the stride-1 chain advance inside the lane.  A warp
// takes a pair of metablocks (32 blocks, one per lane).
//
// Carries come from summing the blocks first instead of a chained
// look-back.  An A task sums the blocks of one metablock pair and publishes
// the block sums and the pair total; the A task that completes a group of
// 64 pairs adds the group up, runs a decoupled look-back over the groups and
// publishes every pair's exclusive prefix.  A B task copies the same pair
// again (from L2), gives every lane its block's carry (pair prefix plus the
// block sums before it in the pair) and decodes and writes each integer
// once.  Warps take tasks from one counter: A tasks alone
// for a lead of pairs, then A and B tasks alternately (A runs a lead ahead of
// B), then the remaining B tasks, so the summing (compute bound) overlaps the
// stores (bandwidth bound).  Every task waits only for tasks taken before
// it, and every published value is a set of 64-bit words tagged with the
// launch epoch, so readers need no fences.
#include <cstddef>

#include "icx_bp128.cuh"
#include "icx_kernels.cuh"

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

// Reads NL tagged words; true if every word carries `tag`.
template <int NL>
__device__ __forceinline__ bool ld_tagged(const unsigned long long* p, uint32_t tag, uint4& v) {
    if (NL == 1) {
        const unsigned long long w = ld_relaxed(p);
        v = make_uint4((uint32_t)w, 0, 0, 0);
        return (uint32_t)(w >> 32) == tag;
    }
    unsigned long long w0, w1, w2, w3;
    ld_relaxed_v2(p, w0, w1);
    ld_relaxed_v2(p + 2, w2, w3);
    v = make_uint4((uint32_t)w0, (uint32_t)w1, (uint32_t)w2, (uint32_t)w3);
    return (uint32_t)(w0 >> 32) == tag && (uint32_t)(w1 >> 32) == tag && (uint32_t)(w2 >> 32) == tag &&
           (uint32_t)(w3 >> 32) == tag;
}

// Waits (bounded) until the NL words at p carry `tag`; returns their values.
template <int NL>
__device__ __forceinline__ uint4 wait_tagged(const unsigned long long* p, uint32_t tag, WsHeader* h) {
    uint4 v;
    if (ld_tagged<NL>(p, tag, v)) return v;
    const unsigned long long t0 = globaltimer();
    while (!ld_tagged<NL>(p, tag, v)) {
        if (globaltimer() - t0 > kWaitLimitNs) {
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

template <int NL>
__device__ __forceinline__ bool check_tagged(const RawTagged& t, uint32_t tag, uint4& v) {
    v = make_uint4((uint32_t)t.w0, (uint32_t)t.w1, (uint32_t)t.w2, (uint32_t)t.w3);
    return (uint32_t)(t.w0 >> 32) == tag &&
           (NL == 1 || ((uint32_t)(t.w1 >> 32) == tag && (uint32_t)(t.w2 >> 32) == tag && (uint32_t)(t.w3 >> 32) == tag));
}

// Output store paths of pass 2.
constexpr int kStoreRestage = 0;  // 8 fields of every block through shared memory, then coalesced 16-byte stores
constexpr int kStoreV8 = 1;       // each lane stores its own 32-byte field pairs (output 32-byte aligned)
constexpr int kStoreV4 = 2;       // each lane stores its own 16-byte fields

// One pair of metablocks as the warp sees it: byte offset of the second
// metablock, total size, number of metablocks (1 or 2) and their blocks.
struct Pair {
    uint64_t start;
    uint32_t off1, size;
    uint32_t mcount, K0, K1;
    bool ok;
};

struct SmemRows {
    const uint8_t* base;
    uint32_t sb;  // shared-window address of base
    __device__ __forceinline__ uint4 operator()(uint32_t off) const {
        return *reinterpret_cast<const uint4*>(base + off);
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

// Rows read straight from the stream (a pair too large for the ring); a row
// past the end of the stream reads as zeros.
struct GlobalRows {
    const uint8_t* base;
    uint64_t avail;
    __device__ __forceinline__ uint4 operator()(uint32_t off) const {
        return (uint64_t)off + 16 <= avail ? __ldg(reinterpret_cast<const uint4*>(base + off)) : make_uint4(0, 0, 0, 0);
    }
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

// One pair: lane L takes block L & 15 of metablock L >> 4.  Pass 1
// (DECODE false) returns the block's sum (stride 4: one per residue, stride
// 1: in .x).  Pass 2 decodes the block with `carry` (its exclusive prefix)
// and writes it.  A metablock whose widths exceed 32 or disagree with its
// size is recorded as corrupt and decoded as zeros.
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

// The 32 fields of the lane's block, FPS fields per window step: with every
// width of the pair at most 32 / FPS, the FPS fields from the current bit
// offset all lie in one 32-bit funnel shift of the window, so the window
// moves once per FPS fields.
template <int DELTA, bool DECODE, int STORE, int FPS, class Rows, class Mid>
__device__ __forceinline__ void walk_block(const Rows& rows, Walk& w, Mid& mid) {
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
                const uint4 f = make_uint4((x.x >> s) & w.mask, (x.y >> s) & w.mask, (x.z >> s) & w.mask,
                                           (x.w >> s) & w.mask);
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

// One pair: lane L takes block L & 15 of metablock L >> 4.  Pass A (DECODE
// false) returns the block's sum (stride 4: one per residue, stride 1: in
// .x).  Pass B decodes the block with `carry` (its exclusive prefix) and
// writes it.  A metablock whose widths exceed 32 or disagree with its size is
// recorded as corrupt and decoded as zeros.  `mid` runs once, after the
// first quarter of the fields (the caller's work that should overlap them).
template <int DELTA, bool DECODE, int STORE, class Rows, class Mid>
__device__ __forceinline__ uint4 pair_blocks(const Rows& rows, const Pair& d, uint4 carry, uint32_t* __restrict__ out,
                                             size_t pair_first, uint8_t* rest, WsHeader* h, int lane, Mid& mid) {
    const int m = lane >> 4, k = lane & 15;
    const uint32_t K = m ? d.K1 : d.K0;
    const bool in_meta = (uint32_t)m < d.mcount;
    const bool active = in_meta && (uint32_t)k < K;
    const uint32_t moff = m ? d.off1 : 0u;
    const uint32_t msize = d.mcount == 2 ? (m ? d.size - d.off1 : d.off1) : d.size;
    const uint4 desc = rows(in_meta ? moff : 0u);
    uint32_t b = active ? desc_width(desc, k) : 0u;
    uint32_t incl = b;
#pragma unroll
    for (int off = 1; off < 16; off <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, incl, off, 16);
        if (k >= off) incl += y;
    }
    const uint32_t tot = __shfl_sync(FULL, incl, 15, 16);
    const unsigned wide = (__ballot_sync(FULL, b > 32) >> (16 * m)) & 0xFFFFu;
    const bool bad = in_meta && (wide != 0 || 16 + 16 * tot != msize);
    if (bad && k == 0) set_error(h, ICX_ECORRUPT);
    uint32_t base = moff + 16 + 16 * (incl - b);
    if (bad || !active) {
        b = 0;
        base = 0;
    }
    Walk w;
    w.b = b;
    w.mask = width_mask(b);
    w.r0 = rows(base);
    w.r1 = rows(base + 16);
    w.nxt = rows.cursor(base + 32);
    w.sh = 0;
    w.acc = DECODE ? carry : make_uint4(0, 0, 0, 0);
    w.prev = make_uint4(0, 0, 0, 0);
    w.live = active && !bad;
    w.dst = out + pair_first + 128 * (size_t)lane;  // this lane's block
    // Restage layout (rest is 128-byte aligned): field i of block kb at row
    // 8 kb + (i ^ (kb & 7)), conflict-free for the lane-per-block writes and
    // the row-per-lane reads.  Write address of field i: wsb ^ 16 i.  Read
    // u (blocks 4u + q, q = lane >> 3; field lane & 7): 512 u + ro[u & 1].
    const uint32_t q = lane >> 3, i7 = lane & 7;
    w.wsb = smem_u32(rest) + 128 * lane + 16 * (lane & 7);
    const uint32_t rsb = smem_u32(rest) + 128 * q;
    w.ro0 = rsb + 16 * (i7 ^ q);
    w.ro1 = rsb + 16 * (i7 ^ (q + 4));
    w.ob = out + pair_first + 128 * q + 4 * i7;
    w.actq = __ballot_sync(FULL, w.live) >> q;
    // fields per window step, the same for the whole warp
    const uint32_t maxb = __reduce_max_sync(FULL, b);
    if (maxb <= 8)
        walk_block<DELTA, DECODE, STORE, 4>(rows, w, mid);
    else if (maxb <= 16)
        walk_block<DELTA, DECODE, STORE, 2>(rows, w, mid);
    else
        walk_block<DELTA, DECODE, STORE, 1>(rows, w, mid);
    if constexpr (DECODE) {
        return make_uint4(0, 0, 0, 0);
    } else {
        if (DELTA == ICX_DELTA_1) w.acc = make_uint4(w.acc.x + w.acc.y + w.acc.z + w.acc.w, 0, 0, 0);
        return w.acc;
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

}  // namespace bl

// The decode (see the top of this file).  A persistent grid; task u (from
// the workspace's tile counter) maps to:
//   u < L0:                              A task of pair u
//   v = u - L0 < 2 (P - L0), v even:     A task of pair L0 + v/2
//   v = u - L0 < 2 (P - L0), v odd:      B task of pair v/2
//   otherwise:                           B task of pair v - (P - L0)
// with B index P the Variable Byte tail (`tail` = n % 128 integers,
// Sec. 2.4).  With L0 >= 128 the A tasks of every pair in the group of a B
// task's pair (and of every earlier group) come before it, so a task only
// waits for tasks taken before it.  The last CTA to finish resets the
// counters and advances the epoch.
template <int DELTA, int STORE>
__global__ void __maxnreg__(96)
    bp128_blocklane_kernel(const uint8_t* __restrict__ in, size_t in_bytes, uint32_t* __restrict__ out, size_t n,
                           const uint64_t* __restrict__ index, WsHeader* h, bl::Scratch sc, uint32_t tail,
                           uint32_t lead, uint32_t sumw) {
    using namespace bl;
    constexpr int NL = DELTA == ICX_DELTA_4 ? 4 : 1;
    extern __shared__ __align__(128) uint8_t smem[];
    Hdr& S = *reinterpret_cast<Hdr*>(smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t* ring = smem + kHdr + (size_t)warp * kWarpSmem;
    uint8_t* rest = ring + kRing + kSlack;
    uint64_t* bar = reinterpret_cast<uint64_t*>(&S.bar[2 * warp]);
    const uint32_t epoch = launch_epoch(h);
    const uint32_t tagA = (epoch << 2) | 1u, tagI = (epoch << 2) | 2u;
    const size_t nb = n / 128, M = (nb + 15) / 16;
    const uint32_t P = (uint32_t)((M + 1) / 2);
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
    if (threadIdx.x == 0) S.last = atomicAdd(&h->aux[4], 1u) == 0 ? 1u : 0u;
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
    // the index entries of pair p (lanes 0..2), then the pair they describe
    auto index_entry = [&](uint32_t p) -> uint64_t {
        return lane < 3 ? __ldg(index + min((size_t)2 * p + lane, M)) : 0ull;
    };
    auto pair_from = [&](uint32_t p, uint64_t e) -> Pair {
        const uint64_t a = __shfl_sync(FULL, e, 0), b1 = __shfl_sync(FULL, e, 1), c = __shfl_sync(FULL, e, 2);
        Pair d;
        const size_t mb = 2 * (size_t)p;
        d.mcount = M - mb >= 2 ? 2u : 1u;
        const uint64_t end = d.mcount == 2 ? c : b1;
        d.K0 = (uint32_t)min((size_t)16, nb - 16 * mb);
        d.K1 = d.mcount == 2 ? (uint32_t)min((size_t)16, nb - 16 * (mb + 1)) : 0u;
        d.ok = a <= b1 && b1 <= end && end <= in_bytes && ((a | b1 | end) & 15) == 0 && b1 - a >= 16 &&
               b1 - a <= (uint64_t)kMetaMax && (d.mcount == 1 || (end - b1 >= 16 && end - b1 <= (uint64_t)kMetaMax));
        d.start = a;
        d.off1 = d.ok ? (uint32_t)(b1 - a) : 0u;
        d.size = d.ok ? (uint32_t)(end - a) : 0u;
        return d;
    };

    // Staging ring: copy number s sits at the left end of the ring when s is
    // even, at the right end when odd, so two consecutive copies share the
    // ring when their sizes add up to at most kRing.  Every copy arms its
    // barrier once (with the copy's bytes, or none for a pair read straight
    // from the stream), so the barrier phases stay in step.
    uint32_t s_iss = 0, s_wt = 0;
    bool broken = false;
    auto space = [&](const Pair& d) -> uint32_t { return d.ok && d.size <= kRing ? d.size : 0u; };
    auto slot = [&](uint32_t s, const Pair& d) -> uint32_t { return (s & 1) ? kRing - space(d) : 0u; };
    auto issue = [&](const Pair& d, uint64_t policy) -> uint32_t {
        const uint32_t s = s_iss;
        if (!broken) {
            if (lane == 0) {
                const uint32_t bytes = space(d);
                fence_proxy_async();
                mbar_expect_tx(bar + (s & 1), bytes);
                if (bytes) bulk_load_hint(ring + slot(s, d), in + d.start, bytes, bar + (s & 1), policy);
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
    auto fits = [&](const Pair& a, const Pair& b) { return space(a) + space(b) <= kRing; };
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
        if (!ok0) v0 = wait_tagged<NL>(sc.ptot + 4 * (size_t)p0, tagA, h);
        if (!ok1) v1 = wait_tagged<NL>(sc.ptot + 4 * (size_t)(p0 + 1), tagA, h);
        const uint4 ls = add4(v0, v1);
        const uint4 li = warp_scan_carry<DELTA>(ls, lane);
        const uint4 agg = shfl4(li, 31);
        if (lane < NL)
            st_relaxed(sc.gst + 4 * (size_t)g + lane, ((unsigned long long)(g ? tagA : tagI) << 32) | comp(agg, lane));
        const uint4 ex = lookback_resolve_at<NL>(sc.gst, h, epoch, g, agg);
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

    uint32_t kc, pc, kn, pn;
    task_of(take_async(), kc, pc);
    Pair dc;
    uint32_t s_cur = 0;
    if (kc <= 1) {
        dc = pair_from(pc, index_entry(pc));
        s_cur = issue(dc, kc == 0 ? keep : drop);
        if (kc == 1) load_b(pc);
    }
    task_of(take_async(), kn, pn);
    uint64_t en = kn <= 1 ? index_entry(pn) : 0ull;
    while (kc != 3) {
        // the current B task's prefix and block sum, loaded an iteration ago
        uint4 pre_c = make_uint4(0, 0, 0, 0), bs_c = pre_c;
        bool pre_ok = true, bs_ok = true;
        if (kc == 1) {
            pre_ok = check_tagged<NL>(pr, tagI, pre_c);
            if (32 * (size_t)pc + lane < nb) bs_ok = check_tagged<NL>(br, tagA, bs_c);
        }
        // the task after next: its id is taken now and read, with its index
        // entries requested, a quarter of the way through the current task
        const uint32_t raw2 = take_async();
        uint32_t kk = 3, pk = 0;
        uint64_t ek = 0;
        bool mid_done = false;
        auto mid = [&]() {
            task_of(raw2, kk, pk);
            ek = kk <= 1 ? index_entry(pk) : 0ull;
            mid_done = true;
        };
        Pair dn;
        uint32_t s_nx = 0;
        bool nx_issued = false;
        if (kn <= 1) {
            dn = pair_from(pn, en);
            if (kc > 1 || fits(dc, dn)) {
                s_nx = issue(dn, kn == 0 ? keep : drop);
                nx_issued = true;
            }
            if (kn == 1) load_b(pn);
        }
        if (kc == 0) {
            // ------------------------------------------------------ A task
            // the pair some warp sums about one round from now goes into L2
            // (its index entries are read now, the prefetch is issued after
            // the sums)
            uint64_t pf_a = 0, pf_e = 0;
            if (lane == 0 && pc + nwarps < P) {
                const size_t pf = 2 * (size_t)(pc + nwarps);
                pf_a = __ldg(index + pf);
                pf_e = __ldg(index + min(pf + 2, M));
            }
            uint4 bs = make_uint4(0, 0, 0, 0);
            if (wait()) {
                if (!dc.ok) {
                    if (lane == 0) set_error(h, ICX_ECORRUPT);
                } else if (space(dc)) {
                    bs = pair_blocks<DELTA, false, 0>(
                        SmemRows{ring + slot(s_cur, dc), smem_u32(ring + slot(s_cur, dc))}, dc, bs, out, 0, rest, h,
                        lane, mid);
                } else {
                    bs = pair_blocks<DELTA, false, 0>(GlobalRows{in + dc.start, in_bytes - dc.start}, dc, bs, out, 0,
                                                      rest, h, lane, mid);
                }
            }
            __syncwarp();
            if (lane == 0 && pf_a < pf_e && pf_e <= in_bytes && pf_e - pf_a <= 2 * (uint64_t)kMetaMax &&
                ((pf_a | pf_e) & 15) == 0)
                prefetch_l2_hint(in + pf_a, (uint32_t)(pf_e - pf_a), keep);
            const size_t blk = 32 * (size_t)pc + lane;
            if (blk < nb) st_tagged<NL>(sc.bst + 4 * blk, tagA, bs);
            const uint4 tot = warp_sum<NL>(bs);
            // the group's counter (zeroed by the first CTA of this launch,
            // which raises aux[3] to epoch + 1 when done)
            if (!counters_ready) {
                if (lane == 0) {
                    const unsigned long long t0 = globaltimer();
                    while (ld_acquire_u32(&h->aux[3]) != epoch + 1u) {
                        if (globaltimer() - t0 > kWaitLimitNs) {
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
            if (!__all_sync(FULL, pre_ok)) pre_c = wait_tagged<NL>(sc.pre + 4 * (size_t)pc, tagI, h);
            if (!bs_ok) bs_c = wait_tagged<NL>(sc.bst + 4 * (32 * (size_t)pc + lane), tagA, h);
            const uint4 bi = warp_scan_carry<DELTA>(bs_c, lane);
            const uint4 carry = add4(pre_c, sub4(bi, bs_c));
            if (wait() && dc.ok) {
                const size_t first = 4096 * (size_t)pc;
                if (space(dc))
                    pair_blocks<DELTA, true, STORE>(SmemRows{ring + slot(s_cur, dc), smem_u32(ring + slot(s_cur, dc))},
                                                    dc, carry, out, first, rest, h, lane, mid);
                else
                    pair_blocks<DELTA, true, STORE>(GlobalRows{in + dc.start, in_bytes - dc.start}, dc, carry, out,
                                                    first, rest, h, lane, mid);
            }
            __syncwarp();
        } else {
            // ---------------------------------------- the Variable Byte tail
            // its carry is the inclusive prefix of the last group
            uint4 carry = make_uint4(0, 0, 0, 0);
            if (P > 0) carry = wait_tagged<NL>(sc.gst + 4 * (size_t)(Gn - 1), tagI, h);
            uint32_t* scratch = reinterpret_cast<uint32_t*>(rest);
            const uint64_t tstart = __ldg(index + M);
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

// ------------------------------------------------------------ launcher

// Output store path of phase B (measured on the 2^26 sorted arrays, 2^26
// uniform stride 4: restaged 0.0864 ms, 32-byte lane stores 0.0967 ms,
// 16-byte lane stores 0.152 ms).
static int g_blocklane_store = bl::kStoreRestage;

void set_bp128_blocklane_store(int v) { g_blocklane_store = (v >= 0 && v <= 2) ? v : bl::kStoreRestage; }

static int g_blocklane_ctas = 0;  // CTAs of the persistent grid (0: as many as are resident)

void set_bp128_blocklane_ctas(int v) { g_blocklane_ctas = v > 0 ? v : 0; }

// Pairs summed before the first decode task (0: two per resident warp; at
// least 128, which keeps every task's dependencies before it).
static int g_blocklane_lead = 0;

void set_bp128_blocklane_lead(int v) { g_blocklane_lead = v > 0 ? v : 0; }

// Warps per CTA that only sum (the others only decode); 0: every warp takes
// both kinds of task from one counter.
static int g_blocklane_sumw = 0;

void set_bp128_blocklane_sumw(int v) { g_blocklane_sumw = (v > 0 && v < bl::kW) ? v : 0; }

// Scratch layout of a decode of n integers inside a workspace of ws_bytes
// bytes at h: the last ws_blocklane_bytes(n) bytes (from a 256-byte
// boundary).  Every region another decoder writes for a length m ends at
// ws_unitmeta_end(m) <= ws_bytes - ws_blocklane_bytes(m), and the region
// grows with the length, so no decoder sharing the workspace writes here.
static bl::Scratch blocklane_scratch(WsHeader* h, size_t n, size_t ws_bytes) {
    const size_t nb = n / 128, M = (nb + 15) / 16, P = (M + 1) / 2, Gn = (P + bl::kGroup - 1) / bl::kGroup;
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

template <int DELTA, int STORE>
static cudaError_t launch_blocklane_t(const uint8_t* in, size_t in_bytes, uint32_t* out, size_t n,
                                      const uint64_t* index, WsHeader* h, size_t ws_bytes, cudaStream_t s) {
    auto kern = bp128_blocklane_kernel<DELTA, STORE>;
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
    const size_t nb = n / 128, M = (nb + 15) / 16, P = (M + 1) / 2;
    const size_t resident = (size_t)blocks_per_sm * sms;
    size_t G = max((size_t)1, min(resident, (P + bl::kW - 1) / bl::kW));
    if (g_blocklane_ctas > 0 && (size_t)g_blocklane_ctas < G) G = (size_t)g_blocklane_ctas;
    const size_t lead = max((size_t)128, g_blocklane_lead > 0 ? (size_t)g_blocklane_lead : 2 * G * bl::kW);
    kern<<<(int)G, bl::kW * 32, smem, s>>>(in, in_bytes, out, n, index, h, blocklane_scratch(h, n, ws_bytes),
                                            (uint32_t)(n - 128 * nb), (uint32_t)min(lead, (size_t)0xFFFFFFFFu),
                                            (uint32_t)g_blocklane_sumw);
    return cudaGetLastError();
}

template <int DELTA>
static cudaError_t launch_blocklane_d(const uint8_t* in, size_t in_bytes, uint32_t* out, size_t n,
                                      const uint64_t* index, WsHeader* h, size_t ws_bytes, cudaStream_t s) {
    int st = g_blocklane_store;
    if (st == bl::kStoreV8 && (reinterpret_cast<uintptr_t>(out) & 31u) != 0) st = bl::kStoreV4;
    if (st == bl::kStoreRestage) return launch_blocklane_t<DELTA, bl::kStoreRestage>(in, in_bytes, out, n, index, h, ws_bytes, s);
    if (st == bl::kStoreV8) return launch_blocklane_t<DELTA, bl::kStoreV8>(in, in_bytes, out, n, index, h, ws_bytes, s);
    return launch_blocklane_t<DELTA, bl::kStoreV4>(in, in_bytes, out, n, index, h, ws_bytes, s);
}

cudaError_t launch_bp128_blocklane(int delta, const uint8_t* in, size_t in_bytes, uint32_t* out, size_t n,
                                   const uint64_t* index, WsHeader* h, size_t ws_bytes, cudaStream_t s) {
    if (delta == ICX_DELTA_4) return launch_blocklane_d<ICX_DELTA_4>(in, in_bytes, out, n, index, h, ws_bytes, s);
    if (delta == ICX_DELTA_1) return launch_blocklane_d<ICX_DELTA_1>(in, in_bytes, out, n, index, h, ws_bytes, s);
    return cudaErrorInvalidValue;
}

}  // namespace icx
