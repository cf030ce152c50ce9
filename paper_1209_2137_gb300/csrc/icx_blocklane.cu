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
// stores (bandwidth bound).  With stride 4 the default lead is every pair:
// all sums first, then every decode task finds its carry published.  Every
// task waits only for tasks taken before
// it, and every published value is a set of 64-bit words tagged with the
// launch epoch, so readers need no fences.
#include "icx_blocklane.cuh"
#include "icx_bp128.cuh"
#include "icx_kernels.cuh"

namespace icx {

namespace bl {

// One pair of metablocks as the warp sees it: byte offset of the second
// metablock, total size, number of metablocks (1 or 2) and their blocks.
struct Pair {
    uint64_t start;
    uint32_t off1, size;
    uint32_t mcount, K0, K1;
    bool ok;
};


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
    NoPatch np;
    if (maxb <= 8)
        walk_block<DELTA, DECODE, STORE, 4>(rows, w, mid, np);
    else if (maxb <= 16)
        walk_block<DELTA, DECODE, STORE, 2>(rows, w, mid, np);
    else
        walk_block<DELTA, DECODE, STORE, 1>(rows, w, mid, np);
    if constexpr (DECODE) {
        return make_uint4(0, 0, 0, 0);
    } else {
        if (DELTA == ICX_DELTA_1) w.acc = make_uint4(w.acc.x + w.acc.y + w.acc.z + w.acc.w, 0, 0, 0);
        return w.acc;
    }
}

// SIMD-BP128 as a block-per-lane codec: pair p is metablocks 2p and 2p+1,
// located by the stream's metablock index (lanes 0..2 load entries 2p,
// 2p+1, 2p+2; the last is the end of the pair).
struct Bp128Codec {
    const uint64_t* index;
    const uint8_t* in;
    size_t in_bytes, nb, M;

    using Pre = uint64_t;
    using Desc = Pair;
    struct Ahead {
        uint64_t a, e;
    };
    __device__ __forceinline__ Pre load(uint32_t p, int lane) const {
        return lane < 3 ? __ldg(index + min((size_t)2 * p + lane, M)) : 0ull;
    }
    __device__ __forceinline__ Pair describe(uint32_t p, Pre e, int lane) const {
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
    }
    __device__ __forceinline__ uint32_t space(const Pair& d) const { return d.ok && d.size <= kRing ? d.size : 0u; }
    __device__ __forceinline__ void issue(const Pair& d, uint8_t* dst, uint64_t* bar, uint64_t policy,
                                          int lane) const {
        const uint32_t bytes = space(d);
        if (lane == 0) {
            fence_proxy_async();
            mbar_expect_tx(bar, bytes);
            if (bytes) bulk_load_hint(dst, in + d.start, bytes, bar, policy);
        }
    }
    __device__ __forceinline__ GlobalRows global_rows(const Pair& d) const {
        return GlobalRows{in + d.start, in_bytes - d.start};
    }
    __device__ __forceinline__ Ahead ahead(uint32_t p, int lane) const {
        Ahead a{0, 0};
        if (lane == 0) {
            const size_t pf = 2 * (size_t)p;
            a.a = __ldg(index + pf);
            a.e = __ldg(index + min(pf + 2, M));
        }
        return a;
    }
    __device__ __forceinline__ void prefetch(const Ahead& a, uint64_t policy, int lane) const {
        if (lane == 0 && a.a < a.e && a.e <= in_bytes && a.e - a.a <= 2 * (uint64_t)kMetaMax && ((a.a | a.e) & 15) == 0)
            prefetch_l2_hint(in + a.a, (uint32_t)(a.e - a.a), policy);
    }
    __device__ __forceinline__ uint64_t tail_start() const { return __ldg(index + M); }
    template <int DELTA, bool DECODE, int STORE, class Rows, class Mid>
    __device__ __forceinline__ uint4 blocks(const Rows& rows, const Pair& d, uint4 carry, uint32_t& /*flag*/,
                                            uint32_t* __restrict__ out, size_t first, uint8_t* rest, WsHeader* h,
                                            int lane, Mid& mid) const {
        return pair_blocks<DELTA, DECODE, STORE>(rows, d, carry, out, first, rest, h, lane, mid);
    }
};

}  // namespace bl

template <int DELTA, int STORE>
__global__ void __maxnreg__(96)
    bp128_blocklane_kernel(const uint8_t* __restrict__ in, size_t in_bytes, uint32_t* __restrict__ out, size_t n,
                           const uint64_t* __restrict__ index, WsHeader* h, bl::Scratch sc, uint32_t tail,
                           uint32_t lead, uint32_t sumw) {
    const size_t nb = n / 128;
    const bl::Bp128Codec codec{index, in, in_bytes, nb, (nb + 15) / 16};
    bl::run<bl::Bp128Codec, DELTA, STORE>(codec, in, in_bytes, out, n, h, sc, tail, lead, sumw);
}

// ------------------------------------------------------------ launcher

// Output store path of phase B (measured on the 2^26 sorted arrays, 2^26
// uniform stride 4: restaged 0.0864 ms, 32-byte lane stores 0.0967 ms,
// 16-byte lane stores 0.152 ms).
static int g_blocklane_store = bl::kStoreRestage;

void set_bp128_blocklane_store(int v) { g_blocklane_store = (v >= 0 && v <= 2) ? v : bl::kStoreRestage; }

static int g_blocklane_ctas = 0;  // CTAs of the persistent grid (0: as many as are resident)

void set_bp128_blocklane_ctas(int v) { g_blocklane_ctas = v > 0 ? v : 0; }

// Pairs summed before the first decode task (0: every pair with stride 4,
// two per resident warp with stride 1; at least 128, which keeps every
// task's dependencies before it).  Measured on the 2^26 uniform and the
// clustered arrays (ms, default / two per warp / 2048): stride 4 summing
// every pair first 0.0815 / 0.0845 / 0.0960 and 0.0692 / 0.0758 / 0.0856;
// stride 1 two per warp 0.0819 (0.0836 with every pair first) and 0.0717
// (0.0717).
static int g_blocklane_lead = 0;

void set_bp128_blocklane_lead(int v) { g_blocklane_lead = v > 0 ? v : 0; }

// Warps per CTA that only sum (the others only decode); 0: every warp takes
// both kinds of task from one counter.
static int g_blocklane_sumw = 0;

void set_bp128_blocklane_sumw(int v) { g_blocklane_sumw = (v > 0 && v < bl::kW) ? v : 0; }

BlocklaneTuning blocklane_tuning() {
    return BlocklaneTuning{g_blocklane_store, g_blocklane_ctas, g_blocklane_lead, g_blocklane_sumw};
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
    const size_t nb = n / 128, P = (nb + 31) / 32;
    const size_t resident = (size_t)blocks_per_sm * sms;
    size_t G = max((size_t)1, min(resident, (P + bl::kW - 1) / bl::kW));
    if (g_blocklane_ctas > 0 && (size_t)g_blocklane_ctas < G) G = (size_t)g_blocklane_ctas;
    const size_t lead = max((size_t)128, g_blocklane_lead > 0        ? (size_t)g_blocklane_lead
                                         : DELTA == ICX_DELTA_4 ? P
                                                                : 2 * G * bl::kW);
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
