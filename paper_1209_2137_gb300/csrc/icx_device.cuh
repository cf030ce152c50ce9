// Device-side building blocks shared by the icx kernels: PTX wrappers for the
// bulk-copy engine and mbarriers, warp scans, and the bounded single-pass
// decoupled look-back that carries the running prefix sum of differential
// decoding (Sec. 3) from one tile to the next.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "icx.h"

namespace icx {

constexpr unsigned FULL = 0xFFFFFFFFu;

// Workspace layout: a 256-byte header, then per look-back tile four 64-bit
// states (one per residue mod 4; differential decoding with stride 1 uses the
// first only).  A state holds (epoch << 2 | flag) in its high word and a
// 32-bit sum in its low word; flag 1 = tile aggregate, 2 = inclusive prefix.
// Any other high word (an older epoch, zero) means "not yet published".
constexpr size_t kWsHeaderBytes = 256;
constexpr int kStatesPerTile = 4;

struct WsHeader {
    unsigned int tile_counter;  // dynamic tile ids handed out by atomicAdd
    unsigned int done_counter;  // CTAs that finished this launch
    unsigned int epoch;         // launch number; tags the tile states
    unsigned int status;        // first data-dependent error (icx_status)
    uint64_t mini_index[2];  // index of a single-metablock/page stream
    uint64_t total;          // encoders: stream length
    unsigned int aux[48];
};
static_assert(sizeof(WsHeader) <= kWsHeaderBytes, "workspace header");

// Workspace regions after the header: look-back tile states, then (for
// SIMD-FastPFOR) one 16-byte record per block and one 144-byte record per page
// written by the page parse and read by the decode.
struct BlockMeta {
    uint32_t packed_off;  // page-relative byte offset of the block's packed low bits
    uint32_t pos_off;     // page-relative byte offset of its exception positions
    uint32_t cursor;      // index of its first exception in array d
    uint8_t b, d, c, flags;
};
static_assert(sizeof(BlockMeta) == 16, "block meta");
constexpr size_t kPageMetaWords = 36;  // arr_off[32] (page-relative), bad flag, pad

// Workspace layout for a decode of n integers in a workspace of ws_bytes
// bytes.  Regions that hold epoch-tagged words (read as "published" only when
// their tag matches the current launch) never share bytes with regions that
// hold plain data, whatever lengths share the workspace:
//   - the header and the look-back tile states, sized for the largest length
//     N the workspace serves (ws_capacity);
//   - after them the plain regions for n: SIMD-FastPFOR block records, page
//     records and per-16-block ranges (page parse), then the prepare
//     kernel's per-block records and tile sums;
//   - at the very end the tagged scratch of the block-per-lane decoders for
//     n (it grows with n, so it stays above every plain region of any length
//     up to N).
__host__ __device__ inline size_t ws_round(size_t x) { return (x + 255) / 256 * 256; }
__host__ __device__ inline size_t ws_tiles(size_t n) { return n / 2048 + 16; }
__host__ __device__ inline size_t ws_head_bytes(size_t n) { return ws_round(kWsHeaderBytes + 32 * ws_tiles(n)); }
// page parse: one BlockMeta per block, kPageMetaWords per page, an 8-byte
// range per unit of 16 blocks
__host__ __device__ inline size_t ws_pagemeta_rel(size_t n) { return 16 * (n / 128 + 1); }
__host__ __device__ inline size_t ws_unitmeta_rel(size_t n) {
    return ws_round(ws_pagemeta_rel(n) + 4 * kPageMetaWords * ((n / 128 + 511) / 512 + 1));
}
__host__ __device__ inline size_t ws_meta_bytes(size_t n) { return ws_round(ws_unitmeta_rel(n) + 8 * (n / 2048 + 2)); }
// prepare kernel: 32 bytes per block, 16 per tile of 256 blocks
__host__ __device__ inline size_t ws_fp2_tiles_rel(size_t n) { return 32 * (n / 128 + 1); }
__host__ __device__ inline size_t ws_fp2_bytes(size_t n) {
    return ws_round(ws_fp2_tiles_rel(n) + 16 * ((n / 128 + 255) / 256 + 1));
}
// Two-phase block-per-lane decoding: per 128-integer block four tagged
// 64-bit words (block sums), per pair of metablocks two groups of four (pair
// total, pair prefix), per group of 64 pairs one group of four (look-back
// state) and a 32-bit counter.
__host__ __device__ inline size_t ws_blocklane_bytes(size_t n) {
    const size_t nb = n / 128, P = ((nb + 15) / 16 + 1) / 2, Gn = (P + 63) / 64;
    return ws_round(32 * (nb + 1) + 64 * (P + 1) + 36 * (Gn + 1));
}
__host__ __device__ inline size_t ws_total_bytes(size_t n) {
    return ws_head_bytes(n) + ws_meta_bytes(n) + ws_fp2_bytes(n) + ws_blocklane_bytes(n);
}
// The largest length a workspace of ws_bytes serves (every size above grows
// with n).
__host__ __device__ inline size_t ws_capacity(size_t ws_bytes) {
    size_t lo = 0, hi = (size_t)1 << 44;
    if (ws_total_bytes(0) > ws_bytes) return 0;
    while (lo < hi) {
        const size_t mid = lo + (hi - lo + 1) / 2;
        if (ws_total_bytes(mid) <= ws_bytes) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}
// Start of the plain regions in a workspace of ws_bytes.
__host__ __device__ inline size_t ws_plain_base(size_t ws_bytes) { return ws_head_bytes(ws_capacity(ws_bytes)); }

// A device wait that sees no progress for this long gives up with ETIMEOUT.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;

// Header word holding a shorter limit for the waits on published values (in
// microseconds; 0 = kWaitLimitNs), set by icx_workspace_set_wait_limit.
constexpr int kAuxWaitLimit = 5;

__device__ __forceinline__ unsigned long long* tile_states(WsHeader* h) {
    return reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(h) + kWsHeaderBytes);
}

__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// The limit of a wait on values other CTAs publish in this workspace.
__device__ __forceinline__ unsigned long long wait_limit_ns(WsHeader* h) {
    const unsigned v = *reinterpret_cast<volatile const unsigned*>(&h->aux[kAuxWaitLimit]);
    return v ? 1000ull * v : kWaitLimitNs;
}

__device__ __forceinline__ void set_error(WsHeader* h, unsigned code) {
    atomicCAS(&h->status, 0u, code);
}

// ---------------------------------------------------------------- bulk copy

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Programmatic dependent launch.  A kernel launched with the
// programmatic-stream-serialization attribute may be scheduled while the
// kernel before it in the stream is still running; grid_dependency_wait()
// returns once that kernel has completed and its writes are visible, so a
// dependent kernel calls it before its first global-memory access and only
// its scheduling overlaps the predecessor's tail.  allow_dependents() lets
// the next kernel be scheduled as soon as every CTA of this grid has run it.
// Both are no-ops for a kernel launched without the attribute.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ void allow_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's earlier generic-proxy accesses to shared memory before
// later bulk-copy (async-proxy) accesses.
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
        "r"(bytes)
        : "memory");
}

// One bulk copy global -> shared (16-byte aligned addresses, size a multiple
// of 16); completion is signalled on `bar` as transaction bytes.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Hint: bring `bytes` (a multiple of 16) at the 16-byte aligned `src` into L2.
__device__ __forceinline__ void prefetch_l2(const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// L2 eviction-priority policies for the cache-hinted copies below.
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// bulk_load and prefetch_l2 with an L2 eviction policy for the source lines.
__device__ __forceinline__ void bulk_load_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                               uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}
__device__ __forceinline__ void prefetch_l2_hint(const void* src, uint32_t bytes, uint64_t policy) {
    asm volatile("cp.async.bulk.prefetch.L2.global.L2::cache_hint [%0], %1, %2;" ::"l"(src), "r"(bytes), "l"(policy)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for phase `parity` of `bar`; false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (globaltimer() - t0 > kWaitLimitNs) return false;
    }
}

// ------------------------------------------------------------- bit fields

__device__ __forceinline__ uint32_t width_mask(uint32_t b) {
    return b ? (0xFFFFFFFFu >> (32u - b)) : 0u;
}

__device__ __forceinline__ uint32_t comp(const uint4& v, int c) {
    return c == 0 ? v.x : c == 1 ? v.y : c == 2 ? v.z : v.w;
}

__device__ __forceinline__ uint4 add4(uint4 a, uint4 b) {
    return make_uint4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}

__device__ __forceinline__ uint4 sub4(uint4 a, uint4 b) {
    return make_uint4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
}

__device__ __forceinline__ uint4 shfl4(uint4 v, int src) {
    return make_uint4(__shfl_sync(FULL, v.x, src), __shfl_sync(FULL, v.y, src),
                      __shfl_sync(FULL, v.z, src), __shfl_sync(FULL, v.w, src));
}

// ------------------------------------------------------------------ scans

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v, int lane) {
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        uint32_t y = __shfl_up_sync(FULL, v, off);
        if (lane >= off) v += y;
    }
    return v;
}

__device__ __forceinline__ uint4 warp_incl_scan4(uint4 v, int lane) {
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        uint32_t a = __shfl_up_sync(FULL, v.x, off), b = __shfl_up_sync(FULL, v.y, off);
        uint32_t c = __shfl_up_sync(FULL, v.z, off), d = __shfl_up_sync(FULL, v.w, off);
        if (lane >= off) {
            v.x += a;
            v.y += b;
            v.z += c;
            v.w += d;
        }
    }
    return v;
}

// Row ownership, stride-4 prefix sum: component c of every lane belongs to
// residue c, so the block is four column scans over the lanes.
__device__ __forceinline__ uint4 row_scan_d4(uint4 v, uint4& carry, int lane) {
    const uint4 incl = warp_incl_scan4(v, lane);
    const uint4 out = add4(incl, carry);
    carry = add4(carry, shfl4(incl, 31));
    return out;
}

// Residue ownership -> row ownership: inside each group of four lanes the
// 4x4 matrix M[m][l] (lane l holds column l) is transposed so lane l' holds
// row l' = integers 16g + 4l' + 0..3.  Two butterfly exchanges.
__device__ __forceinline__ uint4 residue_to_row(uint4 a, int lane) {
    const int l = lane & 3;
    const bool odd = l & 1;
    // stage 1 (partner l^1): keep the rows of my parity, swap the others.
    uint32_t keep0 = odd ? a.y : a.x;  // row p
    uint32_t keep1 = odd ? a.w : a.z;  // row p + 2
    uint32_t x0 = __shfl_xor_sync(FULL, odd ? a.x : a.y, 1);  // row p, column l^1
    uint32_t x1 = __shfl_xor_sync(FULL, odd ? a.z : a.w, 1);  // row p+2, column l^1
    // stage 2 (partner l^2): keep row l, send row l^2.
    const bool hi = l & 2;
    uint32_t own = hi ? keep1 : keep0;         // M[l][l]
    uint32_t own_x = hi ? x1 : x0;             // M[l][l^1]
    uint32_t y0 = __shfl_xor_sync(FULL, hi ? keep0 : keep1, 2);  // M[l][l^2]
    uint32_t y1 = __shfl_xor_sync(FULL, hi ? x0 : x1, 2);        // M[l][l^3]
    // e[c ^ l] = M[l][c]: undo the xor-by-l permutation.
    uint32_t e0 = own, e1 = own_x, e2 = y0, e3 = y1;
    if (odd) {
        uint32_t t = e0; e0 = e1; e1 = t;
        t = e2; e2 = e3; e3 = t;
    }
    if (hi) {
        uint32_t t = e0; e0 = e2; e2 = t;
        t = e1; e1 = e3; e3 = t;
    }
    return make_uint4(e0, e1, e2, e3);
}

// ------------------------------------------------------------- look-back

__device__ __forceinline__ void ld_relaxed_v2(const unsigned long long* p, unsigned long long& a,
                                              unsigned long long& b) {
    asm volatile("ld.relaxed.gpu.global.v2.b64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p) : "memory");
}

// Decoupled look-back for tile `tile`, run by one full warp.  NL is the
// number of independent chains (1 for stride 1, 4 for stride 4); agg holds
// the tile's NL aggregates.  A tile's state is NL 64-bit words, each (epoch
// tag | flag | 32-bit value), written by NL relaxed stores; a reader counts a
// state only if all its NL tags agree (mixed tags mean the owner is between
// its two publications and are waited out).  Every round trip inspects 32*R
// predecessors: lane i reads the state of tile end-1-i-32r with one or two
// 128-bit loads.  Contributions are summed per lane and reduced once at the
// end.  Returns the exclusive prefixes (components 0..NL-1) and publishes the
// inclusive ones.  Every wait is bounded: after wait_limit_ns without progress
// the status word gets ICX_ETIMEOUT and the tile publishes what it has, so no
// other tile can wait forever on it.
// Publishes a tile's aggregate (the first tile publishes it as its inclusive
// prefix).  Lanes 0..NL-1 of the calling warp store one chain each.
template <int NL>
__device__ __forceinline__ void lookback_publish(WsHeader* h, uint32_t epoch, uint32_t tile, uint4 agg) {
    const int lane = threadIdx.x & 31;
    const uint32_t tag = (epoch << 2) | (tile ? 1u : 2u);
    if (lane < NL)
        st_relaxed(tile_states(h) + (size_t)tile * kStatesPerTile + lane,
                   ((unsigned long long)tag << 32) | comp(agg, lane));
}

// Predecessors read per look-back round: 32 x this.  Measured on the 2^26
// sorted workloads, one row (32 predecessors) beats 2 and 4: the window's
// loads and registers cost more than the extra rounds they save.
constexpr int kLookbackRows = 1;

// Resolves the exclusive prefix of `tile` (whose aggregate `agg` is already
// published) from its predecessors' states and, if `publish`, publishes its
// inclusive prefix.  Whole warp.
template <int NL, int R = kLookbackRows>
__device__ uint4 lookback_resolve_at(unsigned long long* st, WsHeader* h, uint32_t epoch, uint32_t tile, uint4 agg,
                                     bool publish = true, const unsigned long long* limit = nullptr) {
    static_assert(NL == 1 || NL == 4, "chains");
    const int lane = threadIdx.x & 31;
    const uint32_t tagA = (epoch << 2) | 1u, tagP = (epoch << 2) | 2u;
    uint4 acc = make_uint4(0, 0, 0, 0);
    if (tile == 0) return acc;
    long long end = tile;
    unsigned long long t0 = 0;
    for (;;) {
        uint32_t flag[R];
        uint4 val[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const long long p = end - 1 - lane - 32 * r;
            flag[r] = 2;
            val[r] = make_uint4(0, 0, 0, 0);
            if (p >= 0) {
                const unsigned long long* sp = st + (size_t)p * kStatesPerTile;
                if (NL == 1) {
                    const unsigned long long s0 = ld_relaxed(sp);
                    const uint32_t t = (uint32_t)(s0 >> 32);
                    flag[r] = t == tagP ? 2u : t == tagA ? 1u : 0u;
                    val[r].x = (uint32_t)s0;
                } else {
                    unsigned long long s0, s1, s2, s3;
                    ld_relaxed_v2(sp, s0, s1);
                    ld_relaxed_v2(sp + 2, s2, s3);
                    const uint32_t t = (uint32_t)(s0 >> 32);
                    const bool same = (uint32_t)(s1 >> 32) == t && (uint32_t)(s2 >> 32) == t &&
                                      (uint32_t)(s3 >> 32) == t;
                    flag[r] = !same ? 0u : t == tagP ? 2u : t == tagA ? 1u : 0u;
                    val[r] = make_uint4((uint32_t)s0, (uint32_t)s1, (uint32_t)s2, (uint32_t)s3);
                }
            }
        }
        // nearest inclusive prefix at distance lane + 32r
        bool wait = false, found = false;
        uint4 c = make_uint4(0, 0, 0, 0);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (found) continue;
            const unsigned pm = __ballot_sync(FULL, flag[r] == 2);
            const unsigned xm = __ballot_sync(FULL, flag[r] == 0);
            const unsigned first = pm ? (unsigned)(__ffs(pm) - 1) : 32u;
            const unsigned upto = first >= 31 ? FULL : ((2u << first) - 1u);
            if (xm & upto) wait = true;
            if ((unsigned)lane <= first) c = add4(c, val[r]);
            if (first < 32) found = true;
        }
        if (wait) {
            if (t0 == 0) t0 = globaltimer();
            if (globaltimer() - t0 > (limit ? *limit : wait_limit_ns(h))) {
                if (lane == 0) set_error(h, ICX_ETIMEOUT);
                break;
            }
            __nanosleep(32);
            continue;
        }
        t0 = 0;
        acc = add4(acc, c);
        if (found) break;
        end -= 32 * R;
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        acc.x += __shfl_xor_sync(FULL, acc.x, off);
        if (NL == 4) {
            acc.y += __shfl_xor_sync(FULL, acc.y, off);
            acc.z += __shfl_xor_sync(FULL, acc.z, off);
            acc.w += __shfl_xor_sync(FULL, acc.w, off);
        }
    }
    if (publish && lane < NL)
        st_relaxed(st + (size_t)tile * kStatesPerTile + lane,
                   ((unsigned long long)tagP << 32) | (comp(acc, lane) + comp(agg, lane)));
    return acc;
}

// The same over the workspace's look-back states.
template <int NL, int R = kLookbackRows>
__device__ __forceinline__ uint4 lookback_resolve(WsHeader* h, uint32_t epoch, uint32_t tile, uint4 agg,
                                                  bool publish = true) {
    return lookback_resolve_at<NL, R>(tile_states(h), h, epoch, tile, agg, publish);
}

// Decoupled look-back of one tile: publish its aggregate, resolve its
// exclusive prefix, publish its inclusive prefix.  Whole warp.
template <int NL, int R = kLookbackRows>
__device__ __forceinline__ uint4 lookback(WsHeader* h, uint32_t epoch, uint32_t tile, uint4 agg) {
    lookback_publish<NL>(h, epoch, tile, agg);
    return lookback_resolve<NL, R>(h, epoch, tile, agg);
}

// Epoch of this launch (constant while it runs).
__device__ __forceinline__ uint32_t launch_epoch(WsHeader* h) {
    return *reinterpret_cast<volatile unsigned int*>(&h->epoch);
}

// Called by every CTA after its last tile: the last CTA to finish resets the
// tile counter and advances the epoch, so the next launch on the same
// workspace starts clean without a memset.
__device__ __forceinline__ void finish_launch(WsHeader* h, uint32_t epoch) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(&h->done_counter, 1u);
        if (prev == gridDim.x - 1) {
            atomicExch(&h->tile_counter, 0u);
            atomicExch(&h->done_counter, 0u);
            atomicExch(&h->epoch, (epoch + 1u) & 0x3FFFFFFFu);
            __threadfence();
        }
    }
}

}  // namespace icx
