// Decoding fused into its consumer (Sec. 7): membership of a sorted query
// list b[0..nb) in the sorted list a SIMD-BP128 / W32 stream decodes to,
// without writing the decoded integers anywhere.  The paper notes that an
// integrated decode can be much faster than decoding and then processing,
// and that intersections of sorted arrays are a consumer that touches many
// integers per query.
//
// bp128_member_kernel runs the decoder's tile pipeline (bulk copy, unpack,
// local scan, decoupled look-back) and replaces the stores with the
// consumer: each warp parks its unit's 2,048 absolute values in its shared
// buffer, finds the first query element >= the unit's first value (a
// directory of the query list in shared memory, then 32-way probes of the
// list), and looks every query element up to the unit's last value up in
// the parked values (a 12-step binary search).  Hits set bit j of the
// result bitmap with one atomicOr per 32 query elements; a short second
// launch counts the set bits, so a query element matched by two units
// (equal values across a unit boundary) counts once.
//
// sorted_member_kernel is the same consumer over an array that is already
// decoded in memory: the unfused path is bp128_decode, then this.
#include "icx_bp128.cuh"
#include "icx_kernels.cuh"


namespace icx {

constexpr int kDir = 4096;           // directory entries of the query list per CTA (16 KB)
constexpr int kMemberHdr = 1024;     // TileShared, then two mbarriers per warp
static_assert(sizeof(TileShared) + 16 * kMaxWarps <= kMemberHdr, "tile header");
static_assert(2048 * 4 <= kBuf, "a unit's values fit its copy buffer");

struct MemberArgs {
    const uint32_t* b;            // the query list, non-decreasing
    size_t nb;                    // > 0
    uint32_t* bits;               // ceil(nb / 32) words, zeroed before the launch
    size_t step;                  // directory spacing, ceil(nb / entries)
};

// CTA-wide: this CTA's share of the query list into L2 (its 16-byte
// aligned interior; the probes of every unit then hit L2), then
// dir[j] = b[min(j * step, nb - 1)] for j < DIR.
template <int DIR>
__device__ __forceinline__ void load_dir(uint32_t* dir, const MemberArgs& a) {
    if (threadIdx.x == 0) {
        const uintptr_t base = reinterpret_cast<uintptr_t>(a.b), bytes = 4 * a.nb;
        const uintptr_t share = ((bytes + gridDim.x - 1) / gridDim.x + 15) & ~(uintptr_t)15;
        const uintptr_t lo = (base + (uintptr_t)blockIdx.x * share + 15) & ~(uintptr_t)15;
        const uintptr_t hi = min(base + (uintptr_t)(blockIdx.x + 1) * share, base + bytes) & ~(uintptr_t)15;
        for (uintptr_t p = lo; p < hi; p += 65536)
            prefetch_l2(reinterpret_cast<const void*>(p), (uint32_t)min(hi - p, (uintptr_t)65536));
    }
    for (int j = threadIdx.x; j < DIR; j += blockDim.x) dir[j] = __ldg(a.b + min((size_t)j * a.step, a.nb - 1));
}

// Whole warp: the first j with b[j] >= y (nb if none).  The directory
// entries below y form a prefix; its length c comes from a 32-way descent
// (windows of DIR, DIR/32, ... entries).  Then 32 probes per round of the
// query list, with the invariant b[j] < y for j < lo and b[j] >= y for
// lo <= hi <= j < nb.
template <int DIR>
__device__ __forceinline__ size_t lower_bound_warp(const MemberArgs& a, const uint32_t* dir, uint32_t y, int lane) {
    static_assert(DIR >= 32 && (DIR & (DIR - 1)) == 0, "a power of two");
    uint32_t c = 0;
#pragma unroll
    for (uint32_t window = DIR; window > 1;) {
        const uint32_t span = window > 32 ? window / 32 : 1;
        const uint32_t q = c + (lane + 1) * span - 1;  // probes inside the window and the directory
        const bool below = (uint32_t)(lane + 1) * span <= window && q < DIR && dir[q] < y;
        c += span * __popc(__ballot_sync(FULL, below));
        window = span;
    }
    size_t lo = c ? min((size_t)(c - 1) * a.step, a.nb - 1) + 1 : 0;
    size_t hi = c < DIR ? min((size_t)c * a.step, a.nb) : a.nb;
    while (hi - lo > 32) {
        const size_t s = (hi - lo + 31) / 32;
        const size_t q = lo + (size_t)(lane + 1) * s - 1;
        const bool below = q < hi && __ldg(a.b + q) < y;
        const size_t nlo = lo + (size_t)__popc(__ballot_sync(FULL, below)) * s;
        hi = min(nlo + s - 1, hi);  // the first probe not below y, if inside
        lo = nlo;
    }
    const size_t q = lo + lane;
    const bool below = q < hi && __ldg(a.b + q) < y;
    return lo + __popc(__ballot_sync(FULL, below));
}

// Whole warp: the query elements in [vals[0], vals[cnt-1]] looked up in
// vals[0..cnt) (non-decreasing, in shared memory; cnt >= 1); a hit sets its
// bit.  The query list is read four words (128 elements) at a time, so
// their loads are in flight together; the bitmap is written with atomicOr
// whose result is not waited for.
template <int DIR>
__device__ __forceinline__ void member_unit(const MemberArgs& a, const uint32_t* dir, const uint32_t* vals,
                                           uint32_t cnt, int lane) {
    constexpr int kWords = 4;
    const uint32_t first = vals[0], last = vals[cnt - 1];
    const size_t j0 = lower_bound_warp<DIR>(a, dir, first, lane);
    for (size_t w0 = j0 / 32; 32 * w0 < a.nb; w0 += kWords) {
        uint32_t y[kWords];
#pragma unroll
        for (int i = 0; i < kWords; ++i) {
            const size_t j = 32 * (w0 + i) + lane;
            y[i] = j < a.nb ? __ldg(a.b + j) : 0xFFFFFFFFu;
        }
        bool past = false;
#pragma unroll
        for (int i = 0; i < kWords; ++i) {
            const size_t j = 32 * (w0 + i) + lane;
            const bool out = j >= a.nb || y[i] > last;
            past = past || out;
            bool hit = false;
            if (j >= j0 && !out) {
                uint32_t p = 0;
#pragma unroll
                for (uint32_t s = 2048; s; s >>= 1)
                    if (p + s <= cnt && vals[p + s - 1] < y[i]) p += s;
                hit = p < cnt && vals[p] == y[i];
            }
            const uint32_t mask = __ballot_sync(FULL, hit);
            if (lane == 0 && mask) atomicOr(a.bits + w0 + i, mask);
        }
        if (__any_sync(FULL, past)) break;
    }
}

// The number of set bits of the bitmap (a query element matched by two
// units, equal values across a unit boundary, counts once).
__global__ void count_bits_kernel(const uint32_t* __restrict__ bits, size_t words,
                                  unsigned long long* __restrict__ count) {
    uint32_t c = 0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (size_t)gridDim.x * blockDim.x)
        c += __popc(__ldg(bits + i));
#pragma unroll
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, (unsigned long long)c);
}

static cudaError_t launch_count_bits(const uint32_t* bits, size_t nb, unsigned long long* count, cudaStream_t s) {
    const size_t words = (nb + 31) / 32;
    const int grid = (int)min((size_t)1216, (words + 255) / 256);
    count_bits_kernel<<<grid, 256, 0, s>>>(bits, words, count);
    return cudaGetLastError();
}

// ------------------------------------------------------------ fused path

// The SIMD-BP128 decoder's pipeline (see bp128_decode_kernel) with the
// consumer in place of the stores.  The next metablock's copy is issued
// after the consumer, because the parked values occupy the copy buffer.
template <int DELTA, int FMT, int W>
__global__ void __launch_bounds__(W * 32, 16 / W)
    bp128_member_kernel(const uint8_t* __restrict__ in, size_t in_bytes, size_t n,
                        const uint64_t* __restrict__ index, MemberArgs ma, WsHeader* h) {
    constexpr int NL = DELTA == ICX_DELTA_4 ? 4 : 1;
    extern __shared__ __align__(128) uint8_t smem_raw[];
    TileShared& S = *reinterpret_cast<TileShared*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + kMemberHdr) - 2 * kMaxWarps + 2 * warp;
    uint8_t* buf = smem_raw + kMemberHdr + (size_t)warp * kBuf;
    uint32_t* vals = reinterpret_cast<uint32_t*>(buf);
    uint32_t* dir = reinterpret_cast<uint32_t*>(smem_raw + kMemberHdr + (size_t)W * kBuf);
    const size_t nb = n / 128;
    const uint32_t M = (uint32_t)((nb + 15) / 16);
    const uint32_t ntiles = (M + 1 + W - 1) / W;
    const uint32_t epoch = launch_epoch(h);
    if (lane == 0) mbar_init(bar, 1);
    fence_mbar_init();
    load_dir<kDir>(dir, ma);
    if (threadIdx.x == 0) S.nx[0] = atomicAdd(&h->tile_counter, 1u);
    __syncthreads();
    uint32_t phase = 0, it = 0;
    bool broken = false;  // a copy of this warp never landed: decode nothing more
    auto issue = [&](uint32_t uu) -> uint32_t {
        uint32_t size = 0;
        if (uu < M && !broken && lane == 0) {
            const uint64_t off = index[uu], end = index[uu + 1];
            const bool ok = off <= end && end <= in_bytes && end - off >= 16 && end - off <= kMetaMax &&
                            ((off | end) & 15) == 0;
            size = ok ? (uint32_t)(end - off) : ~0u;
            if (ok) {
                fence_proxy_async();
                mbar_expect_tx(bar, size);
                bulk_load(buf, in + off, size, bar);
            }
        }
        return __shfl_sync(FULL, size, 0);
    };
    uint32_t tile = S.nx[0];
    uint32_t size = tile < ntiles ? issue(tile * W + warp) : 0u;

    while (tile < ntiles) {
        const uint32_t u = tile * W + warp;
        uint4 v[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = make_uint4(0, 0, 0, 0);
        uint32_t K = 0, cnt = 0;  // blocks and integers of this unit
        bool residue = false, ok = true;
        if (u < M) {
            K = (uint32_t)min((size_t)16, nb - 16 * (size_t)u);
            cnt = 128 * K;
            ok = size != ~0u && !broken;
            if (size == ~0u) {
                if (lane == 0) set_error(h, ICX_ECORRUPT);
            } else if (ok) {
                ok = __all_sync(FULL, mbar_wait(bar, phase));
                phase ^= 1;
                if (!ok) {
                    broken = true;
                    if (lane == 0) set_error(h, ICX_ETIMEOUT);
                }
            }
            if (ok) {
                ok = bp128_unpack_unit<FMT>(buf, size, K, v, h, lane);
                residue = ok && FMT == ICX_FMT_W32;
            }
            __syncwarp();
        } else if (u == M) {
            cnt = (uint32_t)(n - 128 * nb);
            if (cnt) {
                tail_unit(in, in_bytes, index[M], cnt, vals, v, h, lane);  // errors go to the status word
                K = 1;
            }
        }
        uint4 mine = make_uint4(0, 0, 0, 0), incl = mine;
        if (DELTA != ICX_DELTA_NONE) {
            const uint4 agg = unit_sum<DELTA>(v, residue);
            if (lane == 0) S.agg[warp] = agg;
            __syncthreads();
            if (warp == 0) {
                incl = tile_agg_scan<W>(S, mine, lane);
                lookback_publish<NL>(h, epoch, tile, shfl4(incl, W - 1));
            }
        }
        if (DELTA == ICX_DELTA_4 && FMT == ICX_FMT_PAPER)
            unit_scan_d4_smem(v, vals, lane);
        else
            unit_local_scan<DELTA>(v, K, residue, lane);
        if (DELTA != ICX_DELTA_NONE && warp == 0) {
            const uint4 base = lookback_resolve<NL>(h, epoch, tile, shfl4(incl, W - 1));
            if (lane < W) S.pref[lane] = add4(base, sub4(incl, mine));
        }
        ++it;
        if (threadIdx.x == 0) S.nx[it & 1] = atomicAdd(&h->tile_counter, 1u);
        __syncthreads();
        uint4 pref = make_uint4(0, 0, 0, 0);
        if (DELTA != ICX_DELTA_NONE) {
            pref = S.pref[warp];
            if (DELTA == ICX_DELTA_1) pref = make_uint4(pref.x, pref.x, pref.x, pref.x);
        }
        const uint32_t next = S.nx[it & 1];
        if (u <= M && cnt && ok) {
            // park the unit's absolute values in natural order, then consume
            __syncwarp();
#pragma unroll
            for (int k = 0; k < 16; ++k)
                if ((uint32_t)k < K) reinterpret_cast<uint4*>(vals)[32 * k + lane] = add4(v[k], pref);
            __syncwarp();
            member_unit<kDir>(ma, dir, vals, cnt, lane);
        }
        fence_proxy_async();  // the parked values are read before the next copy overwrites them
        __syncwarp();
        size = next < ntiles ? issue(next * W + warp) : 0u;
        tile = next;
    }
    // a copy that never landed must not outlive the CTA's shared memory
    if (broken) mbar_wait(bar, phase ^ 1);  // the parity of the wait that timed out
    finish_launch(h, epoch);
}

template <int DELTA, int FMT, int W>
static cudaError_t launch_member(const uint8_t* in, size_t in_bytes, size_t n, const uint64_t* index,
                                 const MemberArgs& ma, WsHeader* h, cudaStream_t s) {
    auto kern = bp128_member_kernel<DELTA, FMT, W>;
    const int smem = (int)(kMemberHdr + (size_t)W * kBuf + 4 * kDir);
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
    const size_t M = (n / 128 + 15) / 16;
    const size_t ctas = (M + 1 + W - 1) / W;
    const int grid = (int)min((size_t)blocks_per_sm * sms, ctas);
    kern<<<grid, W * 32, smem, s>>>(in, in_bytes, n, index, ma, h);
    return cudaGetLastError();
}

static MemberArgs member_args(const uint32_t* b, size_t nb, uint32_t* bits, int dir_entries) {
    MemberArgs a;
    a.b = b;
    a.nb = nb;
    a.bits = bits;
    a.step = (nb + dir_entries - 1) / dir_entries;
    return a;
}

cudaError_t launch_bp128_member(int delta, int fmt, const uint8_t* in, size_t in_bytes, size_t n,
                                const uint64_t* index, const uint32_t* b, size_t nb, uint32_t* bits,
                                unsigned long long* count, WsHeader* h, cudaStream_t s) {
    const MemberArgs ma = member_args(b, nb, bits, kDir);
    cudaError_t e = cudaErrorInvalidValue;
#define ICX_CASE(D, F, W) \
    if (delta == D && fmt == F) e = launch_member<D, F, W>(in, in_bytes, n, index, ma, h, s);
    ICX_CASE(ICX_DELTA_NONE, ICX_FMT_PAPER, 4)
    ICX_CASE(ICX_DELTA_1, ICX_FMT_PAPER, 4)
    ICX_CASE(ICX_DELTA_4, ICX_FMT_PAPER, 4)
    ICX_CASE(ICX_DELTA_NONE, ICX_FMT_W32, 8)
    ICX_CASE(ICX_DELTA_1, ICX_FMT_W32, 8)
    ICX_CASE(ICX_DELTA_4, ICX_FMT_W32, 8)
#undef ICX_CASE
    return e != cudaSuccess ? e : launch_count_bits(bits, nb, count, s);
}

// ----------------------------------------------------------- unfused path

constexpr int kSortedWarps = 12;  // 2 CTAs of 112 KB per SM

// Units of 2,048 integers of the decoded array, a grid stride apart per
// warp: one 128-bit load per lane and block into the warp's shared buffer,
// then the consumer.
__global__ void __launch_bounds__(kSortedWarps * 32)
    sorted_member_kernel(const uint32_t* __restrict__ a, size_t n, MemberArgs ma) {
    extern __shared__ __align__(128) uint8_t smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t* dir = reinterpret_cast<uint32_t*>(smem_raw);
    uint32_t* vals = reinterpret_cast<uint32_t*>(smem_raw + 4 * kDir) + 2048 * warp;
    load_dir<kDir>(dir, ma);
    __syncthreads();
    const size_t U = (n + 2047) / 2048;
    for (size_t u = (size_t)blockIdx.x * kSortedWarps + warp; u < U; u += (size_t)gridDim.x * kSortedWarps) {
        const size_t first = 2048 * u;
        const uint32_t cnt = (uint32_t)min((size_t)2048, n - first);
        uint4 r[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const size_t p = first + 128 * k + 4 * lane;
            if (p + 4 <= n) {
                r[k] = __ldg(reinterpret_cast<const uint4*>(a + p));
            } else {
                uint32_t t[4];
                for (int c = 0; c < 4; ++c) t[c] = p + c < n ? __ldg(a + p + c) : 0u;
                r[k] = make_uint4(t[0], t[1], t[2], t[3]);
            }
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 16; ++k) reinterpret_cast<uint4*>(vals)[32 * k + lane] = r[k];
        __syncwarp();
        member_unit<kDir>(ma, dir, vals, cnt, lane);
    }
}

cudaError_t launch_sorted_member(const uint32_t* a, size_t n, const uint32_t* b, size_t nb, uint32_t* bits,
                                 unsigned long long* count, cudaStream_t s) {
    const MemberArgs ma = member_args(b, nb, bits, kDir);
    const int smem = 4 * kDir + kSortedWarps * 2048 * 4;
    static int blocks_per_sm = -1;
    static int sms = 0;
    if (blocks_per_sm < 0) {
        cudaError_t e = cudaFuncSetAttribute(sorted_member_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, sorted_member_kernel, kSortedWarps * 32,
                                                          smem);
        if (e != cudaSuccess) return e;
        if (blocks_per_sm < 1) blocks_per_sm = 1;
    }
    const size_t U = (n + 2047) / 2048;
    const int grid = (int)min((size_t)blocks_per_sm * sms, (U + kSortedWarps - 1) / kSortedWarps);
    sorted_member_kernel<<<grid, kSortedWarps * 32, smem, s>>>(a, n, ma);
    const cudaError_t e = cudaGetLastError();
    return e != cudaSuccess ? e : launch_count_bits(bits, nb, count, s);
}

}  // namespace icx
