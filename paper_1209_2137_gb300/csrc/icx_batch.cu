// Batched decoding of many independent lists (posting-list-like arrays of
// uneven length) in one CUDA graph launch.
//
// Every list is cut into units exactly as its single-array decoder cuts it:
// SIMD-BP128 metablocks (2048 integers) or SIMD-FastPFOR units of 16 blocks
// of a page, then the Variable Byte tail if n % 128 != 0.  The plan lays all
// units of all lists out in one work-list (lists contiguous, in a tuned
// order).  One persistent kernel takes tiles of W consecutive work items
// (dynamic tile ids); per tile each warp decodes one unit exactly like the
// single-array kernels, and the carries of differential decoding (Sec. 3)
// come from a segmented scan over the tile plus a decoupled look-back that
// only ever follows the tile's first list:
//   * a tile whose first unit starts a list needs no carry-in;
//   * a tile publishes the running sum of its LAST list: as an inclusive
//     prefix right away when that list starts inside the tile, else as an
//     aggregate that becomes an inclusive prefix after its own look-back.
// So a look-back chain never leaves a list, and short lists never wait.
// Before it, one page-parse launch covers every SIMD-FastPFOR page of every
// list (the same parse as the single-array decoder).
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <string>
#include <vector>

#include "icx_bp128.cuh"
#include "icx_fastpfor.cuh"
#include "icx_kernels.cuh"

namespace icx {

struct __align__(16) ListDev {
    const uint8_t* in;
    uint64_t in_bytes;
    uint32_t* out;
    uint64_t n;
    const uint64_t* index;
    uint32_t page_slot;  // SIMD-FastPFOR: record slot of its first page
    uint32_t units;      // M: metablocks / 16-block units (the tail is unit M)
    uint32_t tail_at;    // index entry where the Variable Byte tail starts
    uint8_t codec, delta, fmt, pad;
    uint32_t item_base;  // its first work item
    uint32_t pad2;
};
static_assert(sizeof(ListDev) == 64, "list record");

constexpr int kBatchHdr = 1024;
constexpr int kBatchBuf = kBuf > kFBuf ? kBuf : kFBuf;
// per warp: staging buffer, 16 block records, exception scratch, unit context
struct WarpCtx {
    ListDev L;
    uint64_t pbase;  // SIMD-FastPFOR: byte offset of the unit's page
    uint32_t u, K, size, slot;
    uint32_t valid, list, pad[4];
};
static_assert(sizeof(WarpCtx) == 112, "warp context");
constexpr int kWarpBytes = kBatchBuf + 16 * 16 + kExScratchBytes + (int)sizeof(WarpCtx) + 128;
static_assert(kWarpBytes % 16 == 0, "warp region");

struct BatchShared {
    uint4 agg[kMaxWarps];
    uint4 pref[kMaxWarps];
    uint32_t list[kMaxWarps];
    uint32_t start[kMaxWarps];
    uint32_t nx[2];
};
static_assert(sizeof(BatchShared) + 8 * kMaxWarps <= kBatchHdr, "batch header");

// ---------------------------------------------------------------- kernels

// Pages of more than kSmallK blocks: one CTA each (items: list, page).
__global__ void __launch_bounds__(kMetaThreads, 7)
    batch_meta_kernel(const ListDev* __restrict__ lists, const uint2* __restrict__ pages,
                      BlockMeta* __restrict__ meta, uint32_t* __restrict__ pmeta, uint2* __restrict__ umeta,
                      ulonglong2* __restrict__ ranges, WsHeader* h) {
    __shared__ MetaSmem S;
    const uint2 pi = pages[blockIdx.x];
    const ListDev& L = lists[pi.x];
    const uint64_t nb = L.n / 128;
    const uint32_t K = (uint32_t)min((uint64_t)kBlocksPerPage, nb - (uint64_t)kBlocksPerPage * pi.y);
    const size_t g = (size_t)L.page_slot + pi.y;
    parse_page(S, L.in, L.in_bytes, L.index[pi.y], L.index[pi.y + 1], K, meta + kBlocksPerPage * g,
               pmeta + kPageMetaWords * g, umeta + kUnitsPerPage * g, h,
               ranges + L.item_base + (size_t)kUnitsPerPage * pi.y);
}

// Pages of at most kSmallK blocks: one warp each.
constexpr int kSmallWarps = 8;

__global__ void __launch_bounds__(kSmallWarps * 32)
    batch_meta_small_kernel(const ListDev* __restrict__ lists, const uint2* __restrict__ pages, uint32_t count,
                            BlockMeta* __restrict__ meta, uint32_t* __restrict__ pmeta, uint2* __restrict__ umeta,
                            ulonglong2* __restrict__ ranges, WsHeader* h) {
    __shared__ SmallPageSmem S[kSmallWarps];
    const int warp = threadIdx.x >> 5;
    const uint32_t j = blockIdx.x * kSmallWarps + warp;
    if (j >= count) return;
    const uint2 pi = pages[j];
    const ListDev& L = lists[pi.x];
    const uint64_t nb = L.n / 128;
    const uint32_t K = (uint32_t)min((uint64_t)kBlocksPerPage, nb - (uint64_t)kBlocksPerPage * pi.y);
    const size_t g = (size_t)L.page_slot + pi.y;
    parse_small_page(S[warp], L.in, L.in_bytes, L.index[pi.y], L.index[pi.y + 1], K, meta + kBlocksPerPage * g,
                     pmeta + kPageMetaWords * g, umeta + kUnitsPerPage * g, h,
                     ranges + L.item_base + (size_t)kUnitsPerPage * pi.y);
}

// Copy range (address, bytes) of every SIMD-BP128 work item: the metablock
// its index entries delimit, bytes = ~0 if they are invalid.  (SIMD-FastPFOR
// items get theirs from the page parse of every launch; tails copy nothing.)
__global__ void batch_ranges_kernel(const ListDev* __restrict__ lists, const uint2* __restrict__ work, uint32_t nwork,
                                    ulonglong2* __restrict__ ranges) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nwork) return;
    const uint2 wi = work[i];
    const ListDev& L = lists[wi.x];
    if (L.codec != ICX_CODEC_BP128 && wi.y < L.units) return;
    ulonglong2 r = make_ulonglong2(0, 0);
    if (wi.y < L.units) {
        const uint64_t off = L.index[wi.y], end = L.index[wi.y + 1];
        const bool ok = off <= end && end <= L.in_bytes && end - off >= 16 && end - off <= kMetaMax &&
                        ((off | end) & 15) == 0;
        r = ok ? make_ulonglong2(reinterpret_cast<uint64_t>(L.in + off), end - off) : make_ulonglong2(0, ~0u);
    }
    ranges[i] = r;
}

// Index of a list stored without one (at most one metablock / page): entry 0
// = 0 and entry 1 = the end of that metablock / page (where the tail starts).
__global__ void batch_mini_index_kernel(const ListDev* __restrict__ lists, const uint32_t* __restrict__ ids,
                                        uint32_t count, uint64_t* __restrict__ mini, WsHeader* h) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= count) return;
    const ListDev& L = lists[ids[j]];
    uint64_t* ix = mini + 2 * (size_t)j;
    const uint64_t nb = L.n / 128;
    uint64_t end = 0;
    bool bad = false;
    if (nb > 0) {
        if (L.codec == ICX_CODEC_BP128) {
            if (L.in_bytes < 16) {
                bad = true;
            } else {
                const uint4 d = *reinterpret_cast<const uint4*>(L.in);
                uint32_t sum = 0;
                for (uint32_t k = 0; k < nb; ++k) {
                    const uint32_t b = desc_width(d, (int)k);
                    bad |= b > 32;
                    sum += b;
                }
                end = L.fmt == ICX_FMT_PAPER ? 16 + 16 * (uint64_t)sum : 16 + 128 * (uint64_t)((4 * sum + 31) / 32);
            }
        } else {
            if (L.in_bytes < 16) {
                bad = true;
            } else {
                const uint64_t len_at = 4 * (uint64_t)ld32(L.in);
                bad = len_at < 16 || (len_at & 15) || len_at + 4 > L.in_bytes;
                uint64_t q = 0;
                if (!bad) {
                    q = len_at + 4 + pad_up(ld32(L.in + len_at), 4);
                    bad = q + 4 > L.in_bytes;
                }
                if (!bad) {
                    const uint32_t bitset = ld32(L.in + q);
                    q += 4;
                    for (int d = 1; d <= 32 && !bad; ++d) {
                        if (!((bitset >> (d - 1)) & 1u)) continue;
                        if (q + 4 > L.in_bytes) {
                            bad = true;
                            break;
                        }
                        const uint64_t cnt = ld32(L.in + q);
                        q = pad_up(q + 4, 16) + 16 * (uint64_t)d * ((cnt + 127) / 128);
                    }
                }
                end = pad_up(q, 16);
            }
        }
        if (end > L.in_bytes) bad = true;
    }
    ix[0] = 0;
    ix[1] = bad ? L.in_bytes : end;
    if (bad) set_error(h, ICX_ECORRUPT);
}

// One look-back state per chain for `tile`: flag 1 = aggregate, 2 = prefix.
__device__ __forceinline__ void publish_state(WsHeader* h, uint32_t epoch, uint32_t tile, uint4 v, bool prefix) {
    const int lane = threadIdx.x & 31;
    const uint32_t tag = (epoch << 2) | (prefix ? 2u : 1u);
    if (lane < 4)
        st_relaxed(tile_states(h) + (size_t)tile * kStatesPerTile + lane,
                   ((unsigned long long)tag << 32) | comp(v, lane));
}

// A decode instance of the serving loop: one list of one request, decoded
// into that request's buffer.
struct InstDev {
    uint32_t list, pad;
    uint32_t* out;
};
// A work item of the serving loop, built on the host: the unit's copy range,
// its instance and unit index.
struct __align__(16) ServeItem {
    uint64_t src;
    uint32_t size, inst, u, pad;
    uint64_t pad2;
};
static_assert(sizeof(ServeItem) == 32, "serve item");

// SERVE = false: work items are (list, unit) of a plan with per-item copy
// ranges; SERVE = true: serving-loop items (ServeItem) whose instances
// (InstDev) name the list and the output, segments are instances.  CODEC:
// -1 = items of both codecs, else only that codec's (the other code path is
// compiled out).
template <int W, bool SERVE, int CODEC = -1>
__global__ void __launch_bounds__(W * 32, 16 / W)
    batch_decode_kernel(const ListDev* __restrict__ lists, const uint2* __restrict__ work, uint32_t nwork,
                        const ulonglong2* __restrict__ ranges, const BlockMeta* __restrict__ meta,
                        const uint32_t* __restrict__ pmeta, bool l2_ahead, WsHeader* h,
                        const ServeItem* __restrict__ items = nullptr, const InstDev* __restrict__ insts = nullptr) {
    extern __shared__ __align__(128) uint8_t smem_raw[];
    BatchShared& S = *reinterpret_cast<BatchShared*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + kBatchHdr) - kMaxWarps + warp;
    uint8_t* wbase = smem_raw + kBatchHdr + (size_t)warp * kWarpBytes;
    uint8_t* buf = wbase;
    BlockMeta* m = reinterpret_cast<BlockMeta*>(wbase + kBatchBuf);
    uint8_t* blk_of = wbase + kBatchBuf + 256;
    WarpCtx& C = *reinterpret_cast<WarpCtx*>(wbase + kBatchBuf + 256 + kExScratchBytes);
    uint32_t* pg = reinterpret_cast<uint32_t*>(wbase + kBatchBuf + 256 + kExScratchBytes + sizeof(WarpCtx));  // array offsets
    const uint32_t ntiles = (nwork + W - 1) / W;
    const uint32_t epoch = launch_epoch(h);
    if (lane == 0) mbar_init(bar, 1);
    fence_mbar_init();
    if (threadIdx.x == 0) S.nx[0] = atomicAdd(&h->tile_counter, 1u);
    __syncthreads();
    uint32_t phase = 0, it = 0;
    bool broken = false;

    // Work item i, step 1: its precomputed copy range; the bulk copy starts
    // at once.  C.size: bytes in flight (0: none, ~0u: invalid).
    auto start_copy = [&](uint32_t i) {
        __syncwarp();
        if (lane == 0) {
            if (i < nwork) {
                uint32_t a, u, size;
                uint64_t src;
                if constexpr (SERVE) {
                    const ServeItem it_ = items[i];
                    a = it_.inst;
                    u = it_.u;
                    size = it_.size;
                    src = it_.src;
                } else {
                    const uint2 wi = work[i];
                    const ulonglong2 rg = ranges[i];
                    a = wi.x;
                    u = wi.y;
                    size = (uint32_t)rg.y;
                    src = rg.x;
                }
                if (!broken && size != 0 && size != ~0u) {
                    fence_proxy_async();
                    mbar_expect_tx(bar, size);
                    bulk_load(buf, reinterpret_cast<const void*>(src), size, bar);
                }
                C.list = a;
                C.u = u;
                C.size = size;
                C.valid = 1;
            } else {
                C.valid = 0;
            }
        }
        __syncwarp();
    };
    // step 2, while the copy is in flight: the list record and, for a
    // SIMD-FastPFOR unit, its block records and page offset
    auto load_context = [&]() {
        if (!C.valid) return;
        if constexpr (SERVE) {
            const InstDev in_ = insts[C.list];
            if (lane < 4) reinterpret_cast<uint4*>(&C.L)[lane] = reinterpret_cast<const uint4*>(lists + in_.list)[lane];
            __syncwarp();
            if (lane == 0) C.L.out = in_.out;
        } else {
            if (lane < 4)
                reinterpret_cast<uint4*>(&C.L)[lane] = reinterpret_cast<const uint4*>(lists + C.list)[lane];
        }
        __syncwarp();
        const uint32_t u = C.u, M = C.L.units;
        const uint64_t nb = C.L.n / 128;
        const uint32_t K = u < M ? (uint32_t)min((uint64_t)16, nb - 16 * (uint64_t)u) : 0u;
        if (CODEC != ICX_CODEC_BP128 && u < M && (CODEC == ICX_CODEC_FASTPFOR || C.L.codec == ICX_CODEC_FASTPFOR)) {
            const uint32_t p = u / kUnitsPerPage, q = u % kUnitsPerPage;
            const uint32_t slot = C.L.page_slot + p;
            if ((uint32_t)lane < K)
                reinterpret_cast<uint4*>(m)[lane] =
                    reinterpret_cast<const uint4*>(meta + (size_t)kBlocksPerPage * slot + 16 * q)[lane];
            pg[lane] = pmeta[(size_t)kPageMetaWords * slot + lane];
            if (lane == 0) {
                C.slot = slot;
                C.pbase = C.L.index[p];
            }
        }
        if (lane == 0) C.K = K;
        __syncwarp();
    };

    uint32_t tile = S.nx[0];
    start_copy(tile < ntiles ? tile * W + warp : nwork);
    load_context();

    while (tile < ntiles) {
        const uint32_t i = tile * W + warp;
        uint4 v[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = make_uint4(0, 0, 0, 0);
        const bool valid = C.valid != 0;
        const uint32_t u = C.u, K = C.K, size = C.size, M = C.L.units;
        const int codec = C.L.codec, delta = C.L.delta, fmt = C.L.fmt;
        uint32_t Ks = 0;  // blocks to scan and store
        bool residue = false;
        ulonglong2 pf = make_ulonglong2(0, 0);
        if (l2_ahead && lane == 0 && i + gridDim.x * W < nwork) {
            if constexpr (SERVE) {
                const ServeItem& a = items[i + gridDim.x * W];
                pf = make_ulonglong2(a.src, a.size);
            } else {
                pf = ranges[i + gridDim.x * W];
            }
        }
        if (valid && u < M) {
            Ks = K;
            bool ok = size != ~0u && !broken;
            if (size == ~0u) {
                if (lane == 0) set_error(h, ICX_ECORRUPT);
            } else if (ok && size != 0) {
                ok = __all_sync(FULL, mbar_wait(bar, phase));
                phase ^= 1;
                if (!ok) {
                    broken = true;
                    if (lane == 0) set_error(h, ICX_ETIMEOUT);
                }
            }
            if (lane == 0 && pf.y && pf.y != ~0ull) prefetch_l2(reinterpret_cast<const void*>(pf.x), (uint32_t)pf.y);
            if (ok) {
                const bool fp = CODEC == ICX_CODEC_FASTPFOR || (CODEC == -1 && codec == ICX_CODEC_FASTPFOR);
                if (CODEC != ICX_CODEC_BP128 && fp) {
                    fp_unit_unpack_patch(C.L.in, C.pbase, pg, m, K, buf, blk_of, v, h, lane);
                } else if (CODEC != ICX_CODEC_FASTPFOR && fmt == ICX_FMT_W32) {
                    ok = bp128_unpack_unit<ICX_FMT_W32>(buf, size, K, v, h, lane);
                    residue = ok;
                } else if (CODEC != ICX_CODEC_FASTPFOR) {
                    bp128_unpack_unit<ICX_FMT_PAPER>(buf, size, K, v, h, lane);
                }
            }
            __syncwarp();
        } else if (valid) {
            const uint32_t count = (uint32_t)(C.L.n % 128);
            if (count) {
                tail_unit(C.L.in, C.L.in_bytes, C.L.index[C.L.tail_at], count, reinterpret_cast<uint32_t*>(buf), v,
                          h, lane);
                Ks = 1;
            }
        }
        // unit aggregate straight after unpacking
        uint4 agg = make_uint4(0, 0, 0, 0);
        if (valid && delta == ICX_DELTA_1) agg = unit_sum<ICX_DELTA_1>(v, residue);
        if (valid && delta == ICX_DELTA_4) agg = unit_sum<ICX_DELTA_4>(v, residue);
        if (lane == 0) {
            S.agg[warp] = agg;
            S.list[warp] = valid ? C.list : 0xFFFFFFFFu - (uint32_t)warp;
            S.start[warp] = valid && u == 0;
        }
        __syncthreads();
        // warp 0: segmented scan of the tile (segments = lists), publish the
        // last list's running sum, look back for the first list if needed
        uint4 a = make_uint4(0, 0, 0, 0), incl = a;
        uint32_t first_b = W;
        bool need_carry = false, single = true;
        if (warp == 0) {
            const bool have = lane < W;
            a = have ? S.agg[lane] : make_uint4(0, 0, 0, 0);
            const uint32_t li = have ? S.list[lane] : 0xFFFFFFF0u - (uint32_t)lane;
            const uint32_t lp = __shfl_up_sync(FULL, li, 1);
            const bool bnd = lane == 0 || li != lp;
            incl = a;
            bool f = bnd;
#pragma unroll
            for (int off = 1; off < W; off <<= 1) {
                const uint4 y = make_uint4(__shfl_up_sync(FULL, incl.x, off), __shfl_up_sync(FULL, incl.y, off),
                                           __shfl_up_sync(FULL, incl.z, off), __shfl_up_sync(FULL, incl.w, off));
                const bool fy = __shfl_up_sync(FULL, f, off);
                if (lane >= off) {
                    if (!f) incl = add4(incl, y);
                    f = f || fy;
                }
            }
            const unsigned bm = __ballot_sync(FULL, bnd && lane > 0 && lane < W);
            first_b = bm ? (uint32_t)(__ffs(bm) - 1) : (uint32_t)W;
            single = bm == 0;
            need_carry = S.start[0] == 0;
            // the last list's running sum: a prefix unless it is the tile's
            // first list and that list started in an earlier tile
            publish_state(h, epoch, tile, shfl4(incl, W - 1), !(single && need_carry));
        }
        if (valid && delta == ICX_DELTA_1) {
            unit_local_scan<ICX_DELTA_1>(v, Ks, residue, lane);
        } else if (valid && delta == ICX_DELTA_4) {
            if (residue)
                unit_local_scan<ICX_DELTA_4>(v, Ks, true, lane);
            else
                unit_scan_d4_smem(v, reinterpret_cast<uint32_t*>(buf), lane);
        } else if (residue) {
#pragma unroll
            for (int k = 0; k < 16; ++k) v[k] = residue_to_row(v[k], lane);
        }
        if (warp == 0) {
            uint4 carry = make_uint4(0, 0, 0, 0);
            if (need_carry) carry = lookback_resolve<4>(h, epoch, tile, shfl4(incl, W - 1), single);
            if (lane < W) {
                uint4 pr = sub4(incl, a);
                if ((uint32_t)lane < first_b) pr = add4(pr, carry);
                S.pref[lane] = pr;
            }
        }
        ++it;
        if (threadIdx.x == 0) S.nx[it & 1] = atomicAdd(&h->tile_counter, 1u);
        __syncthreads();
        uint4 pref = S.pref[warp];
        if (delta == ICX_DELTA_1) pref = make_uint4(pref.x, pref.x, pref.x, pref.x);
        if (delta == ICX_DELTA_NONE) pref = make_uint4(0, 0, 0, 0);
        uint32_t* out = C.L.out;
        const uint64_t n = C.L.n, first = u < M ? 2048 * (uint64_t)u : 128 * (n / 128);
        const uint32_t next = S.nx[it & 1];
        start_copy(next < ntiles ? next * W + warp : nwork);  // lands during the stores
        if (valid && Ks) store_unit(out, first, n, v, Ks, pref, lane);
        load_context();
        tile = next;
    }
    if (broken) mbar_wait(bar, phase ^ 1);  // the parity of the wait that timed out
    finish_launch(h, epoch);
}

// ------------------------------------------------------------------ plan

struct PlanMem {
    ListDev* lists = nullptr;
    uint2* work = nullptr;
    ulonglong2* ranges = nullptr;
    uint2* pages = nullptr;  // large pages, then small pages
    BlockMeta* meta = nullptr;
    uint32_t* pmeta = nullptr;
    uint2* umeta = nullptr;
    uint64_t* mini = nullptr;
    uint32_t* mini_ids = nullptr;
    WsHeader* ws = nullptr;   // page parses and SIMD-FastPFOR items
    WsHeader* ws2 = nullptr;  // SIMD-BP128 items
};

template <int CODEC>
static cudaError_t batch_occupancy(int W, int* blocks, int* sms) {
    const int smem = kBatchHdr + W * kWarpBytes;
    cudaError_t e;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev);
    // the page parse wants 7 CTAs of 30 KB per SM
    e = cudaFuncSetAttribute(batch_meta_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    if (W == 4) {
        e = cudaFuncSetAttribute(batch_decode_kernel<4, false, CODEC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, batch_decode_kernel<4, false, CODEC>, W * 32,
                                                              smem);
    } else {
        e = cudaFuncSetAttribute(batch_decode_kernel<8, false, CODEC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, batch_decode_kernel<8, false, CODEC>, W * 32,
                                                              smem);
    }
    if (*blocks < 1) *blocks = 1;
    return e;
}

template <int CODEC>
static void launch_batch(int W, int grid, cudaStream_t st, const PlanMem& d, const uint2* work, uint32_t nwork,
                         const ulonglong2* ranges, bool l2, WsHeader* ws) {
    const int smem = kBatchHdr + W * kWarpBytes;
    if (W == 4)
        batch_decode_kernel<4, false, CODEC><<<grid, 128, smem, st>>>(d.lists, work, nwork, ranges, d.meta, d.pmeta,
                                                                     l2, ws);
    else
        batch_decode_kernel<8, false, CODEC><<<grid, 256, smem, st>>>(d.lists, work, nwork, ranges, d.meta, d.pmeta,
                                                                     l2, ws);
}

}  // namespace icx

using icx::ListDev;

struct icx_plan {
    int device = 0;
    std::vector<icx_list_desc> lists;
    std::vector<ListDev> host_lists;
    std::vector<uint32_t> items_per_list;  // work items of each list
    size_t nwork = 0, nwork_bp = 0, npages = 0, nlarge = 0, nsmall = 0, nmini = 0;
    size_t max_n = 0;
    void* mem = nullptr;
    icx::PlanMem d;
    icx_tuning tune{8, 0, 1, nullptr};
    cudaStream_t cap = nullptr;   // capture stream
    cudaStream_t cap2 = nullptr;  // second branch of the graph (small pages)
    cudaStream_t cap3 = nullptr;  // third branch (SIMD-BP128 items)
    cudaEvent_t fork = nullptr, join = nullptr, join3 = nullptr;
    cudaGraphExec_t exec = nullptr;
    // per-list baseline
    void* single_ws = nullptr;
    size_t single_ws_bytes = 0;
    cudaGraphExec_t per_list_exec = nullptr;
};

namespace {

thread_local long long g_error_list = -1;

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

icx_status check_list(const icx_list_desc& l) {
    if (!(l.codec == ICX_CODEC_BP128 || l.codec == ICX_CODEC_FASTPFOR)) return ICX_EINVAL;
    if (!(l.delta == ICX_DELTA_NONE || l.delta == ICX_DELTA_1 || l.delta == ICX_DELTA_4)) return ICX_EINVAL;
    if (l.codec == ICX_CODEC_BP128 && !(l.fmt == ICX_FMT_PAPER || l.fmt == ICX_FMT_W32)) return ICX_EINVAL;
    if (l.codec == ICX_CODEC_FASTPFOR && l.fmt != ICX_FMT_PAPER) return ICX_EINVAL;  // SIMD-FastPFOR only
    if (l.n == 0) return ICX_OK;
    if (!l.d_in || !l.d_out) return ICX_EINVAL;
    if (!aligned16(l.d_in) || !aligned16(l.d_out) || (l.d_index && !aligned16(l.d_index))) return ICX_EALIGN;
    if (l.n > ((size_t)1 << 36)) return ICX_EINVAL;
    const size_t nb = l.n / 128;
    if (!l.d_index) {
        const bool small = l.codec == ICX_CODEC_BP128 ? (nb + 15) / 16 <= 1 : (nb + 511) / 512 <= 1;
        if (!small) return ICX_EINVAL;
    }
    return ICX_OK;
}

// Fills the device record of list i, appends its pages (more than kSmallK
// blocks: `large`, else `small`; slots counted by npages) and, without an
// index, its id to mini_ids.  Returns its work items (units, then the tail).
uint32_t layout_list(const icx_list_desc& l, uint32_t i, ListDev& d, size_t& npages, std::vector<uint2>& large,
                     std::vector<uint2>& small, std::vector<uint32_t>& mini_ids) {
    using namespace icx;
    std::memset(&d, 0, sizeof d);
    const size_t nb = l.n / 128, M = (nb + 15) / 16;
    d.in = l.d_in;
    d.in_bytes = l.d_in ? l.in_bytes : 0;
    d.out = l.d_out;
    d.n = l.n;
    d.index = l.d_index;
    d.units = (uint32_t)M;
    d.codec = (uint8_t)l.codec;
    d.delta = (uint8_t)l.delta;
    d.fmt = (uint8_t)(l.codec == ICX_CODEC_BP128 ? l.fmt : 0);
    if (l.codec == ICX_CODEC_FASTPFOR) {
        const size_t P = (nb + kBlocksPerPage - 1) / kBlocksPerPage;
        d.page_slot = (uint32_t)npages;
        d.tail_at = (uint32_t)P;
        for (size_t q = 0; q < P; ++q) {
            const size_t K = std::min<size_t>(kBlocksPerPage, nb - kBlocksPerPage * q);
            (K > kSmallK ? large : small).push_back(make_uint2(i, (uint32_t)q));
        }
        npages += P;
    } else {
        d.tail_at = (uint32_t)M;
    }
    if (l.n && !l.d_index) mini_ids.push_back(i);
    return l.n ? (uint32_t)(M + (l.n % 128 ? 1 : 0)) : 0u;
}

// work-list: lists contiguous, in the tuned order
std::vector<uint2> build_work(const icx_plan& p, int order) {
    const size_t L = p.lists.size();
    std::vector<uint32_t> ids(L);
    for (size_t i = 0; i < L; ++i) ids[i] = (uint32_t)i;
    if (order == 1)
        std::stable_sort(ids.begin(), ids.end(),
                         [&](uint32_t a, uint32_t b) { return p.items_per_list[a] > p.items_per_list[b]; });
    else if (order == 2)
        std::stable_sort(ids.begin(), ids.end(),
                         [&](uint32_t a, uint32_t b) { return p.items_per_list[a] < p.items_per_list[b]; });
    // SIMD-BP128 lists first, then SIMD-FastPFOR lists (one decode kernel each)
    std::vector<uint2> w;
    w.reserve(p.nwork);
    for (int codec : {ICX_CODEC_BP128, ICX_CODEC_FASTPFOR})
        for (uint32_t id : ids)
            if (p.lists[id].codec == codec)
                for (uint32_t u = 0; u < p.items_per_list[id]; ++u) w.push_back(make_uint2(id, u));
    return w;
}

cudaError_t capture(icx_plan* p) {
    using namespace icx;
    if (p->exec) {
        cudaGraphExecDestroy(p->exec);
        p->exec = nullptr;
    }
    const int W = p->tune.warps_per_cta;
    const bool l2 = p->tune.l2_prefetch != 0;
    int b_bp = 1, b_fp = 1, sms = 1;
    cudaError_t e = batch_occupancy<ICX_CODEC_BP128>(W, &b_bp, &sms);
    if (e == cudaSuccess) e = batch_occupancy<ICX_CODEC_FASTPFOR>(W, &b_fp, &sms);
    if (e != cudaSuccess) return e;
    // both decode kernels are persistent over their work-lists with a full
    // grid each: the second one's CTAs take the SMs as the first one's finish
    const size_t n_bp = p->nwork_bp, n_fp = p->nwork - p->nwork_bp;
    const size_t g_bp = std::min<size_t>((size_t)b_bp * sms, (n_bp + W - 1) / W);
    const size_t g_fp = std::min<size_t>((size_t)b_fp * sms, (n_fp + W - 1) / W);
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaEventRecord(p->fork, p->cap);
    // branch 3: SIMD-BP128 items (no page parse needed)
    if (n_bp) {
        cudaStreamWaitEvent(p->cap3, p->fork, 0);
        launch_batch<ICX_CODEC_BP128>(W, (int)g_bp, p->cap3, p->d, p->d.work, (uint32_t)n_bp, p->d.ranges, l2,
                                      p->d.ws2);
        cudaEventRecord(p->join3, p->cap3);
    }
    // branch 2: short pages; main: long pages, then SIMD-FastPFOR items
    if (p->nsmall) {
        cudaStreamWaitEvent(p->cap2, p->fork, 0);
        batch_meta_small_kernel<<<(unsigned)((p->nsmall + kSmallWarps - 1) / kSmallWarps), kSmallWarps * 32, 0,
                                  p->cap2>>>(p->d.lists, p->d.pages + p->nlarge, (uint32_t)p->nsmall, p->d.meta,
                                             p->d.pmeta, p->d.umeta, p->d.ranges, p->d.ws);
        cudaEventRecord(p->join, p->cap2);
    }
    if (p->nlarge)
        batch_meta_kernel<<<(unsigned)p->nlarge, kMetaThreads, 0, p->cap>>>(p->d.lists, p->d.pages, p->d.meta,
                                                                           p->d.pmeta, p->d.umeta, p->d.ranges,
                                                                           p->d.ws);
    if (p->nsmall) cudaStreamWaitEvent(p->cap, p->join, 0);
    if (n_fp)
        launch_batch<ICX_CODEC_FASTPFOR>(W, (int)g_fp, p->cap, p->d, p->d.work + n_bp, (uint32_t)n_fp,
                                         p->d.ranges + n_bp, l2, p->d.ws);
    if (n_bp) cudaStreamWaitEvent(p->cap, p->join3, 0);
    cudaError_t le = cudaGetLastError();
    e = cudaStreamEndCapture(p->cap, &g);
    if (le != cudaSuccess) e = le;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, g, 0);
    if (g) cudaGraphDestroy(g);
    return e;
}

cudaError_t apply_order(icx_plan* p, int order) {
    const std::vector<uint2> w = build_work(*p, order);
    if (w.empty()) return cudaSuccess;
    for (size_t i = 0; i < w.size(); ++i)
        if (w[i].y == 0) p->host_lists[w[i].x].item_base = (uint32_t)i;
    cudaError_t e = cudaMemcpy(p->d.lists, p->host_lists.data(), sizeof(ListDev) * p->host_lists.size(),
                               cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->d.work, w.data(), w.size() * sizeof(uint2), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    icx::batch_ranges_kernel<<<(unsigned)((w.size() + 255) / 256), 256, 0, p->cap>>>(p->d.lists, p->d.work,
                                                                                    (uint32_t)w.size(), p->d.ranges);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->cap);
    return e;
}

// ------------------------------------------------------------ tuning cache

std::string signature(const icx_plan& p) {
    uint64_t hsh = 1469598103934665603ull;  // FNV-1a over (n, codec, delta, fmt)
    auto mix = [&](uint64_t x) {
        for (int b = 0; b < 8; ++b) {
            hsh ^= (x >> (8 * b)) & 0xFF;
            hsh *= 1099511628211ull;
        }
    };
    for (const auto& l : p.lists) {
        mix(l.n);
        mix((uint64_t)l.codec | (uint64_t)l.delta << 8 | (uint64_t)l.fmt << 16);
    }
    char buf[96];
    snprintf(buf, sizeof buf, "lists=%zu;units=%zu;h=%016llx", p.lists.size(), p.nwork, (unsigned long long)hsh);
    return buf;
}

const char* cache_file(const icx_tuning* t) {
    if (t && t->cache_path) return t->cache_path;
    return std::getenv("ICX_TUNE_CACHE");
}

// The cache is a flat JSON object {"<signature>": [W, order, l2], ...}.
bool cache_lookup(const char* path, const std::string& key, int* W, int* order, int* l2) {
    if (!path) return false;
    FILE* f = std::fopen(path, "rb");
    if (!f) return false;
    std::string s;
    char chunk[4096];
    size_t r;
    while ((r = std::fread(chunk, 1, sizeof chunk, f)) > 0) s.append(chunk, r);
    std::fclose(f);
    const std::string k = "\"" + key + "\"";
    const size_t at = s.find(k);
    if (at == std::string::npos) return false;
    const size_t lb = s.find('[', at + k.size());
    if (lb == std::string::npos) return false;
    return std::sscanf(s.c_str() + lb, "[%d, %d, %d]", W, order, l2) == 3 && (*W == 4 || *W == 8) && *order >= 0 &&
           *order <= 2 && (*l2 == 0 || *l2 == 1);
}

void cache_store(const char* path, const std::string& key, int W, int order, int l2) {
    if (!path) return;
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    std::vector<std::pair<std::string, std::string>> entries;
    if (FILE* f = std::fopen(path, "rb")) {
        std::string s;
        char chunk[4096];
        size_t r;
        while ((r = std::fread(chunk, 1, sizeof chunk, f)) > 0) s.append(chunk, r);
        std::fclose(f);
        size_t pos = 0;
        for (;;) {
            const size_t q0 = s.find('"', pos);
            if (q0 == std::string::npos) break;
            const size_t q1 = s.find('"', q0 + 1);
            const size_t lb = s.find('[', q1);
            const size_t rb = s.find(']', lb);
            if (q1 == std::string::npos || lb == std::string::npos || rb == std::string::npos) break;
            entries.emplace_back(s.substr(q0 + 1, q1 - q0 - 1), s.substr(lb, rb - lb + 1));
            pos = rb + 1;
        }
    }
    char val[64];
    snprintf(val, sizeof val, "[%d, %d, %d]", W, order, l2);
    bool found = false;
    for (auto& e : entries)
        if (e.first == key) {
            e.second = val;
            found = true;
        }
    if (!found) entries.emplace_back(key, val);
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "wb");
    if (!f) return;
    std::fputs("{\n", f);
    for (size_t i = 0; i < entries.size(); ++i)
        std::fprintf(f, "  \"%s\": %s%s\n", entries[i].first.c_str(), entries[i].second.c_str(),
                     i + 1 < entries.size() ? "," : "");
    std::fputs("}\n", f);
    std::fclose(f);
    std::rename(tmp.c_str(), path);
}

cudaError_t time_config(icx_plan* p, float* ms) {
    cudaError_t e = capture(p);
    if (e != cudaSuccess) return e;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    e = cudaGraphLaunch(p->exec, p->cap);  // warm-up
    std::vector<float> t;
    for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
        cudaEventRecord(a, p->cap);
        e = cudaGraphLaunch(p->exec, p->cap);
        cudaEventRecord(b, p->cap);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float x = 0;
        cudaEventElapsedTime(&x, a, b);
        t.push_back(x);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return e;
    std::sort(t.begin(), t.end());
    *ms = t[t.size() / 2];
    return cudaSuccess;
}

}  // namespace

extern "C" {

long long icx_plan_error_list(void) { return g_error_list; }

icx_status icx_plan_create(const icx_list_desc* lists, size_t nlists, const icx_tuning* t, icx_plan** out) {
    using namespace icx;
    g_error_list = -1;
    if (!out || (!lists && nlists)) return ICX_EINVAL;
    *out = nullptr;
    if (nlists >= 0x80000000u) return ICX_EINVAL;
    if (t && ((t->warps_per_cta != 0 && t->warps_per_cta != 4 && t->warps_per_cta != 8) || t->order < -1 ||
              t->order > 2 || t->l2_prefetch < -1 || t->l2_prefetch > 1))
        return ICX_EINVAL;
    for (size_t i = 0; i < nlists; ++i) {
        const icx_status st = check_list(lists[i]);
        if (st != ICX_OK) {
            g_error_list = (long long)i;
            return st;
        }
    }
    icx_plan* p = new icx_plan();
    cudaGetDevice(&p->device);
    p->lists.assign(lists, lists + nlists);
    p->host_lists.resize(nlists);
    p->items_per_list.resize(nlists);
    std::vector<uint2> pages, small_pages;
    std::vector<uint32_t> mini_ids;
    for (size_t i = 0; i < nlists; ++i) {
        p->items_per_list[i] = layout_list(lists[i], (uint32_t)i, p->host_lists[i], p->npages, pages, small_pages,
                                           mini_ids);
        p->nwork += p->items_per_list[i];
        if (lists[i].codec == ICX_CODEC_BP128) p->nwork_bp += p->items_per_list[i];
        p->max_n = std::max(p->max_n, lists[i].n);
    }
    p->nlarge = pages.size();
    p->nsmall = small_pages.size();
    pages.insert(pages.end(), small_pages.begin(), small_pages.end());
    p->nmini = mini_ids.size();
    if (p->nwork > 0xFFFFFFF0ull / 2) {
        delete p;
        return ICX_EINVAL;
    }
    // one allocation for everything
    const size_t ntiles_max = (p->nwork + 3) / 4;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = (off + bytes + 255) / 256 * 256;
        return at;
    };
    const size_t o_lists = take(sizeof(ListDev) * nlists), o_work = take(sizeof(uint2) * p->nwork),
                 o_ranges = take(sizeof(ulonglong2) * p->nwork), o_pages = take(sizeof(uint2) * p->npages),
                 o_meta = take(sizeof(BlockMeta) * kBlocksPerPage * p->npages),
                 o_pmeta = take(4 * kPageMetaWords * p->npages), o_umeta = take(8 * kUnitsPerPage * p->npages),
                 o_mini = take(16 * p->nmini), o_ids = take(4 * p->nmini),
                 o_ws = take(kWsHeaderBytes + 32 * (ntiles_max + 16)),
                 o_ws2 = take(kWsHeaderBytes + 32 * (ntiles_max + 16));
    if (cudaMalloc(&p->mem, off) != cudaSuccess) {
        cudaGetLastError();
        delete p;
        return ICX_ENOSPC;
    }
    char* base = static_cast<char*>(p->mem);
    p->d.lists = reinterpret_cast<ListDev*>(base + o_lists);
    p->d.work = reinterpret_cast<uint2*>(base + o_work);
    p->d.ranges = reinterpret_cast<ulonglong2*>(base + o_ranges);
    p->d.pages = reinterpret_cast<uint2*>(base + o_pages);
    p->d.meta = reinterpret_cast<BlockMeta*>(base + o_meta);
    p->d.pmeta = reinterpret_cast<uint32_t*>(base + o_pmeta);
    p->d.umeta = reinterpret_cast<uint2*>(base + o_umeta);
    p->d.mini = reinterpret_cast<uint64_t*>(base + o_mini);
    p->d.mini_ids = reinterpret_cast<uint32_t*>(base + o_ids);
    p->d.ws = reinterpret_cast<WsHeader*>(base + o_ws);
    p->d.ws2 = reinterpret_cast<WsHeader*>(base + o_ws2);
    for (size_t j = 0; j < p->nmini; ++j) p->host_lists[mini_ids[j]].index = p->d.mini + 2 * j;
    auto fail = [&](icx_status st) {
        icx_plan_destroy(p);
        return st;
    };
    if (cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&p->cap2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&p->cap3, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->join3, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->join, cudaEventDisableTiming) != cudaSuccess)
        return fail(ICX_ECUDA);
    if (nlists &&
        cudaMemcpy(p->d.lists, p->host_lists.data(), sizeof(ListDev) * nlists, cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(ICX_ECUDA);
    if (!pages.empty() &&
        cudaMemcpy(p->d.pages, pages.data(), sizeof(uint2) * pages.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(ICX_ECUDA);
    if (cudaMemset(p->d.ws, 0, kWsHeaderBytes + 32 * (ntiles_max + 16)) != cudaSuccess ||
        cudaMemset(p->d.ws2, 0, kWsHeaderBytes + 32 * (ntiles_max + 16)) != cudaSuccess)
        return fail(ICX_ECUDA);
    if (p->nmini) {
        if (cudaMemcpy(p->d.mini_ids, mini_ids.data(), 4 * p->nmini, cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(ICX_ECUDA);
        batch_mini_index_kernel<<<(unsigned)((p->nmini + 127) / 128), 128, 0, p->cap>>>(
            p->d.lists, p->d.mini_ids, (uint32_t)p->nmini, p->d.mini, p->d.ws);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(p->cap) != cudaSuccess) return fail(ICX_ECUDA);
    }
    // tuning: explicit fields, then the cache, then timing
    int W = t ? t->warps_per_cta : 0, order = t ? t->order : -1, l2 = t ? t->l2_prefetch : -1;
    if (!t) {
        W = 0;
        order = -1;
        l2 = -1;
    }
    p->tune.cache_path = nullptr;
    if (W == 0 || order < 0 || l2 < 0) {
        const std::string key = signature(*p);
        const char* path = cache_file(t);
        int cW, cO, cL;
        if (cache_lookup(path, key, &cW, &cO, &cL)) {
            if (W == 0) W = cW;
            if (order < 0) order = cO;
            if (l2 < 0) l2 = cL;
        } else {
            float best = 3.4e38f;
            int bW = 8, bO = 0, bL = 1;
            for (int w : {4, 8}) {
                if (W && w != W) continue;
                for (int o = 0; o <= 2; ++o) {
                    if (order >= 0 && o != order) continue;
                    if (apply_order(p, o) != cudaSuccess) return fail(ICX_ECUDA);
                    for (int q = 0; q <= 1; ++q) {
                        if (l2 >= 0 && q != l2) continue;
                        p->tune.warps_per_cta = w;
                        p->tune.order = o;
                        p->tune.l2_prefetch = q;
                        float ms = 0;
                        if (time_config(p, &ms) != cudaSuccess) return fail(ICX_ECUDA);
                        if (ms < best) {
                            best = ms;
                            bW = w;
                            bO = o;
                            bL = q;
                        }
                    }
                }
            }
            W = bW;
            order = bO;
            l2 = bL;
            cache_store(path, key, W, order, l2);
        }
    }
    p->tune.warps_per_cta = W;
    p->tune.order = order;
    p->tune.l2_prefetch = l2;
    if (apply_order(p, order) != cudaSuccess) return fail(ICX_ECUDA);
    if (capture(p) != cudaSuccess) return fail(ICX_ECUDA);
    *out = p;
    return ICX_OK;
}

icx_status icx_plan_launch(icx_plan* p, icx_stream_t stream) {
    if (!p) return ICX_EINVAL;
    if (!p->nwork && !p->npages) return ICX_OK;
    return cudaGraphLaunch(p->exec, (cudaStream_t)stream) == cudaSuccess ? ICX_OK : ICX_ECUDA;
}

icx_status icx_plan_launch_per_list(icx_plan* p, icx_stream_t stream) {
    using namespace icx;
    if (!p) return ICX_EINVAL;
    if (!p->per_list_exec) {
        p->single_ws_bytes = ws_total_bytes(std::max<size_t>(p->max_n, 1));
        if (!p->single_ws) {
            if (cudaMalloc(&p->single_ws, p->single_ws_bytes) != cudaSuccess) {
                cudaGetLastError();
                return ICX_ENOSPC;
            }
            if (cudaMemset(p->single_ws, 0, p->single_ws_bytes) != cudaSuccess) return ICX_ECUDA;
        }
        WsHeader* h = static_cast<WsHeader*>(p->single_ws);
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return ICX_ECUDA;
        cudaError_t le = cudaSuccess;
        for (size_t i = 0; i < p->lists.size() && le == cudaSuccess; ++i) {
            const icx_list_desc& l = p->lists[i];
            if (!l.n) continue;
            const uint64_t* index = p->host_lists[i].index;
            if (l.codec == ICX_CODEC_BP128)
                le = launch_bp128_decode(l.delta, l.fmt, l.d_in, l.in_bytes, l.d_out, l.n, index, h,
                                         p->single_ws_bytes, p->cap);
            else
                le = launch_fastpfor_decode(l.delta, ICX_FMT_PAPER, l.d_in, l.in_bytes, l.d_out, l.n, index, h,
                                           p->single_ws_bytes, p->cap);
        }
        cudaError_t e = cudaStreamEndCapture(p->cap, &g);
        if (le != cudaSuccess) e = le;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&p->per_list_exec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) return ICX_ECUDA;
    }
    return cudaGraphLaunch(p->per_list_exec, (cudaStream_t)stream) == cudaSuccess ? ICX_OK : ICX_ECUDA;
}

icx_status icx_plan_status(icx_plan* p, icx_stream_t stream, icx_status* out) {
    using namespace icx;
    if (!p || !out) return ICX_EINVAL;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return ICX_ECUDA;
    unsigned a = 0, b = 0, c = 0;
    const size_t at = offsetof(WsHeader, status);
    if (cudaMemcpy(&a, reinterpret_cast<char*>(p->d.ws) + at, 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&c, reinterpret_cast<char*>(p->d.ws2) + at, 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        return ICX_ECUDA;
    if (!a) a = c;
    cudaMemset(reinterpret_cast<char*>(p->d.ws2) + at, 0, 4);
    if (p->single_ws &&
        cudaMemcpy(&b, static_cast<char*>(p->single_ws) + at, 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        return ICX_ECUDA;
    cudaMemset(reinterpret_cast<char*>(p->d.ws) + at, 0, 4);
    if (p->single_ws) cudaMemset(static_cast<char*>(p->single_ws) + at, 0, 4);
    if (cudaDeviceSynchronize() != cudaSuccess) return ICX_ECUDA;
    *out = (icx_status)(a ? a : b);
    return ICX_OK;
}

icx_status icx_plan_tuning(const icx_plan* p, icx_tuning* out) {
    if (!p || !out) return ICX_EINVAL;
    *out = p->tune;
    return ICX_OK;
}

void icx_plan_destroy(icx_plan* p) {
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->per_list_exec) cudaGraphExecDestroy(p->per_list_exec);
    if (p->cap) {
        cudaStreamSynchronize(p->cap);
        cudaStreamDestroy(p->cap);
    }
    if (p->cap2) cudaStreamDestroy(p->cap2);
    if (p->cap3) cudaStreamDestroy(p->cap3);
    if (p->fork) cudaEventDestroy(p->fork);
    if (p->join) cudaEventDestroy(p->join);
    if (p->join3) cudaEventDestroy(p->join3);
    if (p->mem) cudaFree(p->mem);
    if (p->single_ws) cudaFree(p->single_ws);
    delete p;
}

}  // extern "C"

// ---------------------------------------------------------------- serving

namespace {

// First-fit allocator of decode buffers inside the server's arena.
class Arena {
   public:
    void reset(size_t bytes) {
        free_.clear();
        free_[0] = bytes;
        used_ = peak_ = 0;
    }
    // offset of a block of `bytes` (a multiple of 256), or SIZE_MAX
    size_t alloc(size_t bytes) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            const size_t at = it->first, rest = it->second - bytes;
            free_.erase(it);
            if (rest) free_[at + bytes] = rest;
            used_ += bytes;
            peak_ = std::max(peak_, used_);
            return at;
        }
        return SIZE_MAX;
    }
    void release(size_t at, size_t bytes) {
        used_ -= bytes;
        auto next = free_.lower_bound(at);
        if (next != free_.end() && at + bytes == next->first) {
            bytes += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == at) {
                prev->second += bytes;
                return;
            }
        }
        free_[at] = bytes;
    }
    size_t peak() const { return peak_; }

   private:
    std::map<size_t, size_t> free_;
    size_t used_ = 0, peak_ = 0;
};

constexpr size_t kServeMaxItems = (size_t)1 << 20;  // work items of one batch
constexpr size_t kServeMaxInsts = (size_t)1 << 18;  // (request, list) pairs of one batch

size_t pad256(size_t x) { return (x + 255) / 256 * 256; }
size_t out_bytes(size_t n) { return (4 * n + 15) / 16 * 16; }

}  // namespace

struct icx_server {
    int device = 0, W = 8, blocks = 1, sms = 1;
    size_t nlists = 0, budget = 0;
    std::vector<ListDev> host_lists;
    std::vector<uint32_t> items;            // work items per list
    std::vector<uint32_t> item_base;        // first unit of each list in the pool order
    std::vector<ulonglong2> unit_ranges;    // copy range of every unit, pool order
    void* mem = nullptr;                    // lists, page records, ranges, mini index
    icx::PlanMem d;
    uint8_t* arena = nullptr;
    Arena alloc;
    struct Lane {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;   // the batch's work done
        cudaEvent_t ev0 = nullptr;  // before its copies (GPU time of the batch: ev0 -> ev)
        uint64_t t_launch = 0;      // host time the batch was issued
        icx::WsHeader* ws = nullptr;
        icx::ServeItem* d_items = nullptr;
        icx::InstDev* d_insts = nullptr;
        icx::ServeItem* h_items = nullptr;
        icx::InstDev* h_insts = nullptr;
        bool busy = false;
        std::vector<uint32_t> reqs;
        std::vector<size_t> offs;
    };
    std::vector<Lane> lanes;
    void* lane_mem = nullptr;
};

extern "C" {

void icx_server_destroy(icx_server* sv) {
    if (!sv) return;
    for (auto& l : sv->lanes) {
        if (l.st) {
            cudaStreamSynchronize(l.st);
            cudaStreamDestroy(l.st);
        }
        if (l.ev) cudaEventDestroy(l.ev);
        if (l.ev0) cudaEventDestroy(l.ev0);
        if (l.h_items) cudaFreeHost(l.h_items);
        if (l.h_insts) cudaFreeHost(l.h_insts);
    }
    if (sv->lane_mem) cudaFree(sv->lane_mem);
    if (sv->arena) cudaFree(sv->arena);
    if (sv->mem) cudaFree(sv->mem);
    delete sv;
}

icx_status icx_server_create(const icx_list_desc* pool, size_t nlists, size_t budget_bytes, int streams,
                             int warps_per_cta, icx_server** out) {
    using namespace icx;
    g_error_list = -1;
    if (!out || (!pool && nlists) || streams < 2 || streams > 16 || budget_bytes < 256 ||
        (warps_per_cta != 4 && warps_per_cta != 8) || nlists >= 0x80000000u)
        return ICX_EINVAL;
    *out = nullptr;
    for (size_t i = 0; i < nlists; ++i) {
        icx_list_desc l = pool[i];
        l.d_out = reinterpret_cast<uint32_t*>(uintptr_t(256));  // outputs come from the arena
        const icx_status st = check_list(l);
        if (st != ICX_OK) {
            g_error_list = (long long)i;
            return st;
        }
    }
    icx_server* sv = new icx_server();
    auto fail = [&](icx_status st) {
        icx_server_destroy(sv);
        return st;
    };
    cudaGetDevice(&sv->device);
    sv->nlists = nlists;
    sv->budget = budget_bytes / 256 * 256;
    sv->W = warps_per_cta;
    sv->host_lists.resize(nlists);
    sv->items.resize(nlists);
    sv->item_base.resize(nlists);
    std::vector<uint2> pages, small_pages;
    std::vector<uint32_t> mini_ids;
    size_t npages = 0, nunits = 0;
    for (size_t i = 0; i < nlists; ++i) {
        sv->items[i] = layout_list(pool[i], (uint32_t)i, sv->host_lists[i], npages, pages, small_pages, mini_ids);
        sv->host_lists[i].out = nullptr;
        sv->host_lists[i].item_base = (uint32_t)nunits;
        sv->item_base[i] = (uint32_t)nunits;
        nunits += sv->items[i];
    }
    if (nunits >= 0x80000000ull) return fail(ICX_EINVAL);
    const size_t nlarge = pages.size(), nsmall = small_pages.size();
    pages.insert(pages.end(), small_pages.begin(), small_pages.end());
    std::vector<uint2> work;
    work.reserve(nunits);
    for (size_t i = 0; i < nlists; ++i)
        for (uint32_t u = 0; u < sv->items[i]; ++u) work.push_back(make_uint2((uint32_t)i, u));
    // device memory of the pool's records
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = pad256(off + bytes);
        return at;
    };
    const size_t o_lists = take(sizeof(ListDev) * nlists), o_work = take(sizeof(uint2) * nunits),
                 o_ranges = take(sizeof(ulonglong2) * nunits), o_pages = take(sizeof(uint2) * npages),
                 o_meta = take(sizeof(BlockMeta) * kBlocksPerPage * npages), o_pmeta = take(4 * kPageMetaWords * npages),
                 o_umeta = take(8 * kUnitsPerPage * npages), o_mini = take(16 * mini_ids.size()),
                 o_ids = take(4 * mini_ids.size()), o_ws = take(kWsHeaderBytes);
    if (cudaMalloc(&sv->mem, std::max<size_t>(off, 256)) != cudaSuccess) {
        cudaGetLastError();
        return fail(ICX_ENOSPC);
    }
    char* base = static_cast<char*>(sv->mem);
    sv->d.lists = reinterpret_cast<ListDev*>(base + o_lists);
    sv->d.work = reinterpret_cast<uint2*>(base + o_work);
    sv->d.ranges = reinterpret_cast<ulonglong2*>(base + o_ranges);
    sv->d.pages = reinterpret_cast<uint2*>(base + o_pages);
    sv->d.meta = reinterpret_cast<BlockMeta*>(base + o_meta);
    sv->d.pmeta = reinterpret_cast<uint32_t*>(base + o_pmeta);
    sv->d.umeta = reinterpret_cast<uint2*>(base + o_umeta);
    sv->d.mini = reinterpret_cast<uint64_t*>(base + o_mini);
    sv->d.mini_ids = reinterpret_cast<uint32_t*>(base + o_ids);
    sv->d.ws = reinterpret_cast<WsHeader*>(base + o_ws);
    for (size_t j = 0; j < mini_ids.size(); ++j) sv->host_lists[mini_ids[j]].index = sv->d.mini + 2 * j;
    cudaStream_t st0 = nullptr;
    if (cudaStreamCreateWithFlags(&st0, cudaStreamNonBlocking) != cudaSuccess) return fail(ICX_ECUDA);
    bool ok = cudaMemset(sv->d.ws, 0, kWsHeaderBytes) == cudaSuccess;
    if (ok && nlists)
        ok = cudaMemcpy(sv->d.lists, sv->host_lists.data(), sizeof(ListDev) * nlists, cudaMemcpyHostToDevice) ==
             cudaSuccess;
    if (ok && nunits)
        ok = cudaMemcpy(sv->d.work, work.data(), sizeof(uint2) * nunits, cudaMemcpyHostToDevice) == cudaSuccess;
    if (ok && npages)
        ok = cudaMemcpy(sv->d.pages, pages.data(), sizeof(uint2) * npages, cudaMemcpyHostToDevice) == cudaSuccess;
    if (ok && !mini_ids.empty()) {
        ok = cudaMemcpy(sv->d.mini_ids, mini_ids.data(), 4 * mini_ids.size(), cudaMemcpyHostToDevice) == cudaSuccess;
        batch_mini_index_kernel<<<(unsigned)((mini_ids.size() + 127) / 128), 128, 0, st0>>>(
            sv->d.lists, sv->d.mini_ids, (uint32_t)mini_ids.size(), sv->d.mini, sv->d.ws);
    }
    // the pool's copy ranges and page records, once
    if (ok && nunits)
        batch_ranges_kernel<<<(unsigned)((nunits + 255) / 256), 256, 0, st0>>>(sv->d.lists, sv->d.work,
                                                                              (uint32_t)nunits, sv->d.ranges);
    if (ok && nlarge)
        batch_meta_kernel<<<(unsigned)nlarge, kMetaThreads, 0, st0>>>(sv->d.lists, sv->d.pages, sv->d.meta,
                                                                      sv->d.pmeta, sv->d.umeta, sv->d.ranges, sv->d.ws);
    if (ok && nsmall)
        batch_meta_small_kernel<<<(unsigned)((nsmall + kSmallWarps - 1) / kSmallWarps), kSmallWarps * 32, 0, st0>>>(
            sv->d.lists, sv->d.pages + nlarge, (uint32_t)nsmall, sv->d.meta, sv->d.pmeta, sv->d.umeta, sv->d.ranges,
            sv->d.ws);
    ok = ok && cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(st0) == cudaSuccess;
    cudaStreamDestroy(st0);
    if (!ok) return fail(ICX_ECUDA);
    unsigned status = 0;
    cudaMemcpy(&status, &sv->d.ws->status, 4, cudaMemcpyDeviceToHost);
    if (status) return fail((icx_status)status);
    sv->unit_ranges.resize(nunits);
    if (nunits && cudaMemcpy(sv->unit_ranges.data(), sv->d.ranges, sizeof(ulonglong2) * nunits,
                             cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(ICX_ECUDA);
    // decode-buffer arena and per-stream state
    if (cudaMalloc(&sv->arena, sv->budget) != cudaSuccess) {
        cudaGetLastError();
        return fail(ICX_ENOSPC);
    }
    sv->alloc.reset(sv->budget);
    const size_t ws_bytes = pad256(kWsHeaderBytes + 32 * (kServeMaxItems / 4 + 16));
    const size_t per_lane = ws_bytes + pad256(sizeof(ServeItem) * kServeMaxItems) + pad256(sizeof(InstDev) * kServeMaxInsts);
    if (cudaMalloc(&sv->lane_mem, per_lane * streams) != cudaSuccess) {
        cudaGetLastError();
        return fail(ICX_ENOSPC);
    }
    if (cudaMemset(sv->lane_mem, 0, per_lane * streams) != cudaSuccess) return fail(ICX_ECUDA);
    sv->lanes.resize(streams);
    for (int k = 0; k < streams; ++k) {
        auto& l = sv->lanes[k];
        char* b = static_cast<char*>(sv->lane_mem) + per_lane * k;
        l.ws = reinterpret_cast<WsHeader*>(b);
        l.d_items = reinterpret_cast<ServeItem*>(b + ws_bytes);
        l.d_insts = reinterpret_cast<InstDev*>(b + ws_bytes + pad256(sizeof(ServeItem) * kServeMaxItems));
        if (cudaStreamCreateWithFlags(&l.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreate(&l.ev) != cudaSuccess || cudaEventCreate(&l.ev0) != cudaSuccess ||
            cudaMallocHost(&l.h_items, sizeof(ServeItem) * kServeMaxItems) != cudaSuccess ||
            cudaMallocHost(&l.h_insts, sizeof(InstDev) * kServeMaxInsts) != cudaSuccess)
            return fail(ICX_ECUDA);
    }
    const int smem = kBatchHdr + sv->W * kWarpBytes;
    cudaError_t e = cudaFuncSetAttribute(batch_meta_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return fail(ICX_ECUDA);
    if (sv->W == 4) {
        e = cudaFuncSetAttribute(batch_decode_kernel<4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&sv->blocks, batch_decode_kernel<4, true>, 128, smem);
    } else {
        e = cudaFuncSetAttribute(batch_decode_kernel<8, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&sv->blocks, batch_decode_kernel<8, true>, 256, smem);
    }
    if (e != cudaSuccess) return fail(ICX_ECUDA);
    sv->blocks = std::max(sv->blocks, 1);
    cudaDeviceGetAttribute(&sv->sms, cudaDevAttrMultiProcessorCount, sv->device);
    *out = sv;
    return ICX_OK;
}

icx_status icx_server_run(icx_server* sv, size_t nreq, const uint64_t* arrival_ns, const uint64_t* offs,
                          const uint32_t* ids, uint64_t* latency_ns, uint32_t* results, const uint64_t* res_off,
                          icx_server_stats* stats) {
    using namespace icx;
    using clock = std::chrono::steady_clock;
    if (!sv || (nreq && (!arrival_ns || !offs || !ids || !latency_ns)) || (results && !res_off)) return ICX_EINVAL;
    // per request: buffer bytes, work items, instances, integers
    std::vector<size_t> rbytes(nreq), ritems(nreq), rints(nreq);
    for (size_t r = 0; r < nreq; ++r) {
        if (offs[r + 1] < offs[r] || (r && arrival_ns[r] < arrival_ns[r - 1])) return ICX_EINVAL;
        size_t b = 0, it = 0, n = 0;
        for (uint64_t j = offs[r]; j < offs[r + 1]; ++j) {
            if (ids[j] >= sv->nlists) return ICX_EINVAL;
            b += out_bytes(sv->host_lists[ids[j]].n);
            it += sv->items[ids[j]];
            n += sv->host_lists[ids[j]].n;
        }
        rbytes[r] = pad256(std::max<size_t>(b, 16));
        ritems[r] = it;
        rints[r] = n;
        if (rbytes[r] > sv->budget || it > kServeMaxItems || offs[r + 1] - offs[r] > kServeMaxInsts) return ICX_ENOSPC;
    }
    icx_server_stats S{};
    std::deque<uint32_t> pending;
    size_t next = 0, done = 0;
    const int W = sv->W;
    const int smem = kBatchHdr + W * kWarpBytes;
    const auto t0 = clock::now();
    auto now_ns = [&]() { return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(clock::now() - t0).count(); };
    uint64_t first_arrival = nreq ? arrival_ns[0] : 0, last_done = 0;
    icx_status err = ICX_OK;
    auto complete = [&](icx_server::Lane& l) {
        const uint64_t t = now_ns();
        float gpu_ms = 0.f;
        if (cudaEventElapsedTime(&gpu_ms, l.ev0, l.ev) == cudaSuccess) S.gpu_s += 1e-3 * gpu_ms;
        S.service_s += 1e-9 * (double)(t - l.t_launch);
        for (size_t q = 0; q < l.reqs.size(); ++q) {
            const uint32_t r = l.reqs[q];
            latency_ns[r] = t - arrival_ns[r];
            if (results) {
                size_t o = l.offs[q], e = res_off[r];
                for (uint64_t j = offs[r]; j < offs[r + 1]; ++j) {
                    const size_t n = sv->host_lists[ids[j]].n;
                    if (n && cudaMemcpy(results + e, sv->arena + o, 4 * n, cudaMemcpyDeviceToHost) != cudaSuccess)
                        err = ICX_ECUDA;
                    o += out_bytes(n);
                    e += n;
                }
            }
            sv->alloc.release(l.offs[q], rbytes[r]);
            S.ints += rints[r];
        }
        done += l.reqs.size();
        S.requests += l.reqs.size();
        l.reqs.clear();
        l.offs.clear();
        l.busy = false;
        last_done = t;
    };
    auto launch = [&](icx_server::Lane& l) -> bool {
        size_t nitems = 0, ninst = 0;
        while (!pending.empty()) {
            const uint32_t r = pending.front();
            const size_t k = offs[r + 1] - offs[r];
            if (nitems + ritems[r] > kServeMaxItems || ninst + k > kServeMaxInsts) break;
            const size_t at = sv->alloc.alloc(rbytes[r]);
            if (at == SIZE_MAX) break;  // wait for buffers to be freed
            pending.pop_front();
            l.reqs.push_back(r);
            l.offs.push_back(at);
            size_t o = at;
            for (uint64_t j = offs[r]; j < offs[r + 1]; ++j) {
                const uint32_t id = ids[j];
                l.h_insts[ninst] = InstDev{id, 0, reinterpret_cast<uint32_t*>(sv->arena + o)};
                const ulonglong2* rg = sv->unit_ranges.data() + sv->item_base[id];
                for (uint32_t u = 0; u < sv->items[id]; ++u) {
                    ServeItem& it = l.h_items[nitems++];
                    it.src = rg[u].x;
                    it.size = (uint32_t)rg[u].y;
                    it.inst = (uint32_t)ninst;
                    it.u = u;
                }
                ++ninst;
                o += out_bytes(sv->host_lists[id].n);
            }
        }
        if (l.reqs.empty()) return false;
        S.batches++;
        S.max_batch = std::max<uint64_t>(S.max_batch, l.reqs.size());
        l.t_launch = now_ns();
        for (const uint32_t r : l.reqs) S.queue_s += 1e-9 * (double)(l.t_launch - std::min(l.t_launch, arrival_ns[r]));
        cudaEventRecord(l.ev0, l.st);
        cudaMemcpyAsync(l.d_insts, l.h_insts, sizeof(InstDev) * ninst, cudaMemcpyHostToDevice, l.st);
        if (nitems) {
            cudaMemcpyAsync(l.d_items, l.h_items, sizeof(ServeItem) * nitems, cudaMemcpyHostToDevice, l.st);
            const size_t ntiles = (nitems + W - 1) / W;
            const int grid = (int)std::max<size_t>(1, std::min<size_t>((size_t)sv->blocks * sv->sms, ntiles));
            if (W == 4)
                batch_decode_kernel<4, true><<<grid, 128, smem, l.st>>>(sv->d.lists, nullptr, (uint32_t)nitems, nullptr,
                                                                       sv->d.meta, sv->d.pmeta, true, l.ws, l.d_items,
                                                                       l.d_insts);
            else
                batch_decode_kernel<8, true><<<grid, 256, smem, l.st>>>(sv->d.lists, nullptr, (uint32_t)nitems, nullptr,
                                                                       sv->d.meta, sv->d.pmeta, true, l.ws, l.d_items,
                                                                       l.d_insts);
        }
        if (cudaGetLastError() != cudaSuccess || cudaEventRecord(l.ev, l.st) != cudaSuccess) err = ICX_ECUDA;
        l.busy = true;
        return true;
    };
    while (done < nreq && err == ICX_OK) {
        const uint64_t t = now_ns();
        while (next < nreq && arrival_ns[next] <= t) pending.push_back((uint32_t)next++);
        S.max_queue = std::max<uint64_t>(S.max_queue, pending.size());
        bool progressed = false;
        for (auto& l : sv->lanes) {
            if (!l.busy) continue;
            const cudaError_t q = cudaEventQuery(l.ev);
            if (q == cudaSuccess) {
                complete(l);
                progressed = true;
            } else if (q != cudaErrorNotReady) {
                err = ICX_ECUDA;
            }
        }
        for (auto& l : sv->lanes)
            if (!l.busy && !pending.empty() && launch(l)) progressed = true;
        if (!progressed && pending.empty() && next < nreq) {
            bool any = false;
            for (auto& l : sv->lanes) any |= l.busy;
            if (!any) {
                // idle until the next arrival (spin for the last stretch)
                const uint64_t wait = arrival_ns[next] > t ? arrival_ns[next] - t : 0;
                if (wait > 200000) std::this_thread::sleep_for(std::chrono::nanoseconds(wait - 100000));
            }
        }
    }
    for (auto& l : sv->lanes)
        if (l.busy) cudaEventSynchronize(l.ev);
    cudaDeviceSynchronize();
    S.peak_bytes = sv->alloc.peak();
    S.wall_s = nreq ? (double)(last_done - std::min(first_arrival, last_done)) * 1e-9 : 0.0;
    if (stats) *stats = S;
    if (err != ICX_OK) return err;
    for (auto& l : sv->lanes) {
        unsigned status = 0;
        if (cudaMemcpy(&status, &l.ws->status, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return ICX_ECUDA;
        if (status) {
            cudaMemset(&l.ws->status, 0, 4);
            return (icx_status)status;
        }
    }
    return ICX_OK;
}

}  // extern "C"
