// SIMD-FastPFOR decoding (Sec. 5, SIMD variant): page walk, page parse and
// the fused unpack + exception patch + differential decoding.
//
// The byte array of a page (per block b, maxbits and, for blocks with
// exceptions, the count c and c positions) has variable-length records, so
// finding block k's record needs the records before it.  Every decode
// therefore starts with the page parse:
//  1. fastpfor_meta_kernel -- one CTA per page finds the record starts of
//     its byte array (jump tables + an 8-record chain, see below) and writes
//     a fixed 16-byte record per block (packed offset, positions offset,
//     exception cursor, b, d, c) plus the page-relative offsets of the 32
//     exception arrays.
// With a stride (D1, D4) the SIMD layout then goes, by default, through the
// prepare / tile-scan / stream kernels of icx_fp_prep.cu.  This file holds
// the tile decoders that serve the rest (no delta, the scalar and Simple-8b
// layouts, and fastpfor.blocklane = 0):
//  2. fastpfor_decode_kernel (no delta, D1) or fastpfor_decode_pipe_kernel
//     (D4) -- units of 16 blocks exactly like the SIMD-BP128 decoder: one
//     bulk copy of the unit's packed low bits into
//     shared memory, vertical unpacking, then every exception of the unit is
//     fetched by random access into its vertically packed array (element q:
//     chunk q/128, lane q%4, field (q%128)/4) and OR-ed in as high << b
//     (Sec. 5 "patching"), then the tile epilogue (scan, look-back, stores).
#include "icx_fastpfor.cuh"
#include "icx_kernels.cuh"

namespace icx {


// ------------------------------------------------------------- page walk

// Sequential walk over the pages: each page's size follows from its header
// word, byte-array length, bitset and exception counts.
__global__ void fastpfor_index_kernel(const uint8_t* __restrict__ in, size_t in_bytes, size_t n, int fmt,
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
        if (fmt == kSimple) {  // N, W, then W Simple-8b words from a 16-byte boundary
            if (q + 8 > in_bytes) {
                bad = true;
                continue;
            }
            const size_t W = ld32(in + q + 4);
            q = pos + pad_up(q + 8 - pos, 16) + 8 * W;
            const size_t end = pos + pad_up(q - pos, 16);
            if (end > in_bytes) bad = true;
            pos = end;
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
            q = pos + pad_up(q + 4 - pos, 16) +
                (fmt == ICX_FMT_SCALAR ? 4 * (size_t)d * ((cnt + 31) / 32) : 16 * (size_t)d * ((cnt + 127) / 128));
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

template <int LAYOUT>
__device__ __forceinline__ void meta_page(const uint8_t* __restrict__ in, size_t in_bytes, size_t n,
                                          const uint64_t* __restrict__ index, BlockMeta* __restrict__ meta,
                                          uint32_t* __restrict__ pmeta, uint2* __restrict__ umeta, WsHeader* h) {
    __shared__ MetaSmem S;
    const size_t nb = n / 128, p = blockIdx.x;
    const uint32_t K = (uint32_t)min((size_t)kBlocksPerPage, nb - kBlocksPerPage * p);
    parse_page<LAYOUT>(S, in, in_bytes, index[p], index[p + 1], K, meta + kBlocksPerPage * p,
                       pmeta + kPageMetaWords * p, umeta + kUnitsPerPage * p, h);
}

__global__ void __launch_bounds__(kMetaThreads, 7)
    fastpfor_meta_kernel(const uint8_t* __restrict__ in, size_t in_bytes, size_t n, const uint64_t* __restrict__ index,
                         BlockMeta* __restrict__ meta, uint32_t* __restrict__ pmeta, uint2* __restrict__ umeta,
                         WsHeader* h) {
    allow_dependents();  // a prepare kernel launched as a dependent may be scheduled now
    meta_page<ICX_FMT_PAPER>(in, in_bytes, n, index, meta, pmeta, umeta, h);
}

// The same page parse for SimplePFOR (one Simple-8b stream of high parts).
__global__ void __launch_bounds__(kMetaThreads, 7)
    simplepfor_meta_kernel(const uint8_t* __restrict__ in, size_t in_bytes, size_t n,
                           const uint64_t* __restrict__ index, BlockMeta* __restrict__ meta,
                           uint32_t* __restrict__ pmeta, uint2* __restrict__ umeta, WsHeader* h) {
    meta_page<kSimple>(in, in_bytes, n, index, meta, pmeta, umeta, h);
}

// The same page parse for the scalar FastPFOR (exception arrays in groups
// of 32 values).
__global__ void __launch_bounds__(kMetaThreads, 7)
    fastpfor_scalar_meta_kernel(const uint8_t* __restrict__ in, size_t in_bytes, size_t n,
                                const uint64_t* __restrict__ index, BlockMeta* __restrict__ meta,
                                uint32_t* __restrict__ pmeta, uint2* __restrict__ umeta, WsHeader* h) {
    meta_page<ICX_FMT_SCALAR>(in, in_bytes, n, index, meta, pmeta, umeta, h);
}

// ---------------------------------------------------------------- decode


// The page-record word lane `lane` stages for unit uu: the 32 exception-array
// offsets, or for SimplePFOR the unit's first word, the words' offset and
// their count in lanes 0..2.
template <int LAYOUT>
__device__ __forceinline__ uint32_t page_slot(uint32_t uu, int lane) {
    if (LAYOUT != kSimple) return (uint32_t)lane;
    return lane == 0 ? uu % kUnitsPerPage : lane == 1 ? 33u : lane == 2 ? 34u : 35u;
}

template <int W, int LAYOUT>
struct FpSmem {
    TileShared t;
    uint64_t bar[W];
    BlockMeta m[W][16];
    uint32_t pg[W][32];           // the unit's page: offsets of its exception arrays
    uint8_t blk_of[W][kExScratchBytes];  // block of the unit's q-th exception, then its counts
    uint8_t s8[W][LAYOUT == kSimple ? kS8Scratch : 16];  // SimplePFOR: a window of Simple-8b words
};

// No delta and D1: a CTA of W warps takes tiles of W consecutive units of 16
// blocks (then the Variable Byte tail), one look-back per tile, exactly like
// the SIMD-BP128 decoder: per warp its unit's block records, one bulk copy of
// its packed low bits, unpack, exception patch, local scan.
template <int DELTA, int W, int LAYOUT>
__device__ __forceinline__ void fp_decode_units(const uint8_t* __restrict__ in, size_t in_bytes,
                                                uint32_t* __restrict__ out, size_t n,
                                                const uint64_t* __restrict__ index,
                                                const BlockMeta* __restrict__ meta,
                                                const uint32_t* __restrict__ pmeta, const uint2* __restrict__ umeta,
                                                WsHeader* h) {
    static_assert(DELTA != ICX_DELTA_4, "D4 has its own kernel");
    extern __shared__ __align__(128) uint8_t smem_raw[];
    FpSmem<W, LAYOUT>& S = *reinterpret_cast<FpSmem<W, LAYOUT>*>(smem_raw);
    uint8_t* bufs = smem_raw + ((sizeof(FpSmem<W, LAYOUT>) + 127) / 128) * 128;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t* buf = bufs + (size_t)warp * kFBuf;
    uint32_t* buf32 = reinterpret_cast<uint32_t*>(buf);
    uint64_t* bar = &S.bar[warp];
    BlockMeta* m = S.m[warp];
    uint8_t* blk_of = S.blk_of[warp];
    const size_t nb = n / 128;
    const uint32_t U = (uint32_t)((nb + 15) / 16);  // units of 16 blocks
    const uint32_t P = (uint32_t)((nb + kBlocksPerPage - 1) / kBlocksPerPage);
    const uint32_t ntiles = (U + 1 + W - 1) / W;  // then the Variable Byte tail
    const uint32_t epoch = launch_epoch(h);
    if (lane == 0) mbar_init(bar, 1);
    fence_mbar_init();
    __syncthreads();
    // bit 0: parity of the next copy; bit 1: a copy of this warp never
    // landed (decode nothing more)
    uint32_t phase = 0;

    // records of a unit: lane 0 its page base, page flag and packed region,
    // lanes 0..15 its block records
    struct Rec {
        uint64_t pbase;
        uint2 um;
        uint32_t bad;
        uint4 mrec;
        uint32_t arr;  // lane l: offset of exception array l + 1
    };
    auto prefetch = [&](uint32_t t, Rec& r) {
        const uint32_t uu = t * W + warp;
        if (t < ntiles && uu < U) {
            const uint32_t p = uu / kUnitsPerPage;
            const uint32_t K = (uint32_t)min((size_t)16, nb - 16 * (size_t)uu);
            if (lane == 0) {
                r.pbase = index[p];
                r.um = umeta[uu];
                r.bad = pmeta[kPageMetaWords * p + 32];
            }
            if ((uint32_t)lane < K) r.mrec = reinterpret_cast<const uint4*>(meta + 16 * (size_t)uu)[lane];
            r.arr = pmeta[kPageMetaWords * p + page_slot<LAYOUT>(uu, lane)];
        }
    };
    // publishes the records and starts the bulk copy; returns 0 = nothing to
    // wait for, 1 = copy in flight, 2 = bad page
    auto issue = [&](uint32_t t, const Rec& r) -> uint32_t {
        uint32_t res = 0;
        const uint32_t uu = t * W + warp;
        if (t < ntiles && uu < U) {
            if (lane < 16) reinterpret_cast<uint4*>(m)[lane] = r.mrec;
            S.pg[warp][lane] = r.arr;
            __syncwarp();
            if (lane == 0) {
                if (r.bad) {
                    res = 2;
                } else if (r.um.y && !(phase & 2)) {
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
        const uint32_t u = tile * W + warp;
        uint4 v[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = make_uint4(0, 0, 0, 0);
        uint32_t K = 0;
        // the page whose first unit is one grid of tiles ahead: into L2 now
        // (packed bits, byte array and exception arrays), so the copies and
        // exception gathers of its units hit L2
        const uint32_t ahead = u + gridDim.x * W;
        uint64_t pf_a = 0, pf_b = 0;
        if (lane == 0 && ahead < U && ahead % kUnitsPerPage == 0) {
            pf_a = __ldg(index + ahead / kUnitsPerPage);
            pf_b = __ldg(index + ahead / kUnitsPerPage + 1);
        }
        if (u < U) {
            K = (uint32_t)min((size_t)16, nb - 16 * (size_t)u);
            const uint32_t* pg = S.pg[warp];  // staged with the block records
            Rec r{};
            prefetch(tile, r);
            const uint64_t pbase = __shfl_sync(FULL, r.pbase, 0);
            const uint32_t st = issue(tile, r);
            bool ok = st != 2 && !(phase & 2);
            if (st == 2) {
                if (lane == 0) set_error(h, ICX_ECORRUPT);
            } else if (st == 1) {
                ok = __all_sync(FULL, mbar_wait(bar, phase & 1));
                phase ^= 1;
                if (!ok) {
                    phase |= 2;
                    if (lane == 0) set_error(h, ICX_ETIMEOUT);
                }
            }
            if (lane == 0 && pf_a < pf_b && pf_b <= in_bytes && ((pf_a | pf_b) & 15) == 0)
                prefetch_l2(in + pf_a, (uint32_t)min(pf_b - pf_a, (uint64_t)0x7FFFFFF0u));
            if (ok) fp_unit_unpack_patch<LAYOUT>(in, pbase, pg, m, K, buf, blk_of, v, h, lane, S.s8[warp]);
        } else if (u == U) {
            const uint32_t count = (uint32_t)(n - 128 * nb);
            if (count) {
                tail_unit(in, in_bytes, index[P], count, buf32, v, h, lane);
                K = 1;
            }
        }
        __syncwarp();
        const uint4 agg = unit_local_scan<DELTA>(v, K, false, lane);
        const uint4 pref = tile_prefix<DELTA, W>(S.t, agg, tile, epoch, h, warp, lane);
        if (u <= U) store_unit(out, u < U ? 2048 * (size_t)u : 128 * nb, n, v, K, pref, lane);
        if (DELTA == ICX_DELTA_NONE) __syncthreads();
    }
    if (phase & 2) mbar_wait(bar, (phase & 1) ^ 1);  // the parity of the wait that timed out
    finish_launch(h, epoch);
}

// The stride-4 (D4) decode, with the SIMD-BP128 decoder's tile pipeline: the
// unit sums are published for the tile before any local scan; the local scan
// runs while warp 0 resolves the carry and takes the next tile id; each warp
// loads the next unit's block records and starts its copy before its stores.
// Measured on the 2^26 sorted arrays it beats the kernel above by 4-5% for
// D4, but loses 6% for D1, where the register scan of stride 1 spills.
template <int W, int LAYOUT>
__device__ __forceinline__ void fp_decode_units_pipe(const uint8_t* __restrict__ in, size_t in_bytes,
                                                     uint32_t* __restrict__ out, size_t n,
                                                     const uint64_t* __restrict__ index,
                                                     const BlockMeta* __restrict__ meta,
                                                     const uint32_t* __restrict__ pmeta,
                                                     const uint2* __restrict__ umeta, WsHeader* h) {
    extern __shared__ __align__(128) uint8_t smem_raw[];
    FpSmem<W, LAYOUT>& S = *reinterpret_cast<FpSmem<W, LAYOUT>*>(smem_raw);
    uint8_t* bufs = smem_raw + ((sizeof(FpSmem<W, LAYOUT>) + 127) / 128) * 128;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t* buf = bufs + (size_t)warp * kFBuf;
    uint32_t* buf32 = reinterpret_cast<uint32_t*>(buf);
    uint64_t* bar = &S.bar[warp];
    BlockMeta* m = S.m[warp];
    uint8_t* blk_of = S.blk_of[warp];
    const size_t nb = n / 128;
    const uint32_t U = (uint32_t)((nb + 15) / 16);
    const uint32_t P = (uint32_t)((nb + kBlocksPerPage - 1) / kBlocksPerPage);
    const uint32_t ntiles = (U + 1 + W - 1) / W;
    const uint32_t epoch = launch_epoch(h);
    if (lane == 0) mbar_init(bar, 1);
    fence_mbar_init();
    if (threadIdx.x == 0) S.t.nx[0] = atomicAdd(&h->tile_counter, 1u);
    __syncthreads();
    uint32_t phase = 0, it = 0;
    bool broken = false;
    uint64_t pbase = 0;
    // unit uu: its block records and page offsets into shared memory, its
    // packed low bits into buf; returns 0 = nothing to wait for, 1 = copy in
    // flight, 2 = bad page
    auto issue = [&](uint32_t uu) -> uint32_t {
        uint32_t res = 0;
        if (uu < U) {
            const uint32_t p = uu / kUnitsPerPage;
            const uint32_t K = (uint32_t)min((size_t)16, nb - 16 * (size_t)uu);
            uint4 mrec = make_uint4(0, 0, 0, 0);
            uint2 um = make_uint2(0, 0);
            uint32_t bad = 0;
            uint64_t pb = 0;
            if ((uint32_t)lane < K) mrec = reinterpret_cast<const uint4*>(meta + 16 * (size_t)uu)[lane];
            const uint32_t arr = pmeta[kPageMetaWords * p + page_slot<LAYOUT>(uu, lane)];
            if (lane == 0) {
                pb = index[p];
                um = umeta[uu];
                bad = pmeta[kPageMetaWords * p + 32];
            }
            if ((uint32_t)lane < K) reinterpret_cast<uint4*>(m)[lane] = mrec;
            S.pg[warp][lane] = arr;
            __syncwarp();
            if (lane == 0) {
                if (bad) {
                    res = 2;
                } else if (um.y && !broken) {
                    fence_proxy_async();
                    mbar_expect_tx(bar, um.y);
                    bulk_load(buf, in + pb + um.x, um.y, bar);
                    res = 1;
                }
            }
            pbase = __shfl_sync(FULL, pb, 0);
        }
        return __shfl_sync(FULL, res, 0);
    };
    uint32_t tile = S.t.nx[0];
    uint32_t st = tile < ntiles ? issue(tile * W + warp) : 0u;

    while (tile < ntiles) {
        const uint32_t u = tile * W + warp;
        uint4 v[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = make_uint4(0, 0, 0, 0);
        uint32_t K = 0;
        const uint32_t ahead = u + gridDim.x * W;
        uint64_t pf_a = 0, pf_b = 0;
        if (lane == 0 && ahead < U && ahead % kUnitsPerPage == 0) {
            pf_a = __ldg(index + ahead / kUnitsPerPage);
            pf_b = __ldg(index + ahead / kUnitsPerPage + 1);
        }
        if (u < U) {
            K = (uint32_t)min((size_t)16, nb - 16 * (size_t)u);
            bool ok = st != 2 && !broken;
            if (st == 2) {
                if (lane == 0) set_error(h, ICX_ECORRUPT);
            } else if (ok && st == 1) {
                ok = __all_sync(FULL, mbar_wait(bar, phase));
                phase ^= 1;
                if (!ok) {
                    broken = true;
                    if (lane == 0) set_error(h, ICX_ETIMEOUT);
                }
            }
            if (lane == 0 && pf_a < pf_b && pf_b <= in_bytes && ((pf_a | pf_b) & 15) == 0)
                prefetch_l2(in + pf_a, (uint32_t)min(pf_b - pf_a, (uint64_t)0x7FFFFFF0u));
            if (ok) fp_unit_unpack_patch<LAYOUT>(in, pbase, S.pg[warp], m, K, buf, blk_of, v, h, lane, S.s8[warp]);
        } else if (u == U) {
            const uint32_t count = (uint32_t)(n - 128 * nb);
            if (count) {
                tail_unit(in, in_bytes, index[P], count, buf32, v, h, lane);
                K = 1;
            }
        }
        __syncwarp();
        // warp 0 keeps only the tile total across the local scan; the
        // exclusive unit prefixes wait in shared memory
        uint4 total = make_uint4(0, 0, 0, 0);
        const uint4 agg = unit_sum<ICX_DELTA_4>(v, false);
        if (lane == 0) S.t.agg[warp] = agg;
        __syncthreads();
        if (warp == 0) {
            uint4 mine;
            const uint4 incl = tile_agg_scan<W>(S.t, mine, lane);
            total = shfl4(incl, W - 1);
            lookback_publish<4>(h, epoch, tile, total);
            __syncwarp();
            if (lane < W) S.t.agg[lane] = sub4(incl, mine);
        }
        unit_scan_d4_smem(v, buf32, lane);
        if (warp == 0) {
            const uint4 base = lookback_resolve<4>(h, epoch, tile, total);
            if (lane < W) S.t.pref[lane] = add4(base, S.t.agg[lane]);
        }
        ++it;
        if (threadIdx.x == 0) S.t.nx[it & 1] = atomicAdd(&h->tile_counter, 1u);
        __syncthreads();
        const uint4 pref = S.t.pref[warp];
        const uint32_t next = S.t.nx[it & 1];
        __syncwarp();
        st = next < ntiles ? issue(next * W + warp) : 0u;  // lands during the stores
        if (u <= U) store_unit(out, u < U ? 2048 * (size_t)u : 128 * nb, n, v, K, pref, lane);
        tile = next;
    }
    if (broken) mbar_wait(bar, phase ^ 1);  // the parity of the wait that timed out
    finish_launch(h, epoch);
}

// The kernels: SIMD-FastPFOR, and the scalar FastPFOR under its own names.
#define ICX_FP_KERNEL_ARGS                                                                                    \
    const uint8_t *__restrict__ in, size_t in_bytes, uint32_t *__restrict__ out, size_t n,                    \
        const uint64_t *__restrict__ index, const BlockMeta *__restrict__ meta, const uint32_t *__restrict__ pmeta, \
        const uint2 *__restrict__ umeta, WsHeader *h
template <int DELTA, int W>
__global__ void __launch_bounds__(W * 32, 16 / W) fastpfor_decode_kernel(ICX_FP_KERNEL_ARGS) {
    fp_decode_units<DELTA, W, ICX_FMT_PAPER>(in, in_bytes, out, n, index, meta, pmeta, umeta, h);
}
template <int W>
__global__ void __launch_bounds__(W * 32, 16 / W) fastpfor_decode_pipe_kernel(ICX_FP_KERNEL_ARGS) {
    fp_decode_units_pipe<W, ICX_FMT_PAPER>(in, in_bytes, out, n, index, meta, pmeta, umeta, h);
}
template <int DELTA, int W>
__global__ void __launch_bounds__(W * 32, 16 / W) fastpfor_scalar_decode_kernel(ICX_FP_KERNEL_ARGS) {
    fp_decode_units<DELTA, W, ICX_FMT_SCALAR>(in, in_bytes, out, n, index, meta, pmeta, umeta, h);
}
template <int W>
__global__ void __launch_bounds__(W * 32, 16 / W) fastpfor_scalar_decode_pipe_kernel(ICX_FP_KERNEL_ARGS) {
    fp_decode_units_pipe<W, ICX_FMT_SCALAR>(in, in_bytes, out, n, index, meta, pmeta, umeta, h);
}
template <int DELTA, int W>
__global__ void __launch_bounds__(W * 32, 16 / W) simplepfor_decode_kernel(ICX_FP_KERNEL_ARGS) {
    fp_decode_units<DELTA, W, kSimple>(in, in_bytes, out, n, index, meta, pmeta, umeta, h);
}
template <int W>
__global__ void __launch_bounds__(W * 32, 16 / W) simplepfor_decode_pipe_kernel(ICX_FP_KERNEL_ARGS) {
    fp_decode_units_pipe<W, kSimple>(in, in_bytes, out, n, index, meta, pmeta, umeta, h);
}
#undef ICX_FP_KERNEL_ARGS

// ------------------------------------------------------------ launchers

// The page parse of the SIMD layout alone (one CTA per page).
cudaError_t launch_fastpfor_meta(const uint8_t* in, size_t in_bytes, size_t n, const uint64_t* index, BlockMeta* meta,
                                 uint32_t* pmeta, uint2* umeta, WsHeader* h, cudaStream_t s) {
    static bool carveout = false;
    if (!carveout) {
        // the page parse wants 7 CTAs of 30 KB per SM
        const cudaError_t e = cudaFuncSetAttribute(fastpfor_meta_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                                   cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        carveout = true;
    }
    const size_t P = (n / 128 + kBlocksPerPage - 1) / kBlocksPerPage;
    if (P) fastpfor_meta_kernel<<<(unsigned)P, kMetaThreads, 0, s>>>(in, in_bytes, n, index, meta, pmeta, umeta, h);
    return cudaGetLastError();
}

cudaError_t launch_fastpfor_index(const uint8_t* in, size_t in_bytes, size_t n, int fmt, uint64_t* index,
                                  WsHeader* h, cudaStream_t s) {
    fastpfor_index_kernel<<<1, 32, 0, s>>>(in, in_bytes, n, fmt, index, h);
    return cudaGetLastError();
}

// Decoder of the SIMD layout with deltas: 0 = the tile decoder with a
// chained look-back, 1 = the block-per-lane decoder (block sums as tasks of
// the same kernel), 2 (default) = the prepare and stream kernels.
static int g_fp_blocklane = 2;

void set_fastpfor_blocklane(int v) { g_fp_blocklane = v < 0 || v > 2 ? 2 : v; }

template <int DELTA, int W, int LAYOUT>
static cudaError_t launch_fp(const uint8_t* in, size_t in_bytes, uint32_t* out, size_t n, const uint64_t* index,
                             WsHeader* h, size_t ws_bytes, cudaStream_t s) {
    void (*kern)(const uint8_t*, size_t, uint32_t*, size_t, const uint64_t*, const BlockMeta*, const uint32_t*,
                 const uint2*, WsHeader*);
    auto meta_kern = LAYOUT == ICX_FMT_SCALAR ? fastpfor_scalar_meta_kernel
                     : LAYOUT == kSimple      ? simplepfor_meta_kernel
                                              : fastpfor_meta_kernel;
    if constexpr (DELTA == ICX_DELTA_4 && LAYOUT == kSimple)
        kern = simplepfor_decode_pipe_kernel<W>;
    else if constexpr (LAYOUT == kSimple)
        kern = simplepfor_decode_kernel<DELTA, W>;
    else if constexpr (DELTA == ICX_DELTA_4 && LAYOUT == ICX_FMT_SCALAR)
        kern = fastpfor_scalar_decode_pipe_kernel<W>;
    else if constexpr (DELTA == ICX_DELTA_4)
        kern = fastpfor_decode_pipe_kernel<W>;
    else if constexpr (LAYOUT == ICX_FMT_SCALAR)
        kern = fastpfor_scalar_decode_kernel<DELTA, W>;
    else
        kern = fastpfor_decode_kernel<DELTA, W>;
    const int smem = (int)(((sizeof(FpSmem<W, LAYOUT>) + 127) / 128) * 128 + (size_t)W * kFBuf);
    static int blocks_per_sm = -1;
    static int sms = 0;
    if (blocks_per_sm < 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        // the page parse wants 7 CTAs of 30 KB per SM
        e = cudaFuncSetAttribute(meta_kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, W * 32, smem);
        if (e != cudaSuccess) return e;
        if (blocks_per_sm < 1) blocks_per_sm = 1;
    }
    char* ws = reinterpret_cast<char*>(h);
    const size_t plain = ws_plain_base(ws_bytes);
    BlockMeta* meta = reinterpret_cast<BlockMeta*>(ws + plain);
    uint32_t* pmeta = reinterpret_cast<uint32_t*>(ws + plain + ws_pagemeta_rel(n));
    uint2* umeta = reinterpret_cast<uint2*>(ws + plain + ws_unitmeta_rel(n));
    const size_t nb = n / 128, P = (nb + kBlocksPerPage - 1) / kBlocksPerPage, U = (nb + 15) / 16;
    if (LAYOUT == ICX_FMT_PAPER && DELTA != ICX_DELTA_NONE && g_fp_blocklane == 2)
        return launch_fastpfor_two_kernel(DELTA, in, in_bytes, out, n, index, meta, pmeta, umeta, h, ws_bytes, s);
    if (P > 0) {
        meta_kern<<<(unsigned)P, kMetaThreads, 0, s>>>(in, in_bytes, n, index, meta, pmeta, umeta, h);
    }
    if (LAYOUT == ICX_FMT_PAPER && DELTA != ICX_DELTA_NONE && g_fp_blocklane == 1) {
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        return launch_fastpfor_blocklane(DELTA, in, in_bytes, out, n, index, meta, pmeta, umeta, h, ws_bytes, s);
    }
    const size_t ntiles = (U + 1 + W - 1) / W;
    const int grid = (int)min((size_t)blocks_per_sm * sms, ntiles);
    kern<<<grid, W * 32, smem, s>>>(in, in_bytes, out, n, index, meta, pmeta, umeta, h);
    return cudaGetLastError();
}

static int g_fp_warps = 0;  // warps per CTA of the SIMD-FastPFOR decoder (0 = default)

void set_fastpfor_warps(int w) { g_fp_warps = (w == 4 || w == 8) ? w : 0; }

template <int DELTA, int LAYOUT>
static cudaError_t launch_fp_w(const uint8_t* in, size_t in_bytes, uint32_t* out, size_t n, const uint64_t* index,
                               WsHeader* h, size_t ws_bytes, cudaStream_t s) {
    // measured on the 2^26 sorted arrays: 4 warps per CTA for the pipelined
    // SIMD-FastPFOR stride-4 kernel (0.1816 vs 0.1820 ms), 8 for the others
    // (SIMD stride 1: 0.178 vs 0.181 ms; scalar FastPFOR and SimplePFOR
    // stride 4: 0.183 vs 0.198 and 0.197 vs 0.207 ms)
    const int w = g_fp_warps ? g_fp_warps : (DELTA == ICX_DELTA_4 && LAYOUT == ICX_FMT_PAPER ? 4 : 8);
    if (w == 4) return launch_fp<DELTA, 4, LAYOUT>(in, in_bytes, out, n, index, h, ws_bytes, s);
    return launch_fp<DELTA, 8, LAYOUT>(in, in_bytes, out, n, index, h, ws_bytes, s);
}

cudaError_t launch_fastpfor_decode(int delta, int fmt, const uint8_t* in, size_t in_bytes, uint32_t* out, size_t n,
                                   const uint64_t* index, WsHeader* h, size_t ws_bytes, cudaStream_t s) {
#define ICX_CASE(D, L) \
    if (delta == D && fmt == L) return launch_fp_w<D, L>(in, in_bytes, out, n, index, h, ws_bytes, s);
    ICX_CASE(ICX_DELTA_NONE, ICX_FMT_PAPER)
    ICX_CASE(ICX_DELTA_1, ICX_FMT_PAPER)
    ICX_CASE(ICX_DELTA_4, ICX_FMT_PAPER)
    ICX_CASE(ICX_DELTA_NONE, ICX_FMT_SCALAR)
    ICX_CASE(ICX_DELTA_1, ICX_FMT_SCALAR)
    ICX_CASE(ICX_DELTA_4, ICX_FMT_SCALAR)
    ICX_CASE(ICX_DELTA_NONE, kSimple)
    ICX_CASE(ICX_DELTA_1, kSimple)
    ICX_CASE(ICX_DELTA_4, kSimple)
#undef ICX_CASE
    return cudaErrorInvalidValue;
}

}  // namespace icx
