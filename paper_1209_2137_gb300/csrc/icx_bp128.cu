// SIMD-BP128 / W32 decoding (Sec. 6.2 metablocks, Sec. 4 vertical unpacking,
// Sec. 2.4 Variable Byte tail) fused with differential decoding (Sec. 3), the
// sequential index walk, and the standalone differential decoder.
//
// A CTA of W warps takes a tile of W consecutive units; unit u < M is
// metablock u (2048 integers), unit M is the Variable Byte tail.  A warp
// stages its metablock into shared memory with one bulk copy, unpacks the 16
// blocks into registers (64 integers per lane), scans them locally, and the
// CTA obtains its carry-in with one decoupled look-back per tile before the
// 128-bit stores.  Every wait is bounded (see icx_device.cuh).
#include "icx_bp128.cuh"
#include "icx_kernels.cuh"

namespace icx {

// ---------------------------------------------------------------- decode

constexpr int kPipeHdr = 1024;  // TileShared, then two mbarriers per warp
static_assert(sizeof(TileShared) + 16 * kMaxWarps <= kPipeHdr, "tile header");

// A CTA of W warps takes tiles of W consecutive units (unit u < M is
// metablock u, unit M the Variable Byte tail); tile ids come from the
// launch's counter.  Per tile:
//   1. every warp waits for its metablock (one bulk copy into its shared
//      buffer), unpacks it into registers (64 integers per lane) and sums it;
//   2. warp 0 publishes the tile aggregate at once, so that the look-backs of
//      later tiles never wait for this tile's local scans;
//   3. every warp scans its unit locally while warp 0 resolves the tile's
//      carry-in (decoupled look-back) and takes the next tile id;
//   4. every warp starts the bulk copy of its next metablock, then adds its
//      carry and stores (the copy lands during the stores).
template <int DELTA, int FMT, int W>
__global__ void __launch_bounds__(W * 32, 16 / W)
    bp128_decode_kernel(const uint8_t* __restrict__ in, size_t in_bytes, uint32_t* __restrict__ out,
                        size_t n, const uint64_t* __restrict__ index, bool l2_ahead, WsHeader* h) {
    constexpr int NL = DELTA == ICX_DELTA_4 ? 4 : 1;
    extern __shared__ __align__(128) uint8_t smem_raw[];
    TileShared& S = *reinterpret_cast<TileShared*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + kPipeHdr) - 2 * kMaxWarps + 2 * warp;
    uint8_t* buf = smem_raw + kPipeHdr + (size_t)warp * kBuf;
    const size_t nb = n / 128;
    const uint32_t M = (uint32_t)((nb + 15) / 16);
    const uint32_t ntiles = (M + 1 + W - 1) / W;
    const uint32_t epoch = launch_epoch(h);
    if (lane == 0) mbar_init(bar, 1);
    fence_mbar_init();
    if (threadIdx.x == 0) S.nx[0] = atomicAdd(&h->tile_counter, 1u);
    __syncthreads();
    uint32_t phase = 0, it = 0;
    uint32_t shift = 0;   // BP32: the unit's offset inside its 16-byte aligned copy
    bool broken = false;  // a copy of this warp never landed: decode nothing more
    // starts the bulk copy of metablock uu; returns its size, ~0u for an
    // invalid index entry, 0 if there is nothing to copy
    auto issue = [&](uint32_t uu) -> uint32_t {
        uint32_t size = 0;
        if (FMT == ICX_FMT_BP32) {
            // BP32 units are 4-byte aligned: the 16-byte aligned interior
            // [off & ~15, end & ~15) by bulk copy (possibly empty: the barrier
            // is then armed with no bytes), the last end % 16 bytes by plain
            // loads; nothing past `end` is read
            uint64_t off = 0, end = 0;
            if (uu < M && !broken && lane == 0) {
                off = index[uu];
                end = index[uu + 1];
                const bool ok = off <= end && end <= in_bytes && end - off >= 4 &&
                                end - (off & ~15ull) <= (uint64_t)(kBp32UnitMax + 15) && ((off | end) & 3) == 0;
                size = ok ? (uint32_t)(end - off) : ~0u;
                if (ok) {
                    const uint64_t a0 = off & ~15ull, a1 = end & ~15ull;
                    fence_proxy_async();
                    mbar_expect_tx(bar, a1 > a0 ? (uint32_t)(a1 - a0) : 0u);
                    if (a1 > a0) bulk_load(buf, in + a0, (uint32_t)(a1 - a0), bar);
                }
            }
            size = __shfl_sync(FULL, size, 0);
            off = __shfl_sync(FULL, off, 0);
            end = __shfl_sync(FULL, end, 0);
            if (size != 0 && size != ~0u) {
                const uint64_t a0 = off & ~15ull, a1 = end & ~15ull;
                if ((uint64_t)lane < end - a1) buf[a1 - a0 + lane] = __ldg(in + a1 + lane);
                shift = (uint32_t)(off - a0);
            }
            return size;
        }
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
        uint32_t K = 0;        // blocks in this unit
        bool residue = false;  // W32 metablocks arrive in residue ownership
        // the metablock one grid of tiles ahead: some CTA takes it about one
        // tile-time from now; bring it into L2 so that its copy is short
        const uint32_t ahead = u + gridDim.x * W;
        uint64_t pf_off = 0, pf_end = 0;
        if (l2_ahead && lane == 0 && ahead < M) {
            pf_off = __ldg(index + ahead);
            pf_end = __ldg(index + ahead + 1);
        }
        if (u < M) {
            K = (uint32_t)min((size_t)16, nb - 16 * (size_t)u);
            bool ok = size != ~0u && !broken;
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
            if (lane == 0 && pf_off < pf_end && pf_end <= in_bytes && pf_end - pf_off <= kMetaMax &&
                ((pf_off | pf_end) & 15) == 0)
                prefetch_l2(in + pf_off, (uint32_t)(pf_end - pf_off));
            if (ok) {
                __syncwarp();  // BP32: the plainly loaded last bytes
                if (FMT == ICX_FMT_BP32)
                    ok = bp32_unpack_unit(buf + shift, size, K, v, h, lane);
                else
                    ok = bp128_unpack_unit<FMT>(buf, size, K, v, h, lane);
                residue = ok && FMT == ICX_FMT_W32;
            }
            __syncwarp();
        } else if (u == M) {
            // Variable Byte tail: n % 128 integers after the last metablock,
            // decoded into row ownership of one block.
            const uint32_t count = (uint32_t)(n - 128 * nb);
            if (count) {
                tail_unit(in, in_bytes, index[M], count, reinterpret_cast<uint32_t*>(buf), v, h, lane);
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
        if (DELTA == ICX_DELTA_4 && FMT != ICX_FMT_W32)  // row ownership
            unit_scan_d4_smem(v, reinterpret_cast<uint32_t*>(buf), lane);
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
        __syncwarp();
        size = next < ntiles ? issue(next * W + warp) : 0u;  // lands during the stores
        if (u <= M) store_unit(out, u < M ? 2048 * (size_t)u : 128 * nb, n, v, K, pref, lane);
        tile = next;
    }
    // a copy that never landed must not outlive the CTA's shared memory
    if (broken) mbar_wait(bar, phase ^ 1);  // the parity of the wait that timed out
    finish_launch(h, epoch);
}

// -------------------------------------------------------------- index walk

// Sequential walk over the metablocks (each size comes from its descriptor).
__global__ void bp128_index_kernel(const uint8_t* __restrict__ in, size_t in_bytes, size_t n, int fmt,
                                   uint64_t* __restrict__ index, WsHeader* h) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const size_t nb = n / 128, M = (nb + 15) / 16;
    size_t pos = 0;
    bool bad = false;
    for (size_t m = 0; m < M; ++m) {
        index[m] = pos;
        if (bad) continue;
        const size_t K = min((size_t)16, nb - 16 * m);
        if (fmt == ICX_FMT_BP32) {  // K metablocks of 128 integers, each 4 + 4 * (sum of 4 widths) bytes
            for (size_t k = 0; k < K && !bad; ++k) {
                if (pos + 4 > in_bytes) {
                    bad = true;
                    break;
                }
                size_t size = 4;
                for (int j = 0; j < 4; ++j) {
                    const uint32_t b = in[pos + j];
                    if (b > 32) bad = true;
                    size += 4 * (size_t)b;
                }
                if (pos + size > in_bytes) bad = true;
                pos += size;
            }
            continue;
        }
        if (pos + 16 > in_bytes) {
            bad = true;
            continue;
        }
        const uint4 d = __ldg(reinterpret_cast<const uint4*>(in + pos));
        uint32_t sum = 0;
        for (size_t k = 0; k < K; ++k) {
            const uint32_t b = (comp(d, (int)(k >> 2)) >> (8 * (k & 3))) & 255u;
            if (b > 32) bad = true;
            sum += b;
        }
        const size_t size = fmt == ICX_FMT_PAPER ? 16 + 16 * (size_t)sum : 16 + 128 * (size_t)((4 * sum + 31) / 32);
        if (pos + size > in_bytes) bad = true;
        pos += size;
    }
    index[M] = bad ? in_bytes : pos;
    if (bad) set_error(h, ICX_ECORRUPT);
}

// ------------------------------------------------------ standalone delta

// CTA tiles of kWarps x 2048 integers: coalesced 128-bit loads in row
// ownership, local scan, one look-back per tile, stores.  In place is safe:
// every element is read and written by the same lane.
template <int DELTA>
__global__ void __launch_bounds__(kWarps * 32, 2)
    delta_decode_kernel(const uint32_t* in, uint32_t* out, size_t n, WsHeader* h) {
    __shared__ TileShared S;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t ntiles = (uint32_t)((n + 2048 * kWarps - 1) / (2048 * kWarps));
    const uint32_t epoch = launch_epoch(h);
    for (;;) {
        const uint32_t tile = next_tile(S, h);
        if (tile >= ntiles) break;
        const size_t base = ((size_t)tile * kWarps + warp) * 2048;
        uint4 v[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const size_t p = base + 128 * k + 4 * lane;
            if (p + 4 <= n) {
                v[k] = *reinterpret_cast<const uint4*>(in + p);
            } else {
                v[k] = make_uint4(p < n ? in[p] : 0u, p + 1 < n ? in[p + 1] : 0u, p + 2 < n ? in[p + 2] : 0u,
                                  p + 3 < n ? in[p + 3] : 0u);
            }
        }
        const uint4 agg = unit_local_scan<DELTA>(v, 16, false, lane);
        const uint4 pref = tile_prefix<DELTA>(S, agg, tile, epoch, h, warp, lane);
        store_unit(out, base, n, v, 16, pref, lane);
        __syncthreads();
    }
    finish_launch(h, epoch);
}

// ------------------------------------------------------------ launchers

static int g_bp128_warps = 0;          // warps per CTA of the SIMD-BP128 decoder (0 = per-stride default)
static bool g_bp128_l2_ahead = true;  // L2 prefetch one grid of tiles ahead

template <int DELTA, int FMT, int W>
static cudaError_t launch_bp128(const uint8_t* in, size_t in_bytes, uint32_t* out, size_t n,
                                const uint64_t* index, WsHeader* h, cudaStream_t s) {
    auto kern = bp128_decode_kernel<DELTA, FMT, W>;
    const int smem = (int)(kPipeHdr + (size_t)W * kBuf);
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
    kern<<<grid, W * 32, smem, s>>>(in, in_bytes, out, n, index, g_bp128_l2_ahead, h);
    return cudaGetLastError();
}

void set_bp128_warps(int w) { g_bp128_warps = (w == 4 || w == 8 || w == 16) ? w : 0; }


void set_bp128_prefetch(int on) { g_bp128_l2_ahead = on != 0; }

template <int DELTA, int FMT>
static cudaError_t launch_bp128_w(const uint8_t* in, size_t in_bytes, uint32_t* out, size_t n,
                                  const uint64_t* index, WsHeader* h, cudaStream_t s) {
    // measured on the 2^26 sorted workloads: 4 warps per CTA for the paper
    // layout (and BP32, also row ownership), 8 for W32
    const int w = g_bp128_warps ? g_bp128_warps : (FMT == ICX_FMT_W32 ? 8 : 4);
    if (w == 4) return launch_bp128<DELTA, FMT, 4>(in, in_bytes, out, n, index, h, s);
    if (w == 16) return launch_bp128<DELTA, FMT, 16>(in, in_bytes, out, n, index, h, s);
    return launch_bp128<DELTA, FMT, 8>(in, in_bytes, out, n, index, h, s);
}

static bool g_bp128_blocklane = true;  // two-phase block-per-lane decoder for the paper layout with deltas

void set_bp128_blocklane(int on) { g_bp128_blocklane = on != 0; }

cudaError_t launch_bp128_decode(int delta, int fmt, const uint8_t* in, size_t in_bytes, uint32_t* out,
                                size_t n, const uint64_t* index, WsHeader* h, size_t ws_bytes, cudaStream_t s) {
    if (g_bp128_blocklane && fmt == ICX_FMT_PAPER && delta != ICX_DELTA_NONE)
        return launch_bp128_blocklane(delta, in, in_bytes, out, n, index, h, ws_bytes, s);
    return launch_bp128_decode_lookback(delta, fmt, in, in_bytes, out, n, index, h, s);
}

// The single-pass decoder with a decoupled look-back; it uses only the
// workspace header and look-back states.
cudaError_t launch_bp128_decode_lookback(int delta, int fmt, const uint8_t* in, size_t in_bytes, uint32_t* out,
                                         size_t n, const uint64_t* index, WsHeader* h, cudaStream_t s) {
#define ICX_CASE(D, F) \
    if (delta == D && fmt == F) return launch_bp128_w<D, F>(in, in_bytes, out, n, index, h, s);
    ICX_CASE(ICX_DELTA_NONE, ICX_FMT_PAPER)
    ICX_CASE(ICX_DELTA_1, ICX_FMT_PAPER)
    ICX_CASE(ICX_DELTA_4, ICX_FMT_PAPER)
    ICX_CASE(ICX_DELTA_NONE, ICX_FMT_W32)
    ICX_CASE(ICX_DELTA_1, ICX_FMT_W32)
    ICX_CASE(ICX_DELTA_4, ICX_FMT_W32)
    ICX_CASE(ICX_DELTA_NONE, ICX_FMT_BP32)
    ICX_CASE(ICX_DELTA_1, ICX_FMT_BP32)
    ICX_CASE(ICX_DELTA_4, ICX_FMT_BP32)
#undef ICX_CASE
    return cudaErrorInvalidValue;
}

cudaError_t launch_bp128_index(const uint8_t* in, size_t in_bytes, size_t n, int fmt, uint64_t* index,
                               WsHeader* h, cudaStream_t s) {
    bp128_index_kernel<<<1, 32, 0, s>>>(in, in_bytes, n, fmt, index, h);
    return cudaGetLastError();
}

template <int DELTA>
static cudaError_t launch_delta(const uint32_t* in, uint32_t* out, size_t n, WsHeader* h, cudaStream_t s) {
    auto kern = delta_decode_kernel<DELTA>;
    static int blocks_per_sm = -1;
    static int sms = 0;
    if (blocks_per_sm < 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, kWarps * 32, 0);
        if (e != cudaSuccess) return e;
        if (blocks_per_sm < 1) blocks_per_sm = 1;
    }
    const size_t ctas = (n + 2048 * kWarps - 1) / (2048 * kWarps);
    const int grid = (int)min((size_t)blocks_per_sm * sms, ctas);
    kern<<<grid, kWarps * 32, 0, s>>>(in, out, n, h);
    return cudaGetLastError();
}

cudaError_t launch_delta_decode(int delta, const uint32_t* in, uint32_t* out, size_t n, WsHeader* h,
                                cudaStream_t s) {
    if (delta == ICX_DELTA_1) return launch_delta<ICX_DELTA_1>(in, out, n, h, s);
    if (delta == ICX_DELTA_4) return launch_delta<ICX_DELTA_4>(in, out, n, h, s);
    return launch_delta<ICX_DELTA_NONE>(in, out, n, h, s);
}

}  // namespace icx
