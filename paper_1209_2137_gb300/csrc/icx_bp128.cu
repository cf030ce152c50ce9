// SIMD-BP128 / W32 decoding (Sec. 6.2 metablocks, Sec. 4 vertical unpacking,
// Sec. 2.4 Variable Byte tail) fused with differential decoding (Sec. 3), the
// sequential index walk, and the standalone differential decoder.
//
// One CTA of 8 warps takes a tile of 8 consecutive units; unit u < M is
// metablock u (2048 integers), unit M is the Variable Byte tail.  A warp
// stages its metablock into shared memory with one bulk copy, unpacks the 16
// blocks into registers (64 integers per lane), scans them locally, and the
// CTA obtains its carry-in with one decoupled look-back per tile before the
// 128-bit stores.  Every wait is bounded (see icx_device.cuh).
#include "icx_kernels.cuh"

namespace icx {

// ----------------------------------------------------------- tail (VByte)

// Warp-parallel Variable Byte decoder (Sec. 2.4): 32 bytes per step; a
// ballot of the terminating bytes gives every byte its integer and its group
// position.  Decodes `count` (<= 127) integers starting at in[start] into
// vals[0..127] (zero-filled).  Returns false (and records ECORRUPT) on a
// truncated stream or an integer above 32 bits / 5 bytes.
__device__ bool vbyte_decode_warp(const uint8_t* __restrict__ in, size_t start, size_t in_bytes,
                                  uint32_t count, uint32_t* vals, WsHeader* h) {
    const int lane = threadIdx.x & 31;
    for (int i = lane; i < 128; i += 32) vals[i] = 0;
    __syncwarp();
    uint32_t k0 = 0, carry = 0;
    size_t pos = start;
    bool bad = false;
    while (k0 < count) {
        const size_t p = pos + lane;
        const bool have = p < in_bytes;
        const uint32_t byte = have ? in[p] : 0u;
        const unsigned have_mask = __ballot_sync(FULL, have);
        const unsigned term = __ballot_sync(FULL, have && (byte & 0x80u));
        const unsigned before = term & ((1u << lane) - 1u);
        const uint32_t idx = k0 + __popc(before);
        const uint32_t posin = before ? (uint32_t)(lane - (31 - __clz(before)) - 1) : carry + lane;
        if (have && idx < count) {
            if (posin > 4 || (posin == 4 && (byte & 0x70u)))
                bad = true;
            else
                atomicOr(&vals[idx], (byte & 0x7Fu) << (7 * posin));
        }
        k0 += __popc(term);
        carry = term ? (uint32_t)(__clz(term)) : carry + 32;
        pos += 32;
        if (have_mask != FULL) {
            if (k0 < count) bad = true;
            break;
        }
    }
    bad = __any_sync(FULL, bad);
    if (bad && lane == 0) set_error(h, ICX_ECORRUPT);
    __syncwarp();
    return !bad;
}

// ---------------------------------------------------------------- decode

constexpr int kWarps = 8;
constexpr int kMetaMax = 16 + 16 * 16 * 32;  // 8208: every width 32
constexpr int kBuf = kMetaMax + 128;         // slack for reading one row past

struct DecodeSmem {
    uint64_t bar[kWarps];
    uint4 agg[kWarps];
    uint4 pref[kWarps];
    uint32_t tile;
    uint32_t pad[3];
};

template <int FMT>
__device__ __forceinline__ uint4 unpack_block(const uint8_t* buf, uint32_t base_bytes, uint32_t bitbase,
                                              uint32_t b, int lane) {
    const uint32_t mask = width_mask(b);
    if (FMT == ICX_FMT_PAPER) {
        // Fig. 7 generalised: lane t extracts field t of each of the 4 lanes
        // (integers 4t..4t+3) from rows (t*b)/32 and the next one.
        const uint32_t bit = (uint32_t)lane * b;
        const uint4* rows = reinterpret_cast<const uint4*>(buf + base_bytes);
        const uint4 r0 = rows[bit >> 5], r1 = rows[(bit >> 5) + 1];
        const uint32_t s = bit & 31;
        return make_uint4(__funnelshift_r(r0.x, r1.x, s) & mask, __funnelshift_r(r0.y, r1.y, s) & mask,
                          __funnelshift_r(r0.z, r1.z, s) & mask, __funnelshift_r(r0.w, r1.w, s) & mask);
    } else {
        // W32: lane j's own column; fields m = 0..3 at bits bitbase + m*b.
        const uint32_t* col = reinterpret_cast<const uint32_t*>(buf + 16) + lane;
        uint32_t r[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const uint32_t bit = bitbase + (uint32_t)m * b;
            const uint32_t w = bit >> 5;
            r[m] = __funnelshift_r(col[32 * w], col[32 * (w + 1)], bit & 31) & mask;
        }
        return make_uint4(r[0], r[1], r[2], r[3]);
    }
}

template <int DELTA, int FMT>
__global__ void __launch_bounds__(kWarps * 32, 2)
    bp128_decode_kernel(const uint8_t* __restrict__ in, size_t in_bytes, uint32_t* __restrict__ out,
                        size_t n, const uint64_t* __restrict__ index, WsHeader* h) {
    extern __shared__ __align__(128) uint8_t smem_raw[];
    DecodeSmem& S = *reinterpret_cast<DecodeSmem*>(smem_raw);
    uint8_t* bufs = smem_raw + ((sizeof(DecodeSmem) + 127) / 128) * 128;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t* buf = bufs + (size_t)warp * kBuf;
    const size_t nb = n / 128;
    const uint32_t M = (uint32_t)((nb + 15) / 16);
    const uint32_t ntiles = (M + 1 + kWarps - 1) / kWarps;
    const uint32_t epoch = launch_epoch(h);
    if (lane == 0) mbar_init(&S.bar[warp], 1);
    fence_mbar_init();
    __syncthreads();
    uint32_t phase = 0;

    for (;;) {
        if (threadIdx.x == 0) S.tile = atomicAdd(&h->tile_counter, 1u);
        __syncthreads();
        const uint32_t tile = S.tile;
        if (tile >= ntiles) break;
        const uint32_t u = tile * kWarps + warp;
        uint4 v[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = make_uint4(0, 0, 0, 0);
        uint32_t K = 0;          // blocks in this unit
        bool residue = false;    // W32 metablocks arrive in residue ownership
        if (u < M) {
            K = (uint32_t)min((size_t)16, nb - 16 * (size_t)u);
            uint32_t ok = 0, size = 0;
            if (lane == 0) {
                const uint64_t off = index[u], end = index[u + 1];
                size = (uint32_t)(end - off);
                ok = off <= end && end <= in_bytes && end - off >= 16 && end - off <= kMetaMax &&
                     ((off | end) & 15) == 0;
                if (ok) {
                    fence_proxy_async();
                    mbar_expect_tx(&S.bar[warp], size);
                    bulk_load(buf, in + off, size, &S.bar[warp]);
                }
            }
            ok = __shfl_sync(FULL, ok, 0);
            size = __shfl_sync(FULL, size, 0);
            if (ok) {
                ok = mbar_wait(&S.bar[warp], phase);
                phase ^= 1;
                if (!ok && lane == 0) set_error(h, ICX_ETIMEOUT);
            } else if (lane == 0) {
                set_error(h, ICX_ECORRUPT);
            }
            if (ok) {
                const uint4 desc = *reinterpret_cast<const uint4*>(buf);
                uint32_t sum = 0, maxw = 0;
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const uint32_t b = ((uint32_t)k < K) ? (comp(desc, k >> 2) >> (8 * (k & 3))) & 255u : 0u;
                    sum += b;
                    maxw = max(maxw, b);
                }
                const uint32_t want =
                    FMT == ICX_FMT_PAPER ? 16 + 16 * sum : 16 + 128 * ((4 * sum + 31) / 32);
                if (maxw > 32 || want != size) {
                    ok = 0;
                    if (lane == 0) set_error(h, ICX_ECORRUPT);
                }
            }
            if (ok) {
                const uint4 desc = *reinterpret_cast<const uint4*>(buf);
                uint32_t base = 16, bitbase = 0;
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    if ((uint32_t)k < K) {
                        const uint32_t b = (comp(desc, k >> 2) >> (8 * (k & 3))) & 255u;
                        v[k] = unpack_block<FMT>(buf, base, bitbase, b, lane);
                        base += 16 * b;
                        bitbase += 4 * b;
                    }
                }
                residue = FMT == ICX_FMT_W32;
            }
            __syncwarp();
        } else if (u == M) {
            // Variable Byte tail: n % 128 integers after the last metablock,
            // decoded into row ownership of one block.
            const uint32_t count = (uint32_t)(n - 128 * nb);
            if (count) {
                uint32_t* vals = reinterpret_cast<uint32_t*>(buf);
                const uint64_t start = index[M];
                if (start <= in_bytes && vbyte_decode_warp(in, start, in_bytes, count, vals, h))
                    v[0] = *reinterpret_cast<const uint4*>(vals + 4 * lane);
                else if (start > in_bytes && lane == 0)
                    set_error(h, ICX_ECORRUPT);
                __syncwarp();
                K = 1;
            }
        }

        // local scan: values relative to the start of the unit, plus the
        // unit's aggregate (component c = residue c for stride 4).
        uint4 agg = make_uint4(0, 0, 0, 0);
        if (DELTA == ICX_DELTA_4 && residue) {
            uint32_t carry = 0;
#pragma unroll
            for (int k = 0; k < 16; ++k)
                if ((uint32_t)k < K) v[k] = residue_to_row(residue_scan_d4(v[k], carry, lane), lane);
            agg.x = __shfl_sync(FULL, carry, 0);
            agg.y = __shfl_sync(FULL, carry, 1);
            agg.z = __shfl_sync(FULL, carry, 2);
            agg.w = __shfl_sync(FULL, carry, 3);
        } else {
            if (residue) {
#pragma unroll
                for (int k = 0; k < 16; ++k)
                    if ((uint32_t)k < K) v[k] = residue_to_row(v[k], lane);
            }
            if (DELTA == ICX_DELTA_1) {
                uint32_t carry = 0;
#pragma unroll
                for (int k = 0; k < 16; ++k)
                    if ((uint32_t)k < K) v[k] = row_scan_d1(v[k], carry, lane);
                agg.x = carry;
            } else if (DELTA == ICX_DELTA_4) {
                uint4 carry = make_uint4(0, 0, 0, 0);
#pragma unroll
                for (int k = 0; k < 16; ++k)
                    if ((uint32_t)k < K) v[k] = row_scan_d4(v[k], carry, lane);
                agg = carry;
            }
        }

        uint4 pref = make_uint4(0, 0, 0, 0);
        if (DELTA != ICX_DELTA_NONE) {
            if (lane == 0) S.agg[warp] = agg;
            __syncthreads();
            if (warp == 0) {
                // exclusive scan of the 8 warp aggregates, then one look-back
                uint4 mine = lane < kWarps ? S.agg[lane] : make_uint4(0, 0, 0, 0);
                uint4 incl = mine;
#pragma unroll
                for (int off = 1; off < kWarps; off <<= 1) {
                    uint4 y = make_uint4(__shfl_up_sync(FULL, incl.x, off), __shfl_up_sync(FULL, incl.y, off),
                                         __shfl_up_sync(FULL, incl.z, off), __shfl_up_sync(FULL, incl.w, off));
                    if (lane >= off) incl = add4(incl, y);
                }
                const uint4 total = shfl4(incl, kWarps - 1);
                const uint4 base = DELTA == ICX_DELTA_1 ? lookback<1>(h, epoch, tile, total)
                                                        : lookback<4>(h, epoch, tile, total);
                if (lane < kWarps) S.pref[lane] = add4(base, sub4(incl, mine));
            }
            __syncthreads();
            pref = S.pref[warp];
            if (DELTA == ICX_DELTA_1) pref = make_uint4(pref.x, pref.x, pref.x, pref.x);
        }

        if (u < M) {
            uint4* o = reinterpret_cast<uint4*>(out + 2048 * (size_t)u) + lane;
#pragma unroll
            for (int k = 0; k < 16; ++k)
                if ((uint32_t)k < K) o[32 * k] = add4(v[k], pref);
        } else if (u == M && K) {
            const size_t p0 = 128 * nb + 4 * (size_t)lane;
            const uint4 r = add4(v[0], pref);
            if (p0 + 4 <= n) {
                *reinterpret_cast<uint4*>(out + p0) = r;
            } else {
                for (int c = 0; c < 4; ++c)
                    if (p0 + c < n) out[p0 + c] = comp(r, c);
            }
        }
        // keep thread 0 from overwriting S.tile before every warp read it
        if (DELTA == ICX_DELTA_NONE) __syncthreads();
    }
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

// Tile = 8 warps x 2048 integers; lanes load row-owned uint4s (coalesced),
// scan, look back, store.  In place is safe: every element is read and
// written by the same lane.
template <int DELTA>
__global__ void __launch_bounds__(kWarps * 32, 2)
    delta_decode_kernel(const uint32_t* in, uint32_t* out, size_t n, WsHeader* h) {
    __shared__ uint4 s_agg[kWarps], s_pref[kWarps];
    __shared__ uint32_t s_tile;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t ntiles = (uint32_t)((n + 2048 * kWarps - 1) / (2048 * kWarps));
    const uint32_t epoch = launch_epoch(h);
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&h->tile_counter, 1u);
        __syncthreads();
        const uint32_t tile = s_tile;
        if (tile >= ntiles) break;
        const size_t base = (size_t)(tile * kWarps + warp) * 2048;
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
        uint4 agg = make_uint4(0, 0, 0, 0);
        if (DELTA == ICX_DELTA_1) {
            uint32_t carry = 0;
#pragma unroll
            for (int k = 0; k < 16; ++k) v[k] = row_scan_d1(v[k], carry, lane);
            agg.x = carry;
        } else if (DELTA == ICX_DELTA_4) {
            uint4 carry = make_uint4(0, 0, 0, 0);
#pragma unroll
            for (int k = 0; k < 16; ++k) v[k] = row_scan_d4(v[k], carry, lane);
            agg = carry;
        }
        uint4 pref = make_uint4(0, 0, 0, 0);
        if (DELTA != ICX_DELTA_NONE) {
            if (lane == 0) s_agg[warp] = agg;
            __syncthreads();
            if (warp == 0) {
                uint4 mine = lane < kWarps ? s_agg[lane] : make_uint4(0, 0, 0, 0);
                uint4 incl = mine;
#pragma unroll
                for (int off = 1; off < kWarps; off <<= 1) {
                    uint4 y = make_uint4(__shfl_up_sync(FULL, incl.x, off), __shfl_up_sync(FULL, incl.y, off),
                                         __shfl_up_sync(FULL, incl.z, off), __shfl_up_sync(FULL, incl.w, off));
                    if (lane >= off) incl = add4(incl, y);
                }
                const uint4 total = shfl4(incl, kWarps - 1);
                const uint4 b = DELTA == ICX_DELTA_1 ? lookback<1>(h, epoch, tile, total)
                                                     : lookback<4>(h, epoch, tile, total);
                if (lane < kWarps) s_pref[lane] = add4(b, sub4(incl, mine));
            }
            __syncthreads();
            pref = s_pref[warp];
            if (DELTA == ICX_DELTA_1) pref = make_uint4(pref.x, pref.x, pref.x, pref.x);
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const size_t p = base + 128 * k + 4 * lane;
            const uint4 r = add4(v[k], pref);
            if (p + 4 <= n) {
                *reinterpret_cast<uint4*>(out + p) = r;
            } else {
                for (int c = 0; c < 4; ++c)
                    if (p + c < n) out[p + c] = comp(r, c);
            }
        }
        __syncthreads();
    }
    finish_launch(h, epoch);
}

// ------------------------------------------------------------ launchers

template <int DELTA, int FMT>
static cudaError_t launch_bp128(const uint8_t* in, size_t in_bytes, uint32_t* out, size_t n,
                                const uint64_t* index, WsHeader* h, cudaStream_t s) {
    auto kern = bp128_decode_kernel<DELTA, FMT>;
    const int smem = (int)(((sizeof(DecodeSmem) + 127) / 128) * 128 + (size_t)kWarps * kBuf);
    static int blocks_per_sm = -1;
    static int sms = 0;
    if (blocks_per_sm < 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, kWarps * 32, smem);
        if (e != cudaSuccess) return e;
        if (blocks_per_sm < 1) blocks_per_sm = 1;
    }
    const size_t M = (n / 128 + 15) / 16;
    const size_t ntiles = (M + 1 + kWarps - 1) / kWarps;
    const int grid = (int)min((size_t)blocks_per_sm * sms, ntiles);
    kern<<<grid, kWarps * 32, smem, s>>>(in, in_bytes, out, n, index, h);
    return cudaGetLastError();
}

cudaError_t launch_bp128_decode(int delta, int fmt, const uint8_t* in, size_t in_bytes, uint32_t* out,
                                size_t n, const uint64_t* index, WsHeader* h, cudaStream_t s) {
#define ICX_CASE(D, F) \
    if (delta == D && fmt == F) return launch_bp128<D, F>(in, in_bytes, out, n, index, h, s);
    ICX_CASE(ICX_DELTA_NONE, ICX_FMT_PAPER)
    ICX_CASE(ICX_DELTA_1, ICX_FMT_PAPER)
    ICX_CASE(ICX_DELTA_4, ICX_FMT_PAPER)
    ICX_CASE(ICX_DELTA_NONE, ICX_FMT_W32)
    ICX_CASE(ICX_DELTA_1, ICX_FMT_W32)
    ICX_CASE(ICX_DELTA_4, ICX_FMT_W32)
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
    const size_t ntiles = (n + 2048 * kWarps - 1) / (2048 * kWarps);
    const int grid = (int)min((size_t)blocks_per_sm * sms, ntiles);
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
