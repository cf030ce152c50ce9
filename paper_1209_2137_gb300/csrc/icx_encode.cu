// GPU encoders: differential coding (Sec. 3) and SIMD-BP128 / W32 packing
// (Sec. 6.2).  They produce the byte format of the decoders bit for bit:
// block width = largest bit length of the block's deltas, 4-lane vertical
// packing with zero padding, Variable Byte tail (Sec. 2.4).
//
// Three passes: widths and metablock sizes (one warp per metablock), an
// exclusive scan of the sizes into the index, then packing (one warp per
// metablock, fields OR-ed into shared memory, rows copied out) and the tail.
#include "icx_kernels.cuh"

namespace icx {

// ------------------------------------------------------------ delta encode

template <int S>
__global__ void delta_encode_kernel(const uint32_t* __restrict__ x, uint32_t* __restrict__ d, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const uint32_t prev = (S > 0 && i >= (size_t)S) ? x[i - S] : 0u;
        d[i] = x[i] - prev;
    }
}

cudaError_t launch_delta_encode(int delta, const uint32_t* x, uint32_t* d, size_t n, cudaStream_t s) {
    const int grid = (int)min((n + 255) / 256, (size_t)152 * 16);
    if (delta == ICX_DELTA_1)
        delta_encode_kernel<1><<<grid, 256, 0, s>>>(x, d, n);
    else if (delta == ICX_DELTA_4)
        delta_encode_kernel<4><<<grid, 256, 0, s>>>(x, d, n);
    else
        delta_encode_kernel<0><<<grid, 256, 0, s>>>(x, d, n);
    return cudaGetLastError();
}

// ------------------------------------------------------------ helpers

// Deltas of the 4 integers start + 4*lane .. +3 (row ownership).
template <int DELTA>
__device__ __forceinline__ uint4 row_deltas(const uint32_t* __restrict__ x, size_t start, int lane) {
    const uint4 v = *reinterpret_cast<const uint4*>(x + start + 4 * lane);
    if (DELTA == ICX_DELTA_NONE) return v;
    if (DELTA == ICX_DELTA_1) {
        uint32_t prev = __shfl_up_sync(FULL, v.w, 1);
        if (lane == 0) prev = start > 0 ? x[start - 1] : 0u;
        return make_uint4(v.x - prev, v.y - v.x, v.z - v.y, v.w - v.z);
    }
    uint4 prev = make_uint4(__shfl_up_sync(FULL, v.x, 1), __shfl_up_sync(FULL, v.y, 1),
                            __shfl_up_sync(FULL, v.z, 1), __shfl_up_sync(FULL, v.w, 1));
    if (lane == 0) {
        prev = start >= 4 ? *reinterpret_cast<const uint4*>(x + start - 4) : make_uint4(0, 0, 0, 0);
    }
    return sub4(v, prev);
}

template <int DELTA>
__device__ __forceinline__ uint32_t delta_at(const uint32_t* __restrict__ x, size_t p) {
    if (DELTA == ICX_DELTA_NONE) return x[p];
    const uint32_t prev = (DELTA > 0 && p >= (size_t)DELTA) ? x[p - DELTA] : 0u;
    return x[p] - prev;
}

__device__ __forceinline__ uint32_t bitlen32(uint32_t v) { return 32u - (uint32_t)__clz(v); }

// ------------------------------------------------------------ pass 1

template <int DELTA, int FMT>
__global__ void bp128_sizes_kernel(const uint32_t* __restrict__ x, size_t n, uint8_t* __restrict__ widths,
                                   uint32_t* __restrict__ sizes) {
    const int lane = threadIdx.x & 31;
    const size_t nb = n / 128, M = (nb + 15) / 16;
    const size_t warps = (size_t)gridDim.x * (blockDim.x / 32);
    for (size_t m = blockIdx.x * (size_t)(blockDim.x / 32) + (threadIdx.x >> 5); m < M; m += warps) {
        const size_t K = min((size_t)16, nb - 16 * m);
        uint32_t sum = 0;
        for (size_t k = 0; k < K; ++k) {
            const uint4 d = row_deltas<DELTA>(x, 128 * (16 * m + k), lane);
            const uint32_t orv = __reduce_or_sync(FULL, d.x | d.y | d.z | d.w);
            const uint32_t b = bitlen32(orv);  // Sec. 6.2: width of the largest delta
            if (lane == 0) widths[16 * m + k] = (uint8_t)b;
            sum += b;
        }
        if (lane == 0)
            sizes[m] = FMT == ICX_FMT_PAPER ? 16 + 16 * sum : 16 + 128 * ((4 * sum + 31) / 32);
    }
}

// ------------------------------------------------------------ pass 2

// Exclusive scan of `count` sizes into index[0..count]; one CTA of 1024.
__global__ void __launch_bounds__(1024) scan_sizes_kernel(const uint32_t* __restrict__ sizes, size_t count,
                                                          uint64_t* __restrict__ index) {
    __shared__ unsigned long long warp_tot[32];
    __shared__ unsigned long long s_carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (size_t base = 0; base < count; base += 1024) {
        const size_t i = base + threadIdx.x;
        const unsigned long long v = i < count ? sizes[i] : 0ull;
        unsigned long long incl = v;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            unsigned long long y = __shfl_up_sync(FULL, incl, off);
            if (lane >= off) incl += y;
        }
        if (lane == 31) warp_tot[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            unsigned long long t = warp_tot[lane], ti = t;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                unsigned long long y = __shfl_up_sync(FULL, ti, off);
                if (lane >= off) ti += y;
            }
            warp_tot[lane] = ti - t;  // exclusive prefix of warp totals
        }
        __syncthreads();
        const unsigned long long carry = s_carry;
        if (i < count) index[i] = carry + warp_tot[warp] + incl - v;
        __syncthreads();
        if (threadIdx.x == 1023) s_carry = carry + warp_tot[warp] + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) index[count] = s_carry;
}

// ------------------------------------------------------------ pass 3

constexpr int kEncWarps = 4;
constexpr int kColWords = 64 * 32;  // W32: up to 64 rows of 32 lane words

template <int DELTA, int FMT>
__global__ void __launch_bounds__(kEncWarps * 32) bp128_pack_kernel(const uint32_t* __restrict__ x, size_t n,
                                                                    const uint8_t* __restrict__ widths,
                                                                    const uint64_t* __restrict__ index,
                                                                    uint8_t* __restrict__ out) {
    __shared__ uint32_t sm_all[kEncWarps][FMT == ICX_FMT_PAPER ? 128 : kColWords];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* sm = sm_all[warp];
    const size_t nb = n / 128, M = (nb + 15) / 16;
    const size_t warps = (size_t)gridDim.x * kEncWarps;
    for (size_t m = blockIdx.x * (size_t)kEncWarps + warp; m < M; m += warps) {
        const size_t K = min((size_t)16, nb - 16 * m);
        uint8_t* meta = out + index[m];
        // descriptor: byte k = width of block k, unused bytes zero (R1, R4)
        if (lane < 16) meta[lane] = (size_t)lane < K ? widths[16 * m + lane] : 0;
        if (FMT == ICX_FMT_PAPER) {
            uint8_t* blk = meta + 16;
            for (size_t k = 0; k < K; ++k) {
                const uint32_t b = widths[16 * m + k];
                for (int i = lane; i < 128; i += 32) sm[i] = 0;
                __syncwarp();
                const uint4 d = row_deltas<DELTA>(x, 128 * (16 * m + k), lane);
                // lane t holds field t of the four vertical lanes (Figs. 6-7)
                const uint32_t bit = (uint32_t)lane * b, w = bit >> 5, s = bit & 31;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const uint32_t val = comp(d, c);
                    if (b) {
                        atomicOr(&sm[4 * w + c], val << s);
                        if (s + b > 32) atomicOr(&sm[4 * (w + 1) + c], val >> (32 - s));
                    }
                }
                __syncwarp();
                if ((uint32_t)lane < b) reinterpret_cast<uint4*>(blk)[lane] = reinterpret_cast<const uint4*>(sm)[lane];
                __syncwarp();
                blk += 16 * b;
            }
        } else {
            uint32_t sum = 0;
            for (size_t k = 0; k < K; ++k) sum += widths[16 * m + k];
            const uint32_t W = (4 * sum + 31) / 32;
            for (uint32_t i = lane; i < 32 * W; i += 32) sm[i] = 0;
            __syncwarp();
            const int g = lane >> 2, l = lane & 3;
            uint32_t bitbase = 0;
            for (size_t k = 0; k < K; ++k) {
                const uint32_t b = widths[16 * m + k];
                const size_t start = 128 * (16 * m + k);
#pragma unroll
                for (int mm = 0; mm < 4; ++mm) {
                    // lane j = 4g + l holds integer 16g + 4m + l of the block
                    const uint32_t val = delta_at<DELTA>(x, start + 16 * g + 4 * mm + l);
                    const uint32_t bit = bitbase + mm * b, w = bit >> 5, s = bit & 31;
                    if (b) {
                        sm[32 * w + lane] |= val << s;
                        if (s + b > 32) sm[32 * (w + 1) + lane] |= val >> (32 - s);
                    }
                }
                bitbase += 4 * b;
            }
            __syncwarp();
            uint32_t* dst = reinterpret_cast<uint32_t*>(meta + 16);
            for (uint32_t r = 0; r < W; ++r) dst[32 * r + lane] = sm[32 * r + lane];
            __syncwarp();
        }
    }
}

// ------------------------------------------------------------ tail

template <int DELTA>
__global__ void vbyte_tail_encode_kernel(const uint32_t* __restrict__ x, size_t n, const uint64_t* __restrict__ index,
                                         size_t M, uint8_t* __restrict__ out, uint64_t* __restrict__ out_bytes) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const size_t first = 128 * (n / 128);
    size_t pos = index[M];
    for (size_t i = first; i < n; ++i) {
        uint32_t v = delta_at<DELTA>(x, i);
        while (v >= 128) {  // Sec. 2.4: low group first, flag on the last byte
            out[pos++] = (uint8_t)(v & 127u);
            v >>= 7;
        }
        out[pos++] = (uint8_t)(v | 128u);
    }
    *out_bytes = pos;
}

// ------------------------------------------------------------ BP32

// Widths of the 4 blocks of 32 integers of each 128-integer metablock (Sec.
// 6.2, R20) as descriptor words (byte j = width of block j), and the size
// of each unit of 16 metablocks.  Warp per unit; lane t holds integers
// 4t..4t+3 of a metablock, so the 8 lanes 8j..8j+7 hold block j.
template <int DELTA>
__global__ void bp32_sizes_kernel(const uint32_t* __restrict__ x, size_t n, uint32_t* __restrict__ descs,
                                  uint32_t* __restrict__ sizes) {
    const int lane = threadIdx.x & 31;
    const size_t nb = n / 128, M = (nb + 15) / 16;
    const size_t warps = (size_t)gridDim.x * (blockDim.x / 32);
    for (size_t m = blockIdx.x * (size_t)(blockDim.x / 32) + (threadIdx.x >> 5); m < M; m += warps) {
        const size_t K = min((size_t)16, nb - 16 * m);
        uint32_t size = 0;
        for (size_t k = 0; k < K; ++k) {
            const uint4 d = row_deltas<DELTA>(x, 128 * (16 * m + k), lane);
            uint32_t orv = d.x | d.y | d.z | d.w;
            orv |= __shfl_xor_sync(FULL, orv, 1);
            orv |= __shfl_xor_sync(FULL, orv, 2);
            orv |= __shfl_xor_sync(FULL, orv, 4);
            const uint32_t b = bitlen32(orv);  // width of the block's largest delta
            const uint32_t desc = __shfl_sync(FULL, b, 0) | __shfl_sync(FULL, b, 8) << 8 |
                                  __shfl_sync(FULL, b, 16) << 16 | __shfl_sync(FULL, b, 24) << 24;
            if (lane == 0) descs[16 * m + k] = desc;
            size += 4 + 4 * ((desc & 255u) + ((desc >> 8) & 255u) + ((desc >> 16) & 255u) + (desc >> 24));
        }
        if (lane == 0) sizes[m] = size;
    }
}

// Writes each unit at its offset: per metablock the descriptor word, then
// the 4 blocks, integer i of block j at bits [i*b_j, (i+1)*b_j) of the
// block's words (packed in shared memory, stored with 4-byte stores).
template <int DELTA>
__global__ void __launch_bounds__(kEncWarps * 32) bp32_pack_kernel(const uint32_t* __restrict__ x, size_t n,
                                                                   const uint32_t* __restrict__ descs,
                                                                   const uint64_t* __restrict__ index,
                                                                   uint8_t* __restrict__ out) {
    __shared__ uint32_t sm_all[kEncWarps][4 * 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* sm = sm_all[warp];
    const size_t nb = n / 128, M = (nb + 15) / 16;
    const size_t warps = (size_t)gridDim.x * kEncWarps;
    const uint32_t j = (uint32_t)lane >> 3, i0 = 4 * ((uint32_t)lane & 7);
    for (size_t m = blockIdx.x * (size_t)kEncWarps + warp; m < M; m += warps) {
        const size_t K = min((size_t)16, nb - 16 * m);
        uint32_t* dst = reinterpret_cast<uint32_t*>(out + index[m]);  // 4-byte aligned: every size is
        for (size_t k = 0; k < K; ++k) {
            const uint32_t desc = descs[16 * m + k];
            const uint32_t bw[4] = {desc & 255u, (desc >> 8) & 255u, (desc >> 16) & 255u, desc >> 24};
            const uint32_t b = bw[j];
            for (int i = lane; i < 128; i += 32) sm[i] = 0;
            __syncwarp();
            const uint4 d = row_deltas<DELTA>(x, 128 * (16 * m + k), lane);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const uint32_t bit = (i0 + c) * b, w = bit >> 5, sh = bit & 31, val = comp(d, c);
                if (b) {
                    atomicOr(&sm[32 * j + w], val << sh);
                    if (sh + b > 32) atomicOr(&sm[32 * j + w + 1], val >> (32 - sh));
                }
            }
            __syncwarp();
            if (lane == 0) dst[0] = desc;
            uint32_t o = 1;
            for (int jj = 0; jj < 4; ++jj) {
                if ((uint32_t)lane < bw[jj]) dst[o + lane] = sm[32 * jj + lane];
                o += bw[jj];
            }
            __syncwarp();
            dst += o;
        }
    }
}

template <int DELTA>
static cudaError_t launch_bp32_encode_t(const uint32_t* x, size_t n, uint8_t* out, uint64_t* index,
                                        uint64_t* out_bytes, uint32_t* descs, uint32_t* sizes, cudaStream_t s) {
    const size_t nb = n / 128, M = (nb + 15) / 16;
    if (M > 0) {
        const int grid = (int)min((M + 3) / 4, (size_t)152 * 8);
        bp32_sizes_kernel<DELTA><<<grid, 128, 0, s>>>(x, n, descs, sizes);
    }
    scan_sizes_kernel<<<1, 1024, 0, s>>>(sizes, M, index);
    if (M > 0) {
        const int grid = (int)min((M + kEncWarps - 1) / kEncWarps, (size_t)152 * 8);
        bp32_pack_kernel<DELTA><<<grid, kEncWarps * 32, 0, s>>>(x, n, descs, index, out);
    }
    vbyte_tail_encode_kernel<DELTA><<<1, 32, 0, s>>>(x, n, index, M, out, out_bytes);
    return cudaGetLastError();
}

// ------------------------------------------------------------ launcher

template <int DELTA, int FMT>
static cudaError_t launch_bp128_encode_t(const uint32_t* x, size_t n, uint8_t* out, uint64_t* index,
                                         uint64_t* out_bytes, uint8_t* widths, uint32_t* sizes, cudaStream_t s) {
    const size_t nb = n / 128, M = (nb + 15) / 16;
    if (M > 0) {
        const int grid = (int)min((M + 3) / 4, (size_t)152 * 8);
        bp128_sizes_kernel<DELTA, FMT><<<grid, 128, 0, s>>>(x, n, widths, sizes);
    }
    scan_sizes_kernel<<<1, 1024, 0, s>>>(sizes, M, index);
    if (M > 0) {
        const int grid = (int)min((M + kEncWarps - 1) / kEncWarps, (size_t)152 * 8);
        bp128_pack_kernel<DELTA, FMT><<<grid, kEncWarps * 32, 0, s>>>(x, n, widths, index, out);
    }
    vbyte_tail_encode_kernel<DELTA><<<1, 32, 0, s>>>(x, n, index, M, out, out_bytes);
    return cudaGetLastError();
}

cudaError_t launch_bp128_encode(int delta, int fmt, const uint32_t* x, size_t n, uint8_t* out, uint64_t* index,
                                uint64_t* out_bytes, uint8_t* widths, uint32_t* sizes, cudaStream_t s) {
#define ICX_CASE(D, F) \
    if (delta == D && fmt == F) return launch_bp128_encode_t<D, F>(x, n, out, index, out_bytes, widths, sizes, s);
    ICX_CASE(ICX_DELTA_NONE, ICX_FMT_PAPER)
    ICX_CASE(ICX_DELTA_1, ICX_FMT_PAPER)
    ICX_CASE(ICX_DELTA_4, ICX_FMT_PAPER)
    ICX_CASE(ICX_DELTA_NONE, ICX_FMT_W32)
    ICX_CASE(ICX_DELTA_1, ICX_FMT_W32)
    ICX_CASE(ICX_DELTA_4, ICX_FMT_W32)
#undef ICX_CASE
    uint32_t* descs = reinterpret_cast<uint32_t*>(widths);  // 4-byte aligned workspace region
    if (fmt == ICX_FMT_BP32 && delta == ICX_DELTA_NONE)
        return launch_bp32_encode_t<ICX_DELTA_NONE>(x, n, out, index, out_bytes, descs, sizes, s);
    if (fmt == ICX_FMT_BP32 && delta == ICX_DELTA_1)
        return launch_bp32_encode_t<ICX_DELTA_1>(x, n, out, index, out_bytes, descs, sizes, s);
    if (fmt == ICX_FMT_BP32 && delta == ICX_DELTA_4)
        return launch_bp32_encode_t<ICX_DELTA_4>(x, n, out, index, out_bytes, descs, sizes, s);
    return cudaErrorInvalidValue;
}

}  // namespace icx
