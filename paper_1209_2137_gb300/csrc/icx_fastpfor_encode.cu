// SIMD-FastPFOR encoding on the GPU (Sec. 5), byte for byte the format the
// decoder reads (see include/icx.h):
//  1. per block (one warp): deltas, the bit-width histogram as counts
//     c_b = #{v : bitlen(v) > b}, and the b minimising 128*b + c_b*(8 +
//     maxbits - b) (ties to the larger b);
//  2. per page (one warp): record offsets, exception cursors, exception
//     array layout and the page size;
//  3. exclusive scan of page sizes -> index;
//  4. per block (one warp): packed low bits, the byte-array record, and the
//     exceptions' high parts into a scratch array per page and width;
//  5. per page (one warp): header word, length word, padding, bitset,
//     counts, and the exception arrays packed at width d;
//  6. the Variable Byte tail.
#include "icx_kernels.cuh"

namespace icx {

constexpr uint32_t kPageBlocks = 512;
constexpr uint32_t kPageExc = 65536;  // scratch slots per page (>= exceptions)

struct EncMeta {
    uint32_t packed_off;  // page-relative
    uint32_t rec_off;     // offset inside the byte array
    uint32_t cursor;      // first exception's index in array d
    uint8_t b, mb, c, d;
};

struct PageEnc {
    uint32_t len_at, L, bitset, size;
    uint32_t N, W;  // SimplePFOR: exception high parts and Simple-8b words of the page
    uint32_t arr_off[32];  // page-relative offset of array d (d = index + 1)
    uint32_t cnt[32];
    uint32_t arr_base[32];  // first scratch slot of array d
};

__host__ __device__ inline size_t fe_pad(size_t x, size_t a) { return (x + a - 1) / a * a; }

// encode workspace layout
struct FeLayout {
    size_t em, meta, pages, sizes, scratch, total;
    __host__ __device__ FeLayout(size_t n) {
        const size_t nb = n / 128, P = (nb + kPageBlocks - 1) / kPageBlocks;
        em = kWsHeaderBytes;
        meta = fe_pad(em + 4 * (nb + 1), 256);
        pages = fe_pad(meta + sizeof(EncMeta) * (nb + 1), 256);
        sizes = fe_pad(pages + sizeof(PageEnc) * (P + 1), 256);
        scratch = fe_pad(sizes + 4 * (P + 2), 256);
        total = fe_pad(scratch + 4 * (size_t)kPageExc * P, 256);
    }
};

size_t fastpfor_encode_workspace_bytes(size_t n) { return FeLayout(n).total; }

template <int DELTA>
__device__ __forceinline__ uint4 fe_row_deltas(const uint32_t* __restrict__ x, size_t start, int lane) {
    const uint4 v = *reinterpret_cast<const uint4*>(x + start + 4 * lane);
    if (DELTA == ICX_DELTA_NONE) return v;
    if (DELTA == ICX_DELTA_1) {
        uint32_t prev = __shfl_up_sync(FULL, v.w, 1);
        if (lane == 0) prev = start > 0 ? x[start - 1] : 0u;
        return make_uint4(v.x - prev, v.y - v.x, v.z - v.y, v.w - v.z);
    }
    uint4 prev = shfl4(v, lane > 0 ? lane - 1 : 0);
    if (lane == 0) prev = start >= 4 ? *reinterpret_cast<const uint4*>(x + start - 4) : make_uint4(0, 0, 0, 0);
    return sub4(v, prev);
}

__device__ __forceinline__ uint32_t fe_bitlen(uint32_t v) { return 32u - (uint32_t)__clz(v); }

// ---------------------------------------------------------------- pass 1

template <int DELTA>
__global__ void fp_choose_kernel(const uint32_t* __restrict__ x, size_t n, uint32_t* __restrict__ em) {
    const int lane = threadIdx.x & 31;
    const size_t nb = n / 128, warps = (size_t)gridDim.x * (blockDim.x / 32);
    for (size_t k = blockIdx.x * (size_t)(blockDim.x / 32) + (threadIdx.x >> 5); k < nb; k += warps) {
        const uint4 d = fe_row_deltas<DELTA>(x, 128 * k, lane);
        const uint32_t l0 = fe_bitlen(d.x), l1 = fe_bitlen(d.y), l2 = fe_bitlen(d.z), l3 = fe_bitlen(d.w);
        const uint32_t maxbits = fe_bitlen(__reduce_or_sync(FULL, d.x | d.y | d.z | d.w));
        uint32_t best_b = maxbits, best_c = 0;
        unsigned long long best = ~0ull;
        for (uint32_t b = 0; b <= maxbits; ++b) {
            const uint32_t mine = (l0 > b) + (l1 > b) + (l2 > b) + (l3 > b);
            const uint32_t c = __reduce_add_sync(FULL, mine);
            const unsigned long long cost = 128ull * b + (unsigned long long)c * (8 + maxbits - b);
            if (cost <= best) {  // ties move to the larger b
                best = cost;
                best_b = b;
                best_c = c;
            }
        }
        if (lane == 0) em[k] = best_b | (maxbits << 8) | (best_c << 16);
    }
}

// ---------------------------------------------------------------- pass 2

// LAYOUT: ICX_FMT_PAPER = SIMD-FastPFOR (4-lane packing, arrays in chunks of
// 128), ICX_FMT_SCALAR = FastPFOR (one-lane packing, arrays in groups of 32).
template <int LAYOUT>
__global__ void fp_layout_kernel(size_t n, const uint32_t* __restrict__ em, EncMeta* __restrict__ meta,
                                 PageEnc* __restrict__ pages, uint32_t* __restrict__ sizes) {
    __shared__ uint32_t cnt_all[4][33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t nb = n / 128, P = (nb + kPageBlocks - 1) / kPageBlocks;
    const size_t p = (size_t)blockIdx.x * 4 + warp;
    if (p >= P) return;
    uint32_t* cnt = cnt_all[warp];
    cnt[lane] = 0;
    if (lane == 0) cnt[32] = 0;
    __syncwarp();
    const size_t k0 = kPageBlocks * p, K = min((size_t)kPageBlocks, nb - k0);
    if (lane == 0) {
        uint32_t packed = 16, rec = 0;
        for (size_t k = 0; k < K; ++k) {
            const uint32_t e = em[k0 + k];
            const uint32_t b = e & 255u, mb = (e >> 8) & 255u, c = e >> 16;
            EncMeta m;
            m.packed_off = packed;
            m.rec_off = rec;
            m.b = (uint8_t)b;
            m.mb = (uint8_t)mb;
            m.c = (uint8_t)c;
            m.d = (uint8_t)(mb - b);
            m.cursor = 0;
            if (mb > b) {
                // SimplePFOR: one stream in block order (running count in cnt[32])
                const uint32_t slot = LAYOUT == ICX_FMT_SIMPLE8B ? 32u : mb - b;
                m.cursor = cnt[slot];
                cnt[slot] += c;
                rec += 3 + c;
            } else {
                rec += 2;
            }
            meta[k0 + k] = m;
            packed += 16 * b;
        }
        PageEnc& pg = pages[p];
        pg.len_at = packed;
        pg.L = rec;
        pg.N = cnt[32];
        pg.W = 0;
        uint32_t q = packed + 4 + (uint32_t)fe_pad(rec, 4);
        uint32_t bitset = 0, base = 0;
        q += 4;  // bitset word
        for (int d = 1; d <= 32; ++d) {
            const uint32_t nd = cnt[d];
            pg.cnt[d - 1] = nd;
            pg.arr_base[d - 1] = base;
            base += nd;
            pg.arr_off[d - 1] = 0;
            if (nd) {
                bitset |= 1u << (d - 1);
                q = (uint32_t)fe_pad(q + 4, 16);
                pg.arr_off[d - 1] = q;
                q += LAYOUT == ICX_FMT_SCALAR ? 4 * d * ((nd + 31) / 32) : 16 * d * ((nd + 127) / 128);
            }
        }
        pg.bitset = bitset;
        pg.size = (uint32_t)fe_pad(q, 16);
        if (LAYOUT != ICX_FMT_SIMPLE8B) sizes[p] = pg.size;  // SimplePFOR: after its words are counted
    }
}

// ---------------------------------------------------------------- pass 4

// OUT = false: only the exceptions' high parts into the scratch (SimplePFOR
// sizes its pages from them before the index exists).
template <int DELTA, int LAYOUT, bool OUT = true>
__global__ void __launch_bounds__(128) fp_pack_kernel(const uint32_t* __restrict__ x, size_t n,
                                                      const EncMeta* __restrict__ meta,
                                                      const PageEnc* __restrict__ pages,
                                                      const uint64_t* __restrict__ index, uint8_t* __restrict__ out,
                                                      uint32_t* __restrict__ scratch) {
    __shared__ uint32_t sm_all[4][128];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* sm = sm_all[warp];
    const size_t nb = n / 128, warps = (size_t)gridDim.x * 4;
    for (size_t k = blockIdx.x * (size_t)4 + warp; k < nb; k += warps) {
        const size_t p = k / kPageBlocks;
        const EncMeta m = meta[k];
        const PageEnc& pg = pages[p];
        uint8_t* page = OUT ? out + index[p] : nullptr;
        const uint4 d = fe_row_deltas<DELTA>(x, 128 * k, lane);
        const uint32_t b = m.b, mask = width_mask(b);
        // packed low b bits: vertical layout (lane t holds field t of the 4
        // lanes), or one lane (lane t holds fields 4(t%8)..+3 of group t/8,
        // each group b words)
        for (int i = lane; i < 128; i += 32) sm[i] = 0;
        __syncwarp();
        if (LAYOUT == ICX_FMT_SCALAR || LAYOUT == ICX_FMT_SIMPLE8B) {
            const uint32_t g = (uint32_t)lane >> 3, i0 = 4 * ((uint32_t)lane & 7);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const uint32_t val = comp(d, c) & mask, bit = (i0 + c) * b, w = b * g + (bit >> 5), s = bit & 31;
                if (b) {
                    atomicOr(&sm[w], val << s);
                    if (s + b > 32) atomicOr(&sm[w + 1], val >> (32 - s));
                }
            }
        } else {
            const uint32_t bit = (uint32_t)lane * b, w = bit >> 5, s = bit & 31;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const uint32_t val = comp(d, c) & mask;
                if (b) {
                    atomicOr(&sm[4 * w + c], val << s);
                    if (s + b > 32) atomicOr(&sm[4 * (w + 1) + c], val >> (32 - s));
                }
            }
        }
        __syncwarp();
        if (OUT && (uint32_t)lane < b)
            reinterpret_cast<uint4*>(page + m.packed_off)[lane] = reinterpret_cast<const uint4*>(sm)[lane];
        __syncwarp();
        // byte-array record: b, maxbits[, c, positions ascending]
        uint8_t* rec = OUT ? page + pg.len_at + 4 + m.rec_off : nullptr;
        if (OUT && lane == 0) {
            rec[0] = (uint8_t)b;
            rec[1] = m.mb;
            if (m.mb > b) rec[2] = m.c;
        }
        if (m.mb > b) {
            bool f[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) f[c] = fe_bitlen(comp(d, c)) > b;
            unsigned bal[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) bal[c] = __ballot_sync(FULL, f[c]);
            const unsigned below = (1u << lane) - 1u;
            uint32_t rank = 0;
#pragma unroll
            for (int c = 0; c < 4; ++c) rank += __popc(bal[c] & below);
            uint32_t* exc = scratch + (size_t)kPageExc * p + pg.arr_base[m.d - 1] + m.cursor;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                if (f[c]) {
                    if (OUT) rec[3 + rank] = (uint8_t)(4 * lane + c);
                    exc[rank] = comp(d, c) >> b;  // b < maxbits <= 32
                    rank += 1;
                }
            }
        }
    }
}

// ------------------------------------------------- SimplePFOR: Simple-8b

// Simple-8b (Sec. 2, Table 2): integers per 64-bit word and their width, per
// selector (selector in bits 60..63).
__device__ __forceinline__ uint32_t fe_s8_count(uint32_t s) {
    const uint8_t c[16] = {240, 120, 60, 30, 20, 15, 12, 10, 8, 7, 6, 5, 4, 3, 2, 1};
    return c[s & 15];
}
__device__ __forceinline__ uint32_t fe_s8_bits(uint32_t s) {
    const uint8_t b[16] = {0, 0, 1, 2, 3, 4, 5, 6, 7, 8, 10, 12, 15, 20, 30, 60};
    return b[s & 15];
}

// Whole warp: the selector of the word starting at value p of v[0..N): the
// smallest selector whose count next values all exist and fit (Sec. 2's
// greedy rule; lane s tests selector s).
__device__ __forceinline__ uint32_t fe_s8_select(const uint32_t* __restrict__ v, uint32_t N, uint32_t p, int lane) {
    bool ok = false;
    if (lane < 16) {
        const uint32_t cnt = fe_s8_count((uint32_t)lane), b = fe_s8_bits((uint32_t)lane);
        ok = p + cnt <= N;
        for (uint32_t i = 0; i < cnt && ok; ++i) ok = b >= 32 || v[p + i] < (1u << b);
    }
    return (uint32_t)__ffs(__ballot_sync(FULL, ok)) - 1;  // lane 15 (1 value of 60 bits) always fits
}

// Per page (one warp): the number of Simple-8b words of its exception high
// parts, then the page size.
__global__ void __launch_bounds__(128) s8_size_kernel(size_t n, PageEnc* __restrict__ pages,
                                                      const uint32_t* __restrict__ scratch,
                                                      uint32_t* __restrict__ sizes) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t nb = n / 128, P = (nb + kPageBlocks - 1) / kPageBlocks;
    const size_t p = (size_t)blockIdx.x * 4 + warp;
    if (p >= P) return;
    PageEnc& pg = pages[p];
    const uint32_t* v = scratch + (size_t)kPageExc * p;
    const uint32_t N = pg.N;
    uint32_t q = 0, W = 0;
    while (q < N) {
        q += fe_s8_count(fe_s8_select(v, N, q, lane));
        ++W;
    }
    if (lane == 0) {
        const uint32_t words_at = (uint32_t)fe_pad(pg.len_at + 4 + fe_pad(pg.L, 4) + 8, 16);
        pg.W = W;
        pg.size = (uint32_t)fe_pad(words_at + 8 * (size_t)W, 16);
        sizes[p] = pg.size;
    }
}

// ---------------------------------------------------------------- pass 5

template <int LAYOUT>
__global__ void __launch_bounds__(128) fp_finish_kernel(size_t n, const PageEnc* __restrict__ pages,
                                                        const uint64_t* __restrict__ index, uint8_t* __restrict__ out,
                                                        const uint32_t* __restrict__ scratch) {
    __shared__ uint32_t sm_all[4][16 * 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* sm = sm_all[warp];
    const size_t nb = n / 128, P = (nb + kPageBlocks - 1) / kPageBlocks;
    const size_t p = (size_t)blockIdx.x * 4 + warp;
    if (p >= P) return;
    const PageEnc& pg = pages[p];
    uint8_t* page = out + index[p];
    if (lane == 0) {
        *reinterpret_cast<uint32_t*>(page) = pg.len_at / 4;  // offset in words
        *reinterpret_cast<uint32_t*>(page + pg.len_at) = pg.L;
    }
    if (lane >= 4 && lane < 16) page[lane] = 0;
    const uint32_t bytes_at = pg.len_at + 4, Lpad = (uint32_t)fe_pad(pg.L, 4);
    if ((uint32_t)lane < Lpad - pg.L) page[bytes_at + pg.L + lane] = 0;
    uint32_t q = bytes_at + Lpad;
    if (LAYOUT == ICX_FMT_SIMPLE8B) {
        // N, W, zero padding to 16 bytes, the Simple-8b words, zero padding
        if (lane == 0) {
            *reinterpret_cast<uint32_t*>(page + q) = pg.N;
            *reinterpret_cast<uint32_t*>(page + q + 4) = pg.W;
        }
        const uint32_t words_at = (uint32_t)fe_pad(q + 8, 16);
        if ((uint32_t)lane < words_at - (q + 8)) page[q + 8 + lane] = 0;
        const uint32_t* v = scratch + (size_t)kPageExc * p;
        uint64_t* words = reinterpret_cast<uint64_t*>(page + words_at);  // 16-byte aligned
        uint32_t e = 0;
        for (uint32_t w = 0; w < pg.W; ++w) {
            const uint32_t sel = fe_s8_select(v, pg.N, e, lane), cnt = fe_s8_count(sel), b = fe_s8_bits(sel);
            uint64_t word = 0;
            if (sel >= 2)
                for (uint32_t i = lane; i < cnt; i += 32) word |= (uint64_t)v[e + i] << (i * b);
#pragma unroll
            for (int o = 16; o; o >>= 1) word |= __shfl_xor_sync(FULL, word, o);
            if (lane == 0) words[w] = word | (uint64_t)sel << 60;
            e += cnt;
        }
        const uint32_t end = words_at + 8 * pg.W;
        if ((uint32_t)lane < pg.size - end) page[end + lane] = 0;
        return;
    }
    if (lane == 0) *reinterpret_cast<uint32_t*>(page + q) = pg.bitset;
    q += 4;
    for (int d = 1; d <= 32; ++d) {
        const uint32_t nd = pg.cnt[d - 1];
        if (!nd) continue;
        if (lane == 0) *reinterpret_cast<uint32_t*>(page + q) = nd;
        const uint32_t off = pg.arr_off[d - 1];
        if ((uint32_t)lane < off - (q + 4)) page[q + 4 + lane] = 0;
        const uint32_t* src = scratch + (size_t)kPageExc * p + pg.arr_base[d - 1];
        if (LAYOUT == ICX_FMT_SCALAR) {
            // groups of 32 values in one lane: value e of a group at bit e*d
            const uint32_t groups = (nd + 31) / 32;
            for (uint32_t gi = 0; gi < groups; ++gi) {
                for (int i = lane; i < d; i += 32) sm[i] = 0;
                __syncwarp();
                const uint32_t e = 32 * gi + lane, val = e < nd ? src[e] : 0u;
                const uint32_t bit = (uint32_t)lane * d, w = bit >> 5, s = bit & 31;
                atomicOr(&sm[w], val << s);
                if (s + d > 32) atomicOr(&sm[w + 1], val >> (32 - s));
                __syncwarp();
                if (lane < d) reinterpret_cast<uint32_t*>(page + off + 4 * d * gi)[lane] = sm[lane];
                __syncwarp();
            }
            q = off + 4 * d * groups;
            continue;
        }
        const uint32_t chunks = (nd + 127) / 128;
        for (uint32_t ch = 0; ch < chunks; ++ch) {
            for (int i = lane; i < 4 * d; i += 32) sm[i] = 0;
            __syncwarp();
            const uint32_t bit = (uint32_t)lane * d, w = bit >> 5, s = bit & 31;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const uint32_t e = 128 * ch + 4 * lane + c;
                const uint32_t val = e < nd ? src[e] : 0u;
                atomicOr(&sm[4 * w + c], val << s);
                if (s + d > 32) atomicOr(&sm[4 * (w + 1) + c], val >> (32 - s));
            }
            __syncwarp();
            if (lane < d)
                reinterpret_cast<uint4*>(page + off + 16 * d * ch)[lane] = reinterpret_cast<const uint4*>(sm)[lane];
            __syncwarp();
        }
        q = off + 16 * d * chunks;
    }
    if ((uint32_t)lane < pg.size - q) page[q + lane] = 0;
}

// ---------------------------------------------------------------- pass 6

template <int DELTA>
__global__ void fp_tail_kernel(const uint32_t* __restrict__ x, size_t n, const uint64_t* __restrict__ index, size_t P,
                               uint8_t* __restrict__ out, uint64_t* __restrict__ out_bytes) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    size_t pos = index[P];
    for (size_t i = 128 * (n / 128); i < n; ++i) {
        const uint32_t prev = (DELTA > 0 && i >= (size_t)DELTA) ? x[i - DELTA] : 0u;
        uint32_t v = x[i] - prev;
        while (v >= 128) {
            out[pos++] = (uint8_t)(v & 127u);
            v >>= 7;
        }
        out[pos++] = (uint8_t)(v | 128u);
    }
    *out_bytes = pos;
}

__global__ void fp_scan_kernel(const uint32_t* __restrict__ sizes, size_t count, uint64_t* __restrict__ index) {
    // exclusive scan of page sizes (few pages: one thread is enough)
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    unsigned long long run = 0;
    for (size_t i = 0; i < count; ++i) {
        index[i] = run;
        run += sizes[i];
    }
    index[count] = run;
}

template <int DELTA, int LAYOUT>
static cudaError_t fp_encode_t(const uint32_t* x, size_t n, uint8_t* out, uint64_t* index, uint64_t* out_bytes,
                               uint8_t* ws, cudaStream_t s) {
    const FeLayout lay(n);
    const size_t nb = n / 128, P = (nb + kPageBlocks - 1) / kPageBlocks;
    uint32_t* em = reinterpret_cast<uint32_t*>(ws + lay.em);
    EncMeta* meta = reinterpret_cast<EncMeta*>(ws + lay.meta);
    PageEnc* pages = reinterpret_cast<PageEnc*>(ws + lay.pages);
    uint32_t* sizes = reinterpret_cast<uint32_t*>(ws + lay.sizes);
    uint32_t* scratch = reinterpret_cast<uint32_t*>(ws + lay.scratch);
    if (nb) {
        const int g = (int)min((nb + 3) / 4, (size_t)152 * 16);
        fp_choose_kernel<DELTA><<<g, 128, 0, s>>>(x, n, em);
        fp_layout_kernel<LAYOUT><<<(unsigned)((P + 3) / 4), 128, 0, s>>>(n, em, meta, pages, sizes);
        if (LAYOUT == ICX_FMT_SIMPLE8B) {  // the high parts first: they size the pages
            fp_pack_kernel<DELTA, LAYOUT, false><<<g, 128, 0, s>>>(x, n, meta, pages, index, out, scratch);
            s8_size_kernel<<<(unsigned)((P + 3) / 4), 128, 0, s>>>(n, pages, scratch, sizes);
        }
    }
    fp_scan_kernel<<<1, 32, 0, s>>>(sizes, P, index);
    if (nb) {
        const int g = (int)min((nb + 3) / 4, (size_t)152 * 16);
        fp_pack_kernel<DELTA, LAYOUT><<<g, 128, 0, s>>>(x, n, meta, pages, index, out, scratch);
        fp_finish_kernel<LAYOUT><<<(unsigned)((P + 3) / 4), 128, 0, s>>>(n, pages, index, out, scratch);
    }
    fp_tail_kernel<DELTA><<<1, 32, 0, s>>>(x, n, index, P, out, out_bytes);
    return cudaGetLastError();
}

cudaError_t launch_fastpfor_encode(int delta, int fmt, const uint32_t* x, size_t n, uint8_t* out, size_t out_cap,
                                   uint64_t* index, uint64_t* out_bytes, void* ws, size_t ws_bytes, cudaStream_t s) {
    (void)out_cap;
    if (ws_bytes < FeLayout(n).total) return cudaErrorInvalidValue;
    uint8_t* w = static_cast<uint8_t*>(ws);
#define ICX_CASE(D, L) \
    if (delta == D && fmt == L) return fp_encode_t<D, L>(x, n, out, index, out_bytes, w, s);
    ICX_CASE(ICX_DELTA_NONE, ICX_FMT_PAPER)
    ICX_CASE(ICX_DELTA_1, ICX_FMT_PAPER)
    ICX_CASE(ICX_DELTA_4, ICX_FMT_PAPER)
    ICX_CASE(ICX_DELTA_NONE, ICX_FMT_SCALAR)
    ICX_CASE(ICX_DELTA_1, ICX_FMT_SCALAR)
    ICX_CASE(ICX_DELTA_4, ICX_FMT_SCALAR)
    ICX_CASE(ICX_DELTA_NONE, ICX_FMT_SIMPLE8B)
    ICX_CASE(ICX_DELTA_1, ICX_FMT_SIMPLE8B)
    ICX_CASE(ICX_DELTA_4, ICX_FMT_SIMPLE8B)
#undef ICX_CASE
    return cudaErrorInvalidValue;
}

}  // namespace icx
