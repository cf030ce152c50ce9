// C ABI of the icx library (declared in include/icx.h): argument validation
// and launches.  Argument errors return synchronously without launching;
// data-dependent errors land in the workspace status word.
#include <cstdint>
#include <cstring>

#include "icx_kernels.cuh"

using icx::WsHeader;

namespace {

constexpr size_t kMaxN = (size_t)1 << 34;  // bound that keeps every size in range

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
bool valid_delta(int d) { return d == ICX_DELTA_NONE || d == ICX_DELTA_1 || d == ICX_DELTA_4; }
bool valid_fmt(int f) { return f == ICX_FMT_PAPER || f == ICX_FMT_W32 || f == ICX_FMT_BP32; }
bool valid_fp_fmt(int f) { return f == ICX_FMT_PAPER || f == ICX_FMT_SCALAR || f == ICX_FMT_SIMPLE8B; }
size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

icx_status from_cuda(cudaError_t e) { return e == cudaSuccess ? ICX_OK : ICX_ECUDA; }

size_t metablocks(size_t n) { return (n / 128 + 15) / 16; }
size_t pages(size_t n) { return (n / 128 + 511) / 512; }

// encode workspace: header, then widths (1 byte per 128-integer block; BP32:
// one 4-width descriptor word per 128 integers), then sizes (4 bytes per
// metablock or page, plus one).
size_t enc_widths_off() { return icx::kWsHeaderBytes; }
size_t enc_sizes_off(size_t n) { return enc_widths_off() + round_up(4 * (n / 128 + 1), 256); }

}  // namespace

extern "C" {

size_t icx_bp128_index_len(size_t n) { return metablocks(n) + 1; }
size_t icx_fastpfor_index_len(size_t n) { return pages(n) + 1; }

size_t icx_bp128_max_bytes(size_t n, icx_layout fmt) {
    const size_t M = metablocks(n), nb = n / 128;
    const size_t body = fmt == ICX_FMT_W32 ? M * (16 + 128 * 64) : fmt == ICX_FMT_BP32 ? nb * 516 : M * 16 + nb * 512;
    return body + (n % 128) * 5 + 16;
}

size_t icx_fastpfor_max_bytes(size_t n) {
    const size_t nb = n / 128, P = pages(n);
    // per block the exception high parts take <= 512 bytes in arrays, <= 1,024 as Simple-8b words
    return P * (16 + 4 + 3 + 4 + 15 + 32 * (4 + 15 + 16 * 32)) + nb * (512 + 131 + 1024) + (n % 128) * 5 + 16;
}

size_t icx_workspace_bytes(size_t n) { return icx::ws_total_bytes(n); }

icx_status icx_workspace_layout(size_t n, size_t ws_bytes, size_t* out) {
    if (!out || ws_bytes < icx::ws_total_bytes(n)) return ICX_EINVAL;
    const size_t N = icx::ws_capacity(ws_bytes), plain = icx::ws_plain_base(ws_bytes);
    out[0] = N;
    out[1] = icx::kWsHeaderBytes + 32 * icx::ws_tiles(n);  // end of n's look-back states
    out[2] = plain;                                        // page parse records
    out[3] = plain + icx::ws_meta_bytes(n);                // prepare-kernel records
    out[4] = out[3] + icx::ws_fp2_bytes(n);                // end of the plain regions
    out[5] = (ws_bytes - icx::ws_blocklane_bytes(n)) / 256 * 256;  // tagged block-per-lane scratch
    return ICX_OK;
}

size_t icx_encode_workspace_bytes(size_t n) {
    const size_t bp = enc_sizes_off(n) + round_up(4 * (metablocks(n) + 2), 256);
    const size_t fp = icx::fastpfor_encode_workspace_bytes(n);
    return bp > fp ? bp : fp;
}

icx_status icx_workspace_init(void* d_ws, size_t ws_bytes, icx_stream_t stream) {
    if (!d_ws || ws_bytes < icx::kWsHeaderBytes) return ICX_EINVAL;
    return from_cuda(cudaMemsetAsync(d_ws, 0, ws_bytes, (cudaStream_t)stream));
}

icx_status icx_workspace_set_wait_limit(void* d_ws, size_t ws_bytes, unsigned usec, icx_stream_t stream) {
    if (!d_ws || ws_bytes < icx::kWsHeaderBytes) return ICX_EINVAL;
    // from pageable memory: the value is staged before the call returns
    const unsigned v = usec;
    WsHeader* h = static_cast<WsHeader*>(d_ws);
    return from_cuda(cudaMemcpyAsync(&h->aux[icx::kAuxWaitLimit], &v, sizeof(unsigned), cudaMemcpyHostToDevice,
                                     (cudaStream_t)stream));
}

icx_status icx_status_read(void* d_ws, icx_stream_t stream, icx_status* out) {
    if (!d_ws || !out) return ICX_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned int v = 0;
    WsHeader* h = static_cast<WsHeader*>(d_ws);
    if (cudaStreamSynchronize(s) != cudaSuccess) return ICX_ECUDA;
    if (cudaMemcpyAsync(&v, &h->status, sizeof(v), cudaMemcpyDeviceToHost, s) != cudaSuccess) return ICX_ECUDA;
    if (cudaMemsetAsync(&h->status, 0, sizeof(v), s) != cudaSuccess) return ICX_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return ICX_ECUDA;
    *out = (icx_status)v;
    return ICX_OK;
}

icx_status bp128_index(const uint8_t* d_in, size_t in_bytes, size_t n, icx_layout fmt, uint64_t* d_index,
                       void* d_ws, size_t ws_bytes, icx_stream_t stream) {
    if (!valid_fmt(fmt) || !d_index || !d_ws || n > kMaxN) return ICX_EINVAL;
    if (metablocks(n) > 0 && !d_in) return ICX_EINVAL;
    if (d_in && !aligned16(d_in)) return ICX_EALIGN;
    if (ws_bytes < icx::kWsHeaderBytes) return ICX_ENOSPC;
    return from_cuda(icx::launch_bp128_index(d_in, in_bytes, n, fmt, d_index, static_cast<WsHeader*>(d_ws),
                                             (cudaStream_t)stream));
}

icx_status bp128_decode(const uint8_t* d_in, size_t in_bytes, uint32_t* d_out, size_t n, icx_delta delta,
                        icx_layout fmt, const uint64_t* d_index, void* d_ws, size_t ws_bytes,
                        icx_stream_t stream) {
    if (!valid_delta(delta) || !valid_fmt(fmt) || n > kMaxN) return ICX_EINVAL;
    if (n == 0) return ICX_OK;
    if (!d_in || !d_out || !d_ws) return ICX_EINVAL;
    if (!aligned16(d_in) || !aligned16(d_out) || !aligned16(d_ws) || (d_index && !aligned16(d_index)))
        return ICX_EALIGN;
    if (ws_bytes < icx_workspace_bytes(n)) return ICX_ENOSPC;
    WsHeader* h = static_cast<WsHeader*>(d_ws);
    cudaStream_t s = (cudaStream_t)stream;
    if (!d_index) {
        if (metablocks(n) > 1) return ICX_EINVAL;
        const icx_status st = from_cuda(icx::launch_bp128_index(d_in, in_bytes, n, fmt, h->mini_index, h, s));
        if (st != ICX_OK) return st;
        d_index = h->mini_index;
    }
    return from_cuda(icx::launch_bp128_decode(delta, fmt, d_in, in_bytes, d_out, n, d_index, h, ws_bytes, s));
}

// Clears the bitmap and the count of a membership call.
static icx_status member_clear(uint32_t* d_bits, size_t nb, uint64_t* d_count, cudaStream_t s) {
    if (nb && cudaMemsetAsync(d_bits, 0, 4 * ((nb + 31) / 32), s) != cudaSuccess) return ICX_ECUDA;
    return from_cuda(cudaMemsetAsync(d_count, 0, sizeof(uint64_t), s));
}

static bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

icx_status bp128_intersect(const uint8_t* d_in, size_t in_bytes, size_t n, icx_delta delta, icx_layout fmt,
                           const uint64_t* d_index, const uint32_t* d_b, size_t nb, uint32_t* d_bits,
                           uint64_t* d_count, void* d_ws, size_t ws_bytes, icx_stream_t stream) {
    if (!valid_delta(delta) || !valid_fmt(fmt) || fmt == ICX_FMT_BP32 || n > kMaxN || nb > kMaxN || !d_count)
        return ICX_EINVAL;
    if (nb && (!d_b || !d_bits)) return ICX_EINVAL;
    if (!aligned(d_count, 8) || (nb && (!aligned(d_b, 4) || !aligned(d_bits, 4)))) return ICX_EALIGN;
    if (n && (!d_in || !d_ws)) return ICX_EINVAL;
    if (n && (!aligned16(d_in) || !aligned16(d_ws) || (d_index && !aligned16(d_index)))) return ICX_EALIGN;
    if (n && ws_bytes < icx_workspace_bytes(n)) return ICX_ENOSPC;
    cudaStream_t s = (cudaStream_t)stream;
    const icx_status cl = member_clear(d_bits, nb, d_count, s);
    if (cl != ICX_OK || n == 0 || nb == 0) return cl;
    WsHeader* h = static_cast<WsHeader*>(d_ws);
    if (!d_index) {
        if (metablocks(n) > 1) return ICX_EINVAL;
        const icx_status st = from_cuda(icx::launch_bp128_index(d_in, in_bytes, n, fmt, h->mini_index, h, s));
        if (st != ICX_OK) return st;
        d_index = h->mini_index;
    }
    return from_cuda(icx::launch_bp128_member(delta, fmt, d_in, in_bytes, n, d_index, d_b, nb, d_bits,
                                              reinterpret_cast<unsigned long long*>(d_count), h, s));
}

icx_status sorted_intersect(const uint32_t* d_a, size_t n, const uint32_t* d_b, size_t nb, uint32_t* d_bits,
                            uint64_t* d_count, icx_stream_t stream) {
    if (n > kMaxN || nb > kMaxN || !d_count || (n && !d_a)) return ICX_EINVAL;
    if (nb && (!d_b || !d_bits)) return ICX_EINVAL;
    if (!aligned(d_count, 8) || (nb && (!aligned(d_b, 4) || !aligned(d_bits, 4))) || (n && !aligned16(d_a)))
        return ICX_EALIGN;
    cudaStream_t s = (cudaStream_t)stream;
    const icx_status cl = member_clear(d_bits, nb, d_count, s);
    if (cl != ICX_OK || n == 0 || nb == 0) return cl;
    return from_cuda(
        icx::launch_sorted_member(d_a, n, d_b, nb, d_bits, reinterpret_cast<unsigned long long*>(d_count), s));
}

icx_status delta_decode(const uint32_t* d_in, uint32_t* d_out, size_t n, icx_delta delta, void* d_ws,
                        size_t ws_bytes, icx_stream_t stream) {
    if (!valid_delta(delta) || n > kMaxN) return ICX_EINVAL;
    if (n == 0) return ICX_OK;
    if (!d_in || !d_out || !d_ws) return ICX_EINVAL;
    if (!aligned16(d_in) || !aligned16(d_out)) return ICX_EALIGN;
    if (d_in != d_out) {
        const uintptr_t a = reinterpret_cast<uintptr_t>(d_in), b = reinterpret_cast<uintptr_t>(d_out);
        if (a < b + 4 * n && b < a + 4 * n) return ICX_EINVAL;  // partial overlap
    }
    if (ws_bytes < icx_workspace_bytes(n)) return ICX_ENOSPC;
    return from_cuda(
        icx::launch_delta_decode(delta, d_in, d_out, n, static_cast<WsHeader*>(d_ws), (cudaStream_t)stream));
}

icx_status delta_encode(const uint32_t* d_in, uint32_t* d_out, size_t n, icx_delta delta, icx_stream_t stream) {
    if (!valid_delta(delta) || n > kMaxN) return ICX_EINVAL;
    if (n == 0) return ICX_OK;
    if (!d_in || !d_out) return ICX_EINVAL;
    const uintptr_t a = reinterpret_cast<uintptr_t>(d_in), b = reinterpret_cast<uintptr_t>(d_out);
    if (a < b + 4 * n && b < a + 4 * n) return ICX_EINVAL;
    return from_cuda(icx::launch_delta_encode(delta, d_in, d_out, n, (cudaStream_t)stream));
}

icx_status bp128_encode(const uint32_t* d_x, size_t n, icx_delta delta, icx_layout fmt, uint8_t* d_out,
                        size_t out_cap, uint64_t* d_index, uint64_t* d_out_bytes, void* d_ews, size_t ews_bytes,
                        icx_stream_t stream) {
    if (!valid_delta(delta) || !valid_fmt(fmt) || n > kMaxN) return ICX_EINVAL;
    if (!d_out || !d_index || !d_out_bytes || !d_ews || (n > 0 && !d_x)) return ICX_EINVAL;
    if ((d_x && !aligned16(d_x)) || !aligned16(d_out)) return ICX_EALIGN;
    if (out_cap < icx_bp128_max_bytes(n, fmt) || ews_bytes < icx_encode_workspace_bytes(n)) return ICX_ENOSPC;
    uint8_t* base = static_cast<uint8_t*>(d_ews);
    return from_cuda(icx::launch_bp128_encode(delta, fmt, d_x, n, d_out, d_index, d_out_bytes,
                                              base + enc_widths_off(),
                                              reinterpret_cast<uint32_t*>(base + enc_sizes_off(n)),
                                              (cudaStream_t)stream));
}

icx_status fastpfor_index(const uint8_t* d_in, size_t in_bytes, size_t n, icx_layout fmt, uint64_t* d_index,
                          void* d_ws, size_t ws_bytes, icx_stream_t stream) {
    if (!valid_fp_fmt(fmt) || !d_index || !d_ws || n > kMaxN) return ICX_EINVAL;
    if (pages(n) > 0 && !d_in) return ICX_EINVAL;
    if (d_in && !aligned16(d_in)) return ICX_EALIGN;
    if (ws_bytes < icx::kWsHeaderBytes) return ICX_ENOSPC;
    return from_cuda(icx::launch_fastpfor_index(d_in, in_bytes, n, fmt, d_index, static_cast<WsHeader*>(d_ws),
                                                (cudaStream_t)stream));
}

icx_status fastpfor_decode(const uint8_t* d_in, size_t in_bytes, uint32_t* d_out, size_t n, icx_delta delta,
                           icx_layout fmt, const uint64_t* d_index, void* d_ws, size_t ws_bytes,
                           icx_stream_t stream) {
    if (!valid_delta(delta) || !valid_fp_fmt(fmt) || n > kMaxN) return ICX_EINVAL;
    if (n == 0) return ICX_OK;
    if (!d_in || !d_out || !d_ws) return ICX_EINVAL;
    if (!aligned16(d_in) || !aligned16(d_out) || !aligned16(d_ws) || (d_index && !aligned16(d_index)))
        return ICX_EALIGN;
    if (ws_bytes < icx_workspace_bytes(n)) return ICX_ENOSPC;
    WsHeader* h = static_cast<WsHeader*>(d_ws);
    cudaStream_t s = (cudaStream_t)stream;
    if (!d_index) {
        if (pages(n) > 1) return ICX_EINVAL;
        const icx_status st = from_cuda(icx::launch_fastpfor_index(d_in, in_bytes, n, fmt, h->mini_index, h, s));
        if (st != ICX_OK) return st;
        d_index = h->mini_index;
    }
    return from_cuda(icx::launch_fastpfor_decode(delta, fmt, d_in, in_bytes, d_out, n, d_index, h, ws_bytes, s));
}

icx_status fastpfor_encode(const uint32_t* d_x, size_t n, icx_delta delta, icx_layout fmt, uint8_t* d_out,
                           size_t out_cap, uint64_t* d_index, uint64_t* d_out_bytes, void* d_ews, size_t ews_bytes,
                           icx_stream_t stream) {
    if (!valid_delta(delta) || !valid_fp_fmt(fmt) || n > kMaxN) return ICX_EINVAL;
    if (!d_out || !d_index || !d_out_bytes || !d_ews || (n > 0 && !d_x)) return ICX_EINVAL;
    if ((d_x && !aligned16(d_x)) || !aligned16(d_out)) return ICX_EALIGN;
    if (out_cap < icx_fastpfor_max_bytes(n) || ews_bytes < icx_encode_workspace_bytes(n)) return ICX_ENOSPC;
    return from_cuda(icx::launch_fastpfor_encode(delta, fmt, d_x, n, d_out, out_cap, d_index, d_out_bytes, d_ews,
                                                 ews_bytes, (cudaStream_t)stream));
}

const char* icx_version(void) { return "icx 0.1 (sm_103a)"; }

icx_status icx_set_tuning(const char* key, int value) {
    if (!key) return ICX_EINVAL;
    if (!strcmp(key, "bp128.warps_per_cta")) {
        icx::set_bp128_warps(value);
        return ICX_OK;
    }
    if (!strcmp(key, "fastpfor.warps_per_cta")) {
        icx::set_fastpfor_warps(value);
        return ICX_OK;
    }
    if (!strcmp(key, "bp128.blocklane")) {
        icx::set_bp128_blocklane(value);
        return ICX_OK;
    }
    if (!strcmp(key, "fastpfor.stream_warps")) {
        icx::set_fastpfor_stream_warps(value);
        return ICX_OK;
    }
    if (!strcmp(key, "fastpfor.chain_overlap")) {
        icx::set_fastpfor_chain_overlap(value);
        return ICX_OK;
    }
    if (!strcmp(key, "fastpfor.blocklane")) {
        icx::set_fastpfor_blocklane(value);
        return ICX_OK;
    }
    if (!strcmp(key, "bp128.blocklane_store")) {
        icx::set_bp128_blocklane_store(value);
        return ICX_OK;
    }
    if (!strcmp(key, "bp128.blocklane_sum_warps")) {
        icx::set_bp128_blocklane_sumw(value);
        return ICX_OK;
    }
    if (!strcmp(key, "bp128.blocklane_lead")) {
        icx::set_bp128_blocklane_lead(value);
        return ICX_OK;
    }
    if (!strcmp(key, "bp128.blocklane_ctas")) {
        icx::set_bp128_blocklane_ctas(value);
        return ICX_OK;
    }
    if (!strcmp(key, "bp128.l2_prefetch")) {
        icx::set_bp128_prefetch(value);
        return ICX_OK;
    }
    return ICX_EINVAL;
}

}  // extern "C"
