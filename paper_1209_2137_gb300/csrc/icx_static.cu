// bp128_decode_static: SIMD-BP128 / W32 decoding for callers that cannot
// allocate device memory (code that must not call cudaMalloc: allocation-free
// runtimes, callers inside a memory pool they do not own, plugins whose host
// forbids allocations on the hot path).  Instead of a caller-provided
// workspace it uses one file-scope device array, sized for up to
// kStaticMaxN integers.  Every GPU that loads the library holds that array
// until the process exits.
#include <mutex>

#include "icx_kernels.cuh"

namespace {

// Largest n the static workspace serves: 2^28 integers (1 GiB of output).
constexpr size_t kStaticMaxN = (size_t)1 << 28;
// header + look-back states for kStaticMaxN (the SIMD-BP128 decoder uses no
// other workspace region); about 4 MiB.
constexpr size_t kStaticBytes =
    (icx::kWsHeaderBytes + 32 * (kStaticMaxN / 2048 + 16) + 255) / 256 * 256;

__device__ __align__(256) unsigned char g_static_ws[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_ptr[kMaxDevices] = {nullptr};
// Calls per device since the array was last zeroed: its look-back states are
// tagged with a 30-bit launch number, so it is zeroed again (a memset, no
// allocation) before 2^30 launches could reuse a tag.
uint64_t g_calls[kMaxDevices] = {0};
constexpr uint64_t kCallsPerZero = (uint64_t)1 << 29;

// Device address of g_static_ws on the current device.  In host code the
// symbol's name is only a host-side stand-in, so the address is looked up
// with cudaGetSymbolAddress (with that device current) on every call made
// outside stream capture -- after a device reset the module is loaded again
// and the array may sit elsewhere -- and remembered per device for calls made
// while `s` is being captured, when the lookup cannot run.
icx_status static_workspace(cudaStream_t s, void** out, bool* rezero) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ICX_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return ICX_EINVAL;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return ICX_ECUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (cs == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_ws) != cudaSuccess || !p) return ICX_ECUDA;
        g_ptr[dev] = p;
    } else if (!g_ptr[dev]) {
        return ICX_EINVAL;  // no call on this device was made before the capture
    }
    *out = g_ptr[dev];
    *rezero = ++g_calls[dev] % kCallsPerZero == 0;
    return ICX_OK;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" icx_status bp128_decode_static(const uint8_t* d_in, size_t in_bytes, uint32_t* d_out, size_t n,
                                          icx_delta delta, icx_layout fmt, const uint64_t* d_index,
                                          uint32_t* d_status, icx_stream_t stream) {
    if (!(delta == ICX_DELTA_NONE || delta == ICX_DELTA_1 || delta == ICX_DELTA_4)) return ICX_EINVAL;
    if (!(fmt == ICX_FMT_PAPER || fmt == ICX_FMT_W32 || fmt == ICX_FMT_BP32)) return ICX_EINVAL;
    if (n > kStaticMaxN) return ICX_ENOSPC;  // beyond the static workspace
    if (n == 0) return ICX_OK;
    if (!d_in || !d_out) return ICX_EINVAL;
    if (!aligned16(d_in) || !aligned16(d_out) || (d_index && !aligned16(d_index))) return ICX_EALIGN;
    const size_t M = (n / 128 + 15) / 16;
    if (!d_index && M > 1) return ICX_EINVAL;
    void* ws = nullptr;
    bool rezero = false;
    const icx_status st = static_workspace((cudaStream_t)stream, &ws, &rezero);
    if (st != ICX_OK) return st;
    icx::WsHeader* h = static_cast<icx::WsHeader*>(ws);
    cudaStream_t s = (cudaStream_t)stream;
    if (rezero && cudaMemsetAsync(ws, 0, kStaticBytes, s) != cudaSuccess) return ICX_ECUDA;
    // The array keeps the previous call's contents: the unit counters and
    // look-back states reset themselves at the end of every launch (epoch
    // tags), only the status word has to be cleared here.
    if (cudaMemsetAsync(&h->status, 0, sizeof(h->status), s) != cudaSuccess) return ICX_ECUDA;
    if (!d_index) {
        if (icx::launch_bp128_index(d_in, in_bytes, n, fmt, h->mini_index, h, s) != cudaSuccess) return ICX_ECUDA;
        d_index = h->mini_index;
    }
    if (icx::launch_bp128_decode_lookback(delta, fmt, d_in, in_bytes, d_out, n, d_index, h, s) != cudaSuccess)
        return ICX_ECUDA;
    if (d_status &&
        cudaMemcpyAsync(d_status, &h->status, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return ICX_ECUDA;
    return ICX_OK;
}
