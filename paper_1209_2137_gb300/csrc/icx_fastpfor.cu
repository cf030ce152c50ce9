// SIMD-FastPFOR (Sec. 5): page walk, decoding and encoding.
#include "icx_kernels.cuh"

namespace icx {

cudaError_t launch_fastpfor_decode(int, const uint8_t*, size_t, uint32_t*, size_t, const uint64_t*, WsHeader*,
                                   cudaStream_t) {
    return cudaErrorNotSupported;
}
cudaError_t launch_fastpfor_index(const uint8_t*, size_t, size_t, uint64_t*, WsHeader*, cudaStream_t) {
    return cudaErrorNotSupported;
}
cudaError_t launch_fastpfor_encode(int, const uint32_t*, size_t, uint8_t*, size_t, uint64_t*, uint64_t*, void*,
                                   size_t, cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace icx
