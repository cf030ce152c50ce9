// Launchers implemented by the kernel translation units; called by the C ABI
// layer (icx_api.cu) after argument validation.
#pragma once

#include "icx_device.cuh"

namespace icx {

cudaError_t launch_bp128_decode(int delta, int fmt, const uint8_t* in, size_t in_bytes, uint32_t* out,
                                size_t n, const uint64_t* index, WsHeader* h, size_t ws_bytes, cudaStream_t s);
cudaError_t launch_bp128_decode_lookback(int delta, int fmt, const uint8_t* in, size_t in_bytes, uint32_t* out,
                                         size_t n, const uint64_t* index, WsHeader* h, cudaStream_t s);
cudaError_t launch_bp128_blocklane(int delta, const uint8_t* in, size_t in_bytes, uint32_t* out, size_t n,
                                   const uint64_t* index, WsHeader* h, size_t ws_bytes, cudaStream_t s);
cudaError_t launch_bp128_index(const uint8_t* in, size_t in_bytes, size_t n, int fmt, uint64_t* index,
                               WsHeader* h, cudaStream_t s);
cudaError_t launch_delta_decode(int delta, const uint32_t* in, uint32_t* out, size_t n, WsHeader* h,
                                cudaStream_t s);
cudaError_t launch_delta_encode(int delta, const uint32_t* x, uint32_t* d, size_t n, cudaStream_t s);
cudaError_t launch_bp128_encode(int delta, int fmt, const uint32_t* x, size_t n, uint8_t* out, uint64_t* index,
                                uint64_t* out_bytes, uint8_t* widths, uint32_t* sizes, cudaStream_t s);
cudaError_t launch_fastpfor_decode(int delta, int fmt, const uint8_t* in, size_t in_bytes, uint32_t* out, size_t n,
                                   const uint64_t* index, WsHeader* h, size_t ws_bytes, cudaStream_t s);
cudaError_t launch_fastpfor_blocklane(int delta, const uint8_t* in, size_t in_bytes, uint32_t* out, size_t n,
                                      const uint64_t* index, const BlockMeta* meta, const uint32_t* pmeta,
                                      const uint2* umeta, WsHeader* h, size_t ws_bytes, cudaStream_t s);
cudaError_t launch_fastpfor_meta(const uint8_t* in, size_t in_bytes, size_t n, const uint64_t* index, BlockMeta* meta,
                                 uint32_t* pmeta, uint2* umeta, WsHeader* h, cudaStream_t s);
cudaError_t launch_fastpfor_two_kernel(int delta, const uint8_t* in, size_t in_bytes, uint32_t* out, size_t n,
                                       const uint64_t* index, BlockMeta* meta, uint32_t* pmeta, uint2* umeta,
                                       WsHeader* h, size_t ws_bytes, cudaStream_t s);
cudaError_t launch_fastpfor_index(const uint8_t* in, size_t in_bytes, size_t n, int fmt, uint64_t* index,
                                  WsHeader* h, cudaStream_t s);
cudaError_t launch_fastpfor_encode(int delta, int fmt, const uint32_t* x, size_t n, uint8_t* out, size_t out_cap,
                                   uint64_t* index, uint64_t* out_bytes, void* ws, size_t ws_bytes,
                                   cudaStream_t s);
cudaError_t launch_bp128_member(int delta, int fmt, const uint8_t* in, size_t in_bytes, size_t n,
                                const uint64_t* index, const uint32_t* b, size_t nb, uint32_t* bits,
                                unsigned long long* count, WsHeader* h, cudaStream_t s);
cudaError_t launch_sorted_member(const uint32_t* a, size_t n, const uint32_t* b, size_t nb, uint32_t* bits,
                                 unsigned long long* count, cudaStream_t s);

size_t fastpfor_encode_workspace_bytes(size_t n);
void set_bp128_warps(int w);
void set_bp128_prefetch(int on);
void set_bp128_blocklane(int on);
void set_bp128_blocklane_store(int v);
void set_bp128_blocklane_ctas(int v);
void set_bp128_blocklane_lead(int v);
void set_bp128_blocklane_sumw(int v);
void set_fastpfor_warps(int w);
void set_fastpfor_blocklane(int on);
void set_fastpfor_stream_warps(int w);
void set_fastpfor_chain_overlap(int v);

}  // namespace icx
