/*
 * icx -- GPU decoding of SIMD-BP128 / SIMD-FastPFOR integer streams with
 * differential decoding, after Lemire & Boytsov, "Decoding billions of
 * integers per second through vectorization" (arXiv 1209.2137).
 *
 * C ABI.  Every pointer named d_* is a device pointer (CUDA global memory) and
 * every h_* a host pointer; sizes are counts of the stated unit.  The caller
 * owns every buffer; no decode or encode call allocates memory.  Every call is
 * asynchronous on `stream` unless stated otherwise.
 *
 * Errors.  Argument errors (null pointer, bad enum, misaligned pointer, n
 * inconsistent with a size) are returned synchronously and nothing is
 * launched.  Errors that depend on the data (a width byte above 32, a
 * metablock or page that runs past in_bytes, an inconsistent FastPFOR page, a
 * truncated Variable Byte tail, a device wait that gave up) are recorded in a
 * status word inside the workspace; read it with icx_status_read after the
 * stream has reached the call.  A decode that records an error leaves the
 * affected outputs undefined but never reads or writes outside the buffers
 * it was given.
 *
 * Stream formats (integers are uint32, stored little endian; n is never
 * stored in a stream and is passed by the caller):
 *
 *  - SIMD-BP128 (Sec. 6.2): the n/128 full blocks of 128 integers are
 *    grouped 16 per metablock; a metablock is a 16-byte descriptor whose
 *    byte k is the bit width b_k of block k (unused bytes 0), followed by its
 *    blocks, each 16*b_k bytes in the 4-lane vertical layout of Sec. 4
 *    (Figs. 6-7: integer i of a block is field i/4 of lane i%4; word w of lane
 *    l sits at byte 16*w + 4*l).  The n % 128 remaining integers follow the
 *    last metablock in Variable Byte (Sec. 2.4: 7 bits per byte, low group
 *    first, high bit set on the last byte of each integer).
 *  - W32 (ICX_FMT_W32; not in the paper): the same descriptor, then the
 *    metablock's payload as 32 lanes interleaved word by word (word w of lane
 *    j at byte 128*w + 4*j).  Lane j = 4*g + l holds, block after block, the
 *    integers 128*k + 16*g + 4*m + l (m = 0..3) at width b_k; every lane is
 *    ceil(4*sum_k b_k / 32) words long.
 *  - SIMD-FastPFOR (Sec. 5): pages of up to 512 blocks (65536 integers),
 *    each page starting 16-byte aligned: a word giving the offset (in words)
 *    of the byte-array length word, zero padding to byte 16, the blocks'
 *    low b bits packed as above, the byte-array length (unpadded), the byte
 *    array (per block b, maxbits and, when maxbits > b, the exception count
 *    c and c positions; zero-padded to a multiple of 4), a 32-bit bitset whose
 *    bit d-1 flags a non-empty exception array of width d, then for each such
 *    d: its count, zero padding to 16 bytes, and its values packed at width d
 *    in the same vertical layout, padded to a multiple of 128 values.  The
 *    Variable Byte tail follows the last page.
 *  - Differential coding (Sec. 3): ICX_DELTA_1 decodes x_i = delta_i +
 *    x_{i-1}, ICX_DELTA_4 decodes x_i = delta_i + x_{i-4} (the vectorised
 *    variant); values before the start count as 0, arithmetic is modulo 2^32,
 *    and one chain runs over the whole array.
 *
 * An index (uint64 byte offsets of every metablock or page, plus the offset
 * of the Variable Byte tail) gives the decoders random access to the
 * metablocks; the paper's streams have no directory, so it is built once by
 * bp128_index / fastpfor_index or written by the encoders.
 */
#ifndef ICX_H
#define ICX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* The same type as cudaStream_t; 0 is the legacy default stream. */
typedef struct CUstream_st *icx_stream_t;

typedef enum {
    ICX_OK = 0,
    ICX_EINVAL = 1,   /* bad argument */
    ICX_EALIGN = 2,   /* a device pointer is not 16-byte aligned */
    ICX_ECORRUPT = 3, /* the stream does not follow the format */
    ICX_ENOSPC = 4,   /* an output or workspace buffer is too small */
    ICX_ECUDA = 5,    /* a CUDA runtime call failed */
    ICX_ETIMEOUT = 6  /* a device-side wait gave up (no progress for ~2 s) */
} icx_status;

typedef enum { ICX_DELTA_NONE = 0, ICX_DELTA_1 = 1, ICX_DELTA_4 = 4 } icx_delta;
/* Stream layouts of the SIMD-BP128 calls: the paper's SIMD-BP128 (4-lane
 * vertical blocks of 128 integers, 16 per metablock, Sec. 4 and 6.2), the
 * W32 variant (32 lanes interleaved word by word, not in the paper), and the
 * paper's scalar BP32 (Sec. 6.2): metablocks of 128 integers, each a 32-bit
 * little-endian descriptor (byte j = width of 32-integer block j) and four
 * blocks of 32 integers packed LSB-first in b_j words; the n % 128 last
 * integers in Variable Byte.  A BP32 index entry marks every 16th metablock
 * (2,048 integers), so the index lengths agree. */
typedef enum {
    ICX_FMT_PAPER = 0,
    ICX_FMT_W32 = 1,
    ICX_FMT_BP32 = 2,
    ICX_FMT_SCALAR = 2,
    ICX_FMT_SIMPLE8B = 3
} icx_layout;
/* The SIMD-FastPFOR calls take ICX_FMT_PAPER (SIMD-FastPFOR, Sec. 5: 4-lane
 * vertical packing, exception arrays in chunks of 128), ICX_FMT_SCALAR (the
 * paper's scalar FastPFOR: the same pages with a block's low parts packed
 * in one lane as 4 groups of 32 integers and each exception array packed in
 * one lane, padded to a multiple of 32 values) or ICX_FMT_SIMPLE8B (the
 * paper's SimplePFOR: the scalar FastPFOR page with the exception arrays
 * replaced by one Simple-8b stream of the page's exception high parts in
 * block order -- a word N, a word W, then W 64-bit words from the next
 * 16-byte boundary; Simple-8b per Table 2, selector in bits 60..63). */

/* ------------------------------------------------------------- sizes ---- */

/* Entries of a SIMD-BP128 index for n integers: ceil((n/128)/16) + 1. */
size_t icx_bp128_index_len(size_t n);
/* Entries of a SIMD-FastPFOR index for n integers: ceil((n/128)/512) + 1. */
size_t icx_fastpfor_index_len(size_t n);
/* Upper bound on the stream size in bytes. */
size_t icx_bp128_max_bytes(size_t n, icx_layout fmt);
size_t icx_fastpfor_max_bytes(size_t n);
/* Bytes of device workspace a decode, delta_decode or index call on n
 * integers needs (a 256-byte header plus look-back tile states). */
size_t icx_workspace_bytes(size_t n);

/* Where a decode of n integers puts its regions in a workspace of ws_bytes
 * bytes (a diagnostic; the decoders compute the same).  out[0] = the largest
 * length the workspace serves, out[1] = end of n's look-back states (from the
 * start), out[2] = start of the page parse's records, out[3] = start of the
 * SIMD-FastPFOR prepare kernel's records, out[4] = end of those plain regions,
 * out[5] = start of the tagged scratch of the block-per-lane decoders (to the
 * end).  Tagged regions (look-back states, the scratch) of any length the
 * workspace serves never overlap plain regions of any other.  ICX_EINVAL if
 * ws_bytes < icx_workspace_bytes(n) or out is NULL. */
icx_status icx_workspace_layout(size_t n, size_t ws_bytes, size_t *out);
/* Bytes of device workspace an encode call on n integers needs. */
size_t icx_encode_workspace_bytes(size_t n);

/* Zero a workspace before its first use (asynchronous on `stream`).  A
 * workspace resets itself at the end of every launch; one workspace must not
 * be used by two launches that can run at the same time.  Its look-back
 * states are tagged with a 30-bit launch number: a workspace that serves
 * more than 2^30 launches must be zeroed again before then. */
icx_status icx_workspace_init(void *d_workspace, size_t workspace_bytes, icx_stream_t stream);

/* Synchronises `stream`, copies the workspace's status word to *out and
 * clears it.  Returns ICX_ECUDA if the copy fails, else ICX_OK. */
icx_status icx_status_read(void *d_workspace, icx_stream_t stream, icx_status *out);

/* Sets how long a decode's device waits on values other CTAs publish (block
 * sums, look-back states) may see no progress before they give up with
 * ICX_ETIMEOUT, in microseconds; 0 restores the default (2 s).  Kept in the
 * workspace header (icx_workspace_init clears it), so it applies to later
 * launches on that workspace only.  A test aid for the timeout path: a wait
 * that runs out ends the kernel normally, with the status set.  ICX_EINVAL
 * for a null or too small workspace. */
icx_status icx_workspace_set_wait_limit(void *d_workspace, size_t workspace_bytes, unsigned usec,
                                        icx_stream_t stream);

/* ------------------------------------------------------------- index ---- */

/* Walks the metablocks of a SIMD-BP128 (fmt = PAPER), W32 or BP32 stream and
 * writes icx_bp128_index_len(n) byte offsets to d_index: entry m is the
 * offset of metablock m (BP32: of its 16m-th 128-integer metablock), the
 * last entry the offset of the Variable Byte tail (Sec. 6.2).  The walk is
 * sequential (each metablock's size comes from its descriptor). */
icx_status bp128_index(const uint8_t *d_in, size_t in_bytes, size_t n, icx_layout fmt,
                       uint64_t *d_index, void *d_workspace, size_t workspace_bytes,
                       icx_stream_t stream);
/* Same for the pages of a SIMD-FastPFOR (fmt = PAPER) or FastPFOR (fmt =
 * SCALAR) stream (Sec. 5). */
icx_status fastpfor_index(const uint8_t *d_in, size_t in_bytes, size_t n, icx_layout fmt,
                          uint64_t *d_index, void *d_workspace, size_t workspace_bytes,
                          icx_stream_t stream);

/* ------------------------------------------------------------ decode ---- */

/* Decodes n integers from the SIMD-BP128 (or W32, or BP32) stream d_in[0..in_bytes)
 * into d_out[0..n): bit unpacking (Sec. 4, Figs. 6-7), the Variable Byte
 * tail (Sec. 2.4) and differential decoding (Sec. 3) in one pass.
 * d_in and d_out must be 16-byte aligned; d_index is the stream's index
 * (icx_bp128_index_len(n) entries) and may be NULL only when the stream holds
 * at most one metablock (n < 17*128).
 * d_workspace holds workspace_bytes >= icx_workspace_bytes(n) bytes and was
 * initialised once with icx_workspace_init (else ICX_ENOSPC / undefined). */
icx_status bp128_decode(const uint8_t *d_in, size_t in_bytes, uint32_t *d_out, size_t n,
                        icx_delta delta, icx_layout fmt, const uint64_t *d_index,
                        void *d_workspace, size_t workspace_bytes, icx_stream_t stream);

/* Decodes n integers from the SIMD-FastPFOR (fmt = PAPER) or FastPFOR (fmt
 * = SCALAR) stream d_in: per page the exception arrays, the packed low bits
 * of every block, the patch out[p] |= high << b of every exception (Sec. 5),
 * then differential decoding.  d_index may be NULL only when the stream
 * holds at most one page (n < 513*128). */
icx_status fastpfor_decode(const uint8_t *d_in, size_t in_bytes, uint32_t *d_out, size_t n,
                           icx_delta delta, icx_layout fmt, const uint64_t *d_index,
                           void *d_workspace, size_t workspace_bytes, icx_stream_t stream);

/* Differential decoding alone (Sec. 3): d_out[i] = d_in[i] + d_out[i-s] for
 * s = 1 or 4 (ICX_DELTA_NONE copies).  d_out may equal d_in (in place); the
 * buffers must otherwise not overlap.  Both 16-byte aligned. */
icx_status delta_decode(const uint32_t *d_in, uint32_t *d_out, size_t n, icx_delta delta,
                        void *d_workspace, size_t workspace_bytes, icx_stream_t stream);

/* ---------------------------------------------- decode into a consumer -- */

/* Membership of a sorted query list in a compressed sorted list, with the
 * decode fused into the consumer (Sec. 7: an integrated decode, and
 * intersections of sorted arrays as the query that consumes the integers).
 * Let a[0..n) be the integers the SIMD-BP128 / W32 stream d_in decodes to
 * (arguments d_in .. d_index, d_workspace as for bp128_decode).  Bit j of
 * d_bits (bit j%32 of word j/32; ceil(nb/32) words) is set iff d_b[j] equals
 * some a[i], every other bit is cleared, and *d_count (device) receives the
 * number of set bits: the set bits select the intersection of a and b from
 * d_b in order.  The decoded integers are written nowhere.
 * Both a and d_b[0..nb) must be non-decreasing (sorted lists; duplicates are
 * allowed); otherwise the bits are unspecified, but every access stays
 * inside the given buffers.  fmt is ICX_FMT_PAPER or ICX_FMT_W32 (BP32:
 * ICX_EINVAL).  d_b and d_bits need 4-byte, d_count 8-byte,
 * d_in, d_index and the workspace 16-byte alignment.  Data errors of the
 * stream go to the workspace status word as for bp128_decode.  n == 0 or
 * nb == 0 clear the outputs and launch nothing else. */
icx_status bp128_intersect(const uint8_t *d_in, size_t in_bytes, size_t n, icx_delta delta,
                           icx_layout fmt, const uint64_t *d_index, const uint32_t *d_b, size_t nb,
                           uint32_t *d_bits, uint64_t *d_count, void *d_workspace,
                           size_t workspace_bytes, icx_stream_t stream);

/* The same consumer on a list that is already decoded: d_a[0..n)
 * (non-decreasing, 16-byte aligned) in place of the stream.  The unfused
 * path is bp128_decode followed by this call. */
icx_status sorted_intersect(const uint32_t *d_a, size_t n, const uint32_t *d_b, size_t nb,
                            uint32_t *d_bits, uint64_t *d_count, icx_stream_t stream);

/* Allocation-free variant of bp128_decode for callers that cannot allocate
 * device memory -- code that must not call cudaMalloc (an allocation-free
 * runtime, a host application that owns every device allocation, a plugin
 * whose host forbids allocations on its hot path).  The paper has no
 * counterpart: it is a calling convention of this library, not a step of
 * the method.
 *
 * Instead of a caller-provided workspace it uses one file-scope device array
 * of about 4 MiB inside the library, enough for n <= 2^28 integers; a larger
 * n returns ICX_ENOSPC without launching anything.  Every GPU that loads the
 * library holds that array until the process exits.  The caller still passes
 * the stream, its index (NULL allowed for a single metablock, as in
 * bp128_decode), the output and, optionally, d_status: a device word that
 * receives the call's data-dependent status (icx_status) once the stream
 * reaches it.  No allocation happens in this call, and it calls no
 * allocating library routine.
 *
 * The call looks up the array's device address (cudaGetSymbolAddress, with
 * the current device) each time, so it stays valid after a device reset
 * reloads the library's module.  The lookup is skipped while `stream` is
 * capturing; the address from the last call on that device is used then
 * (ICX_EINVAL if there was none).  All calls share the one array: two calls
 * that overlap on the GPU (other streams, other host threads) race and give
 * wrong results; serialise them.
 * Its look-back states are tagged with a 30-bit launch number; the call
 * zeroes the array again (an asynchronous memset on `stream`) every 2^29
 * calls on a device, before a tag could repeat. */
icx_status bp128_decode_static(const uint8_t *d_in, size_t in_bytes, uint32_t *d_out, size_t n,
                               icx_delta delta, icx_layout fmt, const uint64_t *d_index,
                               uint32_t *d_status, icx_stream_t stream);

/* ------------------------------------------------------------ encode ---- */

/* Differential coding (Sec. 3): d_out[i] = d_in[i] - d_in[i-s].  d_out must
 * not overlap d_in. */
icx_status delta_encode(const uint32_t *d_in, uint32_t *d_out, size_t n, icx_delta delta,
                        icx_stream_t stream);

/* Encodes d_x[0..n) as SIMD-BP128 / W32 / BP32 (widths are the largest bit
 * length of each block of deltas, Sec. 6.2) into d_out (capacity out_cap bytes, at
 * least icx_bp128_max_bytes(n, fmt)), writes the index to d_index and the
 * stream length in bytes to *d_out_bytes (device).  The bytes equal those of
 * the format definition above, bit for bit. */
icx_status bp128_encode(const uint32_t *d_x, size_t n, icx_delta delta, icx_layout fmt,
                        uint8_t *d_out, size_t out_cap, uint64_t *d_index,
                        uint64_t *d_out_bytes, void *d_encode_workspace,
                        size_t encode_workspace_bytes, icx_stream_t stream);

/* Encodes d_x[0..n) as SIMD-FastPFOR (fmt = PAPER) or FastPFOR (fmt =
 * SCALAR): per block the width minimising 128*b + c*(8 + maxbits - b), ties
 * to the larger b (Sec. 5). */
icx_status fastpfor_encode(const uint32_t *d_x, size_t n, icx_delta delta, icx_layout fmt, uint8_t *d_out,
                           size_t out_cap, uint64_t *d_index, uint64_t *d_out_bytes,
                           void *d_encode_workspace, size_t encode_workspace_bytes,
                           icx_stream_t stream);

/* Sets a launch parameter of the decoders (not part of the method):
 *   "bp128.warps_per_cta" = 4, 8 or 16 warps per CTA tile of the SIMD-BP128 /
 *       W32 decoder (0 = default: 4 for the paper layout, 8 for W32);
 *   "bp128.l2_prefetch" = 1 (default) / 0: each warp prefetches into L2 the
 *       metablock one grid of tiles ahead;
 *   "fastpfor.warps_per_cta" = 4 or 8 warps per CTA tile of the
 *       SIMD-FastPFOR decoder (0 = default: 4 for SIMD-FastPFOR stride 4, 8 otherwise);
 *   "bp128.blocklane" = 1 (default) / 0: decode the paper layout with
 *       stride 1 or 4 in two passes with one block per lane (0: the
 *       single-pass tile decoder with a chained look-back);
 *   "fastpfor.blocklane" = 2 (default): SIMD-FastPFOR with stride 1 or 4 by
 *       a kernel that parses, sums and prepares every block and one that
 *       streams the integers out; 1: one block-per-lane kernel after the page
 *       parse; 0: the tile decoder with a chained look-back (-1 = default);
 *   "fastpfor.stream_warps" = 4, 5 or 6 warps per CTA of the SIMD-FastPFOR
 *       stream kernel (0 = default: 4 for stride 1, 6 for stride 4);
 *   "fastpfor.chain_overlap" = bits 0, 1, 2: the prepare, scan, stream
 *       kernel of fastpfor.blocklane = 2 is launched as a programmatic
 *       dependent, so it is scheduled while the kernel before it ends (it
 *       waits for its predecessor before it reads or writes memory); 0: plain
 *       stream order (-1 = default, 6: the scan and stream kernels);
 *   "bp128.blocklane_store" = 0 (default: through shared memory, coalesced
 *       16-byte stores), 1 (32-byte stores per lane), 2 (16-byte stores per
 *       lane): output path of the two-pass decoders;
 *   "bp128.blocklane_ctas" = CTAs of their persistent grid (0 = all resident);
 *   "bp128.blocklane_lead" = pairs summed before the first decode task
 *       (0 = every pair with stride 4, two per resident warp with stride 1;
 *       at least 128);
 *   "bp128.blocklane_sum_warps" = warps per CTA that only sum (0 = every
 *       warp takes both kinds of task).
 * The bp128.blocklane_* settings apply to both two-pass decoders.
 * Takes effect for later launches; not thread safe against concurrent
 * launches.  ICX_EINVAL for an unknown key. */
icx_status icx_set_tuning(const char *key, int value);

/* Library version string. */
const char *icx_version(void);

/* ------------------------------------------------------------------------
 * Batched decoding: many independent arrays ("lists", e.g. posting lists)
 * of uneven length decoded by one CUDA graph launch.  No counterpart in the
 * paper, which decodes one array at a time; each list is decoded exactly as
 * bp128_decode / fastpfor_decode would decode it alone.
 *
 * The plan flattens every list into units (a SIMD-BP128 metablock, 16
 * blocks of a SIMD-FastPFOR page, or the Variable Byte tail) in a work-list;
 * one persistent kernel walks the work-list in tiles with a segmented
 * decoupled look-back (the running sum restarts at every list), after one
 * page-parse launch over every SIMD-FastPFOR page.  Both launches are
 * captured in one CUDA graph at plan creation.
 * ---------------------------------------------------------------------- */

typedef enum { ICX_CODEC_BP128 = 0, ICX_CODEC_FASTPFOR = 1 } icx_codec;

/* One list of a batch.  d_in: its stream (16-byte aligned, in_bytes long);
 * d_out: n integers (16-byte aligned, not overlapping any other list's
 * output); d_index: its metablock / page index as built by bp128_index,
 * fastpfor_index or the encoders; it may be NULL where the single-array call
 * allows it (at most one metablock / page).  delta: icx_delta; fmt:
 * icx_layout (SIMD-BP128: ICX_FMT_PAPER or ICX_FMT_W32; SIMD-FastPFOR:
 * ICX_FMT_PAPER; else ICX_EINVAL).  The caller owns all buffers
 * and keeps them alive and unmodified while the plan is in use. */
typedef struct {
    const uint8_t *d_in;
    size_t in_bytes;
    uint32_t *d_out;
    size_t n;
    const uint64_t *d_index;
    int codec;
    int delta;
    int fmt;
} icx_list_desc;

/* Launch parameters of a plan.  warps_per_cta: 4 or 8 (0 = tune); order:
 * work-list order of the lists, 0 = as given, 1 = longest first, 2 =
 * shortest first (-1 = tune); l2_prefetch: 1/0 (-1 = tune).  Any field left
 * to tune is chosen by timing the candidates on this plan's own data at
 * creation (its outputs are written meanwhile); the choice is cached in the
 * JSON file cache_path (NULL: $ICX_TUNE_CACHE, else no cache) under a key
 * made from the lists' lengths, codecs and deltas. */
typedef struct {
    int warps_per_cta;
    int order;
    int l2_prefetch;
    const char *cache_path;
} icx_tuning;

typedef struct icx_plan icx_plan;

/* Creates a plan on the current device: validates every list (arguments as
 * for the single-array calls; ICX_EINVAL / ICX_EALIGN name nothing, see
 * icx_plan_error_list), allocates the plan's device memory once (work-list,
 * page records, look-back states: about 8 bytes per 2048 integers plus 0.5
 * bytes per integer of SIMD-FastPFOR lists), tunes if asked (t NULL = tune
 * everything) and captures the CUDA graph.  Synchronous. */
icx_status icx_plan_create(const icx_list_desc *lists, size_t nlists, const icx_tuning *t, icx_plan **plan);

/* Index of the first list that made icx_plan_create fail, or -1. */
long long icx_plan_error_list(void);

/* Decodes every list: one graph launch on `stream`, asynchronous.  Data
 * errors go to the plan's status word (icx_plan_status). */
icx_status icx_plan_launch(icx_plan *plan, icx_stream_t stream);

/* The same lists decoded by one single-array call per list
 * (bp128_decode / fastpfor_decode, same kernels), all captured in one CUDA
 * graph at the first call: the baseline of the batched launch. */
icx_status icx_plan_launch_per_list(icx_plan *plan, icx_stream_t stream);

/* Synchronises `stream`, returns the first data error of the plan's
 * launches since the last call in *out and clears it. */
icx_status icx_plan_status(icx_plan *plan, icx_stream_t stream, icx_status *out);

/* The launch parameters in use (after tuning). */
icx_status icx_plan_tuning(const icx_plan *plan, icx_tuning *out);

/* Frees the plan's device memory and graphs. */
void icx_plan_destroy(icx_plan *plan);

/* ------------------------------------------------------------------------
 * Serving loop: a pool of lists resident in device memory (with their
 * indexes and, for SIMD-FastPFOR, page records parsed once at creation)
 * answers requests for several lists each.  No counterpart in the paper.
 *
 * A request is admitted, first come first served, when its decode buffers
 * (4 bytes per integer of its lists, each list 16-byte aligned) fit in the
 * budget; admitted requests are batched onto whichever of the server's
 * streams is free (continuous batching: a batch is launched as soon as a
 * stream is free, so batches overlap on the device) and decoded by one
 * launch of the batched kernel per batch.  A request completes when the
 * host observes its batch's completion event; its buffers are freed then.
 * ---------------------------------------------------------------------- */

typedef struct icx_server icx_server;

typedef struct {
    uint64_t requests;        /* completed */
    uint64_t ints;            /* integers decoded */
    uint64_t batches;         /* kernel launches */
    uint64_t max_batch;       /* most requests in one batch */
    uint64_t max_queue;       /* most requests waiting for admission */
    uint64_t peak_bytes;      /* most decode-buffer bytes in use */
    double wall_s;            /* first arrival to last completion */
    double queue_s;           /* summed over requests: arrival to its batch's issue */
    double service_s;         /* summed over batches: issue to completion seen by the host */
    double gpu_s;             /* summed over batches: GPU time, first copy to last kernel */
} icx_server_stats;

/* Creates a server over `pool` (d_out ignored; every other field as for a
 * plan) with `budget_bytes` of decode buffers allocated once and `streams`
 * (>= 2) streams.  warps_per_cta: 4 or 8.  Synchronous. */
icx_status icx_server_create(const icx_list_desc *pool, size_t nlists, size_t budget_bytes, int streams,
                             int warps_per_cta, icx_server **server);

/* Serves an open-loop request schedule and returns when every request has
 * completed.  Request r arrives arrival_ns[r] nanoseconds after the start
 * (non-decreasing) and asks for the lists ids[offs[r] .. offs[r+1]) (pool
 * indexes).  latency_ns[r] receives its completion time minus its arrival
 * time.  If results is not NULL, request r's lists are copied, decoded and
 * back to back without padding, to results + res_off[r] (host memory; slow,
 * for checks).  A request larger than the whole budget fails with
 * ICX_ENOSPC before anything runs; data errors are returned after the run. */
icx_status icx_server_run(icx_server *server, size_t nreq, const uint64_t *arrival_ns, const uint64_t *offs,
                          const uint32_t *ids, uint64_t *latency_ns, uint32_t *results, const uint64_t *res_off,
                          icx_server_stats *stats);

void icx_server_destroy(icx_server *server);

#ifdef __cplusplus
}
#endif
#endif
