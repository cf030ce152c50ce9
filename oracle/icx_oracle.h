/*
 * Scalar CPU oracle for the decoding path of Lemire & Boytsov, "Decoding
 * billions of integers per second through vectorization" (arXiv 1209.2137).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this code; only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code, header, table or constant with the
 * CUDA path.
 *
 * Every routine is a literal, bit-by-bit restatement of the definitions in
 * the paper (section numbers given beside each entry point).  Where the paper
 * is silent, the reading used is named R1..R23; all are stated at the top
 * of icx_oracle.c.
 *
 * All integers are uint32; all delta arithmetic is modulo 2^32.
 * Return codes: 0 = ok, 3 = corrupt stream (same numbering as the library).
 */
#ifndef ICX_ORACLE_H
#define ICX_ORACLE_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_OK 0
#define ORC_ECORRUPT 3

/* Sec. 2: number of binary digits, ceil(log2(x+1)); orc_bitlen(0) == 0. */
int orc_bitlen(uint32_t x);

/* Sec. 4 (Figs. 4-5): tight LSB-first bit packing of `count` fields of `b`
 * bits into 32-bit little-endian words spread over `lanes` interleaved lanes
 * (lanes == 1 is the scalar layout of Fig. 4; lanes == 4 the vertical layout
 * of Figs. 6-7).  Integer i goes to lane i % lanes, field i / lanes.  Only
 * the low b bits of each value are stored (the mask of Sec. 4 / Sec. 6.3).
 * Output is ceil((count/lanes)*b/32) words per lane, word w of lane l at
 * byte 4*(lanes*w + l).  Unused bits are written as zero (R11). */
size_t orc_packed_bytes(size_t count, int lanes, int b);
void orc_pack(const uint32_t *in, size_t count, int lanes, int b, uint8_t *out);
void orc_unpack(const uint8_t *in, size_t count, int lanes, int b, uint32_t *out);

/* Sec. 3: differential coding.  stride 0 = identity, 1 = x_i - x_{i-1}
 * (x_0 := 0), 4 = x_i - x_{i-4} (first four kept). */
void orc_delta_encode(const uint32_t *x, size_t n, int stride, uint32_t *d);
void orc_delta_decode(const uint32_t *d, size_t n, int stride, uint32_t *x);

/* Sec. 2.4: Variable Byte, 7 data bits per byte, least significant group
 * first, high bit set only on the last byte of an integer (R13). */
size_t orc_vbyte_encode(const uint32_t *in, size_t count, uint8_t *out);
/* Returns bytes consumed, or (size_t)-1 if the stream is truncated or an
 * integer needs more than 32 bits / 5 bytes. */
size_t orc_vbyte_decode(const uint8_t *in, size_t in_bytes, size_t count, uint32_t *out);

/* Sec. 6.2: SIMD-BP128.  layout 0 = the paper's 4-lane vertical blocks,
 * layout 1 = the 32-lane word-interleaved variant W32 (R16).  delta is the
 * stride (0, 1, 4).  A stream of n integers holds ceil((n/128)/16)
 * metablocks followed by the Variable Byte tail of n % 128 integers (R1). */
size_t orc_bp128_max_bytes(size_t n);
size_t orc_bp128_encode(const uint32_t *x, size_t n, int delta, int layout, uint8_t *out);
int orc_bp128_decode(const uint8_t *in, size_t in_bytes, size_t n, int delta, int layout,
                     uint32_t *x);
/* Byte offset of every metablock plus the offset of the tail:
 * ceil((n/128)/16) + 1 entries. */
size_t orc_bp128_index_len(size_t n);
int orc_bp128_index(const uint8_t *in, size_t in_bytes, size_t n, int layout, uint64_t *index);

/* Sec. 5: FastPFOR width selection for one block of `len` values: b
 * minimises len*b + c_b*(8 + maxbits - b) over b in [0, maxbits], ties to
 * the larger b (R10).  `costs` (optional, maxbits+1 entries) receives the
 * cost of every candidate b. */
void orc_fastpfor_choose(const uint32_t *v, size_t len, int *b, int *maxbits, int *c,
                         uint64_t *costs);
/* Sec. 5: byte-array record of one block of `len` (<= 256) values and the
 * high parts of its exceptions, for the chosen b.  Returns record length. */
size_t orc_fastpfor_block_record(const uint32_t *v, size_t len, uint8_t *record,
                                 uint32_t *high, size_t *nhigh);

/* Sec. 5: SIMD-FastPFOR.  Pages of at most 512 blocks (65536 integers), then
 * the Variable Byte tail of n % 128 integers (R1, R14). */
size_t orc_fastpfor_max_bytes(size_t n);
size_t orc_fastpfor_encode(const uint32_t *x, size_t n, int delta, uint8_t *out);
int orc_fastpfor_decode(const uint8_t *in, size_t in_bytes, size_t n, int delta, uint32_t *x);
size_t orc_fastpfor_index_len(size_t n);
int orc_fastpfor_index(const uint8_t *in, size_t in_bytes, size_t n, uint64_t *index);
/* The same with a layout (R21): 0 = SIMD-FastPFOR (the calls above), 2 =
 * FastPFOR, the paper's scalar variant (Sec. 5): a block's low parts packed
 * in one lane as 4 groups of 32 integers, each exception array in groups of
 * 32 (padded to a multiple of 32 values), every other part of the page as
 * for SIMD-FastPFOR (16-byte aligned sections). */
size_t orc_fastpfor_encode_layout(const uint32_t *x, size_t n, int delta, int layout, uint8_t *out);
int orc_fastpfor_decode_layout(const uint8_t *in, size_t in_bytes, size_t n, int delta, int layout, uint32_t *x);
int orc_fastpfor_index_layout(const uint8_t *in, size_t in_bytes, size_t n, int layout, uint64_t *index);

/* Sec. 6.2, BP32 (the paper's scalar binary packing; R20): n/128 metablocks
 * of 128 integers, each a 32-bit little-endian descriptor (byte j = width
 * b_j of block j, j = 0..3) followed by blocks 0..3 of 32 integers, block j
 * packed LSB-first into b_j 32-bit words (one lane, orc_pack with lanes = 1);
 * then the n % 128 remaining integers in Variable Byte (R1).  The index has
 * an entry every 16 metablocks (2,048 integers) and one for the tail:
 * orc_bp128_index_len(n) entries. */
size_t orc_bp32_max_bytes(size_t n);
size_t orc_bp32_encode(const uint32_t *x, size_t n, int delta, uint8_t *out);
int orc_bp32_decode(const uint8_t *in, size_t in_bytes, size_t n, int delta, uint32_t *x);
int orc_bp32_index(const uint8_t *in, size_t in_bytes, size_t n, uint64_t *index);

/* Sec. 2 (Table 2), Simple-8b: 64-bit little-endian words, selector s in
 * bits 60..63 (R22); selectors 0 and 1 stand for 240 and 120 zeros (data
 * bits zero); selector s >= 2 packs count(s) integers of bits(s) bits, the
 * i-th at bits [i*b, (i+1)*b).  The encoder is greedy: each word takes the
 * smallest selector whose count(s) next integers all exist and fit (R23).
 * encode returns the number of words; decode returns 0 if the words hold
 * exactly `count` integers (written to out), else ORC_ECORRUPT. */
size_t orc_simple8b_encode(const uint32_t *v, size_t count, uint64_t *words);
int orc_simple8b_decode(const uint64_t *words, size_t nwords, size_t count, uint32_t *out);

/* Sec. 5, SimplePFOR (R22): the scalar FastPFOR page (R21) whose exception
 * high parts, in block order (positions ascending within a block), form one
 * Simple-8b stream: after the byte array, a word N (high parts), a word W
 * (Simple-8b words), zero padding to 16 bytes, the W words; the page padded
 * to 16 bytes.  The index has an entry per page and one for the tail. */
size_t orc_simplepfor_max_bytes(size_t n);
size_t orc_simplepfor_encode(const uint32_t *x, size_t n, int delta, uint8_t *out);
int orc_simplepfor_decode(const uint8_t *in, size_t in_bytes, size_t n, int delta, uint32_t *x);
int orc_simplepfor_index(const uint8_t *in, size_t in_bytes, size_t n, uint64_t *index);

/* Sec. 7 (decoding fused into its consumer; intersections of sorted
 * arrays): membership of the sorted query list b[0..nb) in the sorted list
 * a[0..na), by the textbook merge of two sorted arrays.  Bit j of
 * bits[0..ceil(nb/32)) (bit j%32 of word j/32) is set iff b[j] equals some
 * a[i]; bits past nb stay 0; *count = the number of set bits.  Both lists
 * must be non-decreasing. */
void orc_member_bits(const uint32_t *a, size_t na, const uint32_t *b, size_t nb, uint32_t *bits,
                     uint64_t *count);

#ifdef __cplusplus
}
#endif
#endif
