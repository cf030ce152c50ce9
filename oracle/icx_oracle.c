/*
 * Scalar CPU oracle -- TEST INFRASTRUCTURE ONLY (see icx_oracle.h).
 *
 * Written for clarity, not speed: every field is moved one bit at a time, so
 * that each routine can be checked against the paper's definitions by eye.
 * Section / figure references are to Lemire & Boytsov, arXiv 1209.2137.
 *
 * Readings of points the paper leaves open:
 *  R1  n/128 full blocks are grouped 16 per metablock (the last may hold
 *      fewer, its descriptor stays 16 bytes with unused width bytes 0); the
 *      remaining n % 128 integers are Variable-Byte coded after the last
 *      metablock (or page), unpadded.
 *  R2  n is not stored in any stream; the caller passes it.
 *  R3  one delta chain per array: the 2^16 chunking of Sec. 3 / Sec. 6.2 is a
 *      decode-side cache device and does not restart the chain.
 *  R4  descriptor byte k is the width of block k of the metablock.
 *  R5  the first word of a FastPFOR page is the offset, in 32-bit words from
 *      the page start, of the byte-array length word.
 *  R6  maxbits is stored for every block, even when it equals b.
 *  R7  bit d-1 of the exception bitset flags the array of width d.
 *  R8  each exception array's 32-bit counter holds its unpadded length.
 *  R9  each packed section of a page starts on a 16-byte boundary (zero
 *      padding before the truncated blocks and before every packed array).
 *  R10 FastPFOR width-selection ties go to the larger b (fewer exceptions).
 *  R11 unused and padding bits are zero.
 *  R12 a block's width is max_i bitlen(x_i); the "OR of (x_i+1)" identity
 *      printed in Sec. 6.2 is false (x = {0,3}) and is not used.
 *  R13 the Variable Byte example of Sec. 2.4 is printed most significant
 *      byte first; stored order is least significant group first.
 *  R14 pages start 16-byte aligned: a page is zero-padded to a multiple of 16.
 *  R15 the byte-array length word holds the unpadded length of the array.
 *  R16 W32 (not in the paper): a metablock keeps the 16-byte descriptor; its
 *      payload is 32 lane bitstrings interleaved word by word (word w of lane
 *      j at byte 128*w + 4*j).  Lane j = 4*g + l holds, for every block k in
 *      order, the four integers 128*k + 16*g + 4*m + l (m = 0..3) at width
 *      b_k; the lane is ceil(4*sum(b_k)/32) words long.
 *  R17 a FastPFOR record with more than 128 exceptions is corrupt (a block
 *      holds 128 values).
 *  R18 the width choice costs an exception 8 + (maxbits - b) bits, with the
 *      block length (128) in place of the worked example's 16.
 *  R19 the decode fused into a consumer computes membership of a sorted
 *      query list in the decoded sorted list (bit j set iff b[j] occurs).
 *  R20 BP32: per 128 integers a little-endian descriptor word (byte j = width
 *      of 32-integer block j) and four one-lane blocks; the remainder in
 *      Variable Byte (as R1).
 *  R21 the scalar FastPFOR: the same pages with one-lane packing, exception
 *      arrays padded to 32 values, sections still 16-byte aligned.
 *  R22 SimplePFOR: the scalar page with one Simple-8b stream of the page's
 *      exception high parts (selector in bits 60..63) instead of the arrays.
 *  R23 the Simple-8b encoder takes a selector only when all of its count of
 *      next integers exist (no partial final word).
 */
#include "icx_oracle.h"

#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- bits -- */

int orc_bitlen(uint32_t x) {
    /* Sec. 2: "the binary notation requires ceil(log2(x+1)) bits". */
    int digits = 0;
    while (x != 0) {
        digits += 1;
        x >>= 1;
    }
    return digits;
}

/* Byte and bit of bit `i` of lane `l` when `lanes` lanes are interleaved word
 * by word: lane word w sits at byte 4*(lanes*w + l), little endian. */
static size_t lane_byte(int lanes, int l, size_t i) {
    size_t w = i / 32, j = i % 32;
    return 4 * ((size_t)lanes * w + (size_t)l) + j / 8;
}

static int lane_get_bit(const uint8_t *base, int lanes, int l, size_t i) {
    return (base[lane_byte(lanes, l, i)] >> (i % 8)) & 1;
}

static void lane_set_bit(uint8_t *base, int lanes, int l, size_t i, int bit) {
    size_t byte = lane_byte(lanes, l, i);
    if (bit)
        base[byte] = (uint8_t)(base[byte] | (1u << (i % 8)));
    else
        base[byte] = (uint8_t)(base[byte] & ~(1u << (i % 8)));
}

/* Store the low `b` bits of v, LSB first, at bit `pos` of lane `l`. */
static void put_field(uint8_t *base, int lanes, int l, size_t pos, uint32_t v, int b) {
    for (int k = 0; k < b; ++k) lane_set_bit(base, lanes, l, pos + (size_t)k, (int)((v >> k) & 1u));
}

static uint32_t get_field(const uint8_t *base, int lanes, int l, size_t pos, int b) {
    uint32_t v = 0;
    for (int k = 0; k < b; ++k) v |= (uint32_t)lane_get_bit(base, lanes, l, pos + (size_t)k) << k;
    return v;
}

size_t orc_packed_bytes(size_t count, int lanes, int b) {
    size_t per_lane = count / (size_t)lanes;
    size_t words = (per_lane * (size_t)b + 31) / 32;
    return words * 4 * (size_t)lanes;
}

void orc_pack(const uint32_t *in, size_t count, int lanes, int b, uint8_t *out) {
    memset(out, 0, orc_packed_bytes(count, lanes, b));
    for (size_t i = 0; i < count; ++i) {
        int l = (int)(i % (size_t)lanes);
        size_t field = i / (size_t)lanes;
        put_field(out, lanes, l, field * (size_t)b, in[i], b);
    }
}

void orc_unpack(const uint8_t *in, size_t count, int lanes, int b, uint32_t *out) {
    for (size_t i = 0; i < count; ++i) {
        int l = (int)(i % (size_t)lanes);
        size_t field = i / (size_t)lanes;
        out[i] = get_field(in, lanes, l, field * (size_t)b, b);
    }
}

/* --------------------------------------------------------------- delta -- */

void orc_delta_encode(const uint32_t *x, size_t n, int stride, uint32_t *d) {
    /* Sec. 3: delta_i = x_i - x_{i-s}; elements before the start count as 0,
     * so the first s values are kept as they are. */
    for (size_t i = 0; i < n; ++i) {
        uint32_t prev = 0;
        if (stride > 0 && i >= (size_t)stride) prev = x[i - (size_t)stride];
        d[i] = x[i] - prev;
    }
}

void orc_delta_decode(const uint32_t *d, size_t n, int stride, uint32_t *x) {
    /* Sec. 3: x_i = delta_i + x_{i-s}, in increasing index order. */
    for (size_t i = 0; i < n; ++i) {
        uint32_t prev = 0;
        if (stride > 0 && i >= (size_t)stride) prev = x[i - (size_t)stride];
        x[i] = d[i] + prev;
    }
}

/* --------------------------------------------------------------- vbyte -- */

size_t orc_vbyte_encode(const uint32_t *in, size_t count, uint8_t *out) {
    size_t pos = 0;
    for (size_t i = 0; i < count; ++i) {
        uint32_t v = in[i];
        /* seven data bits per byte, low group first; the eighth bit is one
         * only on the last byte of the integer (Sec. 2.4). */
        while (v >= 128) {
            out[pos++] = (uint8_t)(v & 127u);
            v >>= 7;
        }
        out[pos++] = (uint8_t)(v | 128u);
    }
    return pos;
}

size_t orc_vbyte_decode(const uint8_t *in, size_t in_bytes, size_t count, uint32_t *out) {
    size_t pos = 0;
    for (size_t i = 0; i < count; ++i) {
        uint64_t v = 0;
        int shift = 0;
        for (;;) {
            if (pos >= in_bytes || shift > 28) return (size_t)-1;
            uint8_t byte = in[pos++];
            v |= (uint64_t)(byte & 127u) << shift;
            shift += 7;
            if (byte & 128u) break;
        }
        if (v > 0xFFFFFFFFull) return (size_t)-1;
        out[i] = (uint32_t)v;
    }
    return pos;
}

/* --------------------------------------------------------------- bp128 -- */

static void put_le32(uint8_t *p, uint32_t v) {
    p[0] = (uint8_t)(v & 255u);
    p[1] = (uint8_t)((v >> 8) & 255u);
    p[2] = (uint8_t)((v >> 16) & 255u);
    p[3] = (uint8_t)((v >> 24) & 255u);
}

static uint32_t get_le32(const uint8_t *p) {
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

static int block_width(const uint32_t *v, size_t len) {
    /* R12: the width is the largest bitlen of the block. */
    int w = 0;
    for (size_t i = 0; i < len; ++i) {
        int bl = orc_bitlen(v[i]);
        if (bl > w) w = bl;
    }
    return w;
}

/* W32 lane j = 4*g + l holds integers 16*g + 4*m + l of every block (R16). */
static size_t w32_position(int j, int m) { return (size_t)(16 * (j / 4) + 4 * m + (j % 4)); }

size_t orc_bp128_max_bytes(size_t n) {
    size_t nb = n / 128, meta = (nb + 15) / 16;
    return meta * 16 + nb * 512 + meta * 128 + (n % 128) * 5 + 16;
}

size_t orc_bp128_index_len(size_t n) { return (n / 128 + 15) / 16 + 1; }

size_t orc_bp128_encode(const uint32_t *x, size_t n, int delta, int layout, uint8_t *out) {
    uint32_t *d = (uint32_t *)malloc((n ? n : 1) * sizeof(uint32_t));
    orc_delta_encode(x, n, delta, d);
    size_t nb = n / 128, meta = (nb + 15) / 16, pos = 0;
    for (size_t m = 0; m < meta; ++m) {
        size_t first = 16 * m, k_count = nb - first < 16 ? nb - first : 16;
        uint8_t *desc = out + pos;
        memset(desc, 0, 16);
        int b[16] = {0};
        for (size_t k = 0; k < k_count; ++k) {
            b[k] = block_width(d + 128 * (first + k), 128);
            desc[k] = (uint8_t)b[k]; /* R4 */
        }
        pos += 16;
        if (layout == 0) {
            for (size_t k = 0; k < k_count; ++k) {
                orc_pack(d + 128 * (first + k), 128, 4, b[k], out + pos);
                pos += 16 * (size_t)b[k];
            }
        } else {
            size_t sum_b = 0;
            for (size_t k = 0; k < k_count; ++k) sum_b += (size_t)b[k];
            size_t words = (4 * sum_b + 31) / 32, bytes = 128 * words;
            memset(out + pos, 0, bytes);
            size_t start = 0; /* bit offset of block k inside every lane */
            for (size_t k = 0; k < k_count; ++k) {
                const uint32_t *blk = d + 128 * (first + k);
                for (int j = 0; j < 32; ++j)
                    for (int mm = 0; mm < 4; ++mm)
                        put_field(out + pos, 32, j, start + (size_t)(mm * b[k]), blk[w32_position(j, mm)], b[k]);
                start += 4 * (size_t)b[k];
            }
            pos += bytes;
        }
    }
    pos += orc_vbyte_encode(d + 128 * nb, n - 128 * nb, out + pos);
    free(d);
    return pos;
}

/* Walks one metablock starting at `pos`; returns its size or 0 if corrupt. */
static size_t bp128_meta_size(const uint8_t *in, size_t in_bytes, size_t pos, size_t k_count, int layout) {
    if (pos + 16 > in_bytes) return 0;
    size_t sum_b = 0;
    for (size_t k = 0; k < k_count; ++k) {
        if (in[pos + k] > 32) return 0;
        sum_b += in[pos + k];
    }
    size_t size = layout == 0 ? 16 + 16 * sum_b : 16 + 128 * ((4 * sum_b + 31) / 32);
    if (pos + size > in_bytes) return 0;
    return size;
}

int orc_bp128_index(const uint8_t *in, size_t in_bytes, size_t n, int layout, uint64_t *index) {
    size_t nb = n / 128, meta = (nb + 15) / 16, pos = 0;
    for (size_t m = 0; m < meta; ++m) {
        size_t k_count = nb - 16 * m < 16 ? nb - 16 * m : 16;
        size_t size = bp128_meta_size(in, in_bytes, pos, k_count, layout);
        if (size == 0) return ORC_ECORRUPT;
        index[m] = pos;
        pos += size;
    }
    index[meta] = pos;
    return ORC_OK;
}

int orc_bp128_decode(const uint8_t *in, size_t in_bytes, size_t n, int delta, int layout, uint32_t *x) {
    uint32_t *d = (uint32_t *)malloc((n ? n : 1) * sizeof(uint32_t));
    size_t nb = n / 128, meta = (nb + 15) / 16, pos = 0;
    int rc = ORC_OK;
    for (size_t m = 0; m < meta && rc == ORC_OK; ++m) {
        size_t first = 16 * m, k_count = nb - first < 16 ? nb - first : 16;
        size_t size = bp128_meta_size(in, in_bytes, pos, k_count, layout);
        if (size == 0) {
            rc = ORC_ECORRUPT;
            break;
        }
        const uint8_t *desc = in + pos, *payload = in + pos + 16;
        if (layout == 0) {
            size_t off = 0;
            for (size_t k = 0; k < k_count; ++k) {
                orc_unpack(payload + off, 128, 4, desc[k], d + 128 * (first + k));
                off += 16 * (size_t)desc[k];
            }
        } else {
            size_t start = 0;
            for (size_t k = 0; k < k_count; ++k) {
                uint32_t *blk = d + 128 * (first + k);
                for (int j = 0; j < 32; ++j)
                    for (int mm = 0; mm < 4; ++mm)
                        blk[w32_position(j, mm)] = get_field(payload, 32, j, start + (size_t)(mm * desc[k]), desc[k]);
                start += 4 * (size_t)desc[k];
            }
        }
        pos += size;
    }
    if (rc == ORC_OK) {
        size_t used = orc_vbyte_decode(in + pos, in_bytes - pos, n - 128 * nb, d + 128 * nb);
        if (used == (size_t)-1) rc = ORC_ECORRUPT;
    }
    if (rc == ORC_OK) orc_delta_decode(d, n, delta, x);
    free(d);
    return rc;
}

/* ------------------------------------------------------------ fastpfor -- */

void orc_fastpfor_choose(const uint32_t *v, size_t len, int *b_out, int *maxbits_out, int *c_out,
                         uint64_t *costs) {
    /* Sec. 5: histogram of bit widths (33 bins), then try every b. */
    size_t hist[33] = {0};
    for (size_t i = 0; i < len; ++i) hist[orc_bitlen(v[i])] += 1;
    int maxbits = 0;
    for (int w = 0; w <= 32; ++w)
        if (hist[w] > 0) maxbits = w;
    int best_b = maxbits;
    uint64_t best_cost = (uint64_t)-1;
    size_t best_c = 0;
    for (int b = 0; b <= maxbits; ++b) {
        size_t c = 0; /* values that need more than b bits */
        for (int w = b + 1; w <= 32; ++w) c += hist[w];
        uint64_t cost = (uint64_t)len * (uint64_t)b + (uint64_t)c * (uint64_t)(8 + maxbits - b);
        if (costs) costs[b] = cost;
        if (cost <= best_cost) { /* R10: a tie moves to the larger b */
            best_cost = cost;
            best_b = b;
            best_c = c;
        }
    }
    *b_out = best_b;
    *maxbits_out = maxbits;
    *c_out = (int)best_c;
}

size_t orc_fastpfor_block_record(const uint32_t *v, size_t len, uint8_t *record, uint32_t *high,
                                 size_t *nhigh) {
    int b, maxbits, c;
    orc_fastpfor_choose(v, len, &b, &maxbits, &c, NULL);
    size_t r = 0;
    record[r++] = (uint8_t)b;
    record[r++] = (uint8_t)maxbits; /* R6 */
    *nhigh = 0;
    if (maxbits > b) {
        record[r++] = (uint8_t)c;
        for (size_t i = 0; i < len; ++i) {
            if (orc_bitlen(v[i]) > b) {
                record[r++] = (uint8_t)i;
                high[(*nhigh)++] = v[i] >> b; /* b < maxbits <= 32 here */
            }
        }
    }
    return r;
}

size_t orc_fastpfor_max_bytes(size_t n) {
    size_t nb = n / 128, pages = (nb + 511) / 512;
    /* per page: 16-byte header, length word, bitset and end padding; per
     * block <= 512 packed bytes, <= 131 record bytes and <= 128 exceptions of
     * <= 4 bytes; per exception array a count, <= 15 padding bytes and <= one
     * chunk of padding values (16*d bytes). */
    return pages * (16 + 4 + 3 + 4 + 15 + 32 * (4 + 15 + 16 * 32)) + nb * (512 + 131 + 512) +
           (n % 128) * 5 + 16;
}

size_t orc_fastpfor_index_len(size_t n) { return (n / 128 + 511) / 512 + 1; }

static size_t pad_to(size_t x, size_t a) { return (x + a - 1) / a * a; }

static uint32_t low_bits(uint32_t v, int b) { return b >= 32 ? v : (v & ((1u << b) - 1u)); }

/* Packing of a page's bit-packed sections (R21): layout 0 = SIMD-FastPFOR
 * (4 interleaved lanes, exception arrays in chunks of 128), layout 2 =
 * FastPFOR (one lane: a block's 128 low parts as 4 groups of 32, exception
 * arrays in groups of 32).  Everything else is shared. */
static int fp_lanes(int layout) { return layout == 2 ? 1 : 4; }
static size_t fp_chunk(int layout) { return layout == 2 ? 32 : 128; }

/* Encode `k_count` blocks of 128 values into one page at `out`. */
static size_t fastpfor_page_encode(const uint32_t *v, size_t k_count, int layout, uint8_t *out) {
    int *b = (int *)malloc(k_count * sizeof(int));
    uint8_t *bytes = (uint8_t *)malloc(k_count * 131 + 4);
    uint32_t *exc[33];
    size_t exc_n[33];
    for (int w = 0; w <= 32; ++w) {
        exc[w] = (uint32_t *)malloc((k_count * 128 + 1) * sizeof(uint32_t));
        exc_n[w] = 0;
    }
    size_t L = 0;
    for (size_t k = 0; k < k_count; ++k) {
        uint32_t high[128];
        size_t nh = 0;
        const uint32_t *blk = v + 128 * k;
        size_t r = orc_fastpfor_block_record(blk, 128, bytes + L, high, &nh);
        b[k] = bytes[L];
        int maxbits = bytes[L + 1];
        for (size_t e = 0; e < nh; ++e) {
            int dd = maxbits - b[k];
            exc[dd][exc_n[dd]++] = high[e];
        }
        L += r;
    }
    /* Header word, then zero padding up to byte 16 (R9). */
    size_t pos = 16;
    memset(out, 0, 16);
    uint32_t masked[128];
    for (size_t k = 0; k < k_count; ++k) {
        for (int i = 0; i < 128; ++i) masked[i] = low_bits(v[128 * k + (size_t)i], b[k]);
        orc_pack(masked, 128, fp_lanes(layout), b[k], out + pos); /* 16 * b bytes either way */
        pos += 16 * (size_t)b[k];
    }
    put_le32(out, (uint32_t)(pos / 4)); /* R5 */
    put_le32(out + pos, (uint32_t)L);   /* R15 */
    pos += 4;
    memcpy(out + pos, bytes, L);
    memset(out + pos + L, 0, pad_to(L, 4) - L);
    pos += pad_to(L, 4);
    uint32_t bitset = 0;
    for (int dd = 1; dd <= 32; ++dd)
        if (exc_n[dd] > 0) bitset |= 1u << (dd - 1); /* R7 */
    put_le32(out + pos, bitset);
    pos += 4;
    for (int dd = 1; dd <= 32; ++dd) {
        if (exc_n[dd] == 0) continue;
        put_le32(out + pos, (uint32_t)exc_n[dd]); /* R8 */
        pos += 4;
        size_t aligned = pad_to(pos, 16); /* R9 */
        memset(out + pos, 0, aligned - pos);
        pos = aligned;
        const size_t chunk = fp_chunk(layout);
        size_t chunks = (exc_n[dd] + chunk - 1) / chunk;
        for (size_t ch = 0; ch < chunks; ++ch) {
            uint32_t vals[128];
            for (size_t i = 0; i < chunk; ++i) {
                size_t q = chunk * ch + i;
                vals[i] = q < exc_n[dd] ? exc[dd][q] : 0u;
            }
            orc_pack(vals, chunk, fp_lanes(layout), dd, out + pos);
            pos += chunk / 8 * (size_t)dd; /* chunk values of dd bits */
        }
    }
    size_t end = pad_to(pos, 16); /* R14 */
    memset(out + pos, 0, end - pos);
    for (int w = 0; w <= 32; ++w) free(exc[w]);
    free(bytes);
    free(b);
    return end;
}

/* Walk one page: fills `v` (k_count*128 values) if v != NULL; returns the page
 * size, or 0 if the page is corrupt or runs past `avail`. */
static size_t fastpfor_page_decode(const uint8_t *page, size_t avail, size_t k_count, int layout, uint32_t *v) {
    const size_t chunk = fp_chunk(layout);
    if (avail < 16) return 0;
    size_t len_at = 4 * (size_t)get_le32(page);
    if (len_at < 16 || len_at + 4 > avail) return 0;
    size_t L = get_le32(page + len_at);
    size_t bytes_at = len_at + 4;
    if (bytes_at + pad_to(L, 4) + 4 > avail) return 0;
    const uint8_t *bytes = page + bytes_at;
    size_t pos = bytes_at + pad_to(L, 4);
    uint32_t bitset = get_le32(page + pos);
    pos += 4;
    const uint8_t *arr[33] = {0};
    size_t arr_n[33] = {0};
    for (int dd = 1; dd <= 32; ++dd) {
        if (!((bitset >> (dd - 1)) & 1u)) continue;
        if (pos + 4 > avail) return 0;
        arr_n[dd] = get_le32(page + pos);
        pos = pad_to(pos + 4, 16);
        size_t size = chunk / 8 * (size_t)dd * ((arr_n[dd] + chunk - 1) / chunk);
        if (pos + size > avail) return 0;
        arr[dd] = page + pos;
        pos += size;
    }
    size_t end = pad_to(pos, 16);
    if (end > avail) return 0;
    size_t packed = 16, r = 0, cursor[33] = {0};
    for (size_t k = 0; k < k_count; ++k) {
        if (r + 2 > L) return 0;
        int b = bytes[r], maxbits = bytes[r + 1];
        r += 2;
        if (b > 32 || maxbits > 32 || maxbits < b) return 0;
        if (packed + 16 * (size_t)b > len_at) return 0;
        if (v) orc_unpack(page + packed, 128, fp_lanes(layout), b, v + 128 * k);
        packed += 16 * (size_t)b;
        if (maxbits > b) {
            if (r + 1 > L) return 0;
            size_t c = bytes[r++];
            if (c > 128 || r + c > L) return 0; /* a block has 128 values */
            int dd = maxbits - b;
            if (cursor[dd] + c > arr_n[dd]) return 0;
            for (size_t e = 0; e < c; ++e) {
                size_t p = bytes[r + e];
                if (p >= 128) return 0;
                size_t q = cursor[dd] + e;
                /* element q of a vertically packed array: chunk q/128, then
                 * the ordinary 4-lane position inside that chunk; of a
                 * one-lane array: field q of the single bit string. */
                uint32_t hi = layout == 2 ? get_field(arr[dd], 1, 0, q * (size_t)dd, dd)
                                          : get_field(arr[dd] + 16 * (size_t)dd * (q / 128), 4, (int)(q % 4),
                                                      ((q % 128) / 4) * (size_t)dd, dd);
                if (v) v[128 * k + p] |= hi << b; /* b < 32 here */
            }
            cursor[dd] += c;
            r += c;
        }
    }
    if (packed != len_at) return 0;
    return end;
}

size_t orc_fastpfor_encode_layout(const uint32_t *x, size_t n, int delta, int layout, uint8_t *out) {
    uint32_t *d = (uint32_t *)malloc((n ? n : 1) * sizeof(uint32_t));
    orc_delta_encode(x, n, delta, d);
    size_t nb = n / 128, pages = (nb + 511) / 512, pos = 0;
    for (size_t p = 0; p < pages; ++p) {
        size_t k_count = nb - 512 * p < 512 ? nb - 512 * p : 512;
        pos += fastpfor_page_encode(d + 65536 * p, k_count, layout, out + pos);
    }
    pos += orc_vbyte_encode(d + 128 * nb, n - 128 * nb, out + pos);
    free(d);
    return pos;
}

int orc_fastpfor_index_layout(const uint8_t *in, size_t in_bytes, size_t n, int layout, uint64_t *index) {
    size_t nb = n / 128, pages = (nb + 511) / 512, pos = 0;
    for (size_t p = 0; p < pages; ++p) {
        size_t k_count = nb - 512 * p < 512 ? nb - 512 * p : 512;
        size_t size = fastpfor_page_decode(in + pos, in_bytes - pos, k_count, layout, NULL);
        if (size == 0) return ORC_ECORRUPT;
        index[p] = pos;
        pos += size;
    }
    index[pages] = pos;
    return ORC_OK;
}

int orc_fastpfor_decode_layout(const uint8_t *in, size_t in_bytes, size_t n, int delta, int layout, uint32_t *x) {
    uint32_t *d = (uint32_t *)malloc((n ? n : 1) * sizeof(uint32_t));
    size_t nb = n / 128, pages = (nb + 511) / 512, pos = 0;
    int rc = ORC_OK;
    for (size_t p = 0; p < pages; ++p) {
        size_t k_count = nb - 512 * p < 512 ? nb - 512 * p : 512;
        size_t size = fastpfor_page_decode(in + pos, in_bytes - pos, k_count, layout, d + 65536 * p);
        if (size == 0) {
            rc = ORC_ECORRUPT;
            break;
        }
        pos += size;
    }
    if (rc == ORC_OK) {
        size_t used = orc_vbyte_decode(in + pos, in_bytes - pos, n - 128 * nb, d + 128 * nb);
        if (used == (size_t)-1) rc = ORC_ECORRUPT;
    }
    if (rc == ORC_OK) orc_delta_decode(d, n, delta, x);
    free(d);
    return rc;
}

size_t orc_fastpfor_encode(const uint32_t *x, size_t n, int delta, uint8_t *out) {
    return orc_fastpfor_encode_layout(x, n, delta, 0, out);
}

int orc_fastpfor_index(const uint8_t *in, size_t in_bytes, size_t n, uint64_t *index) {
    return orc_fastpfor_index_layout(in, in_bytes, n, 0, index);
}

int orc_fastpfor_decode(const uint8_t *in, size_t in_bytes, size_t n, int delta, uint32_t *x) {
    return orc_fastpfor_decode_layout(in, in_bytes, n, delta, 0, x);
}

/* ------------------------------------------------------- Sec. 6.2: BP32 */

size_t orc_bp32_max_bytes(size_t n) { return (n / 128) * (4 + 4 * 4 * 32) + 5 * (n % 128) + 16; }

size_t orc_bp32_encode(const uint32_t *x, size_t n, int delta, uint8_t *out) {
    uint32_t *d = (uint32_t *)malloc((n ? n : 1) * sizeof(uint32_t));
    orc_delta_encode(x, n, delta, d);
    size_t meta = n / 128, pos = 0;
    for (size_t m = 0; m < meta; ++m) {
        uint8_t *desc = out + pos;
        int b[4];
        for (int j = 0; j < 4; ++j) {
            b[j] = block_width(d + 128 * m + 32 * j, 32);
            desc[j] = (uint8_t)b[j]; /* byte j of the little-endian descriptor word */
        }
        pos += 4;
        for (int j = 0; j < 4; ++j) {
            orc_pack(d + 128 * m + 32 * j, 32, 1, b[j], out + pos);
            pos += 4 * (size_t)b[j];
        }
    }
    pos += orc_vbyte_encode(d + 128 * meta, n - 128 * meta, out + pos);
    free(d);
    return pos;
}

/* Size of the BP32 metablock at `pos`, or 0 if it is corrupt or truncated. */
static size_t bp32_meta_size(const uint8_t *in, size_t in_bytes, size_t pos) {
    if (pos + 4 > in_bytes) return 0;
    size_t size = 4;
    for (int j = 0; j < 4; ++j) {
        if (in[pos + j] > 32) return 0;
        size += 4 * (size_t)in[pos + j];
    }
    return pos + size <= in_bytes ? size : 0;
}

int orc_bp32_index(const uint8_t *in, size_t in_bytes, size_t n, uint64_t *index) {
    size_t meta = n / 128, pos = 0;
    for (size_t m = 0; m < meta; ++m) {
        size_t size = bp32_meta_size(in, in_bytes, pos);
        if (size == 0) return ORC_ECORRUPT;
        if (m % 16 == 0) index[m / 16] = pos;
        pos += size;
    }
    index[(meta + 15) / 16] = pos;
    return ORC_OK;
}

int orc_bp32_decode(const uint8_t *in, size_t in_bytes, size_t n, int delta, uint32_t *x) {
    uint32_t *d = (uint32_t *)malloc((n ? n : 1) * sizeof(uint32_t));
    size_t meta = n / 128, pos = 0;
    int rc = ORC_OK;
    for (size_t m = 0; m < meta; ++m) {
        size_t size = bp32_meta_size(in, in_bytes, pos);
        if (size == 0) {
            rc = ORC_ECORRUPT;
            break;
        }
        size_t off = pos + 4;
        for (int j = 0; j < 4; ++j) {
            orc_unpack(in + off, 32, 1, in[pos + j], d + 128 * m + 32 * j);
            off += 4 * (size_t)in[pos + j];
        }
        pos += size;
    }
    if (rc == ORC_OK) {
        size_t used = orc_vbyte_decode(in + pos, in_bytes - pos, n - 128 * meta, d + 128 * meta);
        if (used == (size_t)-1) rc = ORC_ECORRUPT;
    }
    if (rc == ORC_OK) orc_delta_decode(d, n, delta, x);
    free(d);
    return rc;
}

/* ------------------------------------------------- Sec. 2: Simple-8b -- */

static const size_t s8_count[16] = {240, 120, 60, 30, 20, 15, 12, 10, 8, 7, 6, 5, 4, 3, 2, 1};
static const int s8_bits[16] = {0, 0, 1, 2, 3, 4, 5, 6, 7, 8, 10, 12, 15, 20, 30, 60};

size_t orc_simple8b_encode(const uint32_t *v, size_t count, uint64_t *words) {
    size_t p = 0, w = 0;
    while (p < count) {
        int sel = 15;
        for (int s = 0; s < 16; ++s) {
            if (p + s8_count[s] > count) continue; /* R23: the whole count must exist */
            int ok = 1;
            for (size_t i = 0; i < s8_count[s] && ok; ++i)
                if (s8_bits[s] < 32 && (uint64_t)v[p + i] >= ((uint64_t)1 << s8_bits[s])) ok = 0;
            if (ok) {
                sel = s;
                break;
            }
        }
        uint64_t word = (uint64_t)sel << 60;
        if (sel >= 2)
            for (size_t i = 0; i < s8_count[sel]; ++i) word |= (uint64_t)v[p + i] << (i * (size_t)s8_bits[sel]);
        words[w++] = word;
        p += s8_count[sel];
    }
    return w;
}

int orc_simple8b_decode(const uint64_t *words, size_t nwords, size_t count, uint32_t *out) {
    size_t p = 0;
    for (size_t w = 0; w < nwords; ++w) {
        const int sel = (int)(words[w] >> 60);
        const size_t c = s8_count[sel];
        if (p + c > count) return ORC_ECORRUPT;
        for (size_t i = 0; i < c; ++i) {
            uint64_t x = sel < 2 ? 0 : (words[w] >> (i * (size_t)s8_bits[sel])) & (((uint64_t)1 << s8_bits[sel]) - 1);
            if (x >> 32) return ORC_ECORRUPT; /* the stream holds 32-bit integers */
            out[p + i] = (uint32_t)x;
        }
        p += c;
    }
    return p == count ? ORC_OK : ORC_ECORRUPT;
}

/* ------------------------------------------------- Sec. 5: SimplePFOR -- */

size_t orc_simplepfor_max_bytes(size_t n) {
    size_t nb = n / 128, pages = (nb + 511) / 512;
    /* per page: header, length, N, W, paddings; per block <= 512 packed
     * bytes, <= 131 record bytes, <= 128 high parts of one word each */
    return pages * (16 + 4 + 3 + 8 + 15 + 15) + nb * (512 + 131 + 128 * 8) + (n % 128) * 5 + 16;
}

static size_t simplepfor_page_encode(const uint32_t *v, size_t k_count, uint8_t *out) {
    uint8_t *bytes = (uint8_t *)malloc(k_count * 131 + 4);
    uint32_t *high = (uint32_t *)malloc((k_count * 128 + 1) * sizeof(uint32_t));
    uint64_t *words = (uint64_t *)malloc((k_count * 128 + 1) * sizeof(uint64_t));
    int *b = (int *)malloc(k_count * sizeof(int));
    size_t L = 0, N = 0;
    for (size_t k = 0; k < k_count; ++k) {
        size_t nh = 0;
        size_t r = orc_fastpfor_block_record(v + 128 * k, 128, bytes + L, high + N, &nh);
        b[k] = bytes[L];
        L += r;
        N += nh; /* block order, positions ascending */
    }
    size_t pos = 16;
    memset(out, 0, 16);
    uint32_t masked[128];
    for (size_t k = 0; k < k_count; ++k) {
        for (int i = 0; i < 128; ++i) masked[i] = low_bits(v[128 * k + (size_t)i], b[k]);
        orc_pack(masked, 128, 1, b[k], out + pos); /* one lane, as the scalar FastPFOR */
        pos += 16 * (size_t)b[k];
    }
    put_le32(out, (uint32_t)(pos / 4)); /* R5 */
    put_le32(out + pos, (uint32_t)L);   /* R15 */
    pos += 4;
    memcpy(out + pos, bytes, L);
    memset(out + pos + L, 0, pad_to(L, 4) - L);
    pos += pad_to(L, 4);
    size_t W = orc_simple8b_encode(high, N, words);
    put_le32(out + pos, (uint32_t)N);
    put_le32(out + pos + 4, (uint32_t)W);
    pos += 8;
    size_t aligned = pad_to(pos, 16);
    memset(out + pos, 0, aligned - pos);
    pos = aligned;
    for (size_t w = 0; w < W; ++w) {
        put_le32(out + pos, (uint32_t)words[w]);
        put_le32(out + pos + 4, (uint32_t)(words[w] >> 32));
        pos += 8;
    }
    size_t end = pad_to(pos, 16); /* R14 */
    memset(out + pos, 0, end - pos);
    free(bytes);
    free(high);
    free(words);
    free(b);
    return end;
}

/* Walk one SimplePFOR page: fills `v` if v != NULL; returns the page size,
 * or 0 if it is corrupt or runs past `avail`. */
static size_t simplepfor_page_decode(const uint8_t *page, size_t avail, size_t k_count, uint32_t *v) {
    if (avail < 16) return 0;
    size_t len_at = 4 * (size_t)get_le32(page);
    if (len_at < 16 || len_at + 4 > avail) return 0;
    size_t L = get_le32(page + len_at);
    size_t bytes_at = len_at + 4;
    if (bytes_at + pad_to(L, 4) + 8 > avail) return 0;
    const uint8_t *bytes = page + bytes_at;
    size_t pos = bytes_at + pad_to(L, 4);
    size_t N = get_le32(page + pos), W = get_le32(page + pos + 4);
    pos = pad_to(pos + 8, 16);
    if (W > avail / 8 || pos + 8 * W > avail) return 0;
    size_t end = pad_to(pos + 8 * W, 16);
    if (end > avail) return 0;
    uint32_t *high = (uint32_t *)malloc((N + 1) * sizeof(uint32_t));
    uint64_t *words = (uint64_t *)malloc((W + 1) * sizeof(uint64_t));
    for (size_t w = 0; w < W; ++w)
        words[w] = (uint64_t)get_le32(page + pos + 8 * w) | (uint64_t)get_le32(page + pos + 8 * w + 4) << 32;
    int bad = orc_simple8b_decode(words, W, N, high) != ORC_OK;
    size_t packed = 16, r = 0, q = 0;
    for (size_t k = 0; k < k_count && !bad; ++k) {
        if (r + 2 > L) { bad = 1; break; }
        int bb = bytes[r], maxbits = bytes[r + 1];
        r += 2;
        if (bb > 32 || maxbits > 32 || maxbits < bb || packed + 16 * (size_t)bb > len_at) { bad = 1; break; }
        if (v) orc_unpack(page + packed, 128, 1, bb, v + 128 * k);
        packed += 16 * (size_t)bb;
        if (maxbits > bb) {
            if (r + 1 > L) { bad = 1; break; }
            size_t c = bytes[r++];
            if (c > 128 || r + c > L || q + c > N) { bad = 1; break; }
            for (size_t e = 0; e < c; ++e) {
                size_t p = bytes[r + e];
                if (p >= 128) { bad = 1; break; }
                if (v) v[128 * k + p] |= high[q + e] << bb; /* bb < 32 here */
            }
            q += c;
            r += c;
        }
    }
    free(high);
    free(words);
    if (bad || packed != len_at || q != N) return 0;
    return end;
}

size_t orc_simplepfor_encode(const uint32_t *x, size_t n, int delta, uint8_t *out) {
    uint32_t *d = (uint32_t *)malloc((n ? n : 1) * sizeof(uint32_t));
    orc_delta_encode(x, n, delta, d);
    size_t nb = n / 128, pages = (nb + 511) / 512, pos = 0;
    for (size_t p = 0; p < pages; ++p) {
        size_t k_count = nb - 512 * p < 512 ? nb - 512 * p : 512;
        pos += simplepfor_page_encode(d + 65536 * p, k_count, out + pos);
    }
    pos += orc_vbyte_encode(d + 128 * nb, n - 128 * nb, out + pos);
    free(d);
    return pos;
}

int orc_simplepfor_index(const uint8_t *in, size_t in_bytes, size_t n, uint64_t *index) {
    size_t nb = n / 128, pages = (nb + 511) / 512, pos = 0;
    for (size_t p = 0; p < pages; ++p) {
        size_t k_count = nb - 512 * p < 512 ? nb - 512 * p : 512;
        size_t size = simplepfor_page_decode(in + pos, in_bytes - pos, k_count, NULL);
        if (size == 0) return ORC_ECORRUPT;
        index[p] = pos;
        pos += size;
    }
    index[pages] = pos;
    return ORC_OK;
}

int orc_simplepfor_decode(const uint8_t *in, size_t in_bytes, size_t n, int delta, uint32_t *x) {
    uint32_t *d = (uint32_t *)malloc((n ? n : 1) * sizeof(uint32_t));
    size_t nb = n / 128, pages = (nb + 511) / 512, pos = 0;
    int rc = ORC_OK;
    for (size_t p = 0; p < pages; ++p) {
        size_t k_count = nb - 512 * p < 512 ? nb - 512 * p : 512;
        size_t size = simplepfor_page_decode(in + pos, in_bytes - pos, k_count, d + 65536 * p);
        if (size == 0) {
            rc = ORC_ECORRUPT;
            break;
        }
        pos += size;
    }
    if (rc == ORC_OK) {
        size_t used = orc_vbyte_decode(in + pos, in_bytes - pos, n - 128 * nb, d + 128 * nb);
        if (used == (size_t)-1) rc = ORC_ECORRUPT;
    }
    if (rc == ORC_OK) orc_delta_decode(d, n, delta, x);
    free(d);
    return rc;
}

/* ---------------------------------------------------------------- Sec. 7 */

void orc_member_bits(const uint32_t *a, size_t na, const uint32_t *b, size_t nb, uint32_t *bits,
                     uint64_t *count) {
    size_t i = 0;
    uint64_t c = 0;
    for (size_t w = 0; w < (nb + 31) / 32; ++w) bits[w] = 0;
    for (size_t j = 0; j < nb; ++j) {
        while (i < na && a[i] < b[j]) ++i; /* a[i] is the first element >= b[j] */
        if (i < na && a[i] == b[j]) {
            bits[j / 32] |= 1u << (j % 32);
            ++c;
        }
    }
    *count = c;
}
