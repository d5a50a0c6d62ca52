// SHA-256 (FIPS 180-4) for one thread, streaming, plus the hash-to-Fr used for every
// Fiat-Shamir challenge: HFr(tag, data) = SHA256(tag || 0x00 || data) || SHA256(tag || 0x01 || data)
// read as a 512-bit big-endian integer and reduced mod r.
#pragma once
#include "fp.cuh"

struct sha256_ctx {
    uint32_t h[8];
    alignas(16) uint8_t buf[64];
    uint32_t nbuf;
    uint64_t total;
};

FPG_DEV uint32_t sha_rotr(uint32_t x, int n) { return (x >> n) | (x << (32 - n)); }

FPG_NOINL void sha256_compress(uint32_t* h, const uint8_t* blk) {
    uint32_t w[16];
    if (((uintptr_t)blk & 3) == 0) {                  // word loads, byte-swapped to big-endian
        const uint32_t* b4 = reinterpret_cast<const uint32_t*>(blk);
#pragma unroll
        for (int t = 0; t < 16; t++) w[t] = __byte_perm(b4[t], 0, 0x0123);
    } else {
#pragma unroll
        for (int t = 0; t < 16; t++)
            w[t] = ((uint32_t)blk[4 * t] << 24) | ((uint32_t)blk[4 * t + 1] << 16) | ((uint32_t)blk[4 * t + 2] << 8) |
                   blk[4 * t + 3];
    }
    uint32_t a = h[0], b = h[1], c = h[2], d = h[3], e = h[4], f = h[5], g = h[6], hh = h[7];
#pragma unroll
    for (int t = 0; t < 64; t++) {
        uint32_t wt;
        if (t < 16) {
            wt = w[t];
        } else {
            uint32_t w15 = w[(t - 15) & 15], w2 = w[(t - 2) & 15];
            uint32_t s0 = sha_rotr(w15, 7) ^ sha_rotr(w15, 18) ^ (w15 >> 3);
            uint32_t s1 = sha_rotr(w2, 17) ^ sha_rotr(w2, 19) ^ (w2 >> 10);
            wt = w[t & 15] = w[t & 15] + s0 + w[(t - 7) & 15] + s1;
        }
        uint32_t S1 = sha_rotr(e, 6) ^ sha_rotr(e, 11) ^ sha_rotr(e, 25);
        uint32_t ch = (e & f) ^ (~e & g);
        uint32_t t1 = hh + S1 + ch + SHA256_K[t] + wt;
        uint32_t S0 = sha_rotr(a, 2) ^ sha_rotr(a, 13) ^ sha_rotr(a, 22);
        uint32_t mj = (a & b) ^ (a & c) ^ (b & c);
        uint32_t t2 = S0 + mj;
        hh = g; g = f; f = e; e = d + t1; d = c; c = b; b = a; a = t1 + t2;
    }
    h[0] += a; h[1] += b; h[2] += c; h[3] += d; h[4] += e; h[5] += f; h[6] += g; h[7] += hh;
}

FPG_DEV void sha256_init(sha256_ctx& c) {
#pragma unroll
    for (int i = 0; i < 8; i++) c.h[i] = SHA256_H0[i];
    c.nbuf = 0;
    c.total = 0;
}
// whole 64-byte blocks of the input are compressed in place; only partial blocks are buffered.
// When the buffered length and the input address are multiples of 4 (long inputs after a header
// of whole words: statements, tree nodes), the input moves into the buffer a word at a time.
FPG_DEV void sha256_update(sha256_ctx& c, const uint8_t* data, uint32_t n) {
    c.total += n;
    if (((c.nbuf | (uint32_t)(uintptr_t)data) & 3) == 0) {
        const uint32_t* d32 = reinterpret_cast<const uint32_t*>(data);
        uint32_t* b32 = reinterpret_cast<uint32_t*>(c.buf);
        while (n >= 4) {
            if (c.nbuf == 0 && n >= 64) {
                sha256_compress(c.h, reinterpret_cast<const uint8_t*>(d32));
                d32 += 16;
                n -= 64;
                continue;
            }
            const uint32_t o = c.nbuf >> 2, take = min(16u - o, n >> 2);
            for (uint32_t i = 0; i < take; i++) b32[o + i] = d32[i];
            d32 += take;
            n -= 4 * take;
            c.nbuf += 4 * take;
            if (c.nbuf == 64) {
                sha256_compress(c.h, c.buf);
                c.nbuf = 0;
            }
        }
        data = reinterpret_cast<const uint8_t*>(d32);
    }
    while (n) {
        if (c.nbuf == 0 && n >= 64) {
            sha256_compress(c.h, data);
            data += 64;
            n -= 64;
            continue;
        }
        const uint32_t take = min(64u - c.nbuf, n);
        for (uint32_t i = 0; i < take; i++) c.buf[c.nbuf + i] = data[i];
        c.nbuf += take;
        data += take;
        n -= take;
        if (c.nbuf == 64) {
            sha256_compress(c.h, c.buf);
            c.nbuf = 0;
        }
    }
}
FPG_DEV void sha256_byte(sha256_ctx& c, uint8_t b) { sha256_update(c, &b, 1); }
FPG_DEV void sha256_final(sha256_ctx& c, uint8_t* out) {
    uint64_t bits = c.total * 8;
    c.buf[c.nbuf++] = 0x80;
    if (c.nbuf > 56) {
        while (c.nbuf < 64) c.buf[c.nbuf++] = 0;
        sha256_compress(c.h, c.buf);
        c.nbuf = 0;
    }
    while (c.nbuf < 56) c.buf[c.nbuf++] = 0;
    for (int i = 0; i < 8; i++) c.buf[56 + i] = (uint8_t)(bits >> (56 - 8 * i));
    sha256_compress(c.h, c.buf);
    for (int i = 0; i < 8; i++) {
        out[4 * i] = (uint8_t)(c.h[i] >> 24); out[4 * i + 1] = (uint8_t)(c.h[i] >> 16);
        out[4 * i + 2] = (uint8_t)(c.h[i] >> 8); out[4 * i + 3] = (uint8_t)c.h[i];
    }
}
FPG_DEV void sha256(uint8_t* out, const uint8_t* data, uint32_t n) {
    sha256_ctx c; sha256_init(c); sha256_update(c, data, n); sha256_final(c, out);
}

// HFr over the concatenation of up to three byte ranges (pieces may be empty) followed by
// `nsuffix` bytes 0x01 (the re-hash rule for a challenge that must be invertible)
FPG_NOINL fr hash_to_fr(const char* tag, uint32_t taglen, const uint8_t* d0, uint32_t n0,
                        const uint8_t* d1, uint32_t n1, const uint8_t* d2, uint32_t n2,
                        uint32_t nsuffix = 0) {
    uint8_t wide[64];
    for (int half = 0; half < 2; half++) {
        sha256_ctx c;
        sha256_init(c);
        sha256_update(c, (const uint8_t*)tag, taglen);
        sha256_byte(c, (uint8_t)half);
        if (n0) sha256_update(c, d0, n0);
        if (n1) sha256_update(c, d1, n1);
        if (n2) sha256_update(c, d2, n2);
        for (uint32_t k = 0; k < nsuffix; k++) sha256_byte(c, 0x01);
        sha256_final(c, wide + 32 * half);
    }
    return fr_from_be64(wide);
}

// HFr that never returns 0: re-hash with one more 0x01 byte appended while the value is 0
FPG_NOINL fr hash_to_fr_nonzero(const char* tag, uint32_t taglen, const uint8_t* d0, uint32_t n0,
                                const uint8_t* d1, uint32_t n1, const uint8_t* d2, uint32_t n2) {
    fr v = hash_to_fr(tag, taglen, d0, n0, d1, n1, d2, n2, 0);
    for (uint32_t k = 1; fr_is_zero(v) && k < 64; k++) v = hash_to_fr(tag, taglen, d0, n0, d1, n1, d2, n2, k);
    return v;
}
