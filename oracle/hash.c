/*
 * Oracle hashing and PRNG.  TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 *  - SHA-256 as specified in FIPS 180-4 (Sec. 4.1.2 functions, Sec. 4.2.2 constants,
 *    Sec. 5.1.1 padding, Sec. 6.2.2 compression).
 *  - The random oracles H, H' -> Fr of the paper (Sec. 2, "random oracle model"; used in
 *    FC.BOpen, Eq. b and Eq. folding, and for the Step-2 challenges) are not instantiated
 *    by the paper.  Reading used here: HFr(tag, data) = the 512-bit big-endian integer
 *    SHA256(tag || 0x00 || data) || SHA256(tag || 0x01 || data), reduced mod r.  A challenge
 *    that must be inverted and comes out 0 is re-hashed with 0x01 appended to the data.
 *  - SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): state += 0x9e3779b97f4a7c15, then the
 *    variant-13 finaliser of MurmurHash3.  Fr draws: four outputs little-endian, the top one
 *    masked to 63 bits, redrawn while >= r.
 */
#include "oracle.h"
#include <stdlib.h>
#include <string.h>

static const u32 K256[64] = {
    0x428a2f98, 0x71374491, 0xb5c0fbcf, 0xe9b5dba5, 0x3956c25b, 0x59f111f1, 0x923f82a4, 0xab1c5ed5,
    0xd807aa98, 0x12835b01, 0x243185be, 0x550c7dc3, 0x72be5d74, 0x80deb1fe, 0x9bdc06a7, 0xc19bf174,
    0xe49b69c1, 0xefbe4786, 0x0fc19dc6, 0x240ca1cc, 0x2de92c6f, 0x4a7484aa, 0x5cb0a9dc, 0x76f988da,
    0x983e5152, 0xa831c66d, 0xb00327c8, 0xbf597fc7, 0xc6e00bf3, 0xd5a79147, 0x06ca6351, 0x14292967,
    0x27b70a85, 0x2e1b2138, 0x4d2c6dfc, 0x53380d13, 0x650a7354, 0x766a0abb, 0x81c2c92e, 0x92722c85,
    0xa2bfe8a1, 0xa81a664b, 0xc24b8b70, 0xc76c51a3, 0xd192e819, 0xd6990624, 0xf40e3585, 0x106aa070,
    0x19a4c116, 0x1e376c08, 0x2748774c, 0x34b0bcb5, 0x391c0cb3, 0x4ed8aa4a, 0x5b9cca4f, 0x682e6ff3,
    0x748f82ee, 0x78a5636f, 0x84c87814, 0x8cc70208, 0x90befffa, 0xa4506ceb, 0xbef9a3f7, 0xc67178f2};

static u32 rotr(u32 x, int n) { return (x >> n) | (x << (32 - n)); }

static void compress(u32 H[8], const u8 block[64]) {
    u32 W[64];
    for (int t = 0; t < 16; t++)
        W[t] = ((u32)block[4 * t] << 24) | ((u32)block[4 * t + 1] << 16) | ((u32)block[4 * t + 2] << 8) | block[4 * t + 3];
    for (int t = 16; t < 64; t++) {
        u32 s0 = rotr(W[t - 15], 7) ^ rotr(W[t - 15], 18) ^ (W[t - 15] >> 3);
        u32 s1 = rotr(W[t - 2], 17) ^ rotr(W[t - 2], 19) ^ (W[t - 2] >> 10);
        W[t] = s1 + W[t - 7] + s0 + W[t - 16];
    }
    u32 a = H[0], b = H[1], c = H[2], d = H[3], e = H[4], f = H[5], g = H[6], h = H[7];
    for (int t = 0; t < 64; t++) {
        u32 S1 = rotr(e, 6) ^ rotr(e, 11) ^ rotr(e, 25);
        u32 ch = (e & f) ^ (~e & g);
        u32 T1 = h + S1 + ch + K256[t] + W[t];
        u32 S0 = rotr(a, 2) ^ rotr(a, 13) ^ rotr(a, 22);
        u32 maj = (a & b) ^ (a & c) ^ (b & c);
        u32 T2 = S0 + maj;
        h = g; g = f; f = e; e = d + T1; d = c; c = b; b = a; a = T1 + T2;
    }
    H[0] += a; H[1] += b; H[2] += c; H[3] += d; H[4] += e; H[5] += f; H[6] += g; H[7] += h;
}

void sha256(u8 out[32], const u8* msg, size_t len) {
    u32 H[8] = {0x6a09e667, 0xbb67ae85, 0x3c6ef372, 0xa54ff53a, 0x510e527f, 0x9b05688c, 0x1f83d9ab, 0x5be0cd19};
    size_t full = len / 64;
    for (size_t i = 0; i < full; i++) compress(H, msg + 64 * i);
    u8 tail[128]; memset(tail, 0, sizeof tail);
    size_t rem = len - 64 * full;
    memcpy(tail, msg + 64 * full, rem);
    tail[rem] = 0x80;
    size_t tl = (rem + 1 + 8 <= 64) ? 64 : 128;
    u64 bits = (u64)len * 8;
    for (int i = 0; i < 8; i++) tail[tl - 1 - i] = (u8)(bits >> (8 * i));
    compress(H, tail);
    if (tl == 128) compress(H, tail + 64);
    for (int i = 0; i < 8; i++) {
        out[4 * i] = (u8)(H[i] >> 24); out[4 * i + 1] = (u8)(H[i] >> 16);
        out[4 * i + 2] = (u8)(H[i] >> 8); out[4 * i + 3] = (u8)H[i];
    }
}

void hfr(fe* out, const char* tag, const u8* data, size_t len) {
    size_t tl = strlen(tag);
    u8* buf = (u8*)malloc(tl + 1 + len + 1);
    memcpy(buf, tag, tl);
    if (len) memcpy(buf + tl + 1, data, len);
    u8 wide[64];
    buf[tl] = 0x00; sha256(wide, buf, tl + 1 + len);
    buf[tl] = 0x01; sha256(wide + 32, buf, tl + 1 + len);
    free(buf);
    fr_from_be_wide(out, wide, 64);
}

void hfr_nonzero(fe* out, const char* tag, const u8* data, size_t len) {
    u8* buf = (u8*)malloc(len + 64);
    memcpy(buf, data, len);
    size_t l = len;
    hfr(out, tag, buf, l);
    while (f_is_zero(&FR, out)) {          /* probability 2^-254; re-hash with 0x01 appended */
        buf = (u8*)realloc(buf, l + 1);
        buf[l++] = 0x01;
        hfr(out, tag, buf, l);
    }
    free(buf);
}

u64 splitmix_next(splitmix* s) {
    u64 z = (s->state += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

void splitmix_fr(splitmix* s, u64 limbs[4]) {
    for (;;) {
        for (int i = 0; i < 4; i++) limbs[i] = splitmix_next(s);
        limbs[3] &= 0x7fffffffffffffffull;
        int ge = 1;                              /* limbs >= r ? */
        for (int i = 3; i >= 0; i--)
            if (limbs[i] != FR.mod[i]) { ge = limbs[i] > FR.mod[i]; break; }
        if (!ge) return;
    }
}
