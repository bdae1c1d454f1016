// sha512.cuh -- SHA-512 (FIPS 180-4) on the device.
#pragma once
#include <cstdint>

namespace snt {

// Round constants of FIPS 180-4 Sec. 4.2.3 (first 64 bits of the fractional
// parts of the cube roots of the first 80 primes).
static __constant__ uint64_t c_sha512_k[80] = {
    0x428a2f98d728ae22ULL, 0x7137449123ef65cdULL, 0xb5c0fbcfec4d3b2fULL, 0xe9b5dba58189dbbcULL,
    0x3956c25bf348b538ULL, 0x59f111f1b605d019ULL, 0x923f82a4af194f9bULL, 0xab1c5ed5da6d8118ULL,
    0xd807aa98a3030242ULL, 0x12835b0145706fbeULL, 0x243185be4ee4b28cULL, 0x550c7dc3d5ffb4e2ULL,
    0x72be5d74f27b896fULL, 0x80deb1fe3b1696b1ULL, 0x9bdc06a725c71235ULL, 0xc19bf174cf692694ULL,
    0xe49b69c19ef14ad2ULL, 0xefbe4786384f25e3ULL, 0x0fc19dc68b8cd5b5ULL, 0x240ca1cc77ac9c65ULL,
    0x2de92c6f592b0275ULL, 0x4a7484aa6ea6e483ULL, 0x5cb0a9dcbd41fbd4ULL, 0x76f988da831153b5ULL,
    0x983e5152ee66dfabULL, 0xa831c66d2db43210ULL, 0xb00327c898fb213fULL, 0xbf597fc7beef0ee4ULL,
    0xc6e00bf33da88fc2ULL, 0xd5a79147930aa725ULL, 0x06ca6351e003826fULL, 0x142929670a0e6e70ULL,
    0x27b70a8546d22ffcULL, 0x2e1b21385c26c926ULL, 0x4d2c6dfc5ac42aedULL, 0x53380d139d95b3dfULL,
    0x650a73548baf63deULL, 0x766a0abb3c77b2a8ULL, 0x81c2c92e47edaee6ULL, 0x92722c851482353bULL,
    0xa2bfe8a14cf10364ULL, 0xa81a664bbc423001ULL, 0xc24b8b70d0f89791ULL, 0xc76c51a30654be30ULL,
    0xd192e819d6ef5218ULL, 0xd69906245565a910ULL, 0xf40e35855771202aULL, 0x106aa07032bbd1b8ULL,
    0x19a4c116b8d2d0c8ULL, 0x1e376c085141ab53ULL, 0x2748774cdf8eeb99ULL, 0x34b0bcb5e19b48a8ULL,
    0x391c0cb3c5c95a63ULL, 0x4ed8aa4ae3418acbULL, 0x5b9cca4f7763e373ULL, 0x682e6ff3d6b2b8a3ULL,
    0x748f82ee5defb2fcULL, 0x78a5636f43172f60ULL, 0x84c87814a1f0ab72ULL, 0x8cc702081a6439ecULL,
    0x90befffa23631e28ULL, 0xa4506cebde82bde9ULL, 0xbef9a3f7b2c67915ULL, 0xc67178f2e372532bULL,
    0xca273eceea26619cULL, 0xd186b8c721c0c207ULL, 0xeada7dd6cde0eb1eULL, 0xf57d4f7fee6ed178ULL,
    0x06f067aa72176fbaULL, 0x0a637dc5a2c898a6ULL, 0x113f9804bef90daeULL, 0x1b710b35131c471bULL,
    0x28db77f523047d84ULL, 0x32caab7b40c72493ULL, 0x3c9ebe0a15c9bebcULL, 0x431d67c49c100d4cULL,
    0x4cc5d4becb3e42b6ULL, 0x597f299cfc657e2aULL, 0x5fcb6fab3ad6faecULL, 0x6c44198c4a475817ULL};

__device__ __forceinline__ uint64_t rotr(uint64_t x, int n) { return (x >> n) | (x << (64 - n)); }

// One 128-byte block: W[16] holds the big-endian message words on entry.
//
// The round is arranged for a short dependency chain: h + K_t + W_t and
// d + h + K_t + W_t do not depend on the previous round's new e and a, so
// they are formed early and the new e is one three-input add after Sigma1(e)
// and Ch; the new a adds Sigma0(a) + Maj to the same partial sum.
__device__ __forceinline__ void sha512_block(uint64_t (&H)[8], uint64_t (&W)[16]) {
    uint64_t a = H[0], b = H[1], c = H[2], d = H[3], e = H[4], f = H[5], g = H[6], h = H[7];
#pragma unroll 1
    for (int r = 0; r < 80; r += 16) {
#pragma unroll
        for (int tt = 0; tt < 16; ++tt) {
            if (r > 0) {
                const uint64_t w15 = W[(tt + 1) & 15], w2 = W[(tt + 14) & 15];
                const uint64_t s0 = rotr(w15, 1) ^ rotr(w15, 8) ^ (w15 >> 7);
                const uint64_t s1 = rotr(w2, 19) ^ rotr(w2, 61) ^ (w2 >> 6);
                W[tt] += s0 + W[(tt + 9) & 15] + s1;
            }
            const uint64_t hkw = h + (c_sha512_k[r + tt] + W[tt]);
            const uint64_t dhkw = d + hkw;
            const uint64_t S1 = rotr(e, 14) ^ rotr(e, 18) ^ rotr(e, 41);
            const uint64_t ch = (e & f) ^ (~e & g);
            const uint64_t S0 = rotr(a, 28) ^ rotr(a, 34) ^ rotr(a, 39);
            const uint64_t mj = (a & b) ^ (a & c) ^ (b & c);
            const uint64_t t1 = hkw + S1 + ch;
            h = g; g = f; f = e; e = dhkw + S1 + ch;
            d = c; c = b; b = a; a = t1 + (S0 + mj);
        }
    }
    H[0] += a; H[1] += b; H[2] += c; H[3] += d;
    H[4] += e; H[5] += f; H[6] += g; H[7] += h;
}

// The 80 rounds of one block with W_t + K_t given per round (wk[t][lane]):
// the same round as sha512_block, the schedule computed elsewhere.  The 16
// table entries of a group of rounds are read before the group runs.
__device__ __forceinline__ void sha512_rounds_wk(uint64_t (&H)[8], const uint64_t (*wk)[32],
                                                 int lane) {
    uint64_t a = H[0], b = H[1], c = H[2], d = H[3], e = H[4], f = H[5], g = H[6], h = H[7];
#pragma unroll 1
    for (int r = 0; r < 80; r += 16) {
        uint64_t kw[16];
#pragma unroll
        for (int tt = 0; tt < 16; ++tt) kw[tt] = wk[r + tt][lane];
#pragma unroll
        for (int tt = 0; tt < 16; ++tt) {
            const uint64_t hkw = h + kw[tt];
            const uint64_t dhkw = d + hkw;
            const uint64_t S1 = rotr(e, 14) ^ rotr(e, 18) ^ rotr(e, 41);
            const uint64_t ch = (e & f) ^ (~e & g);
            const uint64_t S0 = rotr(a, 28) ^ rotr(a, 34) ^ rotr(a, 39);
            const uint64_t mj = (a & b) ^ (a & c) ^ (b & c);
            const uint64_t t1 = hkw + S1 + ch;
            h = g; g = f; f = e; e = dhkw + S1 + ch;
            d = c; c = b; b = a; a = t1 + (S0 + mj);
        }
    }
    H[0] += a; H[1] += b; H[2] += c; H[3] += d;
    H[4] += e; H[5] += f; H[6] += g; H[7] += h;
}

// First 32 bytes of SHA-512(prefix | s1[0..l1) | s2[0..l2)), by one thread
// (the Hash_prefix of the NTRU Prime KEM).  s1 / s2 may be in any memory.
static __device__ __noinline__ void sha512_prefixed(uint8_t prefix, const uint8_t *s1, int l1,
                                             const uint8_t *s2, int l2, uint8_t *out32) {
    const int len = 1 + l1 + l2;
    const int nblk = (len + 1 + 16 + 127) / 128;
    const uint64_t bitlen = (uint64_t)len * 8u;
    uint64_t H[8] = {0x6a09e667f3bcc908ULL, 0xbb67ae8584caa73bULL, 0x3c6ef372fe94f82bULL,
                     0xa54ff53a5f1d36f1ULL, 0x510e527fade682d1ULL, 0x9b05688c2b3e6c1fULL,
                     0x1f83d9abfb41bd6bULL, 0x5be0cd19137e2179ULL};
    for (int blk = 0; blk < nblk; ++blk) {
        uint64_t W[16];
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            uint64_t v = 0;
            for (int b = 0; b < 8; ++b) {
                const int q = 128 * blk + 8 * t + b;
                uint32_t byte;
                if (q == 0) byte = prefix;
                else if (q <= l1) byte = s1[q - 1];
                else if (q < len) byte = s2[q - 1 - l1];
                else if (q == len) byte = 0x80u;
                else if (q >= nblk * 128 - 8) byte = (uint32_t)(bitlen >> (8 * (nblk * 128 - 1 - q))) & 255u;
                else byte = 0;
                v = (v << 8) | byte;
            }
            W[t] = v;
        }
        sha512_block(H, W);
    }
    for (int i = 0; i < 4; ++i)
        for (int b = 0; b < 8; ++b) out32[8 * i + b] = (uint8_t)(H[i] >> (56 - 8 * b));
}

}  // namespace snt
