// sample.cu -- Short f sampling, the product-tree leaves 3f, Small_encode(f)
// and rho, one CTA per key.
//
// Sec. 3.1 KeyGen step 3 / Algorithm 1 line "f <- Short": f has exactly w
// nonzero coefficients, each +-1.  Reading of the uniform draw: p words of
// stream 1; the first w have bit 0 cleared (low bits decode to -1 or +1),
// the rest have low bits forced to 01 (decode to 0); the words are sorted as
// unsigned integers and coefficient j is (word_j mod 4) - 1.  The sort is a
// 1024-slot bitonic network in shared memory, padded with 0xFFFFFFFF
// (no real word can equal it: bit 0 or bit 1 is cleared).
#include "common.cuh"
#include "kernels.h"

namespace snt {

template <int P>
__global__ void __launch_bounds__(256)
k_sample_f(uint64_t seed, uint64_t first, int B, int16_t *__restrict__ leaves,
           uint8_t *__restrict__ sk, int sk_bytes, int rho_off) {
    using G = Geo<P>;
    __shared__ uint32_t s[1024];
    const int key = blockIdx.x;
    if (key >= B) return;
    const uint64_t k = first + (uint64_t)key;
    const int tid = threadIdx.x;

    // words of stream 1, low bits forced; sentinels above p
    for (int blk = tid; blk < 256; blk += blockDim.x) {
        uint32_t r[4] = {0u, 0u, 0u, 0u};
        if (4 * blk < G::p) rand_block(seed, k, STREAM_F, 0u, (uint32_t)blk, r);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int idx = 4 * blk + j;
            uint32_t v;
            if (idx < G::w) v = r[j] & ~1u;
            else if (idx < G::p) v = (r[j] & ~3u) | 1u;
            else v = 0xFFFFFFFFu;
            s[idx] = v;
        }
    }
    __syncthreads();

    // ascending bitonic sort of 1024 words
    for (int size = 2; size <= 1024; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = tid; t < 512; t += blockDim.x) {
                const int lo = 2 * t - (t & (stride - 1));
                const int hi = lo + stride;
                const bool asc = (lo & size) == 0;
                const uint32_t a = s[lo], b = s[hi];
                if ((a > b) == asc) { s[lo] = b; s[hi] = a; }
            }
            __syncthreads();
        }
    }

    // leaves a = 3f (centred int16), zero padded to G::pad
    int16_t *leaf = leaves + (size_t)key * G::pad;
    for (int j = tid; j < G::pad; j += blockDim.x)
        leaf[j] = (int16_t)(j < G::p ? 3 * ((int)(s[j] & 3u) - 1) : 0);

    // Small_encode(f): byte b packs coefficients 4b..4b+3 as (c + 1) in 2 bits
    uint8_t *skk = sk + (size_t)key * sk_bytes;
    for (int b = tid; b < G::small_bytes; b += blockDim.x) {
        uint32_t byte = 0;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int idx = 4 * b + t;
            if (idx < G::p) byte |= (s[idx] & 3u) << (2 * t);
        }
        skk[b] = (uint8_t)byte;
    }

    // rho: small_bytes bytes of stream 2, little-endian within each word
    for (int blk = tid; 16 * blk < G::small_bytes; blk += blockDim.x) {
        uint32_t r[4];
        rand_block(seed, k, STREAM_RHO, 0u, (uint32_t)blk, r);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int idx = 16 * blk + j;
            if (idx < G::small_bytes) skk[rho_off + idx] = (uint8_t)(r[j >> 2] >> (8 * (j & 3)));
        }
    }
}

template <int P>
cudaError_t launch_sample_f(uint64_t seed, uint64_t first, int B, int16_t *leaves,
                            uint8_t *sk, int sk_bytes, int rho_off, cudaStream_t st) {
    k_sample_f<P><<<B, 256, 0, st>>>(seed, first, B, leaves, sk, sk_bytes, rho_off);
    return cudaGetLastError();
}

template cudaError_t launch_sample_f<653>(uint64_t, uint64_t, int, int16_t *, uint8_t *, int, int, cudaStream_t);
template cudaError_t launch_sample_f<761>(uint64_t, uint64_t, int, int16_t *, uint8_t *, int, int, cudaStream_t);
template cudaError_t launch_sample_f<857>(uint64_t, uint64_t, int, int16_t *, uint8_t *, int, int, cudaStream_t);

}  // namespace snt
