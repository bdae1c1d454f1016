// sample.cu -- Short f sampling, the product-tree leaves 3f, Small_encode(f)
// and rho, one CTA per key.
//
// Sec. 3.1 KeyGen step 3 / Algorithm 1 line "f <- Short": f has exactly w
// nonzero coefficients, each +-1.  Reading of the uniform draw: p words of
// stream 1; the first w have bit 0 cleared (low bits decode to -1 or +1),
// the rest have low bits forced to 01 (decode to 0); the words are sorted as
// unsigned integers and coefficient j is (word_j mod 4) - 1.  The sort is a
// 1024-slot bitonic network, padded with 0xFFFFFFFF
// (no real word can equal it: bit 0 or bit 1 is cleared).
#include "common.cuh"
#include "kernels.h"
#include "short.cuh"

namespace snt {

// One CTA of 256 threads per key; thread t holds elements 4t .. 4t+3 of the
// 1024-slot network in registers.  Compare-exchange partners closer than 4
// slots are in the same thread, closer than 128 in the same warp (shuffles),
// farther ones in another warp (exchanged through shared memory, 6 of the 55
// stages).
template <int P>
__global__ void __launch_bounds__(256)
k_sample_f(KeyMap km, int nkeys, int16_t *__restrict__ leaves, int sk_bytes, int rho_off) {
    using G = Geo<P>;
    __shared__ __align__(16) uint32_t xs[1024];
    const int key = blockIdx.x;
    if (key >= nkeys) return;
    const BatchDesc d = key_batch(km, key);
    const uint64_t seed = d.seed;
    const uint64_t k = d.first + (uint64_t)(key - d.key_base);
    const int t = threadIdx.x;

    uint32_t v[4];
    short_sorted_words<P>(seed, k, STREAM_F, v, xs);

    // leaves a = 3f (centred int16), zero padded to G::pad
    int16_t *leaf = leaves + (size_t)key * G::pad;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int j = 4 * t + r;
        if (j < G::pad) leaf[j] = (int16_t)(j < G::p ? 3 * ((int)(v[r] & 3u) - 1) : 0);
    }
    // Small_encode(f): byte t packs coefficients 4t..4t+3 as (c + 1) in 2 bits
    uint8_t *skk = d.sk + (size_t)(key - d.key_base) * sk_bytes;
    if (t < G::small_bytes) {
        uint32_t byte = 0;
#pragma unroll
        for (int r = 0; r < 4; ++r)
            if (4 * t + r < G::p) byte |= (v[r] & 3u) << (2 * r);
        skk[t] = (uint8_t)byte;
    }

    // rho: small_bytes bytes of stream 2, little-endian within each word
    for (int blk = t; 16 * blk < G::small_bytes; blk += blockDim.x) {
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
cudaError_t launch_sample_f(const KeyMap &km, int nkeys, int16_t *leaves, int sk_bytes,
                            int rho_off, cudaStream_t st) {
    k_sample_f<P><<<nkeys, 256, 0, st>>>(km, nkeys, leaves, sk_bytes, rho_off);
    return cudaGetLastError();
}

template cudaError_t launch_sample_f<653>(const KeyMap &, int, int16_t *, int, int, cudaStream_t);
template cudaError_t launch_sample_f<761>(const KeyMap &, int, int16_t *, int, int, cudaStream_t);
template cudaError_t launch_sample_f<857>(const KeyMap &, int, int16_t *, int, int, cudaStream_t);

}  // namespace snt
