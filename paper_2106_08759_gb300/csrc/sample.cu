// sample.cu -- Short f sampling, the product-tree leaves 3f, Small_encode(f),
// rho and (optionally) the first draw of g, one CTA per key.
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
// With g_out: also g's attempt-0 draw (the R/3 kernel's formula, stream 0,
// or the injected test draw) as int8 rows of stride pad, so that h can be
// formed before the R/3 inversions finish; and the resampling list's count
// is reset for this call.
template <int P>
__global__ void __launch_bounds__(256)
k_sample_f(KeyMap km, int nkeys, int16_t *__restrict__ leaves, int sk_bytes, int rho_off,
           int8_t *__restrict__ g_out, const uint64_t *__restrict__ inj_idx,
           const int8_t *__restrict__ inj_g, int n_inj, int *__restrict__ fix_count,
           int16_t *__restrict__ g16_out) {
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

    if (g_out) {
        __shared__ int inj;
        if (t == 0) {
            inj = -1;
            for (int j = 0; j < n_inj; ++j)
                if (inj_idx[j] == k) inj = j;
            if (key == 0) *fix_count = 0;
        }
        __syncthreads();
        int8_t *grow = g_out + (size_t)key * G::pad;
        int16_t *g16 = g16_out ? g16_out + (size_t)key * G::pad : nullptr;
        if (inj >= 0) {
            for (int i = t; i < G::pad; i += blockDim.x) {
                const int8_t c = (i < G::p) ? inj_g[(size_t)inj * G::p + i] : (int8_t)0;
                grow[i] = c;
                if (g16) g16[i] = c;
            }
        } else {
            // g_i = floor(3 (u_i mod 2^30) / 2^30) - 1 for word u_i of stream 0, attempt 0
            for (int blk = t; 4 * blk < G::pad; blk += blockDim.x) {
                uint32_t r[4];
                rand_block(seed, k, STREAM_G, 0u, (uint32_t)blk, r);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int i = 4 * blk + j;
                    const int8_t c = (i < G::p)
                        ? (int8_t)((int)(((unsigned long long)(r[j] & 0x3fffffffu) * 3u) >> 30) - 1)
                        : (int8_t)0;
                    grow[i] = c;
                    if (g16) g16[i] = c;
                }
            }
        }
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
                            int rho_off, cudaStream_t st, int8_t *g_out,
                            const uint64_t *inj_idx, const int8_t *inj_g, int n_inj,
                            int *fix_count, int16_t *g16_out) {
    k_sample_f<P><<<nkeys, 256, 0, st>>>(km, nkeys, leaves, sk_bytes, rho_off, g_out, inj_idx,
                                         inj_g, n_inj, fix_count, g16_out);
    return cudaGetLastError();
}

#define SNT_SAMPLE_INST(P)                                                                  \
    template cudaError_t launch_sample_f<P>(const KeyMap &, int, int16_t *, int, int,       \
                                            cudaStream_t, int8_t *, const uint64_t *,       \
                                            const int8_t *, int, int *, int16_t *);
SNT_SAMPLE_INST(653)
SNT_SAMPLE_INST(761)
SNT_SAMPLE_INST(857)

}  // namespace snt
