// sample.cu -- Short f sampling, the product-tree leaves 3f, Small_encode(f),
// rho and (optionally) the first draw of g, one warp per key.
//
// Sec. 3.1 KeyGen step 3 / Algorithm 1 line "f <- Short": f has exactly w
// nonzero coefficients, each +-1.  Reading of the uniform draw: p words of
// stream 1; the first w have bit 0 cleared (low bits decode to -1 or +1),
// the rest have low bits forced to 01 (decode to 0); the words are sorted as
// unsigned integers and coefficient j is (word_j mod 4) - 1.  The sort is a
// 1024-slot bitonic network, padded with 0xFFFFFFFF
// (no real word can equal it: bit 0 or bit 1 is cleared), run by one warp.
#include "common.cuh"
#include "kernels.h"
#include "short.cuh"
#include "pdl.cuh"

namespace snt {

// One warp per key (four keys per CTA): the sort is the one-warp network of
// short.cuh (32 slots per lane, shuffles only), the leaves are written as
// 16-byte stores, Small_encode(f) byte 8L + b by lane L.
// With g_out: also g's attempt-0 draw (the R/3 kernel's formula, stream 0,
// or the injected test draw) as int8 rows of stride pad, so that h can be
// formed before the R/3 inversions finish; and the resampling list's count
// is reset for this call.
template <int P>
__global__ void __launch_bounds__(128, 4)
k_sample_f(KeyMap km, int nkeys, int16_t *__restrict__ leaves, int sk_bytes, int rho_off,
           int8_t *__restrict__ g_out, const uint64_t *__restrict__ inj_idx,
           const int8_t *__restrict__ inj_g, int n_inj, int *__restrict__ fix_count,
           int16_t *__restrict__ g16_out) {
    pdl_enter();
    using G = Geo<P>;
    static_assert(G::pad % 32 == 0 && G::pad <= 1024, "row padding");
    const int lane = threadIdx.x & 31;
    const int key = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (key >= nkeys) return;  // the whole warp
    const BatchDesc d = key_batch(km, key);
    const uint64_t seed = d.seed;
    const uint64_t k = d.first + (uint64_t)(key - d.key_base);

    uint32_t v[32];
    short_sorted_warp<P>(seed, k, STREAM_F, v);

    // leaves a = 3f (centred int16), zero padded to G::pad
    int16_t *leaf = leaves + (size_t)key * G::pad;
    if (32 * lane < G::pad) {
#pragma unroll
        for (int s4 = 0; s4 < 4; ++s4) {
            uint32_t w4[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int r = 8 * s4 + 2 * h, j = 32 * lane + r;
                const int c0 = j < G::p ? 3 * ((int)(v[r] & 3u) - 1) : 0;
                const int c1 = j + 1 < G::p ? 3 * ((int)(v[r + 1] & 3u) - 1) : 0;
                w4[h] = (uint32_t)(uint16_t)c0 | ((uint32_t)(uint16_t)c1 << 16);
            }
            *reinterpret_cast<uint4 *>(leaf + 32 * lane + 8 * s4) = make_uint4(w4[0], w4[1], w4[2], w4[3]);
        }
    }
    // Small_encode(f): byte b packs coefficients 4b..4b+3 as (c + 1) in 2 bits
    uint8_t *skk = d.sk + (size_t)(key - d.key_base) * sk_bytes;
#pragma unroll
    for (int b8 = 0; b8 < 8; ++b8) {
        const int b = 8 * lane + b8;
        if (b < G::small_bytes) {
            uint32_t byte = 0;
#pragma unroll
            for (int rr = 0; rr < 4; ++rr)
                if (4 * b + rr < G::p) byte |= (v[4 * b8 + rr] & 3u) << (2 * rr);
            skk[b] = (uint8_t)byte;
        }
    }

    if (g_out) {
        int inj = -1;
        if (lane == 0) {
            for (int j = 0; j < n_inj; ++j)
                if (inj_idx[j] == k) inj = j;
            if (key == 0) *fix_count = 0;
        }
        inj = __shfl_sync(0xffffffffu, inj, 0);
        int8_t *grow = g_out + (size_t)key * G::pad;
        int16_t *g16 = g16_out ? g16_out + (size_t)key * G::pad : nullptr;
        if (inj >= 0) {
            for (int i = lane; i < G::pad; i += 32) {
                const int8_t c = (i < G::p) ? inj_g[(size_t)inj * G::p + i] : (int8_t)0;
                grow[i] = c;
                if (g16) g16[i] = c;
            }
        } else {
            // g_i = floor(3 (u_i mod 2^30) / 2^30) - 1 for word u_i of stream 0, attempt 0
            for (int blk = lane; 4 * blk < G::pad; blk += 32) {
                uint32_t r[4];
                rand_block(seed, k, STREAM_G, 0u, (uint32_t)blk, r);
                int c[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int i = 4 * blk + j;
                    c[j] = (i < G::p) ? (int)(((unsigned long long)(r[j] & 0x3fffffffu) * 3u) >> 30) - 1 : 0;
                }
                *reinterpret_cast<uint32_t *>(grow + 4 * blk) =
                    (uint32_t)(uint8_t)c[0] | ((uint32_t)(uint8_t)c[1] << 8) |
                    ((uint32_t)(uint8_t)c[2] << 16) | ((uint32_t)(uint8_t)c[3] << 24);
                if (g16)
                    *reinterpret_cast<uint2 *>(g16 + 4 * blk) =
                        make_uint2((uint32_t)(uint16_t)c[0] | ((uint32_t)(uint16_t)c[1] << 16),
                                   (uint32_t)(uint16_t)c[2] | ((uint32_t)(uint16_t)c[3] << 16));
            }
        }
    }

    // rho: small_bytes bytes of stream 2, little-endian within each word
    for (int blk = lane; 16 * blk < G::small_bytes; blk += 32) {
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
    SNT_LAUNCH(k_sample_f<P>, (nkeys + 3) / 4, 128, 0, st, km, nkeys, leaves, sk_bytes, rho_off,
        g_out, inj_idx, inj_g, n_inj, fix_count, g16_out);
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
