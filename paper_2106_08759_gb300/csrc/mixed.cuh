// mixed.cuh -- the mixed-radix encoding of the NTRU Prime formats on the
// device (Rq_encode with radix q for public keys, radix (q+2)/3 for the
// rounded ciphertext body), for one CTA, following a host-computed schedule
// (EncSched): within a pass every entry but the last has the same radix, so
// each pair's byte count and output offset are fixed.
#pragma once
#include "kernels.h"

namespace snt {

// Values R[cur][0..p) -> bytes.  Contains barriers (all threads call it).
template <int PAD>
__device__ __forceinline__ void mixed_encode(uint32_t (*R)[PAD], const EncSched &S, uint8_t *ob) {
    int cur = 0;
    for (int l = 0; l < S.nlev; ++l) {
        const EncLevel L = S.lev[l];
        const uint32_t *rin = R[cur];
        uint32_t *rout = R[cur ^ 1];
        for (int i = threadIdx.x; 2 * i < L.n; i += blockDim.x) {
            if (2 * i + 1 < L.n) {
                uint32_t r = rin[2 * i] + L.mu * rin[2 * i + 1];
                const int e = (2 * i + 1 == L.n - 1) ? L.elast : L.eu;
                const int off = L.boff + i * L.eu;
                for (int b = 0; b < e; ++b) { ob[off + b] = (uint8_t)(r & 255u); r >>= 8; }
                rout[i] = r;
            } else {
                rout[i] = rin[2 * i];
            }
        }
        __syncthreads();
        cur ^= 1;
    }
    if (threadIdx.x == 0) {
        uint32_t r = R[cur][0];
        for (int b = 0; b < S.efinal; ++b) { ob[S.foff + b] = (uint8_t)(r & 255u); r >>= 8; }
    }
    __syncthreads();
}

// Two value arrays at once (R0 -> ob0, R1 -> ob1), half of the threads on
// each, one barrier per level.  Contains barriers (all threads call it).
template <int PAD>
__device__ __forceinline__ void mixed_encode2(uint32_t (*R0)[PAD], uint32_t (*R1)[PAD],
                                              const EncSched &S, uint8_t *ob0, uint8_t *ob1) {
    const int half = blockDim.x / 2;
    const bool second = (int)threadIdx.x >= half;
    const int t = second ? threadIdx.x - half : threadIdx.x;
    uint32_t(*R)[PAD] = second ? R1 : R0;
    uint8_t *ob = second ? ob1 : ob0;
    int cur = 0;
    for (int l = 0; l < S.nlev; ++l) {
        const EncLevel L = S.lev[l];
        const uint32_t *rin = R[cur];
        uint32_t *rout = R[cur ^ 1];
        for (int i = t; 2 * i < L.n; i += half) {
            if (2 * i + 1 < L.n) {
                uint32_t r = rin[2 * i] + L.mu * rin[2 * i + 1];
                const int e = (2 * i + 1 == L.n - 1) ? L.elast : L.eu;
                const int off = L.boff + i * L.eu;
                for (int b = 0; b < e; ++b) { ob[off + b] = (uint8_t)(r & 255u); r >>= 8; }
                rout[i] = r;
            } else {
                rout[i] = rin[2 * i];
            }
        }
        __syncthreads();
        cur ^= 1;
    }
    if (t == 0) {
        uint32_t r = R[cur][0];
        for (int b = 0; b < S.efinal; ++b) { ob[S.foff + b] = (uint8_t)(r & 255u); r >>= 8; }
    }
    __syncthreads();
}

// bytes -> values (the inverse, reducing every value modulo its radix as the
// format's decoder does, so any byte string decodes to in-range values).
// Returns the buffer index holding R[0..p).  Contains barriers.
template <int PAD>
__device__ __forceinline__ int mixed_decode(const uint8_t *in, const EncSched &S,
                                            uint32_t (*R)[PAD]) {
    int cur = 0;
    if (threadIdx.x == 0) {
        uint32_t r = 0;
        for (int b = S.efinal - 1; b >= 0; --b) r = (r << 8) | in[S.foff + b];
        R[0][0] = S.mfinal ? r % S.mfinal : 0;
    }
    __syncthreads();
    for (int l = S.nlev - 1; l >= 0; --l) {
        const EncLevel L = S.lev[l];
        const uint32_t *rin = R[cur];
        uint32_t *rout = R[cur ^ 1];
        for (int i = threadIdx.x; 2 * i < L.n; i += blockDim.x) {
            if (2 * i + 1 < L.n) {
                const bool last = (2 * i + 1 == L.n - 1);
                uint32_t r = rin[i];
                const int e = last ? L.elast : L.eu;
                const int off = L.boff + i * L.eu;
                for (int b = e - 1; b >= 0; --b) r = (r << 8) | in[off + b];
                const uint32_t mb = last ? L.mlast : L.mu;
                rout[2 * i] = r % L.mu;
                rout[2 * i + 1] = (r / L.mu) % mb;
            } else {
                rout[2 * i] = rin[i];
            }
        }
        __syncthreads();
        cur ^= 1;
    }
    return cur;
}

}  // namespace snt
