// short.cuh -- sampling of a Short element (weight w, coefficients +-1 at
// uniform positions) by sorting forced-low-bit random words; one CTA of (at
// least) 256 threads.  Reading of the uniform draw (Sec. 3.1 KeyGen step 3):
// p words of the given stream; the first w have bit 0 cleared (low bits
// decode to -1 or +1), the rest get low bits 01 (decode to 0); the words are
// sorted as unsigned integers and coefficient j is (word_j mod 4) - 1.  The
// sort is a 1024-slot bitonic network padded with 0xFFFFFFFF (no real word
// can equal it): thread t holds slots 4t .. 4t+3 in registers; partners closer
// than 4 slots are in the same thread, closer than 128 in the same warp
// (shuffles), farther ones in another warp (through shared memory xs[1024]).
#pragma once
#include "common.cuh"

namespace snt {

// On return thread t (< 256) holds sorted slots 4t .. 4t+3 in v; threads
// >= 256 only join the barriers.  All threads of the CTA must call it.
template <int P>
__device__ __forceinline__ void short_sorted_words(uint64_t seed, uint64_t k, uint32_t stream,
                                                   uint32_t (&v)[4], uint32_t *xs) {
    using G = Geo<P>;
    const int t = threadIdx.x;
    const bool mine = t < 256;
    // words of the stream, low bits forced; sentinels above p
    v[0] = v[1] = v[2] = v[3] = 0u;
    if (mine && 4 * t < G::p) rand_block(seed, k, stream, 0u, (uint32_t)t, v);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int idx = 4 * t + r;
        if (idx < G::w) v[r] = v[r] & ~1u;
        else if (idx < G::p) v[r] = (v[r] & ~3u) | 1u;
        else v[r] = 0xFFFFFFFFu;
    }

    // ascending bitonic sort of the 1024 slots
#pragma unroll 1
    for (int size = 2; size <= 1024; size <<= 1) {
#pragma unroll 1
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride >= 4) {
                uint32_t o[4];
                if (stride >= 128) {
                    if (mine) *reinterpret_cast<uint4 *>(&xs[4 * t]) = make_uint4(v[0], v[1], v[2], v[3]);
                    __syncthreads();
                    const uint4 q = mine ? *reinterpret_cast<const uint4 *>(&xs[4 * (t ^ (stride >> 2))])
                                         : make_uint4(0u, 0u, 0u, 0u);
                    o[0] = q.x; o[1] = q.y; o[2] = q.z; o[3] = q.w;
                    __syncthreads();
                } else {
#pragma unroll
                    for (int r = 0; r < 4; ++r) o[r] = __shfl_xor_sync(0xffffffffu, v[r], stride >> 2);
                }
                const int i = 4 * t;  // same relation for all four slots of this thread
                const bool asc = (i & size) == 0;
                const bool low = (i & stride) == 0;  // this slot is the lower one of its pair
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const uint32_t mn = min(v[r], o[r]), mx = max(v[r], o[r]);
                    v[r] = (low == asc) ? mn : mx;
                }
            } else {
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const bool asc = ((4 * t + r) & size) == 0;  // size 2 depends on r
                    if ((r & stride) == 0) {
                        const uint32_t a = v[r], b = v[r | stride];
                        const bool sw = (a > b) == asc;
                        v[r] = sw ? b : a;
                        v[r | stride] = sw ? a : b;
                    }
                }
            }
        }
    }

}

// One compare-exchange stage inside a lane: slots r and r | S (r & S == 0)
// of v, ascending when SIZE > 0 and (r & SIZE) == 0 (the direction of small
// bitonic blocks is fixed by the slot) or, when SIZE == 0, when asc.
template <int S, int SIZE>
__device__ __forceinline__ void bitonic_lane_stage(uint32_t (&v)[32], bool asc) {
#pragma unroll
    for (int r = 0; r < 32; ++r)
        if ((r & S) == 0) {
            const bool a = SIZE ? ((r & SIZE) == 0) : asc;
            const uint32_t x = v[r], y = v[r | S];
            const uint32_t mn = min(x, y), mx = max(x, y);
            v[r] = a ? mn : mx;
            v[r | S] = a ? mx : mn;
        }
}

// The same Short draw by one warp: lane L holds slots 32L .. 32L+31 of the
// 1024-slot network in registers, so partners closer than 32 slots are in
// the same lane (compare-exchanges, their direction a constant for blocks
// up to 16 slots) and the rest one lane-xor shuffle away; no shared memory
// and no barrier.  On return lane L holds sorted slots 32L .. 32L+31.
template <int P>
__device__ __forceinline__ void short_sorted_warp(uint64_t seed, uint64_t k, uint32_t stream,
                                                  uint32_t (&v)[32]) {
    using G = Geo<P>;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        uint32_t r[4] = {0u, 0u, 0u, 0u};
        const int blk = 8 * lane + b;
        if (4 * blk < G::p) rand_block(seed, k, stream, 0u, (uint32_t)blk, r);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int idx = 4 * blk + j;
            uint32_t x = r[j];
            if (idx < G::w) x &= ~1u;
            else if (idx < G::p) x = (x & ~3u) | 1u;
            else x = 0xFFFFFFFFu;
            v[4 * b + j] = x;
        }
    }
    bitonic_lane_stage<1, 2>(v, true);
    bitonic_lane_stage<2, 4>(v, true);
    bitonic_lane_stage<1, 4>(v, true);
    bitonic_lane_stage<4, 8>(v, true);
    bitonic_lane_stage<2, 8>(v, true);
    bitonic_lane_stage<1, 8>(v, true);
    bitonic_lane_stage<8, 16>(v, true);
    bitonic_lane_stage<4, 16>(v, true);
    bitonic_lane_stage<2, 16>(v, true);
    bitonic_lane_stage<1, 16>(v, true);
#pragma unroll 1
    for (int size = 32; size <= 1024; size <<= 1) {
        const bool asc = ((32 * lane) & size) == 0;
#pragma unroll 1
        for (int stride = size >> 1; stride >= 32; stride >>= 1) {
            const int m = stride >> 5;
            const bool keep_min = ((lane & m) == 0) == asc;  // lower slot of an ascending pair
#pragma unroll
            for (int r = 0; r < 32; ++r) {
                const uint32_t o = __shfl_xor_sync(0xffffffffu, v[r], m);
                v[r] = keep_min ? min(v[r], o) : max(v[r], o);
            }
        }
        bitonic_lane_stage<16, 0>(v, asc);
        bitonic_lane_stage<8, 0>(v, asc);
        bitonic_lane_stage<4, 0>(v, asc);
        bitonic_lane_stage<2, 0>(v, asc);
        bitonic_lane_stage<1, 0>(v, asc);
    }
}

}  // namespace snt
