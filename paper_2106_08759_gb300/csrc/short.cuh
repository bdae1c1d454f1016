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

// The warp sort below runs the bitonic network in its all-ascending form:
// to merge two sorted halves of a block of `size` slots, slot i is first
// compared with its mirror i ^ (size - 1) (the upper half read backwards),
// then the block's halves, quarters, ... are cleaned with partners i ^ S,
// every comparator putting the minimum at the lower slot.  It sorts the same
// values into the same order as the alternating-direction network, and no
// comparator's direction depends on the slot.

// In-lane flip stage of blocks of SIZE <= 32 slots: slots r and r ^ (SIZE - 1).
template <int SIZE>
__device__ __forceinline__ void bitonic_lane_flip(uint32_t (&v)[32]) {
#pragma unroll
    for (int r = 0; r < 32; ++r)
        if ((r & (SIZE >> 1)) == 0) {
            const int o = r ^ (SIZE - 1);
            const uint32_t x = v[r], y = v[o];
            v[r] = min(x, y);
            v[o] = max(x, y);
        }
}

// In-lane half-cleaner stage: slots r and r | S (r & S == 0), ascending.
template <int S>
__device__ __forceinline__ void bitonic_lane_stage(uint32_t (&v)[32]) {
#pragma unroll
    for (int r = 0; r < 32; ++r)
        if ((r & S) == 0) {
            const uint32_t x = v[r], y = v[r | S];
            v[r] = min(x, y);
            v[r | S] = max(x, y);
        }
}

// The half-cleaners of an in-lane block of SIZE slots after its flip.
template <int SIZE>
__device__ __forceinline__ void bitonic_lane_clean(uint32_t (&v)[32]) {
    if constexpr (SIZE >= 4) {
        bitonic_lane_stage<SIZE / 4>(v);
        bitonic_lane_clean<SIZE / 2>(v);
    }
}

// The same Short draw by one warp: lane L holds slots 32L .. 32L+31 of the
// 1024-slot network in registers, so partners closer than 32 slots are in
// the same lane (compare-exchanges whose slots are constants) and the rest
// one lane-xor shuffle away; no shared memory and no barrier.  On return
// lane L holds sorted slots 32L .. 32L+31.
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
    // blocks of 2 .. 32 slots: inside the lane
    bitonic_lane_flip<2>(v);
    bitonic_lane_flip<4>(v);
    bitonic_lane_clean<4>(v);
    bitonic_lane_flip<8>(v);
    bitonic_lane_clean<8>(v);
    bitonic_lane_flip<16>(v);
    bitonic_lane_clean<16>(v);
    bitonic_lane_flip<32>(v);
    bitonic_lane_clean<32>(v);
    // blocks of 64 .. 1024 slots: the flip and the half-cleaners of 32 slots
    // and more across lanes, then the in-lane half-cleaners
#pragma unroll 1
    for (int size = 64; size <= 1024; size <<= 1) {
        {
            // mirror of slot 32 L + r: lane L ^ (size / 32 - 1), register 31 - r;
            // the lower slot is in the lane whose bit size / 64 is clear
            const int m = (size >> 5) - 1;
            const bool keep_min = (lane & (size >> 6)) == 0;
            uint32_t o[32];
#pragma unroll
            for (int r = 0; r < 32; ++r) o[r] = __shfl_xor_sync(0xffffffffu, v[31 - r], m);
#pragma unroll
            for (int r = 0; r < 32; ++r) v[r] = keep_min ? min(v[r], o[r]) : max(v[r], o[r]);
        }
#pragma unroll 1
        for (int stride = size >> 2; stride >= 32; stride >>= 1) {
            const int m = stride >> 5;
            const bool keep_min = (lane & m) == 0;
#pragma unroll
            for (int r = 0; r < 32; ++r) {
                const uint32_t o = __shfl_xor_sync(0xffffffffu, v[r], m);
                v[r] = keep_min ? min(v[r], o) : max(v[r], o);
            }
        }
        bitonic_lane_stage<16>(v);
        bitonic_lane_stage<8>(v);
        bitonic_lane_stage<4>(v);
        bitonic_lane_stage<2>(v);
        bitonic_lane_stage<1>(v);
    }
}

}  // namespace snt
