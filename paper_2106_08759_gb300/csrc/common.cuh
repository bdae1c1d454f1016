// common.cuh -- parameter traits and small device helpers shared by the
// sntrup GB300 kernels.  (CUDA path only; nothing here is shared with the
// CPU oracle.)
//
// Rings (arXiv 2106.08759, Sec. 2.1): R/q = (Z/q)[x]/(x^p - x - 1) and
// R/3 = (Z/3)[x]/(x^p - x - 1); (p, q, w) = (653, 4621, 288),
// (761, 4591, 286), (857, 5167, 322).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace snt {

template <int P> struct Prm;
template <> struct Prm<653> { static constexpr int p = 653, q = 4621, w = 288; };
template <> struct Prm<761> { static constexpr int p = 761, q = 4591, w = 286; };
template <> struct Prm<857> { static constexpr int p = 857, q = 5167, w = 322; };

// Whether h can be formed from the inverses of the level-1 nodes (the leaf
// level of the down-sweep skipped): h_L = 3 inv(P) (g_L f_R) with
// |g_L f_R| <= 2w taken as one f16 limb against inv(P)'s 6-bit limbs needs
// every limb sum, at most p * h_max * 2w, below 2^24 (h_max the high limb of
// a centred residue).
template <int P> struct FuseLeaf {
    static constexpr long long hmax = ((Prm<P>::q - 1) / 2 + 32) / 64;
    static constexpr bool ok = (long long)Prm<P>::p * hmax * 2 * Prm<P>::w < (1LL << 24);
};

// Geometry of one polynomial in device memory.
//   words: 32-trit words holding the p + 1 trits a divstep state needs
//   pad:   coefficient stride of every stored polynomial (words * 32), so
//          int16 rows are multiples of 64 bytes and int8 rows of 32 bytes
//   p8:    p rounded up to a multiple of 8 (register tile of the products)
template <int P> struct Geo {
    static constexpr int p = Prm<P>::p;
    static constexpr int q = Prm<P>::q;
    static constexpr int w = Prm<P>::w;
    static constexpr int half = (q - 1) / 2;
    static constexpr int words = (p + 1 + 31) / 32;
    static constexpr int pad = words * 32;
    static constexpr int p8 = (p + 7) / 8 * 8;
    static constexpr int small_bytes = (p + 3) / 4;
};

// Device error word bits (read and cleared by snt_ctx_sync).
enum : int {
    ERR_RESAMPLE = 1,     // a key exhausted its g attempts
    ERR_ROOT = 2,         // product-tree root not invertible (cannot happen in a field)
    ERR_TIMEOUT = 4,      // a bounded wait gave up
};

constexpr int kMaxGAttempts = 32;

// Centred representative of x modulo Q, for any int32 x.
template <int Q> __device__ __forceinline__ int cmod(int x) {
    int r = x % Q;                    // (-Q, Q), sign of x
    r += (r < -(Q - 1) / 2) ? Q : 0;
    r -= (r > (Q - 1) / 2) ? Q : 0;
    return r;
}

// Representative in [0, Q) of x in [-Q, 2Q).
template <int Q> __device__ __forceinline__ int freeze_lazy(int x) {
    x += (x < 0) ? Q : 0;
    x -= (x >= Q) ? Q : 0;
    return x;
}

// Lazy reduction for |x| < 2^27: returns r == x (mod Q) with -Q <= r < 2Q.
// quotient estimate floor(x * floor(2^32/Q) / 2^32) is off by at most one.
template <int Q> __device__ __forceinline__ int lazy_red(int x) {
    constexpr int M = (int)((1ull << 32) / (unsigned long long)Q);
    int t = __mulhi(x, M);
    return x - t * Q;
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds on a 128-bit
// counter with a 64-bit key advanced by the Weyl constants each round.
__device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                              uint32_t c3, uint32_t k0, uint32_t k1,
                                              uint32_t out[4]) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// Random block `blk` (words 4*blk .. 4*blk+3) of stream s, attempt a, key k.
// Counter layout: ((s << 16) | blk, a, k mod 2^32, k >> 32); key = seed halves.
__device__ __forceinline__ void rand_block(uint64_t seed, uint64_t k, uint32_t s,
                                           uint32_t a, uint32_t blk, uint32_t out[4]) {
    philox4x32_10((s << 16) | blk, a, (uint32_t)k, (uint32_t)(k >> 32),
                  (uint32_t)seed, (uint32_t)(seed >> 32), out);
}

enum : uint32_t { STREAM_G = 0, STREAM_F = 1, STREAM_RHO = 2, STREAM_ENC = 3 };

}  // namespace snt
#include "kernels.h"
namespace snt {

// Batch of key j of a launch (binary search over the batch table).
__device__ __forceinline__ BatchDesc key_batch(const KeyMap &km, int j) {
    if (km.nb == 0) return km.one;
    int lo = 0, hi = km.nb - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (km.tab[mid].key_base <= j) lo = mid; else hi = mid - 1;
    }
    return km.tab[lo];
}

// Index in the batch table of the batch of key j (0 for a single batch).
__device__ __forceinline__ int key_batch_index(const KeyMap &km, int j) {
    int lo = 0, hi = km.nb - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (km.tab[mid].key_base <= j) lo = mid; else hi = mid - 1;
    }
    return km.nb > 0 ? lo : 0;
}

// Flag index of key j's subtree: sub_size keys per subtree, or (sub_size 0)
// one subtree per batch of the table.
__device__ __forceinline__ int key_subtree(const KeyMap &km, int j, int sub_size) {
    return sub_size > 0 ? j / sub_size : key_batch_index(km, j);
}

// Batch owning node j of a forest level (pre: nb + 1 prefix sums).
__device__ __forceinline__ int level_batch(const int *pre, int nb, int j) {
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= j) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Node j of a level: its index in its own tree (idx), the first child row of
// that tree in the input level (base) and the tree's input count (n_in).
__device__ __forceinline__ void lm_node(const LevelMap &lm, int j, int &idx, int &base,
                                        int &n_in) {
    idx = j; base = 0; n_in = lm.n_in;
    if (lm.nb > 0) {
        const int b = level_batch(lm.pre_out, lm.nb, j);
        idx = j - lm.pre_out[b];
        base = lm.pre_in[b];
        n_in = lm.pre_in[b + 1] - base;
    } else if (lm.sub_out > 0) {
        const int b = j / lm.sub_out;
        idx = j - b * lm.sub_out;
        base = b * lm.n_in;
    }
}

}  // namespace snt
