// toeplitz.cuh -- R/q multiplication c = a * b in (Z/q)[x]/(x^p - x - 1)
// for one CTA of p8/8 threads, each thread owning 8 consecutive outputs.
//
// With x^p = x + 1 (Sec. 2.1) every term a_i b_m of the schoolbook product
// lands in output j = i + m, or, when i + m >= p, in outputs i + m - p and
// i + m - p + 1.  Grouped by d = j - i this gives, for every output j >= 1,
//     c_j = sum_{i=0}^{p-1} a_i E[d + p - 1]  +  a_j b_{p-1},
//     E[d + p - 1] = b_d                      for d >= 0,
//                  = b_{p+d} + b_{p+d-1}      for d < 0,
// i.e. exactly p terms per output (a Toeplitz matrix-vector product), so all
// threads do the same work and no separate reduction pass is needed.  Output
// 0 gets one correction from output p - 1 (toeplitz_finish).
//
// Range: operands are centred, |a_i|, |E| <= (q-1)/2 = 2295 for sntrup761, so
// one term is below 5.27e6 and 256 terms below 1.35e9 < 2^31: the int32
// accumulators are reduced mod q after every 256 terms (the paper's bound
// 2295 * 2295 * 761 > 2^31, Sec. 3.3, is why a single pass would overflow).
#pragma once
#include "common.cuh"

namespace snt {

template <int P> struct Tp {
    static constexpr int p8 = Geo<P>::p8;
    static constexpr int OFF = 8;                                   // zero guard below E
    static constexpr int ESZ = (OFF + P + p8 - 1 + 3) / 4 * 4;      // E table length
    static constexpr int NT = p8 / 8;                               // threads per product
    static_assert((P & 3) == 1, "16-byte aligned windows need p = 1 mod 4");
};

// E table of b (centred, any stride) into shared memory; Q is the
// coefficient modulus (q for R/q, 3 for R/3).
template <int P, typename T, int Q = Geo<P>::q>
__device__ __forceinline__ void fill_E(const T *__restrict__ b, int *Es) {
    for (int idx = threadIdx.x; idx < Tp<P>::ESZ; idx += blockDim.x) {
        const int t = idx - Tp<P>::OFF;
        int e = 0;
        if (t >= 0 && t <= 2 * P - 2) {
            const int d = t - (P - 1);
            e = (d >= 0) ? (int)b[d] : cmod<Q>((int)b[P + d] + (int)b[P + d - 1]);
        }
        Es[idx] = e;
    }
}

// a (int16 or int8, first p entries) into shared int32, zero up to p8.
template <int P, typename T>
__device__ __forceinline__ void fill_A(const T *__restrict__ a, int *As) {
    for (int i = threadIdx.x; i < Tp<P>::p8; i += blockDim.x) As[i] = (i < P) ? (int)a[i] : 0;
}

// acc[k][t] = sum_i A_k[i] E[j0 + t - i + p - 1] over i in [ib_lo, ib_hi)
// (multiples of 8) for NA operands sharing E, j0 = 8 * tloc; reduced mod q
// every 256 terms and at the end (centred).
template <int P, int NA, int Q = Geo<P>::q>
__device__ __forceinline__ void toeplitz_tile(const int *const (&As)[NA], const int *Es, int tloc,
                                              int ib_lo, int ib_hi, int (&acc)[NA][8]) {
    const int j0 = 8 * tloc;
    const int base = Tp<P>::OFF + P - 9 + j0;  // window start for i-block 0
#pragma unroll
    for (int k = 0; k < NA; ++k)
#pragma unroll
        for (int t = 0; t < 8; ++t) acc[k][t] = 0;
    int whi[8];
    {
        const int4 h0 = *reinterpret_cast<const int4 *>(&Es[base - ib_lo + 8]);
        const int4 h1 = *reinterpret_cast<const int4 *>(&Es[base - ib_lo + 12]);
        whi[0] = h0.x; whi[1] = h0.y; whi[2] = h0.z; whi[3] = h0.w;
        whi[4] = h1.x; whi[5] = h1.y; whi[6] = h1.z; whi[7] = h1.w;
    }
#pragma unroll 2
    for (int ib = ib_lo; ib < ib_hi; ib += 8) {
        int wlo[8];
        const int4 l0 = *reinterpret_cast<const int4 *>(&Es[base - ib]);
        const int4 l1 = *reinterpret_cast<const int4 *>(&Es[base - ib + 4]);
        wlo[0] = l0.x; wlo[1] = l0.y; wlo[2] = l0.z; wlo[3] = l0.w;
        wlo[4] = l1.x; wlo[5] = l1.y; wlo[6] = l1.z; wlo[7] = l1.w;
#pragma unroll
        for (int k = 0; k < NA; ++k) {
            const int4 a0 = *reinterpret_cast<const int4 *>(&As[k][ib]);
            const int4 a1 = *reinterpret_cast<const int4 *>(&As[k][ib + 4]);
            const int a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const int wi = 8 + t - u;  // 1 .. 15
                    const int e = (wi >= 8) ? whi[wi - 8] : wlo[wi];
                    acc[k][t] += a[u] * e;
                }
        }
#pragma unroll
        for (int z = 0; z < 8; ++z) whi[z] = wlo[z];
        if (((ib + 8 - ib_lo) & 255) == 0) {
#pragma unroll
            for (int k = 0; k < NA; ++k)
#pragma unroll
                for (int t = 0; t < 8; ++t) acc[k][t] = cmod<Q>(acc[k][t]);
        }
    }
#pragma unroll
    for (int k = 0; k < NA; ++k)
#pragma unroll
        for (int t = 0; t < 8; ++t) acc[k][t] = cmod<Q>(acc[k][t]);
}

// K-way split of the i-range: thread tid = grp * NT + tloc sums i-blocks
// [grp * per, (grp + 1) * per); group 0 ends with the full centred sums.
// Every thread of the CTA must call it (it contains barriers when K > 1).
// Threads beyond NT * K take no part (they only join the barriers).
template <int P, int NA, int K, int Q = Geo<P>::q>
__device__ __forceinline__ void toeplitz_split(const int *const (&As)[NA], const int *Es,
                                               int *part, int (&acc)[NA][8]) {
    constexpr int NT = Tp<P>::NT;
    constexpr int per = (NT + K - 1) / K;  // i-blocks of 8 per group
    const int tloc = threadIdx.x % NT, grp = threadIdx.x / NT;
    const int ib_lo = min(grp * per, NT) * 8, ib_hi = min((grp + 1) * per, NT) * 8;
    toeplitz_tile<P, NA, Q>(As, Es, tloc, ib_lo, ib_hi, acc);
    if (K > 1) {
        const int j0 = 8 * tloc;
#pragma unroll
        for (int k = 0; k < NA; ++k) {
            if (grp > 0 && grp < K)
#pragma unroll
                for (int t = 0; t < 8; ++t) part[(grp - 1) * Tp<P>::p8 + j0 + t] = acc[k][t];
            __syncthreads();
            if (grp == 0) {
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    int sum = acc[k][t];
                    for (int g = 0; g < K - 1; ++g) sum += part[g * Tp<P>::p8 + j0 + t];
                    acc[k][t] = cmod<Q>(sum);
                }
            }
            __syncthreads();
        }
    }
}

// Adds the [j >= 1] a_j b_{p-1} term, reduces, fixes output 0 and returns
// centred values (zero for j >= p) in the threads with active = true (one
// thread per 8 outputs, tloc = its tile).  Output 0 needs a fix: the E table
// also folds the x^(p-1) coefficient c_{p-1} = sum_{i+m=p-1} a_i b_m into row
// 0, although x^(p-1) is not reduced.  The row-(p-1) result is exactly
// c_{p-1} + a_{p-1} b_{p-1}, so
//     c_0 = (row 0) - (row p-1) + (a_0 + a_{p-1}) b_{p-1}.
// Contains a __syncthreads(): every thread of the CTA must call it.
template <int P, int NA, int Q = Geo<P>::q>
__device__ __forceinline__ void toeplitz_finish(const int *const (&As)[NA], const int (&blast)[NA],
                                                int (&acc)[NA][8], int tloc, bool active) {
    __shared__ int last_row[NA];
    const int j0 = 8 * tloc;
    if (active) {
#pragma unroll
        for (int k = 0; k < NA; ++k)
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int j = j0 + t;
                int v = acc[k][t];
                if (j >= 1 && j < P) v += As[k][j] * blast[k];
                acc[k][t] = (j < P) ? cmod<Q>(v) : 0;
                if (j == P - 1) last_row[k] = acc[k][t];
            }
    }
    __syncthreads();
    if (active && tloc == 0) {
#pragma unroll
        for (int k = 0; k < NA; ++k)
            acc[k][0] = cmod<Q>(acc[k][0] - last_row[k] + (As[k][0] + As[k][P - 1]) * blast[k]);
    }
}

// Output-split form, for the narrow tree levels whose few products would
// each keep one SM busy for the whole level: the NT output tiles are cut into
// S segments of TS tiles, each segment is one CTA (so a product spreads over
// S SMs), and each CTA splits the i-range over K thread groups (TS * K
// threads).  No barrier is needed between CTAs: every segment reads all of A
// and E and writes only its own outputs.  The output-0 fix needs row p - 1,
// which lives in the last segment, so segment 0 recomputes that one row as a
// dot product (warp 0).
template <int P, int S> struct SegGeo {
    static constexpr int NT = Tp<P>::NT;
    static constexpr int TS = (NT + S - 1) / S;  // tiles per segment
};

// Finished, centred outputs of tile tloc = seg * TS + (thread % TS) for the
// threads that return active = true (group 0, tloc < NT); the a_j b_{p-1}
// term and the output-0 fix are included, outputs j >= p are zero.  Every
// thread of the CTA must call it (it contains barriers).
template <int P, int NA, int S, int K, int Q = Geo<P>::q>
__device__ __forceinline__ void toeplitz_seg(const int *const (&As)[NA], const int *Es,
                                             const int (&blast)[NA], int *part, int seg,
                                             int (&acc)[NA][8], int &tloc, bool &active) {
    constexpr int NT = Tp<P>::NT, TS = SegGeo<P, S>::TS;
    constexpr int per = (NT + K - 1) / K;  // i-blocks of 8 per group
    __shared__ int last_row[NA];
    const int tl = threadIdx.x % TS, grp = threadIdx.x / TS;
    tloc = seg * TS + tl;
    const bool tile = tloc < NT && grp < K;
    if (tile) {
        const int ib_lo = min(grp * per, NT) * 8, ib_hi = min((grp + 1) * per, NT) * 8;
        toeplitz_tile<P, NA, Q>(As, Es, tloc, ib_lo, ib_hi, acc);
    } else {
#pragma unroll
        for (int k = 0; k < NA; ++k)
#pragma unroll
            for (int t = 0; t < 8; ++t) acc[k][t] = 0;
    }
    if (seg == 0 && threadIdx.x < 32) {
        // row p-1: sum_i A_i E[2p - 2 - i]; at most ceil(p/32) <= 27 terms of
        // <= (q-1)^2/4 per lane before the reduction, below 2^31
#pragma unroll
        for (int k = 0; k < NA; ++k) {
            int r = 0;
            for (int i = threadIdx.x; i < P; i += 32) r += As[k][i] * Es[Tp<P>::OFF + 2 * P - 2 - i];
            r = cmod<Q>(r);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
            if (threadIdx.x == 0) last_row[k] = cmod<Q>(r + As[k][P - 1] * blast[k]);
        }
    }
    const int j0 = 8 * tloc;
#pragma unroll
    for (int k = 0; k < NA; ++k) {
        if (K > 1 && tile && grp > 0)
#pragma unroll
            for (int t = 0; t < 8; ++t) part[((grp - 1) * TS + tl) * 8 + t] = acc[k][t];
        __syncthreads();
        if (K > 1 && tile && grp == 0)
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                int sum = acc[k][t];
                for (int g = 0; g < K - 1; ++g) sum += part[(g * TS + tl) * 8 + t];
                acc[k][t] = cmod<Q>(sum);
            }
        __syncthreads();
    }
    active = tile && grp == 0;
    if (active) {
#pragma unroll
        for (int k = 0; k < NA; ++k) {
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int j = j0 + t;
                int v = acc[k][t];
                if (j >= 1 && j < P) v += As[k][j] * blast[k];
                acc[k][t] = (j < P) ? cmod<Q>(v) : 0;
            }
            if (tloc == 0)
                acc[k][0] = cmod<Q>(acc[k][0] - last_row[k] + (As[k][0] + As[k][P - 1]) * blast[k]);
        }
    }
}

// Stores 8 outputs (j0 .. j0+7) as int16; pads from p8 to `pad` are zeroed by
// the threads that own the last tile.
template <int P>
__device__ __forceinline__ void store_tile(int16_t *__restrict__ c, const int (&v)[8], int pad,
                                           int tloc) {
    const int j0 = 8 * tloc;
    int4 pk;
    pk.x = (v[0] & 0xffff) | (v[1] << 16);
    pk.y = (v[2] & 0xffff) | (v[3] << 16);
    pk.z = (v[4] & 0xffff) | (v[5] << 16);
    pk.w = (v[6] & 0xffff) | (v[7] << 16);
    *reinterpret_cast<int4 *>(&c[j0]) = pk;
    if (tloc == Tp<P>::NT - 1)
        for (int j = Tp<P>::p8; j < pad; ++j) c[j] = 0;
}

}  // namespace snt
