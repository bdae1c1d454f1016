// mma_mul.cuh -- R/q multiplication on the tensor cores, exact.
//
// The product is the same Toeplitz matrix-vector form as toeplitz.cuh (with
// x^p = x + 1, Sec. 2.1): for j >= 1
//     c_j = row_j + a_j b_{p-1},   row_j = sum_i a_i E[j - i + p - 1],
//     E[d + p - 1] = b_d (d >= 0),  b_{p+d} + b_{p+d-1} (d < 0),
// and c_0 = row_0 - row_{p-1} + a_0 b_{p-1}.
//
// Blocking.  With 16-coefficient blocks (j = 16 J + r, i = 16 I + k) the
// matrix block (J, I) depends only on D = J - I:
//     T_D[r][k] = E[16 D + r - k + p - 1],
// so for a fixed D, output blocks J_0 .. J_0 + 7 receive T_D * [a_{J_0 - D}
// .. a_{J_0 + 7 - D}]: one warp-level m16n8k16 MMA whose A operand is T_D
// and whose 8 columns are 8 input blocks.  An "MMA tile" is 8 output blocks
// (128 outputs); a warp owns NT consecutive tiles and runs D over the union
// of their ranges.  Input blocks outside [0, NBLK) are zero padding, so a
// tile outside its own D range only adds zeros and no bounds test is needed.
//
// Fragments straight from the E table.  In the m16n8k16 A fragment the
// thread (g = lane / 4, tig = lane % 4) holds the pairs (row g, cols 2tig,
// 2tig + 1), (g + 8, same cols), (g, 2tig + 8, 2tig + 9), (g + 8, 2tig + 8,
// 2tig + 9).  In T_D these are (E[x], E[x-1]), (E[x+8], E[x+7]),
// (E[x-8], E[x-9]) and (E[x], E[x-1]) again, x = 16D + g - 2 tig + p - 1:
// a table PE[x] holding the pair (E[x], E[x-1]) of both limbs gives one
// 64-bit shared load per register position, and no Toeplitz block is
// materialised.  The B fragment of a block of a (pairs 2tig, 2tig + 1 and
// 2tig + 8, 2tig + 9) of both limbs is likewise one 128-bit load.
//
// Exactness.  fp16 holds integers up to 2048 exactly; centred residues reach
// (q - 1) / 2 = 2583, so both operands are split into limbs
//     x = 64 h + l,  h = floor((x + 32) / 64) in [-41, 41], l in [-32, 31],
// and the limb products are accumulated in three sums: P_hh = sum h h',
// P_x = sum (h l' + l h') and P_ll = sum l l'.  Each is an integer below
// 2 * 768 * 41 * 32 < 2^24 in magnitude, so the f32 accumulation is exact in
// any order; then
//     row = 4096 P_hh + 64 P_x + P_ll
// is formed from the residues of the three sums mod q.  Four MMAs per step
// rather than the three of Karatsuba's (h + l)(h' + l'): the loop is bound by
// shared-memory wavefronts, and dropping the h + l limb from both tables
// takes a step from 20 wavefronts and 12 tensor-pipe cycles (two products
// per CTA) to 12 wavefronts and 16 cycles.
//
// One wide limb on the vector side (MODE_GW).  Every residue mod q has a
// representative that f16 holds exactly: the integers up to 2048 and the
// even ones up to 4096; an odd residue above 2048 in magnitude moves by q
// (odd) to an even value of magnitude at most q - 2049 (3118 for sntrup857).  With that
// value as the vector side's only limb, P_1 = sum h_E b' and P_2 = sum l_E b'
// need two MMAs per step (row = 64 P_1 + P_2), but a term now reaches
// 40 * 3118, so the f32 sums are exact only over 128 terms (8 steps:
// 128 * 40 * 3118 < 2^24): every 8 steps they are converted (exactly) and
// added into int32 sums.
//
// Small operands.  A leaf of the tree is 3f with coefficients in {-3, 0, 3}:
// its high limb is zero.  MODE_SA (vector side small) needs only
// P_1 = sum h_E l_a and P_2 = sum l_E l_a (row = 64 P_1 + P_2, two MMAs);
// MODE_SAE (both small) only P = sum l_E l_a (one MMA).
#pragma once
#include <cuda_fp16.h>

#include "common.cuh"

namespace snt {

enum : int { MODE_GEN = 0, MODE_SA = 1, MODE_SAE = 2, MODE_GW = 3 };

// Steps between the f32-to-int32 conversions of MODE_GW.
constexpr int kGwFlush = 8;

template <int P, int NT> struct MmaGeo {
    static constexpr int p = Prm<P>::p, q = Prm<P>::q;
    static constexpr int NBLK = (p + 15) / 16;       // 16-coefficient blocks
    static constexpr int NTILE = (NBLK + 7) / 8;     // MMA tiles (8 output blocks)
    static constexpr int NW = (NTILE + NT - 1) / NT; // warps per product
    static constexpr int AN = 16 * NBLK;             // padded coefficient count
    static constexpr int DMIN = 1 - NBLK, DMAX = 8 * NW * NT - 1;
    static constexpr int XLO = 16 * DMIN + p - 16;   // x of table entry 0
    static constexpr int PWN = 16 * (DMAX - DMIN) + 32;
    static constexpr int PADB = 8 * NT;              // zero blocks on each side of a
    static constexpr int VBN = (NBLK + 2 * PADB) * 4;  // B records (block, tig)
};

// E side of one product: per x the pairs (E[x], E[x-1]) of the h and l
// limbs (f16x2 words), and the operand E is built from.
template <int P, int NT> struct MmaE {
    union {
        uint2 pe[MmaGeo<P, NT>::PWN];
        uint32_t pl[MmaGeo<P, NT>::PWN];  // MODE_SAE: the l pairs only
    } t;
    int16_t b[MmaGeo<P, NT>::AN];
};
// Vector side of one product: per (block, tig) the B words (h01, h89, l01,
// l89), then (after the MMA loop) the staged row sums.
template <int P, int NT> struct MmaA {
    union {
        uint4 hl[MmaGeo<P, NT>::VBN];
        uint2 sl[MmaGeo<P, NT>::VBN];  // MODE_SA / MODE_SAE: the l words (l01, l89)
        int stage[MmaGeo<P, NT>::AN + MmaGeo<P, NT>::AN / 4];  // at stage_slot(j)
    } u;
    int16_t a[MmaGeo<P, NT>::AN];
};

// Slot of row sum j in the staging array: 8 padding words after every 32,
// so the four lanes of a fragment column (rows 32 apart) hit distinct banks.
__device__ __forceinline__ int stage_slot(int j) { return j + 8 * (j >> 5); }

__device__ __forceinline__ void limbs64(int x, int &h, int &l) {
    h = (x + 32) >> 6;
    l = x - 64 * h;
}

// f16x2 of two small integers |lo|, |hi| < 512: 1536 + v lies in [1024,
// 2048), where f16 steps by one, so its bit pattern is 0x6600 + v; one f16x2
// subtraction of 1536 leaves v exactly.
__device__ __forceinline__ uint32_t h2_small(int lo, int hi) {
    const uint32_t biased = 0x66006600u + (uint32_t)lo + ((uint32_t)hi << 16);
    uint32_t d;
    asm("add.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(biased), "r"(0xE600E600u));
    return d;
}

__device__ __forceinline__ void mma16816(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// E table value t in [0, 2p - 2], zero elsewhere; b centred in shared memory
// (so a folded sum b_{t+1} + b_t needs at most one correction by q).  Q is
// the coefficient modulus: q for R/q, 3 for R/3.
template <int P, int Q = Prm<P>::q> __device__ __forceinline__ int mma_E(const int16_t *b, int t) {
    constexpr int p = Prm<P>::p, q = Q, h = (q - 1) / 2;
    if (t < 0 || t > 2 * p - 2) return 0;
    if (t >= p - 1) return b[t - p + 1];
    int v = (int)b[t + 1] + (int)b[t];
    v -= (v > h) ? q : 0;
    v += (v < -h) ? q : 0;
    return v;
}

// f16x2 of two integers exact in f16: |x| <= 2048, or x even and |x| <= 4096.
__device__ __forceinline__ uint32_t h2_int(int lo, int hi) {
    const __half2 h = __halves2half2(__int2half_rn(lo), __int2half_rn(hi));
    return *reinterpret_cast<const uint32_t *>(&h);
}

// A representative of the centred residue x (|x| <= (Q-1)/2) exact in f16:
// x itself unless x is odd and |x| > 2048, then x -+ Q (even, |.| <= Q - 2049).
template <int Q> __device__ __forceinline__ int f16_rep(int x) {
    static_assert(Q % 2 == 1 && Q - 2049 <= 4096, "representative must be exact in f16");
    const bool move = (x & 1) && (x > 2048 || x < -2048);
    return move ? (x > 0 ? x - Q : x + Q) : x;
}

// Vector side: a (global, centred int16 or int8, first p entries) into
// shared memory, threads tid = 0 .. nth-1 of the group.
template <int P, int NT, int MODE = MODE_GEN, typename T = int16_t>
__device__ __forceinline__ void mma_fill_a(const T *__restrict__ a, MmaA<P, NT> &s, int tid,
                                           int nth) {
    using M = MmaGeo<P, NT>;
    for (int r = tid; r < M::VBN; r += nth) {  // record (block I, tig)
        const int I = r / 4 - M::PADB, tig = r & 3;
        int v[4] = {0, 0, 0, 0};  // coefficients 2tig, 2tig+1, 2tig+8, 2tig+9
        if (I >= 0 && I < M::NBLK) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int k = 16 * I + 2 * tig + (u & 1) + 8 * (u >> 1);
                v[u] = k < M::p ? (int)a[k] : 0;
                s.a[k] = (int16_t)v[u];
            }
        }
        if constexpr (MODE == MODE_GW) {  // one wide limb: a representative exact in f16
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = f16_rep<Prm<P>::q>(v[u]);
            s.u.sl[r] = make_uint2(h2_int(v[0], v[1]), h2_int(v[2], v[3]));
        } else if constexpr (MODE != MODE_GEN) {  // small coefficients: the value is its own l limb
            s.u.sl[r] = make_uint2(h2_small(v[0], v[1]), h2_small(v[2], v[3]));
        } else {
            int h[4], l[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) limbs64(v[u], h[u], l[u]);
            s.u.hl[r] = make_uint4(h2_small(h[0], h[1]), h2_small(h[2], h[3]), h2_small(l[0], l[1]),
                                   h2_small(l[2], l[3]));
        }
    }
}


// Vector side with one limb of magnitude up to 2048 (a product of two small
// elements), from int16 in any memory: the MODE_SA records with the value
// itself in the l slot.
template <int P, int NT>
__device__ __forceinline__ void mma_fill_a_wide(const int16_t *a, MmaA<P, NT> &s, int tid, int nth) {
    using M = MmaGeo<P, NT>;
    for (int r = tid; r < M::VBN; r += nth) {
        const int I = r / 4 - M::PADB, tig = r & 3;
        int v[4] = {0, 0, 0, 0};
        if (I >= 0 && I < M::NBLK) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int k = 16 * I + 2 * tig + (u & 1) + 8 * (u >> 1);
                v[u] = k < M::p ? (int)a[k] : 0;
                s.a[k] = (int16_t)v[u];
            }
        }
        s.u.sl[r] = make_uint2(h2_int(v[0], v[1]), h2_int(v[2], v[3]));
    }
}

// E side, step 1: b into shared memory.
template <int P, int NT>
__device__ __forceinline__ void mma_fill_b(const int16_t *__restrict__ b, MmaE<P, NT> &s, int tid,
                                           int nth) {
    using M = MmaGeo<P, NT>;
    for (int k = tid; k < M::AN; k += nth) s.b[k] = k < M::p ? b[k] : 0;
}

// E side, step 2 (after a barrier): the limb pair table, two neighbouring
// entries per thread (three E values, one 16-byte store).
template <int P, int NT, int MODE = MODE_GEN, int Q = Prm<P>::q>
__device__ __forceinline__ void mma_fill_pe(MmaE<P, NT> &s, int tid, int nth) {
    using M = MmaGeo<P, NT>;
    static_assert(M::PWN % 2 == 0, "pair table of even length");
    for (int w = 2 * tid; w < M::PWN; w += 2 * nth) {
        const int x = w + M::XLO;
        const int em = mma_E<P, Q>(s.b, x - 1), e0 = mma_E<P, Q>(s.b, x), e1 = mma_E<P, Q>(s.b, x + 1);
        if (MODE == MODE_SAE) {  // small E: the value is its own l limb
            *reinterpret_cast<uint2 *>(&s.t.pl[w]) = make_uint2(h2_small(e0, em), h2_small(e1, e0));
            continue;
        }
        int hm, lm, h0, l0, h1, l1;
        limbs64(em, hm, lm);
        limbs64(e0, h0, l0);
        limbs64(e1, h1, l1);
        *reinterpret_cast<uint4 *>(&s.t.pe[w]) =
            make_uint4(h2_small(h0, hm), h2_small(l0, lm), h2_small(h1, h0), h2_small(l1, l0));
    }
}

// Tiles [T0, T0 + NT) of NPR products sharing one E side, by one warp:
// accumulates the limb sums of every (tile, product): P_hh, P_x, P_ll
// (MODE_GEN), P_1, P_2 (MODE_SA) or P (MODE_SAE).  A2 of step D + 1 is A1 of
// step D (x advances by 16), so two table loads per step suffice.
// ks / nks: this warp's share of the D range when a tile's sum is split over
// nks warps (contiguous parts, reduced by mma_ksplit_reduce).
template <int P, int NT, int NPR, int MODE = MODE_GEN>
__device__ __forceinline__ void mma_tiles(const MmaE<P, NT> &E, const MmaA<P, NT> *const (&A)[NPR],
                                          int T0, int lane, float (&acc)[NT][NPR][3][4],
                                          int ks = 0, int nks = 1) {
    using M = MmaGeo<P, NT>;
    const int g = lane >> 2, tig = lane & 3;
#pragma unroll
    for (int tt = 0; tt < NT; ++tt)
#pragma unroll
        for (int pr = 0; pr < NPR; ++pr)
#pragma unroll
            for (int m = 0; m < 3; ++m)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[tt][pr][m][c] = 0.f;
    const int dall = 8 * T0 - (M::NBLK - 1);          // first D of the tiles
    const int dn = 8 * (NT - 1) + 7 + M::NBLK;        // D values of the tiles
    const int part = (dn + nks - 1) / nks;
    const int dlo = dall + ks * part;
    const int dhi = min(dall + dn, dlo + part) - 1;
    const int x0 = 16 * dlo + g - 2 * tig + M::p - 1 - M::XLO;  // table index at D = dlo
    int rec = 4 * (8 * T0 + g - dlo + M::PADB) + tig;            // B record of tile T0
    if (MODE == MODE_SAE) {
        const uint32_t *pl = E.t.pl + x0;
        uint32_t a2 = pl[-8];
#pragma unroll 2
        for (int D = dlo; D <= dhi; ++D, pl += 16, rec -= 4) {
            const uint32_t a0 = pl[0], a1 = pl[8];
#pragma unroll
            for (int tt = 0; tt < NT; ++tt)
#pragma unroll
                for (int pr = 0; pr < NPR; ++pr) {
                    const uint2 b = A[pr]->u.sl[rec + 32 * tt];
                    mma16816(acc[tt][pr][0], a0, a1, a2, a0, b.x, b.y);
                }
            a2 = a1;
        }
        return;
    }
    const uint2 *pe = E.t.pe + x0;
    uint2 A2 = pe[-8];
#pragma unroll 2
    for (int D = dlo; D <= dhi; ++D, pe += 16, rec -= 4) {
        const uint2 A0 = pe[0], A1 = pe[8];
#pragma unroll
        for (int tt = 0; tt < NT; ++tt)
#pragma unroll
            for (int pr = 0; pr < NPR; ++pr) {
                if (MODE == MODE_SA) {
                    const uint2 b = A[pr]->u.sl[rec + 32 * tt];
                    mma16816(acc[tt][pr][0], A0.x, A1.x, A2.x, A0.x, b.x, b.y);
                    mma16816(acc[tt][pr][1], A0.y, A1.y, A2.y, A0.y, b.x, b.y);
                } else {
                    const uint4 b = A[pr]->u.hl[rec + 32 * tt];
                    mma16816(acc[tt][pr][0], A0.x, A1.x, A2.x, A0.x, b.x, b.y);  // h h'
                    mma16816(acc[tt][pr][1], A0.x, A1.x, A2.x, A0.x, b.z, b.w);  // h l'
                    mma16816(acc[tt][pr][1], A0.y, A1.y, A2.y, A0.y, b.x, b.y);  // l h'
                    mma16816(acc[tt][pr][2], A0.y, A1.y, A2.y, A0.y, b.z, b.w);  // l l'
                }
            }
        A2 = A1;
    }
}

// MODE_GW: tiles [T0, T0 + NT) of NPR products sharing one E side, by one
// warp, into int32 sums P_1 = sum h_E b', P_2 = sum l_E b' (f32 partial sums
// over kGwFlush steps, converted exactly).  ks / nks as for mma_tiles.
template <int P, int NT, int NPR>
__device__ __forceinline__ void mma_tiles_gw(const MmaE<P, NT> &E, const MmaA<P, NT> *const (&A)[NPR],
                                             int T0, int lane, int (&iacc)[NT][NPR][2][4], int ks = 0,
                                             int nks = 1) {
    using M = MmaGeo<P, NT>;
    const int g = lane >> 2, tig = lane & 3;
#pragma unroll
    for (int tt = 0; tt < NT; ++tt)
#pragma unroll
        for (int pr = 0; pr < NPR; ++pr)
#pragma unroll
            for (int m = 0; m < 2; ++m)
#pragma unroll
                for (int c = 0; c < 4; ++c) iacc[tt][pr][m][c] = 0;
    const int dall = 8 * T0 - (M::NBLK - 1);
    const int dn = 8 * (NT - 1) + 7 + M::NBLK;
    const int part = (dn + nks - 1) / nks;
    const int dlo = dall + ks * part;
    const int dhi = min(dall + dn, dlo + part) - 1;
    const int x0 = 16 * dlo + g - 2 * tig + M::p - 1 - M::XLO;
    int rec = 4 * (8 * T0 + g - dlo + M::PADB) + tig;
    const uint2 *pe = E.t.pe + x0;
    uint2 A2 = pe[-8];
    for (int d0 = dlo; d0 <= dhi; d0 += kGwFlush) {
        float acc[NT][NPR][2][4];
#pragma unroll
        for (int tt = 0; tt < NT; ++tt)
#pragma unroll
            for (int pr = 0; pr < NPR; ++pr)
#pragma unroll
                for (int m = 0; m < 2; ++m)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[tt][pr][m][c] = 0.f;
        const int d1 = min(d0 + kGwFlush - 1, dhi);
#pragma unroll 2
        for (int D = d0; D <= d1; ++D, pe += 16, rec -= 4) {
            const uint2 A0 = pe[0], A1 = pe[8];
#pragma unroll
            for (int tt = 0; tt < NT; ++tt)
#pragma unroll
                for (int pr = 0; pr < NPR; ++pr) {
                    const uint2 b = A[pr]->u.sl[rec + 32 * tt];
                    mma16816(acc[tt][pr][0], A0.x, A1.x, A2.x, A0.x, b.x, b.y);  // h_E b'
                    mma16816(acc[tt][pr][1], A0.y, A1.y, A2.y, A0.y, b.x, b.y);  // l_E b'
                }
            A2 = A1;
        }
#pragma unroll
        for (int tt = 0; tt < NT; ++tt)
#pragma unroll
            for (int pr = 0; pr < NPR; ++pr)
#pragma unroll
                for (int m = 0; m < 2; ++m)
#pragma unroll
                    for (int c = 0; c < 4; ++c) iacc[tt][pr][m][c] += __float2int_rn(acc[tt][pr][m][c]);
    }
}

// K-split sum of MODE_GW's int32 sums (same layout of red as
// mma_ksplit_reduce; 8 of its 12 words per tile and product).  Contains a
// barrier: every thread of the CTA must call it.
template <int NT, int NPR>
__device__ __forceinline__ void mma_ksplit_reduce_gw(int (&iacc)[NT][NPR][2][4], int *red, int ks,
                                                     int nks, int tw, int nw, int lane) {
    constexpr int NV = NT * NPR * 8, NR = NT * NPR * 12;
    int *flat = &iacc[0][0][0][0];
    if (ks > 0) {
        int *dst = red + ((size_t)((ks - 1) * nw + tw) * 32 + lane) * NR;
#pragma unroll
        for (int v = 0; v < NV; ++v) dst[v] = flat[v];
    }
    __syncthreads();
    if (ks == 0)
        for (int k = 1; k < nks; ++k) {
            const int *src = red + ((size_t)((k - 1) * nw + tw) * 32 + lane) * NR;
#pragma unroll
            for (int v = 0; v < NV; ++v) flat[v] += src[v];
        }
}

// MODE_GW row sums of tiles [T0, T0 + NT) of product pr into A.u.stage.
template <int P, int NT, int NPR>
__device__ __forceinline__ void mma_stage_gw(MmaA<P, NT> &A, int T0, int lane, int pr,
                                             const int (&iacc)[NT][NPR][2][4]) {
    using M = MmaGeo<P, NT>;
    constexpr int Q = Prm<P>::q;
    const int g = lane >> 2, tig = lane & 3;
#pragma unroll
    for (int tt = 0; tt < NT; ++tt)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int J = 8 * (T0 + tt) + 2 * tig + (c & 1);
            if (J >= M::NBLK) continue;
            const int j = 16 * J + g + 8 * (c >> 1);
            // |P_1| <= 864 * 40 * 3118 < 2^27: reduced before the factor 64
            A.u.stage[stage_slot(j)] = cmod<Q>(64 * cmod<Q>(iacc[tt][pr][0][c]) + iacc[tt][pr][1][c]);
        }
}

// Sum of a K-split: warps with ks > 0 store their partial sums in red
// (floats, (nks - 1) x nw x 32 lanes x NT*NPR*12, nw = warps per part), warps
// with ks = 0 add them (exact: every partial sum is an integer below 2^24).
// Contains a barrier: every thread of the CTA must call it.
template <int NT, int NPR>
__device__ __forceinline__ void mma_ksplit_reduce(float (&acc)[NT][NPR][3][4], float *red, int ks,
                                                  int nks, int tw, int nw, int lane) {
    constexpr int NV = NT * NPR * 12;
    float *flat = &acc[0][0][0][0];
    if (ks > 0) {
        float *dst = red + ((size_t)((ks - 1) * nw + tw) * 32 + lane) * NV;
#pragma unroll
        for (int v = 0; v < NV; ++v) dst[v] = flat[v];
    }
    __syncthreads();
    if (ks == 0)
        for (int k = 1; k < nks; ++k) {
            const float *src = red + ((size_t)((k - 1) * nw + tw) * 32 + lane) * NV;
#pragma unroll
            for (int v = 0; v < NV; ++v) flat[v] += src[v];
        }
}

// Row sums of tiles [T0, T0 + NT) of product pr into A.u.stage (centred).
// The caller must have synchronised every warp reading A.u.hl since the loop.
template <int P, int NT, int NPR, int MODE = MODE_GEN, int Q = Prm<P>::q>
__device__ __forceinline__ void mma_stage(MmaA<P, NT> &A, int T0, int lane, int pr,
                                          const float (&acc)[NT][NPR][3][4]) {
    using M = MmaGeo<P, NT>;
    const int g = lane >> 2, tig = lane & 3;
#pragma unroll
    for (int tt = 0; tt < NT; ++tt)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int J = 8 * (T0 + tt) + 2 * tig + (c & 1);
            if (J >= M::NBLK) continue;
            const int j = 16 * J + g + 8 * (c >> 1);
            const int p0 = __float2int_rn(acc[tt][pr][0][c]);
            const int p1 = __float2int_rn(acc[tt][pr][1][c]);
            const int p2 = __float2int_rn(acc[tt][pr][2][c]);
            int v;
            if (MODE == MODE_GEN) v = 4096 * cmod<Q>(p0) + 64 * cmod<Q>(p1) + cmod<Q>(p2);
            else if (MODE == MODE_SA) v = 64 * p0 + p1;  // |P_1| <= 123 * 16 * NBLK, |P_2| < 2^24
            else v = p0;
            A.u.stage[stage_slot(j)] = cmod<Q>(v);
        }
}

// Final outputs c_0 .. c_{nout-1} (centred int16, zero beyond p) from the
// staged rows, by threads tid = 0 .. nth-1; two outputs per thread when c is
// 4-byte aligned and nout even.
template <int P, int NT, int Q = Prm<P>::q>
__device__ __forceinline__ void mma_finish(const MmaA<P, NT> &A, int blast,
                                           int16_t *__restrict__ c, int nout, int tid, int nth) {
    using M = MmaGeo<P, NT>;
    auto out = [&](int j, int r) -> int {
        if (j >= M::p) return 0;
        if (j == 0) r -= A.u.stage[stage_slot(M::p - 1)];
        return cmod<Q>(r + (int)A.a[j] * blast);
    };
    if (((reinterpret_cast<uintptr_t>(c) & 3) == 0) && (nout % 2 == 0)) {
        for (int j = 2 * tid; j < nout; j += 2 * nth) {
            int v0 = 0, v1 = 0;
            if (j < M::AN) {
                const int2 r = *reinterpret_cast<const int2 *>(&A.u.stage[stage_slot(j)]);
                v0 = out(j, r.x);
                v1 = out(j + 1, r.y);
            }
            *reinterpret_cast<uint32_t *>(c + j) = (uint32_t)(uint16_t)v0 | ((uint32_t)v1 << 16);
        }
        return;
    }
    for (int j = tid; j < nout; j += nth) c[j] = (int16_t)(j < M::AN ? out(j, A.u.stage[stage_slot(j)]) : 0);
}

}  // namespace snt
