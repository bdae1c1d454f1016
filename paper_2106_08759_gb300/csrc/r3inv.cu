// r3inv.cu -- inversion in R/3 = (Z/3)[x]/(x^p - x - 1) by constant-time
// divsteps, bit-sliced, 32 / LK elements per warp (LK lanes per element).
//
// Sec. 3.1 KeyGen steps 1-2 (sample small g until invertible in R/3, then
// 1/g); the paper cites Bernstein-Yang's constant-time extended gcd for this
// and notes that invertibility falls out of it as a side effect.  Here the
// divstep iteration runs on reversed polynomials: F = 1 - x^(p-1) - x^p
// (the reversal of x^p - x - 1), G = x^(p-1) g(1/x), V = 0, R = 1, delta = 1,
// and 2p - 1 steps of
//     V <- x V;
//     if delta > 0 and G(0) != 0: swap (F, G), (V, R), delta <- -delta;
//     delta <- delta + 1;
//     c = -G(0)/F(0);  G <- (G + c F)/x;  R <- R + c V.
// g is invertible iff delta = 0 at the end, and then 1/g has coefficient i
// equal to V(p-1-i) / F(0).  (The usual form f0*G - g0*F differs from this by
// the unit factor 1/f0 on (G, R), which the final division by F(0) absorbs.)
//
// Layout: an element's p + 1 trits of F, G, V, R are spread over a group of
// LK lanes (4, 8 or 32), WL 32-trit words per lane (lane s holds trits
// 32*WL*s .. 32*WL*(s+1) - 1), each word as two bit planes: m (trit nonzero)
// and s (trit is -1; meaningless where m = 0).  F_3 addition is 4 logic ops
// per 32 trits.  One-trit shifts are funnel shifts inside a lane plus one
// shuffle (two packed carry bits) across the lanes of the group.  Per-step
// control (G(0), F(0), delta, the swap) is uniform within a group and
// branch-free.  32 / LK elements share a warp, so every shuffle and control
// instruction serves all of them.
#include "common.cuh"
#include "kernels.h"

namespace snt {

constexpr unsigned FULL = 0xffffffffu;

template <int P, int LK_> struct R3Geo {
    static constexpr int WORDS = (P + 1 + 31) / 32;      // 21 / 24 / 27
    static constexpr int LK = LK_;                        // lanes per element: 4, 8 or 32
    static constexpr int WL = (WORDS + LK - 1) / LK;      // words per lane
    static constexpr int EPW = 32 / LK;                   // elements per warp
    static constexpr int WARPS = 4;                       // warps per CTA
    static constexpr int EPB = EPW * WARPS;               // elements per CTA
};

// (am, as) + (bm, bs) in F_3 on 32 trits at once (s is don't-care where m = 0):
//   one operand zero        -> the other;
//   both nonzero, same sign -> nonzero with the opposite sign (1+1 = -1);
//   both nonzero, opposite  -> zero.
__device__ __forceinline__ void f3_add(uint32_t am, uint32_t as, uint32_t bm, uint32_t bs,
                                       uint32_t &rm, uint32_t &rs) {
    const uint32_t both = am & bm;
    rm = (am | bm) & ~(both & (as ^ bs));
    rs = (am & (as ^ bm)) | (~am & bs);
}

// (a, b) <- (b, a) if sw == 1, unchanged if sw == 0, with three IMADs.
// neg1 holds 0xffffffff in a register the compiler cannot see through, so
// the first product stays an IMAD too.
__device__ __forceinline__ void cswap_fma(uint32_t &a, uint32_t &b, uint32_t sw, uint32_t neg1) {
    uint32_t d, na, nb;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(neg1), "r"(b));     // b - a
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(na) : "r"(d), "r"(sw), "r"(a));      // a + d sw
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(nb) : "r"(d), "r"(0u - sw), "r"(b)); // b - d sw
    a = na;
    b = nb;
}

// 2p - 1 divsteps on this group's state.  In: planes of G (reversed g).
// Out: planes of 1/g in reversed order (trit j is coefficient p-1-j of 1/g).
// Returns true iff g is invertible.  All 32 lanes of the warp must call it.
template <int P, int LKT>
__device__ __forceinline__ bool r3_divsteps(uint32_t (&gm)[R3Geo<P, LKT>::WL],
                                            uint32_t (&gs)[R3Geo<P, LKT>::WL],
                                            uint32_t (&vm)[R3Geo<P, LKT>::WL],
                                            uint32_t (&vs)[R3Geo<P, LKT>::WL]) {
    constexpr int WL = R3Geo<P, LKT>::WL, LK = LKT;
    const int sub = threadIdx.x & (LK - 1);
    uint32_t fm[WL], fs[WL], rm[WL], rs[WL];
#pragma unroll
    for (int w = 0; w < WL; ++w) {
        const int t0 = 32 * (WL * sub + w);  // first trit of this word
        uint32_t m = 0, s = 0;
        if (t0 == 0) m |= 1u;
        if (P - 1 >= t0 && P - 1 < t0 + 32) { m |= 1u << (P - 1 - t0); s |= 1u << (P - 1 - t0); }
        if (P >= t0 && P < t0 + 32) { m |= 1u << (P - t0); s |= 1u << (P - t0); }
        fm[w] = m; fs[w] = s;
        vm[w] = 0; vs[w] = 0;
        rm[w] = (t0 == 0) ? 1u : 0u; rs[w] = 0;
    }
    int delta = 1;
    uint32_t f0s = 0;  // sign bit of F(0); F(0) is never zero
    uint32_t neg1;
    asm volatile("mov.u32 %0, 0xffffffff;" : "=r"(neg1));
#pragma unroll 1
    for (int step = 0; step < 2 * P - 1; ++step) {
        // V <- x V: carry the top trit of each lane into the next lane
        uint32_t cv = (vm[WL - 1] >> 31) | ((vs[WL - 1] >> 30) & 2u);
        cv = __shfl_up_sync(FULL, cv, 1, LK);
        if (sub == 0) cv = 0;
#pragma unroll
        for (int w = WL - 1; w > 0; --w) {
            vm[w] = __funnelshift_l(vm[w - 1], vm[w], 1);
            vs[w] = __funnelshift_l(vs[w - 1], vs[w], 1);
        }
        vm[0] = (vm[0] << 1) | (cv & 1u);
        vs[0] = (vs[0] << 1) | (cv >> 1);
        // G(0), uniform within the group
        const uint32_t g0 = __shfl_sync(FULL, (gm[0] & 1u) | ((gs[0] & 1u) << 1), 0, LK);
        const uint32_t g0m = g0 & 1u, g0s = g0 >> 1;
        const uint32_t sw = (uint32_t)(delta > 0) & g0m;
        // Conditional swaps as integer multiply-adds, a + (b - a) * sw with sw
        // in {0, 1} (exact modulo 2^32): they run on the FMA pipe, which the
        // bit operations of the F_3 arithmetic leave idle.
#pragma unroll
        for (int w = 0; w < WL; ++w) {
            cswap_fma(fm[w], gm[w], sw, neg1);
            cswap_fma(fs[w], gs[w], sw, neg1);
            cswap_fma(vm[w], rm[w], sw, neg1);
            cswap_fma(vs[w], rs[w], sw, neg1);
        }
        const uint32_t nf0s = sw ? g0s : f0s;
        const uint32_t ng0s = sw ? f0s : g0s;  // G(0) stays nonzero iff it was
        f0s = nf0s;
        delta = (sw ? -delta : delta) + 1;
        // c = -G(0) F(0) (= -G(0)/F(0) in F_3)
        const uint32_t cm = 0u - g0m;
        const uint32_t cs = 0u - ((ng0s ^ f0s ^ 1u) & 1u);
#pragma unroll
        for (int w = 0; w < WL; ++w) {
            f3_add(gm[w], gs[w], fm[w] & cm, fs[w] ^ cs, gm[w], gs[w]);
            f3_add(rm[w], rs[w], vm[w] & cm, vs[w] ^ cs, rm[w], rs[w]);
        }
        // G <- G / x (trit 0 is zero now): bring in bit 0 of the next lane
        uint32_t cg = __shfl_down_sync(FULL, (gm[0] & 1u) | ((gs[0] & 1u) << 1), 1, LK);
        if (sub == LK - 1) cg = 0;
#pragma unroll
        for (int w = 0; w < WL - 1; ++w) {
            gm[w] = __funnelshift_r(gm[w], gm[w + 1], 1);
            gs[w] = __funnelshift_r(gs[w], gs[w + 1], 1);
        }
        gm[WL - 1] = __funnelshift_r(gm[WL - 1], cg, 1);
        gs[WL - 1] = __funnelshift_r(gs[WL - 1], cg >> 1, 1);
    }
#pragma unroll
    for (int w = 0; w < WL; ++w) vs[w] ^= 0u - f0s;
    return delta == 0;
}

// This lane's planes of G (trit t = g[p-1-t]) from int8 coefficients g[0..p)
// in shared memory.
template <int P, int LKT>
__device__ __forceinline__ void planes_from_reversed(const int8_t *gsm, uint32_t (&gm)[R3Geo<P, LKT>::WL],
                                                     uint32_t (&gs)[R3Geo<P, LKT>::WL]) {
    constexpr int WL = R3Geo<P, LKT>::WL, LK = LKT;
    const int sub = threadIdx.x & (LK - 1);
#pragma unroll
    for (int w = 0; w < WL; ++w) {
        uint32_t m = 0, s = 0;
        const int t0 = 32 * (WL * sub + w);
#pragma unroll 8
        for (int b = 0; b < 32; ++b) {
            const int src = P - 1 - (t0 + b);
            const int c = (src >= 0) ? gsm[src] : 0;
            m |= (uint32_t)(c != 0) << b;
            s |= (uint32_t)(c < 0) << b;
        }
        gm[w] = m; gs[w] = s;
    }
}

// Natural-order coefficients of the (reversed) output planes into shared
// memory: out[i] = trit p-1-i.
template <int P, int LKT>
__device__ __forceinline__ void reversed_to_smem(const uint32_t (&om)[R3Geo<P, LKT>::WL],
                                                 const uint32_t (&os)[R3Geo<P, LKT>::WL], int8_t *osm) {
    constexpr int WL = R3Geo<P, LKT>::WL, LK = LKT;
    const int sub = threadIdx.x & (LK - 1);
#pragma unroll
    for (int w = 0; w < WL; ++w) {
        const int t0 = 32 * (WL * sub + w);
#pragma unroll 8
        for (int b = 0; b < 32; ++b) {
            const int i = P - 1 - (t0 + b);
            if (i >= 0) {
                const int m = (om[w] >> b) & 1, s = (os[w] >> b) & 1;
                osm[i] = (int8_t)(m ? (s ? -1 : 1) : 0);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Keygen form: sample g (stream 0, attempt a) until invertible, write g
// (int8, zero padded, stride pad) for the h product and Small_encode(1/g)
// into the secret key at sk_off.  A warp keeps retrying while any of its
// elements still needs an invertible g (each retry costs the warp a full
// divstep run; a random g fails with probability about 3^-19).
// ---------------------------------------------------------------------------
template <int P, int LKT>
__global__ void __launch_bounds__(32 * R3Geo<P, LKT>::WARPS)
k_r3_keygen(KeyMap km, int B, int8_t *__restrict__ g_out, int sk_bytes, int sk_off,
            const uint64_t *__restrict__ inj_idx, const int8_t *__restrict__ inj_g,
            int n_inj, int *__restrict__ err) {
    using Gm = Geo<P>;
    using RG = R3Geo<P, LKT>;
    constexpr int WL = RG::WL, LK = RG::LK, EPW = RG::EPW;
    __shared__ int8_t smem[RG::EPB][1024];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sub = lane & (LK - 1), grp = lane / LK;
    const int ebase = blockIdx.x * RG::EPB + warp * EPW;  // first element of this warp
    if (ebase >= B) return;                               // warp-uniform
    const int key = ebase + grp;
    const bool live = key < B;
    const BatchDesc bd = key_batch(km, live ? key : ebase);
    const uint64_t seed = bd.seed;
    const uint64_t k = bd.first + (uint64_t)(key - bd.key_base);
    int8_t *gsm = smem[warp * EPW + grp];

    // optional injected attempt-0 draw (test hook)
    int inj = -1;
    if (live)
        for (int j = sub; j < n_inj; j += LK)
            if (inj_idx[j] == k) inj = j;
    for (int off = LK / 2; off > 0; off >>= 1) inj = max(inj, __shfl_xor_sync(FULL, inj, off, LK));

    bool ok = !live;
    uint32_t om[WL], os[WL];
#pragma unroll
    for (int w = 0; w < WL; ++w) { om[w] = 0; os[w] = 0; }
    for (int att = 0; att < kMaxGAttempts; ++att) {
        if (__all_sync(FULL, ok)) break;
        if (!ok) {
            if (att == 0 && inj >= 0) {
                for (int i = sub; i < P; i += LK) gsm[i] = inj_g[(size_t)inj * Gm::p + i];
            } else {
                // g_i = floor(3 (u_i mod 2^30) / 2^30) - 1 for word u_i of stream 0
                for (int blk = sub; 4 * blk < P; blk += LK) {
                    uint32_t r[4];
                    rand_block(seed, k, STREAM_G, (uint32_t)att, (uint32_t)blk, r);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int i = 4 * blk + j;
                        if (i < P)
                            gsm[i] = (int8_t)((int)(((unsigned long long)(r[j] & 0x3fffffffu) * 3u) >> 30) - 1);
                    }
                }
            }
        }
        __syncwarp();
        uint32_t gm[WL], gs[WL], vm[WL], vs[WL];
        planes_from_reversed<P, LKT>(gsm, gm, gs);
        const bool good = r3_divsteps<P, LKT>(gm, gs, vm, vs);
        if (!ok && good) {
#pragma unroll
            for (int w = 0; w < WL; ++w) { om[w] = vm[w]; os[w] = vs[w]; }
        }
        ok = ok || good;
        __syncwarp();
    }
    if (live && !ok) {
        if (sub == 0) atomicOr(err, ERR_RESAMPLE);
#pragma unroll
        for (int w = 0; w < WL; ++w) { om[w] = 0; os[w] = 0; }
    }
    // g (natural order) for h = g * (3f)^-1: the warp writes its rows together
    __syncwarp();
    for (int e = 0; e < EPW; ++e) {
        if (ebase + e >= B) break;
        const int8_t *src = smem[warp * EPW + e];
        int8_t *gk = g_out + (size_t)(ebase + e) * Gm::pad;
        for (int i = lane; i < Gm::pad; i += 32) gk[i] = (i < P) ? src[i] : (int8_t)0;
    }
    __syncwarp();
    reversed_to_smem<P, LKT>(om, os, gsm);
    __syncwarp();
    // Small_encode(1/g)
    for (int e = 0; e < EPW; ++e) {
        if (ebase + e >= B) break;
        const int8_t *src = smem[warp * EPW + e];
        const BatchDesc be = key_batch(km, ebase + e);
        uint8_t *skk = be.sk + (size_t)(ebase + e - be.key_base) * sk_bytes + sk_off;
        for (int b = lane; b < Gm::small_bytes; b += 32) {
            uint32_t byte = 0;
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int i = 4 * b + t;
                if (i < P) byte |= (uint32_t)(src[i] + 1) << (2 * t);
            }
            skk[b] = (uint8_t)byte;
        }
    }
}

// ---------------------------------------------------------------------------
// Batch form for the kernel microbenchmark: out_i = 1/g_i, ok_i.
// g, out: n x p int8 (stride p).
// ---------------------------------------------------------------------------
template <int P, int LKT>
__global__ void __launch_bounds__(32 * R3Geo<P, LKT>::WARPS)
k_r3_inv(int n, const int8_t *__restrict__ g, int8_t *__restrict__ out,
         int32_t *__restrict__ okv) {
    using RG = R3Geo<P, LKT>;
    constexpr int WL = RG::WL, LK = RG::LK, EPW = RG::EPW;
    __shared__ int8_t smem[RG::EPB][1024];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sub = lane & (LK - 1), grp = lane / LK;
    const int ebase = blockIdx.x * RG::EPB + warp * EPW;
    if (ebase >= n) return;
    const int e = ebase + grp;
    const bool live = e < n;
    int8_t *gsm = smem[warp * EPW + grp];
    for (int i = sub; i < P; i += LK) gsm[i] = live ? g[(size_t)e * P + i] : (int8_t)0;
    __syncwarp();
    uint32_t gm[WL], gs[WL], vm[WL], vs[WL];
    planes_from_reversed<P, LKT>(gsm, gm, gs);
    const bool ok = r3_divsteps<P, LKT>(gm, gs, vm, vs);
    if (!ok)
#pragma unroll
        for (int w = 0; w < WL; ++w) { vm[w] = 0; vs[w] = 0; }
    __syncwarp();
    reversed_to_smem<P, LKT>(vm, vs, gsm);
    __syncwarp();
    if (live) {
        for (int i = sub; i < P; i += LK) out[(size_t)e * P + i] = gsm[i];
        if (sub == 0) okv[e] = ok ? 1 : 0;
    }
}

template <int P, int LK>
cudaError_t launch_r3_keygen_lk(const KeyMap &km, int B, int8_t *g_out, int sk_bytes, int sk_off,
                                const uint64_t *inj_idx, const int8_t *inj_g, int n_inj, int *err,
                                cudaStream_t st) {
    constexpr int EPB = R3Geo<P, LK>::EPB;
    k_r3_keygen<P, LK><<<(B + EPB - 1) / EPB, 32 * R3Geo<P, LK>::WARPS, 0, st>>>(
        km, B, g_out, sk_bytes, sk_off, inj_idx, inj_g, n_inj, err);
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_r3_keygen(const KeyMap &km, int B, int8_t *g_out, int sk_bytes, int sk_off,
                             const uint64_t *inj_idx, const int8_t *inj_g, int n_inj, int *err,
                             cudaStream_t st, int lanes) {
    switch (lanes) {
        case 4: return launch_r3_keygen_lk<P, 4>(km, B, g_out, sk_bytes, sk_off, inj_idx, inj_g, n_inj, err, st);
        case 8: return launch_r3_keygen_lk<P, 8>(km, B, g_out, sk_bytes, sk_off, inj_idx, inj_g, n_inj, err, st);
        default: return launch_r3_keygen_lk<P, 32>(km, B, g_out, sk_bytes, sk_off, inj_idx, inj_g, n_inj, err, st);
    }
}

template <int P, int LK>
cudaError_t launch_r3_inv_lk(int n, const int8_t *g, int8_t *out, int32_t *ok, cudaStream_t st) {
    constexpr int EPB = R3Geo<P, LK>::EPB;
    k_r3_inv<P, LK><<<(n + EPB - 1) / EPB, 32 * R3Geo<P, LK>::WARPS, 0, st>>>(n, g, out, ok);
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_r3_inv(int n, const int8_t *g, int8_t *out, int32_t *ok, cudaStream_t st,
                          int lanes) {
    switch (lanes) {
        case 4: return launch_r3_inv_lk<P, 4>(n, g, out, ok, st);
        case 8: return launch_r3_inv_lk<P, 8>(n, g, out, ok, st);
        default: return launch_r3_inv_lk<P, 32>(n, g, out, ok, st);
    }
}

#define SNT_R3_INST(P)                                                                      \
    template cudaError_t launch_r3_keygen<P>(const KeyMap &, int, int8_t *, int, int,       \
                                             const uint64_t *, const int8_t *, int, int *,  \
                                             cudaStream_t, int);                            \
    template cudaError_t launch_r3_inv<P>(int, const int8_t *, int8_t *, int32_t *, cudaStream_t, int);
SNT_R3_INST(653)
SNT_R3_INST(761)
SNT_R3_INST(857)

}  // namespace snt
