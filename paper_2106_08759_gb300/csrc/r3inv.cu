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
// branch-free.  32 / LK element groups share a warp, and each group may run
// KPT elements at once (their words interleaved in the same registers' step
// loop, their shuffled bits packed into the same shuffles), so every shuffle
// serves 32 KPT / LK elements and each lane has KPT independent chains.
#include "common.cuh"
#include "kernels.h"
#include "pdl.cuh"

namespace snt {

constexpr unsigned FULL = 0xffffffffu;

template <int P, int LK_, int KPT_ = 1> struct R3Geo {
    static constexpr int WORDS = (P + 1 + 31) / 32;      // 21 / 24 / 27
    static constexpr int LK = LK_;                        // lanes per element: 4, 8 or 32
    static constexpr int KPT = KPT_;                      // elements per lane group: 1 or 2
    static constexpr int WL = (WORDS + LK - 1) / LK;      // words per lane
    static constexpr int GPW = 32 / LK;                   // lane groups per warp
    static constexpr int EPW = GPW * KPT;                 // elements per warp
    static constexpr int WARPS = 4 / KPT;                 // warps per CTA
    static constexpr int EPB = EPW * WARPS;               // elements per CTA
    static constexpr int ROW = Geo<P>::pad;               // shared bytes per element
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

// 2p - 1 divsteps on this group's KPT states.  In: planes of G (reversed g).
// Out: planes of 1/g in reversed order (trit j is coefficient p-1-j of 1/g).
// good[k] = g_k invertible.  All 32 lanes of the warp must call it.
template <int P, int LKT, int KPT>
__device__ __forceinline__ void r3_divsteps(uint32_t (&gm)[KPT][R3Geo<P, LKT>::WL],
                                            uint32_t (&gs)[KPT][R3Geo<P, LKT>::WL],
                                            uint32_t (&vm)[KPT][R3Geo<P, LKT>::WL],
                                            uint32_t (&vs)[KPT][R3Geo<P, LKT>::WL],
                                            bool (&good)[KPT]) {
    constexpr int WL = R3Geo<P, LKT>::WL, LK = LKT;
    const int sub = threadIdx.x & (LK - 1);
    uint32_t fm[KPT][WL], fs[KPT][WL], rm[KPT][WL], rs[KPT][WL];
#pragma unroll
    for (int w = 0; w < WL; ++w) {
        const int t0 = 32 * (WL * sub + w);  // first trit of this word
        uint32_t m = 0, s = 0;
        if (t0 == 0) m |= 1u;
        if (P - 1 >= t0 && P - 1 < t0 + 32) { m |= 1u << (P - 1 - t0); s |= 1u << (P - 1 - t0); }
        if (P >= t0 && P < t0 + 32) { m |= 1u << (P - t0); s |= 1u << (P - t0); }
#pragma unroll
        for (int k = 0; k < KPT; ++k) {
            fm[k][w] = m; fs[k][w] = s;
            vm[k][w] = 0; vs[k][w] = 0;
            rm[k][w] = (t0 == 0) ? 1u : 0u; rs[k][w] = 0;
        }
    }
    int delta[KPT];
    uint32_t f0s[KPT];  // sign bit of F(0); F(0) is never zero
#pragma unroll
    for (int k = 0; k < KPT; ++k) { delta[k] = 1; f0s[k] = 0; }
    uint32_t neg1;
    asm volatile("mov.u32 %0, 0xffffffff;" : "=r"(neg1));
#pragma unroll 1
    for (int step = 0; step < 2 * P - 1; ++step) {
        // V <- x V: carry the top trit of each lane into the next lane (two
        // bits per element, all elements in one shuffle)
        uint32_t cv = 0;
#pragma unroll
        for (int k = 0; k < KPT; ++k)
            cv |= ((vm[k][WL - 1] >> 31) | ((vs[k][WL - 1] >> 30) & 2u)) << (2 * k);
        cv = __shfl_up_sync(FULL, cv, 1, LK);
        if (sub == 0) cv = 0;
        // G(0) of every element, uniform within the group
        uint32_t g0 = 0;
#pragma unroll
        for (int k = 0; k < KPT; ++k) g0 |= ((gm[k][0] & 1u) | ((gs[k][0] & 1u) << 1)) << (2 * k);
        g0 = __shfl_sync(FULL, g0, 0, LK);
#pragma unroll
        for (int k = 0; k < KPT; ++k) {
#pragma unroll
            for (int w = WL - 1; w > 0; --w) {
                vm[k][w] = __funnelshift_l(vm[k][w - 1], vm[k][w], 1);
                vs[k][w] = __funnelshift_l(vs[k][w - 1], vs[k][w], 1);
            }
            vm[k][0] = (vm[k][0] << 1) | ((cv >> (2 * k)) & 1u);
            vs[k][0] = (vs[k][0] << 1) | ((cv >> (2 * k + 1)) & 1u);
            const uint32_t g0m = (g0 >> (2 * k)) & 1u, g0s = (g0 >> (2 * k + 1)) & 1u;
            const uint32_t sw = (uint32_t)(delta[k] > 0) & g0m;
            // Conditional swaps as integer multiply-adds, a + (b - a) * sw with
            // sw in {0, 1} (exact modulo 2^32): they run on the FMA pipe, which
            // the bit operations of the F_3 arithmetic leave idle.
#pragma unroll
            for (int w = 0; w < WL; ++w) {
                cswap_fma(fm[k][w], gm[k][w], sw, neg1);
                cswap_fma(fs[k][w], gs[k][w], sw, neg1);
                cswap_fma(vm[k][w], rm[k][w], sw, neg1);
                cswap_fma(vs[k][w], rs[k][w], sw, neg1);
            }
            const uint32_t nf0s = sw ? g0s : f0s[k];
            const uint32_t ng0s = sw ? f0s[k] : g0s;  // G(0) stays nonzero iff it was
            f0s[k] = nf0s;
            delta[k] = (sw ? -delta[k] : delta[k]) + 1;
            // c = -G(0) F(0) (= -G(0)/F(0) in F_3)
            const uint32_t cm = 0u - g0m;
            const uint32_t cs = 0u - ((ng0s ^ f0s[k] ^ 1u) & 1u);
#pragma unroll
            for (int w = 0; w < WL; ++w) {
                f3_add(gm[k][w], gs[k][w], fm[k][w] & cm, fs[k][w] ^ cs, gm[k][w], gs[k][w]);
                f3_add(rm[k][w], rs[k][w], vm[k][w] & cm, vs[k][w] ^ cs, rm[k][w], rs[k][w]);
            }
        }
        // G <- G / x (trit 0 is zero now): bring in bit 0 of the next lane
        uint32_t cg = 0;
#pragma unroll
        for (int k = 0; k < KPT; ++k) cg |= ((gm[k][0] & 1u) | ((gs[k][0] & 1u) << 1)) << (2 * k);
        cg = __shfl_down_sync(FULL, cg, 1, LK);
        if (sub == LK - 1) cg = 0;
#pragma unroll
        for (int k = 0; k < KPT; ++k) {
#pragma unroll
            for (int w = 0; w < WL - 1; ++w) {
                gm[k][w] = __funnelshift_r(gm[k][w], gm[k][w + 1], 1);
                gs[k][w] = __funnelshift_r(gs[k][w], gs[k][w + 1], 1);
            }
            gm[k][WL - 1] = __funnelshift_r(gm[k][WL - 1], cg >> (2 * k), 1);
            gs[k][WL - 1] = __funnelshift_r(gs[k][WL - 1], cg >> (2 * k + 1), 1);
        }
    }
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
#pragma unroll
        for (int w = 0; w < WL; ++w) vs[k][w] ^= 0u - f0s[k];
        good[k] = delta[k] == 0;
    }
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
//
// Deferred form (gfix != null): attempt 0 of g is already in g_out (written
// by the sampling kernel, read by the h kernel while this one runs), so it
// is read from there and g_out is left untouched; a key that needs another
// attempt is appended to the resampling list (fix_keys[i], its final g in
// row i of gfix) for the fix-up kernel that runs after both.
// ---------------------------------------------------------------------------
template <int P, int LKT, int KPT>
__global__ void __launch_bounds__(32 * R3Geo<P, LKT, KPT>::WARPS)
k_r3_keygen(KeyMap km, int B, int8_t *__restrict__ g_out, int sk_bytes, int sk_off,
            const uint64_t *__restrict__ inj_idx, const int8_t *__restrict__ inj_g,
            int n_inj, int *__restrict__ err, int8_t *__restrict__ gfix,
            int *__restrict__ fix_count, int *__restrict__ fix_keys,
            const int *__restrict__ sub_ok, int sub_size, const int *__restrict__ fix_slot) {
    pdl_enter();
    using Gm = Geo<P>;
    using RG = R3Geo<P, LKT, KPT>;
    constexpr int WL = RG::WL, LK = RG::LK, EPW = RG::EPW, GPW = RG::GPW;
    static_assert(EPW <= 32, "one lane per key of the warp");
    __shared__ __align__(16) int8_t smem[RG::EPB][RG::ROW];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sub = lane & (LK - 1), grp = lane / LK;
    const int ebase = blockIdx.x * RG::EPB + warp * EPW;  // first element of this warp
    if (ebase >= B) return;                               // warp-uniform
    if (sub_ok) {  // fall-back form: only warps with a key in a failed subtree
        // lane e tests the warp's key e (the table searches run in parallel)
        const bool mine = lane >= EPW || ebase + lane >= B ||
                          sub_ok[key_subtree(km, ebase + lane, sub_size)] != 0;
        if (__all_sync(FULL, mine)) return;
    }
    // this group's elements: warp slots grp + k GPW
    const bool deferred = gfix != nullptr;
    bool ok[KPT], first_ok[KPT];
    uint64_t seed[KPT], kidx[KPT];
    int inj[KPT];
    int8_t *gsm[KPT];
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
        const int e = ebase + grp + k * GPW;
        const bool live = e < B;
        const BatchDesc bd = key_batch(km, live ? e : ebase);
        seed[k] = bd.seed;
        kidx[k] = bd.first + (uint64_t)((live ? e : ebase) - bd.key_base);
        gsm[k] = smem[warp * EPW + grp + k * GPW];
        ok[k] = !live;
        first_ok[k] = true;
        // optional injected attempt-0 draw (test hook)
        int j0 = -1;
        if (live)
            for (int j = sub; j < n_inj; j += LK)
                if (inj_idx[j] == kidx[k]) j0 = j;
        for (int off = LK / 2; off > 0; off >>= 1) j0 = max(j0, __shfl_xor_sync(FULL, j0, off, LK));
        inj[k] = j0;
    }
    uint32_t om[KPT][WL], os[KPT][WL];
#pragma unroll
    for (int k = 0; k < KPT; ++k)
#pragma unroll
        for (int w = 0; w < WL; ++w) { om[k][w] = 0; os[k][w] = 0; }
    for (int att = 0; att < kMaxGAttempts; ++att) {
        bool all_ok = true;
#pragma unroll
        for (int k = 0; k < KPT; ++k) all_ok = all_ok && ok[k];
        if (__all_sync(FULL, all_ok)) break;
#pragma unroll
        for (int k = 0; k < KPT; ++k) {
            if (ok[k]) continue;
            if (att == 0 && deferred) {
                const int8_t *g0 = g_out + (size_t)(ebase + grp + k * GPW) * Gm::pad;
                for (int i = sub; i < P; i += LK) gsm[k][i] = g0[i];
            } else if (att == 0 && inj[k] >= 0) {
                for (int i = sub; i < P; i += LK) gsm[k][i] = inj_g[(size_t)inj[k] * Gm::p + i];
            } else {
                // g_i = floor(3 (u_i mod 2^30) / 2^30) - 1 for word u_i of stream 0
                for (int blk = sub; 4 * blk < P; blk += LK) {
                    uint32_t r[4];
                    rand_block(seed[k], kidx[k], STREAM_G, (uint32_t)att, (uint32_t)blk, r);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int i = 4 * blk + j;
                        if (i < P)
                            gsm[k][i] = (int8_t)((int)(((unsigned long long)(r[j] & 0x3fffffffu) * 3u) >> 30) - 1);
                    }
                }
            }
        }
        __syncwarp();
        uint32_t gm[KPT][WL], gs[KPT][WL], vm[KPT][WL], vs[KPT][WL];
#pragma unroll
        for (int k = 0; k < KPT; ++k) planes_from_reversed<P, LKT>(gsm[k], gm[k], gs[k]);
        bool good[KPT];
        r3_divsteps<P, LKT, KPT>(gm, gs, vm, vs, good);
#pragma unroll
        for (int k = 0; k < KPT; ++k) {
            if (!ok[k] && good[k]) {
#pragma unroll
                for (int w = 0; w < WL; ++w) { om[k][w] = vm[k][w]; os[k][w] = vs[k][w]; }
            }
            if (att == 0) first_ok[k] = ok[k] || good[k];
            ok[k] = ok[k] || good[k];
        }
        __syncwarp();
    }
#pragma unroll
    for (int k = 0; k < KPT; ++k)
        if (!ok[k]) {  // (dead slots start ok)
            if (sub == 0) atomicOr(err, ERR_RESAMPLE);
#pragma unroll
            for (int w = 0; w < WL; ++w) { om[k][w] = 0; os[k][w] = 0; }
        }
    __syncwarp();
    if (deferred) {
        // resampled keys: final g to the resampling list (one slot per key)
#pragma unroll
        for (int k = 0; k < KPT; ++k) {
            const int e = ebase + grp + k * GPW;
            int slot = 0;
            const bool fix = e < B && ok[k] && !first_ok[k];
            if (fix && sub == 0) {
                const int prev = fix_slot ? fix_slot[e] : -1;  // listed by the screen
                slot = prev >= 0 ? prev : atomicAdd(fix_count, 1);
                fix_keys[slot] = e;
            }
            slot = __shfl_sync(FULL, slot, 0, LK);
            if (fix)
                for (int i = sub; i < Gm::pad; i += LK)
                    gfix[(size_t)slot * Gm::pad + i] = (i < P) ? gsm[k][i] : (int8_t)0;
        }
    } else {
        // g (natural order) for h = g * (3f)^-1: the warp writes its rows together
        for (int e = 0; e < EPW; ++e) {
            if (ebase + e >= B) break;
            const int8_t *src = smem[warp * EPW + e];
            int8_t *gk = g_out + (size_t)(ebase + e) * Gm::pad;
            for (int i = lane; i < Gm::pad; i += 32) gk[i] = (i < P) ? src[i] : (int8_t)0;
        }
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < KPT; ++k) reversed_to_smem<P, LKT>(om[k], os[k], gsm[k]);
    __syncwarp();
    // Small_encode(1/g); lane e looks up the sk row of the warp's key e (the
    // table searches run in parallel, not one per loop step)
    unsigned long long skrow = 0;
    if (lane < EPW && ebase + lane < B) {
        const BatchDesc be = key_batch(km, ebase + lane);
        skrow = reinterpret_cast<unsigned long long>(
            be.sk + (size_t)(ebase + lane - be.key_base) * sk_bytes + sk_off);
    }
    for (int e = 0; e < EPW; ++e) {
        if (ebase + e >= B) break;
        const int8_t *src = smem[warp * EPW + e];
        uint8_t *skk = reinterpret_cast<uint8_t *>(__shfl_sync(FULL, skrow, e));
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
template <int P, int LKT, int KPT>
__global__ void __launch_bounds__(32 * R3Geo<P, LKT, KPT>::WARPS)
k_r3_inv(int n, const int8_t *__restrict__ g, int8_t *__restrict__ out,
         int32_t *__restrict__ okv) {
    using RG = R3Geo<P, LKT, KPT>;
    constexpr int WL = RG::WL, LK = RG::LK, EPW = RG::EPW, GPW = RG::GPW;
    __shared__ __align__(16) int8_t smem[RG::EPB][RG::ROW];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sub = lane & (LK - 1), grp = lane / LK;
    const int ebase = blockIdx.x * RG::EPB + warp * EPW;
    if (ebase >= n) return;
    uint32_t gm[KPT][WL], gs[KPT][WL], vm[KPT][WL], vs[KPT][WL];
    int8_t *gsm[KPT];
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
        const int e = ebase + grp + k * GPW;
        gsm[k] = smem[warp * EPW + grp + k * GPW];
        for (int i = sub; i < P; i += LK) gsm[k][i] = (e < n) ? g[(size_t)e * P + i] : (int8_t)0;
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < KPT; ++k) planes_from_reversed<P, LKT>(gsm[k], gm[k], gs[k]);
    bool ok[KPT];
    r3_divsteps<P, LKT, KPT>(gm, gs, vm, vs, ok);
#pragma unroll
    for (int k = 0; k < KPT; ++k)
        if (!ok[k])
#pragma unroll
            for (int w = 0; w < WL; ++w) { vm[k][w] = 0; vs[k][w] = 0; }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < KPT; ++k) reversed_to_smem<P, LKT>(vm[k], vs[k], gsm[k]);
    __syncwarp();
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
        const int e = ebase + grp + k * GPW;
        if (e < n) {
            for (int i = sub; i < P; i += LK) out[(size_t)e * P + i] = gsm[k][i];
            if (sub == 0) okv[e] = ok[k] ? 1 : 0;
        }
    }
}

template <int P, int LK, int KPT>
cudaError_t launch_r3_keygen_lk(const KeyMap &km, int B, int8_t *g_out, int sk_bytes, int sk_off,
                                const uint64_t *inj_idx, const int8_t *inj_g, int n_inj, int *err,
                                cudaStream_t st, int8_t *gfix, int *fix_count, int *fix_keys,
                                const int *sub_ok, int sub_size, const int *fix_slot) {
    using RG = R3Geo<P, LK, KPT>;
    SNT_LAUNCH(k_r3_keygen<P, LK, KPT>, (B + RG::EPB - 1) / RG::EPB, 32 * RG::WARPS, 0, st, km, B,
        g_out, sk_bytes, sk_off, inj_idx, inj_g, n_inj, err, gfix, fix_count, fix_keys, sub_ok,
        sub_size, fix_slot);
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_r3_keygen(const KeyMap &km, int B, int8_t *g_out, int sk_bytes, int sk_off,
                             const uint64_t *inj_idx, const int8_t *inj_g, int n_inj, int *err,
                             cudaStream_t st, int lanes, int kpt, int8_t *gfix, int *fix_count,
                             int *fix_keys, const int *sub_ok, int sub_size,
                             const int *fix_slot) {
#define SNT_R3K(LK, KP)                                                                     \
    launch_r3_keygen_lk<P, LK, KP>(km, B, g_out, sk_bytes, sk_off, inj_idx, inj_g, n_inj, err, st, \
                                   gfix, fix_count, fix_keys, sub_ok, sub_size, fix_slot)
    if (kpt == 2) {
        switch (lanes) {
            case 4: return SNT_R3K(4, 2);
            case 8: return SNT_R3K(8, 2);
            default: return SNT_R3K(32, 2);
        }
    }
    switch (lanes) {
        case 4: return SNT_R3K(4, 1);
        case 8: return SNT_R3K(8, 1);
        default: return SNT_R3K(32, 1);
    }
#undef SNT_R3K
}

template <int P, int LK, int KPT>
cudaError_t launch_r3_inv_lk(int n, const int8_t *g, int8_t *out, int32_t *ok, cudaStream_t st) {
    using RG = R3Geo<P, LK, KPT>;
    k_r3_inv<P, LK, KPT><<<(n + RG::EPB - 1) / RG::EPB, 32 * RG::WARPS, 0, st>>>(n, g, out, ok);
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_r3_inv(int n, const int8_t *g, int8_t *out, int32_t *ok, cudaStream_t st,
                          int lanes, int kpt) {
    if (kpt == 2) {
        switch (lanes) {
            case 4: return launch_r3_inv_lk<P, 4, 2>(n, g, out, ok, st);
            case 8: return launch_r3_inv_lk<P, 8, 2>(n, g, out, ok, st);
            default: return launch_r3_inv_lk<P, 32, 2>(n, g, out, ok, st);
        }
    }
    switch (lanes) {
        case 4: return launch_r3_inv_lk<P, 4, 1>(n, g, out, ok, st);
        case 8: return launch_r3_inv_lk<P, 8, 1>(n, g, out, ok, st);
        default: return launch_r3_inv_lk<P, 32, 1>(n, g, out, ok, st);
    }
}

#define SNT_R3_INST(P)                                                                      \
    template cudaError_t launch_r3_keygen<P>(const KeyMap &, int, int8_t *, int, int,       \
                                             const uint64_t *, const int8_t *, int, int *,  \
                                             cudaStream_t, int, int, int8_t *, int *, int *, \
                                             const int *, int, const int *);                 \
    template cudaError_t launch_r3_inv<P>(int, const int8_t *, int8_t *, int32_t *, cudaStream_t, int, \
                                          int);
SNT_R3_INST(653)
SNT_R3_INST(761)
SNT_R3_INST(857)

}  // namespace snt
