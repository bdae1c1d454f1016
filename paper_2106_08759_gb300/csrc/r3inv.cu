// r3inv.cu -- inversion in R/3 = (Z/3)[x]/(x^p - x - 1) by constant-time
// divsteps, one warp per element, bit-sliced across the 32 lanes.
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
// Layout: lane L holds trits 32L .. 32L+31 of F, G, V, R as two bit planes
// each: m (trit nonzero) and s (trit is -1; meaningless where m = 0).  All
// trits at or above p + 1 are zero, so the one-trit shifts are lane
// rotations: the bit G loses at trit 0 is zero after the update, and V never
// reaches lane 31.  Every step is branch-free; per-step control (G(0),
// F(0), delta, the swap flag) is warp-uniform.
#include "common.cuh"
#include "kernels.h"

namespace snt {

constexpr unsigned FULL = 0xffffffffu;

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

// Runs the 2p-1 divsteps on this warp's state.  In: G planes (reversed g).
// Out: planes of 1/g in reversed order (trit j of the output planes is
// coefficient p-1-j of 1/g).  Returns true iff g is invertible.
template <int P>
__device__ __forceinline__ bool r3_divsteps(uint32_t gm, uint32_t gs, uint32_t &om,
                                            uint32_t &os) {
    const int lane = threadIdx.x & 31;
    uint32_t fm = 0, fs = 0;
    if (lane == 0) fm |= 1u;
    if (lane == (P - 1) / 32) { fm |= 1u << ((P - 1) % 32); fs |= 1u << ((P - 1) % 32); }
    if (lane == P / 32) { fm |= 1u << (P % 32); fs |= 1u << (P % 32); }
    uint32_t vm = 0, vs = 0, rm = (lane == 0) ? 1u : 0u, rs = 0;
    int delta = 1;
    uint32_t f0s = 0;  // sign bit of F(0); F(0) is never zero
    const int below = (lane + 31) & 31, above = (lane + 1) & 31;

#pragma unroll 2
    for (int step = 0; step < 2 * P - 1; ++step) {
        // V <- x V
        const uint32_t pm = __shfl_sync(FULL, vm, below);
        const uint32_t ps = __shfl_sync(FULL, vs, below);
        vm = __funnelshift_l(pm, vm, 1);
        vs = __funnelshift_l(ps, vs, 1);
        // G(0), warp-uniform
        const uint32_t g0m = __shfl_sync(FULL, gm, 0) & 1u;
        const uint32_t g0s = __shfl_sync(FULL, gs, 0) & 1u;
        const uint32_t sw = (uint32_t)(delta > 0) & g0m;
        const uint32_t msk = 0u - sw;
        uint32_t t;
        t = (fm ^ gm) & msk; fm ^= t; gm ^= t;
        t = (fs ^ gs) & msk; fs ^= t; gs ^= t;
        t = (vm ^ rm) & msk; vm ^= t; rm ^= t;
        t = (vs ^ rs) & msk; vs ^= t; rs ^= t;
        const uint32_t nf0s = sw ? g0s : f0s;
        const uint32_t ng0s = sw ? f0s : g0s;  // G(0) stays nonzero iff it was
        f0s = nf0s;
        delta = (sw ? -delta : delta) + 1;
        // c = -G(0) F(0) (= -G(0)/F(0) in F_3)
        const uint32_t cm = 0u - g0m;
        const uint32_t cs = 0u - ((ng0s ^ f0s ^ 1u) & 1u);
        f3_add(gm, gs, fm & cm, fs ^ cs, gm, gs);
        f3_add(rm, rs, vm & cm, vs ^ cs, rm, rs);
        // G <- G / x
        const uint32_t nm = __shfl_sync(FULL, gm, above);
        const uint32_t ns = __shfl_sync(FULL, gs, above);
        gm = __funnelshift_r(gm, nm, 1);
        gs = __funnelshift_r(gs, ns, 1);
    }
    om = vm;
    os = vs ^ (0u - f0s);
    return delta == 0;
}

// Builds this lane's planes of G (trit j = g[p-1-j]) from int8 coefficients in
// shared memory (g[0..p) in {-1,0,1}).
template <int P>
__device__ __forceinline__ void planes_from_reversed(const int8_t *gsm, uint32_t &gm,
                                                     uint32_t &gs) {
    const int lane = threadIdx.x & 31;
    gm = 0; gs = 0;
#pragma unroll 8
    for (int b = 0; b < 32; ++b) {
        const int j = 32 * lane + b;
        const int src = P - 1 - j;
        const int c = (src >= 0) ? gsm[src] : 0;
        gm |= (uint32_t)(c != 0) << b;
        gs |= (uint32_t)(c < 0) << b;
    }
}

// Writes the natural-order coefficients of the output planes (reversed) to
// shared memory: out[i] = trit (p-1-i).
template <int P>
__device__ __forceinline__ void reversed_to_smem(uint32_t om, uint32_t os, int8_t *osm) {
    const int lane = threadIdx.x & 31;
#pragma unroll 8
    for (int b = 0; b < 32; ++b) {
        const int j = 32 * lane + b;
        const int i = P - 1 - j;
        if (i >= 0) {
            const int m = (om >> b) & 1, s = (os >> b) & 1;
            osm[i] = (int8_t)(m ? (s ? -1 : 1) : 0);
        }
    }
}

// ---------------------------------------------------------------------------
// Keygen form: sample g (stream 0, attempt a) until invertible, write g
// (int8, zero padded, stride pad) for the h product and Small_encode(1/g)
// into the secret key at sk_off.  One warp per key, 4 keys per CTA.
// ---------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(128)
k_r3_keygen(uint64_t seed, uint64_t first, int B, int8_t *__restrict__ g_out,
            uint8_t *__restrict__ sk, int sk_bytes, int sk_off,
            const uint64_t *__restrict__ inj_idx, const int8_t *__restrict__ inj_g,
            int n_inj, int *__restrict__ err) {
    using Gm = Geo<P>;
    __shared__ int8_t smem[4][1024];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int key = blockIdx.x * 4 + warp;
    if (key >= B) return;
    const uint64_t k = first + (uint64_t)key;
    int8_t *gsm = smem[warp];

    // optional injected attempt-0 draw (test hook)
    int inj = -1;
    for (int j = lane; j < n_inj; j += 32)
        if (inj_idx[j] == k) inj = j;
    for (int off = 16; off > 0; off >>= 1) inj = max(inj, __shfl_xor_sync(FULL, inj, off));

    bool ok = false;
    uint32_t om = 0, os = 0;
    for (int att = 0; att < kMaxGAttempts && !ok; ++att) {
        if (att == 0 && inj >= 0) {
            for (int i = lane; i < P; i += 32) gsm[i] = inj_g[(size_t)inj * Gm::p + i];
        } else {
            // g_i = floor(3 (u_i mod 2^30) / 2^30) - 1 for word u_i of stream 0
            for (int blk = lane; 4 * blk < P; blk += 32) {
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
        __syncwarp();
        uint32_t gm, gs;
        planes_from_reversed<P>(gsm, gm, gs);
        ok = r3_divsteps<P>(gm, gs, om, os);
    }
    if (!ok) {
        if (lane == 0) atomicOr(err, ERR_RESAMPLE);
        om = 0; os = 0;
    }
    // g (natural order) for h = g * (3f)^-1
    int8_t *gk = g_out + (size_t)key * Gm::pad;
    for (int i = lane; i < Gm::pad; i += 32) gk[i] = (i < P) ? gsm[i] : (int8_t)0;
    __syncwarp();
    reversed_to_smem<P>(om, os, gsm);
    __syncwarp();
    // Small_encode(1/g)
    uint8_t *skk = sk + (size_t)key * sk_bytes + sk_off;
    for (int b = lane; b < Gm::small_bytes; b += 32) {
        uint32_t byte = 0;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int i = 4 * b + t;
            if (i < P) byte |= (uint32_t)(gsm[i] + 1) << (2 * t);
        }
        skk[b] = (uint8_t)byte;
    }
}

// ---------------------------------------------------------------------------
// Batch form for the kernel microbenchmark: out_i = 1/g_i, ok_i.
// g, out: n x p int8 (stride p).
// ---------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(128)
k_r3_inv(int n, const int8_t *__restrict__ g, int8_t *__restrict__ out,
         int32_t *__restrict__ okv) {
    __shared__ int8_t smem[4][1024];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int e = blockIdx.x * 4 + warp;
    if (e >= n) return;
    int8_t *gsm = smem[warp];
    for (int i = lane; i < P; i += 32) gsm[i] = g[(size_t)e * P + i];
    __syncwarp();
    uint32_t gm, gs, om, os;
    planes_from_reversed<P>(gsm, gm, gs);
    const bool ok = r3_divsteps<P>(gm, gs, om, os);
    if (!ok) { om = 0; os = 0; }
    __syncwarp();
    reversed_to_smem<P>(om, os, gsm);
    __syncwarp();
    for (int i = lane; i < P; i += 32) out[(size_t)e * P + i] = gsm[i];
    if (lane == 0) okv[e] = ok ? 1 : 0;
}

template <int P>
cudaError_t launch_r3_keygen(uint64_t seed, uint64_t first, int B, int8_t *g_out,
                             uint8_t *sk, int sk_bytes, int sk_off, const uint64_t *inj_idx,
                             const int8_t *inj_g, int n_inj, int *err, cudaStream_t st) {
    k_r3_keygen<P><<<(B + 3) / 4, 128, 0, st>>>(seed, first, B, g_out, sk, sk_bytes, sk_off,
                                                inj_idx, inj_g, n_inj, err);
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_r3_inv(int n, const int8_t *g, int8_t *out, int32_t *ok, cudaStream_t st) {
    k_r3_inv<P><<<(n + 3) / 4, 128, 0, st>>>(n, g, out, ok);
    return cudaGetLastError();
}

#define SNT_R3_INST(P)                                                                      \
    template cudaError_t launch_r3_keygen<P>(uint64_t, uint64_t, int, int8_t *, uint8_t *,  \
                                             int, int, const uint64_t *, const int8_t *,    \
                                             int, int *, cudaStream_t);                     \
    template cudaError_t launch_r3_inv<P>(int, const int8_t *, int8_t *, int32_t *, cudaStream_t);
SNT_R3_INST(653)
SNT_R3_INST(761)
SNT_R3_INST(857)

}  // namespace snt
