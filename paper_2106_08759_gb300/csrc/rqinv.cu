// rqinv.cu -- inversion in R/q = (Z/q)[x]/(x^p - x - 1) by divsteps, one CTA
// per element.
//
// Used for the single root inversion of the batch-inversion tree (Sec. 2.2,
// Montgomery's trick: "compute the single multiplicative inverse"; the paper
// reports 785909 Haswell cycles for it in sntrup761, Sec. 3.4), for the
// per-key path (Sec. 3.1 KeyGen step 4 without batching) and for the kernel
// microbenchmark.  The paper cites Bernstein-Yang divsteps; the iteration on
// reversed polynomials is
//     F = 1 - x^(p-1) - x^p,  G = x^(p-1) a(1/x),  V = 0,  R = 1,  delta = 1;
//     2p - 1 times:  V <- x V;
//                    if delta > 0 and G(0) != 0: swap (F,G), (V,R), delta <- -delta;
//                    delta <- delta + 1;
//                    G <- (F(0) G - G(0) F) / x;  R <- F(0) R - G(0) V;
//     a is invertible iff delta = 0; then (1/a)_i = V(p-1-i) / F(0).
//
// Layout: the four state polynomials live in shared memory as int32 in the
// lazy range [-q, 2q).  A swap exchanges two buffer pointers, G <- G/x moves
// G's base up one slot and V <- x V moves V's base down one slot, so no data
// moves except the two multiply-reduce updates per coefficient.  A buffer's
// base only moves while it plays G (up) or V (down), at most 2p - 1 times, so
// 3p slots per buffer suffice; slots are zeroed once and the slots a moving
// base uncovers were never written.  One barrier per step.
#include "common.cuh"
#include "kernels.h"
#include "mma_mul.cuh"
#include "pdl.cuh"

namespace snt {

template <int P> struct InvGeo {
    static constexpr int LEN = 3 * P;     // slots per state buffer
    static constexpr int V0 = 2 * P - 1;  // initial base of the V/R buffers
};

template <int Q> __device__ __forceinline__ int mulmod_pos(int a, int b) {
    return (int)(((long long)a * b) % Q);  // a, b in [0, Q)
}

template <int Q> __device__ __forceinline__ int inv_mod(int a) {  // a^(Q-2), a in [1, Q)
    int acc = 1, base = a;
    for (int e = Q - 2; e > 0; e >>= 1) {
        if (e & 1) acc = mulmod_pos<Q>(acc, base);
        base = mulmod_pos<Q>(base, base);
    }
    return acc;
}

// in: p centred coefficients (stride-free); out: p centred coefficients.
template <int P, int NT, typename TIn>
__device__ __forceinline__ bool rq_inv_cta(const TIn *__restrict__ in, int16_t *__restrict__ out,
                                           int (*buf)[InvGeo<P>::LEN]) {
    constexpr int Q = Geo<P>::q;
    constexpr int LEN = InvGeo<P>::LEN;
    const int tid = threadIdx.x;
    for (int i = tid; i < 4 * LEN; i += NT) (&buf[0][0])[i] = 0;
    __syncthreads();
    // buffers 0/1 play F/G, 2/3 play V/R
    int *Fb = buf[0], *Gb = buf[1], *Vb = buf[2], *Rb = buf[3];
    int bf = 0, bg = 0, bv = InvGeo<P>::V0, br = InvGeo<P>::V0;
    for (int i = tid; i < P; i += NT) Gb[i] = (int)in[P - 1 - i];
    if (tid == 0) {
        Fb[0] = 1;
        Fb[P - 1] = -1;
        Fb[P] = -1;
        Rb[br] = 1;
    }
    __syncthreads();
    int delta = 1;
    for (int step = 0; step < 2 * P - 1; ++step) {
        --bv;  // V <- x V (the uncovered slot is zero)
        int f0 = freeze_lazy<Q>(Fb[bf]);
        int g0 = freeze_lazy<Q>(Gb[bg]);
        if (delta > 0 && g0 != 0) {  // warp-uniform (all threads read the same values)
            int *t = Fb; Fb = Gb; Gb = t;
            int tb = bf; bf = bg; bg = tb;
            t = Vb; Vb = Rb; Rb = t;
            tb = bv; bv = br; br = tb;
            const int tv = f0; f0 = g0; g0 = tv;
            delta = -delta;
        }
        ++delta;
        const int ng0 = g0 ? Q - g0 : 0;  // -g0 in [0, Q)
#pragma unroll 4
        for (int i = tid; i <= P; i += NT) {
            if (i >= 1) Gb[bg + i] = lazy_red<Q>(f0 * Gb[bg + i] + ng0 * Fb[bf + i]);
            Rb[br + i] = lazy_red<Q>(f0 * Rb[br + i] + ng0 * Vb[bv + i]);
        }
        ++bg;  // G <- G / x (G(0) is zero now)
        __syncthreads();
    }
    const bool ok = (delta == 0);
    const int f0 = freeze_lazy<Q>(Fb[bf]);
    const int s = ok ? inv_mod<Q>(f0) : 0;
    for (int i = tid; i < P; i += NT) {
        const int v = freeze_lazy<Q>(Vb[bv + P - 1 - i]);
        out[i] = (int16_t)cmod<Q>(s * v);
    }
    return ok;
}

template <int P> constexpr int inv_threads() { return 256; }

// Element e of n: in + e*in_stride -> out + e*out_stride (p coefficients each;
// the pads of the output rows are left untouched).  ok[e] = invertible.
// In-place use (in == out) is safe: the input is read before any output store.
template <int P, int NT, typename TIn>
__global__ void __launch_bounds__(NT)
k_rq_inv(int n, const TIn *in, long in_stride, int16_t *out, long out_stride,
         int32_t *__restrict__ okv, int *__restrict__ err, int err_bit) {
    pdl_enter();
    __shared__ int buf[4][InvGeo<P>::LEN];
    const int e = blockIdx.x;
    if (e >= n) return;
    const bool ok = rq_inv_cta<P, NT, TIn>(in + (size_t)e * in_stride,
                                           out + (size_t)e * out_stride, buf);
    if (threadIdx.x == 0) {
        if (okv) okv[e] = ok ? 1 : 0;
        if (!ok && err) atomicOr(err, err_bit);
    }
}

// ---------------------------------------------------------------------------
// Jump divsteps (latency-optimised form for the single root inversion).
//
// The first m divsteps of (delta, F, G) depend only on delta and the low m
// coefficients of F and G.  A leader warp runs a chunk of m <= 31 steps on
// those coefficients alone (one coefficient per lane, shuffles for the shifts
// and G(0)) and accumulates the chunk's transition matrix
//     x^m (F', G') = A (F, G),   A = [[u, v], [w, z]],  deg <= m,
// built step by step as  row1 <- x * row1,  row2 <- F(0) row2 - G(0) row1
// (rows exchanged first when the step swaps).  The other warps apply A:
//     F' = (u F + v G) / x^m,   G' = (w F + z G) / x^m,
//     V' = u V + (v / x) R,     R' = x w V + z R,
// the last two because V is multiplied by x before each step's swap, which
// conjugates A by diag(1, x).  The chunks are pipelined: while the appliers
// apply chunk c, the leader (with the helper warps) computes the 32 low
// coefficients of F', G' and runs the divsteps of chunk c + 1, so a chunk
// costs about the larger of the two.  One barrier per chunk,
// ceil((2p-1)/31) chunks.
//
// Live extents.  A chunk's matrix entries have degree at most m, so F', G'
// are zero wherever F and G are (index i of F' reads F at i + m - k, k <= m),
// and V', R' reach at most m + 1 past V and R.  The block keeps the extent
// of each state (one past the highest nonzero coefficient of F or G, and of
// V or R, found by the appliers as they write) and computes only the live
// outputs, zeroing what the older state left above them in the target
// buffer.  F, G shrink while V, R grow, their extents summing to about
// p + 2, so a chunk applies the matrix to about p + 34 coefficients rather
// than to four full-length polynomials.  The appliers run on the three
// schedulers that are not the leader's; the other warps on the leader's
// scheduler (the helpers) compute half of the leader's prologue (the low
// coefficients of F', G') beside it, then wait for its next matrix and
// build that matrix's limb pair tables, so that the appliers find them
// ready.  Measured on one sntrup761 root alone (clock stamps, cycles per
// chunk): 3663 with the leader alone on its scheduler (prologue 786, steps
// 2609), 3651 with the helpers' prologue (516 and 2168: the appliers, ~480
// of set-up and ~2600 for the scheduler that holds three of the usual seven
// tiles, then set the chunk), 3404 with the tables built ahead (set-up 331),
// 3302 with the F, G tiles on that scheduler.  Giving the helpers tiles too
// (so that no scheduler holds three) slowed the leader back to 83 cycles per
// step and the chunk to ~3730.
//
// The application on the tensor cores.  Each output of a pair is a sum of
// two Toeplitz products with the chunk matrix: with T_e[i][j] = e[i - j + o],
//     F' = T_u F + T_v G,  G' = T_w F + T_z G   (o = m for all four),
//     V' = T_u V + T_v R,  R' = T_w V + T_z R   (o = 0, +1, -1, 0),
// the form of the tensor-core R/q product (mma_mul.cuh): for 16-coefficient
// blocks the block (I, J) of T_e depends only on D = I - J, so an m16n8k16
// MMA takes A from a pair table of e ((e[x], e[x-1]) per x as 6-bit limbs
// h, l in f16, built by the applier warps from the matrix at the start of
// the chunk) and as B eight 16-coefficient blocks of the state.  The state
// is kept as one f16 value per coefficient, a representative of its residue
// that f16 holds exactly (the residue itself, or the residue -+ q when it is
// odd and above 2048 in magnitude: at most q - 2049), written once by the
// application that produces it and laid out so that a lane's B fragment is
// one 8-byte load (spos); the leader reads an int copy of the low 64
// coefficients of F and G, and the inverse is read back from V at the end.
// An item is one 128-output tile of one pair (at most eight per chunk, one
// per applier warp, two per scheduler): D runs over the 3 or 4 values where
// some T_e block is nonzero, two MMAs per operand pair (h_e b' and l_e b';
// one, l_e b', when every value is in {-1, 0, 1}); a sum has at most 64
// terms, 64 * 41 * 3118 < 2^24, so every limb sum is exact in f32, and
// 64 P_h + P_l stays below 2^31.
//
// Ranges: inside the leader's steps values are lazily reduced to [-q, 2q)
// (G(0) = 0 mod q iff G(0) is -q, 0 or q); the matrix and the state are
// centred between chunks, so a 64-term application sum stays below 2^31.
// ---------------------------------------------------------------------------
template <int P, int Q = Geo<P>::q> struct JumpGeo {
    static constexpr int M = 31;                        // steps per chunk
    static constexpr int OFF = 32;                      // zero margin below index 0
    // applier warps on the three schedulers that are not the leader's, so
    // that its divstep chain has a scheduler to itself: in R/q ids 1-3, 5-7,
    // 9-11 (seven or eight tiles per chunk for sntrup761), in R/3, where an
    // operand pair is one MMA, ids 1-3, 5-7; the other warps on the leader's
    // scheduler (4 and 8, or 4) compute part of the leader's prologue and
    // build the pair tables of its next matrix
    static constexpr int NW = Q < 64 ? 8 : 12;          // leader, appliers, helpers
    static constexpr int NWA = NW - NW / 4;
    static constexpr int NA = 32 * NWA;                 // applier threads
    static constexpr int NH = NW / 4 - 1;               // helper warps
    static constexpr int LG = 2, HG = 2 / NH;           // prologue groups of 8 terms: leader, helper
    static constexpr int NT = 32 * NW;
    // a tile reads blocks up to two past its last output block (D >= -2)
    static constexpr int LEN = (OFF + P + 160 + 31) / 32 * 32;  // slots per polynomial
    static constexpr int PTX = 112;                     // pair-table entries per matrix entry
    static constexpr int PT0 = 48;                      // table index of coefficient 0
};

template <int Q> __device__ __forceinline__ bool is_zero_lazy(int x) {  // x in [-Q, 2Q)
    return x == 0 || x == Q || x == -Q;
}

// The leader's chunk: m divsteps from (fl, gl) (lane i = coefficient i),
// matrix returned centred in (u, v, w, z) (lane k = coefficient k).
//
// Each step forms the new G row as f0 g - g0 f from the values before the
// swap. When the step swaps, that is minus the divstep's new G (Section 3's
// divstep sends (f, g) to (g, (g0 f - f0 g)/x)), so a row of the returned
// matrix may differ from the divstep matrix's row by a sign. Nothing
// downstream depends on that sign: the swap test looks only at delta and
// whether g0 is zero, F and V (G and R) are always updated by the same row,
// and the inverse is V / F(0) at the end. Dropping the sign takes the swap
// off the step's dependency chain, which is then the product, the
// reduction and one shuffle.
//
// Lane 31 of G after the shift keeps its own value instead of the unknown
// coefficient 32: step s reads only coefficient 0, which depends on
// coefficients 0..s of the chunk's input, so the error never reaches it
// within 31 steps. The matrix entries have degree at most s at step s, so
// lane 31 of u and v is zero before every shift and a rotation by one lane
// is the multiplication by x.
template <int Q>
__device__ __forceinline__ void leader_step(int from, int &delta, int &f0, int &g0, int &fl, int &gl,
                                            int &u, int &v, int &w, int &z) {
    // the chain: new G, then its shift and its coefficient 0 (read straight
    // from lane 1) issued first; the rest of the step runs in the shuffles'
    // shadow
    const int ng = lazy_red<Q>(f0 * gl - g0 * fl);
    const int g0n = __shfl_sync(0xffffffffu, ng, 1);
    const int gln = __shfl_down_sync(0xffffffffu, ng, 1);
    const int nw = lazy_red<Q>(f0 * w - g0 * u);
    const int nz = lazy_red<Q>(f0 * z - g0 * v);
    const bool sw = (delta > 0) & !is_zero_lazy<Q>(g0);  // warp-uniform
    delta = (sw ? -delta : delta) + 1;
    fl = sw ? gl : fl;
    f0 = sw ? g0 : f0;
    // u, v (lazy, inside int16) shifted together as one packed word
    const int uv = __shfl_sync(0xffffffffu, __byte_perm(sw ? w : u, sw ? z : v, 0x5410), from);
    u = (uv << 16) >> 16;
    v = uv >> 16;
    w = nw;
    z = nz;
    g0 = g0n;
    gl = gln;
}

// A full chunk (M steps) is unrolled so consecutive steps interleave; the
// last, shorter chunk runs the same step in a loop.
template <int Q, int M>
__device__ __forceinline__ void leader_chunk(int m, int &delta, int fl, int gl, int &u, int &v,
                                             int &w, int &z) {
    const int lane = threadIdx.x & 31, from = (lane + 31) & 31;
    u = (lane == 0); v = 0; w = 0; z = (lane == 0);
    int f0 = __shfl_sync(0xffffffffu, fl, 0);
    int g0 = __shfl_sync(0xffffffffu, gl, 0);
    if (m == M) {
#pragma unroll
        for (int s = 0; s < M; ++s) leader_step<Q>(from, delta, f0, g0, fl, gl, u, v, w, z);
    } else {
        for (int s = 0; s < m; ++s) leader_step<Q>(from, delta, f0, g0, fl, gl, u, v, w, z);
    }
    u = cmod<Q>(u); v = cmod<Q>(v); w = cmod<Q>(w); z = cmod<Q>(z);
}

// Eight consecutive matrix coefficients from a 16-byte aligned address.
__device__ __forceinline__ void load8(int (&c)[8], const int *p) {
    const int4 a = reinterpret_cast<const int4 *>(p)[0], b = reinterpret_cast<const int4 *>(p)[1];
    c[0] = a.x; c[1] = a.y; c[2] = a.z; c[3] = a.w;
    c[4] = b.x; c[5] = b.y; c[6] = b.z; c[7] = b.w;
}

// Lane k's coefficients of the chunk matrix: coefficient k of u, v, w, z at
// 4 + k of its row (zero outside k = 0..31 from the block's start).
__device__ __forceinline__ void put_matrix(int (*An)[40], int lane, int u, int v, int w, int z) {
    An[0][4 + lane] = u; An[1][4 + lane] = v;
    An[2][4 + lane] = w; An[3][4 + lane] = z;
}

// Position of state coefficient j in its row: within each block of 16
// coefficients, 2t, 2t + 1, 2t + 8 and 2t + 9 sit at 4t .. 4t + 3, so the B
// fragment of a lane (those four coefficients of one block) is one 8-byte
// load and the loads of a half-warp (four consecutive tig, two blocks) are
// one contiguous 128-byte run.
__device__ __forceinline__ int spos(int j) {
    const int k = j & 15;
    return (j & ~15) | (((k & 7) >> 1) << 2) | (k & 1) | ((k >> 3) << 1);
}

// A coefficient as stored: the f16 bits of a representative of the centred
// residue x that f16 holds exactly (x itself, or x -+ Q when x is odd and
// above 2048 in magnitude).
template <int Q> __device__ __forceinline__ uint16_t state_half(int x) {
    return __half_as_ushort(__int2half_rn(f16_rep<Q>(x)));
}
__device__ __forceinline__ int half_value(uint16_t h) { return __half2int_rn(__ushort_as_half(h)); }

// acc[0] += l_e b' and (unless SMALL) acc[1] += h_e b': A from the pair-table
// words at x, x + 8, x - 8 of e's limbs, B the block's four state values.
template <bool SMALL>
__device__ __forceinline__ void jump_mma(float (&acc)[SMALL ? 1 : 2][4], const uint2 *pt, int x,
                                         uint2 b) {
    const uint2 a0 = pt[x], a1 = pt[x + 8], a2 = pt[x - 8];
    mma16816(acc[0], a0.y, a1.y, a2.y, a0.y, b.x, b.y);
    if (!SMALL) mma16816(acc[SMALL ? 0 : 1], a0.x, a1.x, a2.x, a0.x, b.x, b.y);
}

// Part of the leader's prologue: for lane i, the sums over the matrix
// coefficients k = kb0 .. kb0 + 8 NG - 1 of u_k F[hi - k] + v_k G[hi - k]
// (into sf) and w_k F[hi - k] + z_k G[hi - k] (into sg).
template <int NG>
__device__ __forceinline__ void prologue_part(const int (*A)[40], const int *F, const int *G,
                                              int hi, int kb0, int &sf, int &sg) {
    int af[2] = {0, 0}, ag[2] = {0, 0};
#pragma unroll
    for (int gi = 0; gi < NG; ++gi) {
        const int kb = kb0 + 8 * gi;
        int c0[8], c1[8], c2[8], c3[8];
        load8(c0, &A[0][4 + kb]); load8(c1, &A[1][4 + kb]);
        load8(c2, &A[2][4 + kb]); load8(c3, &A[3][4 + kb]);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int fv = F[hi - kb - j], gv = G[hi - kb - j];
            af[j & 1] += c0[j] * fv + c1[j] * gv;
            ag[j & 1] += c2[j] * fv + c3[j] * gv;
        }
    }
    sf = af[0] + af[1];
    sg = ag[0] + ag[1];
}

// The limb pair tables of a chunk matrix (rows u, v, w, z of A) into P,
// entries k = 0 .. 32 of each (the rest stay zero), by threads t0, t0 + nt, ...
template <int PTX, int PT0>
__device__ __forceinline__ void build_pair_tables(const int (*A)[40], uint2 (*P)[PTX], int t0,
                                                  int nt) {
    for (int pe = t0; pe < 4 * 33; pe += nt) {
        const int en = pe / 33, k = pe % 33;
        const int e0 = A[en][4 + k], e1 = A[en][3 + k];  // e[k], e[k-1]; zero at 32 and -1
        int h0, l0, h1, l1;
        limbs64(e0, h0, l0);
        limbs64(e1, h1, l1);
        P[en][PT0 + k] = make_uint2(h2_small(h0, h1), h2_small(l0, l1));
    }
}

// Q: the coefficient modulus (q: R/q; 3: R/3, for the root inversions of
// the R/3 batch inversion).
template <int P, int Q = Geo<P>::q>
__global__ void __launch_bounds__(JumpGeo<P, Q>::NT, 1)
k_rq_inv_jump(int n, const int16_t *in, long in_stride, int16_t *out, long out_stride,
              int32_t *__restrict__ okv, int *__restrict__ err, int err_bit, const int *idx) {
    pdl_enter();
    using JG = JumpGeo<P, Q>;
    constexpr int LEN = JG::LEN, OFF = JG::OFF, NT = JG::NT;
    constexpr bool SMALL = Q < 64;  // every value in {-1, 0, 1}: the l limbs only
    constexpr int NCH = (2 * P - 1 + JG::M - 1) / JG::M;
    // state values (f16) [buffer][F, G, V, R][spos(index + OFF)], and int
    // copies of F, G at indices -32 .. 63 for the leader's prologue
    __shared__ __align__(16) uint16_t st[2][4][LEN];
    __shared__ int lowfg[2][2][96];
    // chunk matrix [buffer][u, v, w, z][4 + k], 16-byte rows for vector
    // loads, zero outside k = 0..31
    __shared__ __align__(16) int mat[2][4][40];
    // limb pair tables of u, v, w, z for the appliers, [buffer][u, v, w, z]:
    // entry PT0 + x holds (h, l) of (e[x], e[x-1]) as f16x2 words, zero
    // outside x = 0..32; chunk c's in pt[c & 1], built by the helpers while
    // the appliers apply chunk c - 1
    __shared__ __align__(16) uint2 pt[2][4][JG::PTX];
    // extents of the state after chunk c - 1 in ext[c % 4]: [0] F, G and
    // [1] V, R (one past the highest nonzero coefficient)
    __shared__ int ext[4][2];
    __shared__ int pro[2][2][32];  // the helpers' prologue sums [helper][F', G'][lane]
    __shared__ int s_ok;
    const int e = blockIdx.x;
    if (e >= n) return;
    const int tid = threadIdx.x, lane = tid & 31;
    const bool leader = tid < 32;
    const int row = idx ? idx[e] : e;
    const int16_t *a = in + (size_t)row * in_stride;
    for (int i = tid; i < 2 * 4 * LEN; i += NT) (&st[0][0][0])[i] = 0;  // f16 zeros
    for (int i = tid; i < 2 * 2 * 96; i += NT) (&lowfg[0][0][0])[i] = 0;
    for (int i = tid; i < 2 * 4 * 40; i += NT) (&mat[0][0][0])[i] = 0;
    for (int i = tid; i < 2 * 4 * JG::PTX; i += NT) (&pt[0][0][0])[i] = make_uint2(0u, 0u);
    if (tid < 8) (&ext[0][0])[tid] = 0;
    __syncthreads();
    for (int i = tid; i < P; i += NT) {
        const int g = (int)a[P - 1 - i];
        st[0][1][spos(OFF + i)] = state_half<Q>(g);
        if (i < 64) lowfg[0][1][32 + i] = g;
    }
    if (tid == 0) {
        st[0][0][spos(OFF)] = state_half<Q>(1);
        st[0][0][spos(OFF + P - 1)] = state_half<Q>(-1);
        st[0][0][spos(OFF + P)] = state_half<Q>(-1);
        st[0][3][spos(OFF)] = state_half<Q>(1);
        lowfg[0][0][32] = 1;
        ext[0][0] = P + 1;
        ext[0][1] = 1;
    }
    __syncthreads();
    int delta = 1;  // leader only
    if (leader) {
        int u, v, w, z;
        leader_chunk<Q, JG::M>(min(JG::M, 2 * P - 1), delta, lowfg[0][0][32 + lane],
                               lowfg[0][1][32 + lane], u, v, w, z);
        put_matrix(mat[0], lane, u, v, w, z);
    }
    __syncthreads();
    build_pair_tables<JG::PTX, JG::PT0>(mat[0], pt[0], tid, NT);
    __syncthreads();
    int cur = 0;
    for (int c = 0; c < NCH; ++c) {
        const int m = min(JG::M, 2 * P - 1 - c * JG::M);
        const int(*A)[40] = mat[c & 1];
        const uint2(*PT)[JG::PTX] = pt[c & 1];
        if (leader) {
            if (c + 1 < NCH) {
                // low 32 coefficients of F', G' (lane i): the first LG groups
                // of matrix terms here, the rest from the helpers; then chunk
                // c + 1
                int sf, sg;
                prologue_part<JG::LG>(A, lowfg[cur][0], lowfg[cur][1], 32 + lane + m, 0, sf, sg);
                asm volatile("bar.sync 2, %0;" ::"n"(32 * (1 + JG::NH)) : "memory");
#pragma unroll
                for (int h = 0; h < JG::NH; ++h) {
                    sf += pro[h][0][lane];
                    sg += pro[h][1][lane];
                }
                const int m1 = min(JG::M, 2 * P - 1 - (c + 1) * JG::M);
                int u, v, w, z;
                leader_chunk<Q, JG::M>(m1, delta, cmod<Q>(sf), cmod<Q>(sg), u, v, w, z);
                put_matrix(mat[(c + 1) & 1], lane, u, v, w, z);
                asm volatile("bar.arrive 3, %0;" ::"n"(32 * (1 + JG::NH)) : "memory");
            } else if (lane == 0) {
                s_ok = (delta == 0);
            }
        } else if ((tid >> 5) & 3) {
            const int w = tid >> 5, ai = w - 1 - (w - 1) / 4;
            const int at = 32 * ai + lane;
            // live ranges of the outputs and what the target buffer held
            const int rfg = ext[c & 3][0], rvr = min(ext[c & 3][1] + m + 1, P + 1);
            const int ofg = ext[(c + 3) & 3][0], ovr = ext[(c + 3) & 3][1];
            uint16_t *T = &st[cur ^ 1][0][0];
            for (int i = rfg + at; i < ofg; i += JG::NA) {
                T[spos(OFF + i)] = 0; T[LEN + spos(OFF + i)] = 0;
                if (i < 64) { lowfg[cur ^ 1][0][32 + i] = 0; lowfg[cur ^ 1][1][32 + i] = 0; }
            }
            for (int i = rvr + at; i < ovr; i += JG::NA) {
                T[2 * LEN + spos(OFF + i)] = 0; T[3 * LEN + spos(OFF + i)] = 0;
            }
            if (at == 0) { ext[(c + 2) & 3][0] = 0; ext[(c + 2) & 3][1] = 0; }
            const int g = lane >> 2, tig = lane & 3;
            const int nfg = (rfg + 127) / 128, nit = nfg + (rvr + 127) / 128;
            int top_fg = 0, top_vr = 0;
            for (int sl = ai; sl < nit; sl += JG::NWA) {  // one tile of one pair per warp
                // with seven tiles (the usual count) the scheduler of slots 0,
                // 3 and 6 holds three: give it tiles 0, 1, 2, the F, G tiles
                // while there are three (three D steps, against four for V, R)
                const int it = (nit == 7 && sl < 7) ? (0x2641530 >> (4 * sl)) & 15 : sl;
                const int pr = it >= nfg;
                const int T0 = pr ? it - nfg : it, r = pr ? rvr : rfg;
                const uint2 *X = reinterpret_cast<const uint2 *>(st[cur][2 * pr]);
                const uint2 *Y = reinterpret_cast<const uint2 *>(st[cur][2 * pr + 1]);
                // offsets o of T_u, T_v, T_w, T_z and the D range where some
                // block is nonzero: 0 <= 16 D + (row - col) + o <= 31
                const int ou = pr ? 0 : m, ov = pr ? 1 : m, ow = pr ? -1 : m;
                const int dlo = pr ? -1 : -((15 + m) >> 4), dhi = pr ? 2 : (46 - m) >> 4;
                constexpr int NL = SMALL ? 1 : 2;  // limb products l_e b', h_e b'
                float acc[2][NL][4];                // [output][limb product]
#pragma unroll
                for (int o = 0; o < 2; ++o)
#pragma unroll
                    for (int t = 0; t < NL; ++t)
#pragma unroll
                        for (int q = 0; q < 4; ++q) acc[o][t][q] = 0.f;
#pragma unroll
                for (int dd = 0; dd < 4; ++dd) {  // at most four D values
                    const int D = dlo + dd;
                    if (D > dhi) break;
                    const int jb = 4 * ((OFF >> 4) + 8 * T0 + g - D) + tig;  // input block I - D
                    const uint2 bx = X[jb], by = Y[jb];
                    const int x = JG::PT0 + 16 * D + g - 2 * tig;
                    // X terms of both outputs first, so the two MMAs that
                    // meet in one accumulator are apart
                    jump_mma<SMALL>(acc[0], PT[0], x + ou, bx);
                    jump_mma<SMALL>(acc[1], PT[2], x + ow, bx);
                    jump_mma<SMALL>(acc[0], PT[1], x + ov, by);
                    jump_mma<SMALL>(acc[1], PT[3], x + ou, by);
                }
                uint16_t *X2 = st[cur ^ 1][2 * pr], *Y2 = st[cur ^ 1][2 * pr + 1];
                int top = 0;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int i = 16 * (8 * T0 + 2 * tig + (q & 1)) + g + 8 * (q >> 1);
                    if (i < r) {
                        int v[2];
#pragma unroll
                        for (int o = 0; o < 2; ++o) {
                            // integer-valued sums below 2^24: the f32 arithmetic is exact
                            if (SMALL) {
                                v[o] = cmod<Q>(__float2int_rn(acc[o][0][q]));
                            } else {
                                v[o] = cmod<Q>(64 * __float2int_rn(acc[o][1][q]) +
                                               __float2int_rn(acc[o][0][q]));
                            }
                        }
                        X2[spos(OFF + i)] = state_half<Q>(v[0]);
                        Y2[spos(OFF + i)] = state_half<Q>(v[1]);
                        if (!pr && i < 64) { lowfg[cur ^ 1][0][32 + i] = v[0]; lowfg[cur ^ 1][1][32 + i] = v[1]; }
                        if (v[0] | v[1]) top = max(top, i + 1);
                    }
                }
                if (pr) top_vr = max(top_vr, top); else top_fg = max(top_fg, top);
            }
            top_fg = __reduce_max_sync(0xffffffffu, top_fg);
            top_vr = __reduce_max_sync(0xffffffffu, top_vr);
            if (lane == 0) {
                atomicMax(&ext[(c + 1) & 3][0], top_fg);
                atomicMax(&ext[(c + 1) & 3][1], top_vr);
            }
        } else if (c + 1 < NCH) {  // helper h: groups LG + h HG .. of the leader's prologue
            const int h = (tid >> 5) / 4 - 1;
            int sf, sg;
            prologue_part<JG::HG>(A, lowfg[cur][0], lowfg[cur][1], 32 + lane + m,
                                  8 * (JG::LG + h * JG::HG), sf, sg);
            pro[h][0][lane] = sf;
            pro[h][1][lane] = sg;
            asm volatile("bar.arrive 2, %0;" ::"n"(32 * (1 + JG::NH)) : "memory");
            // then, once the leader has the next matrix, its pair tables
            asm volatile("bar.sync 3, %0;" ::"n"(32 * (1 + JG::NH)) : "memory");
            build_pair_tables<JG::PTX, JG::PT0>(mat[(c + 1) & 1], pt[(c + 1) & 1], 32 * h + lane,
                                                32 * JG::NH);
        }
        __syncthreads();
        cur ^= 1;
    }
    const bool ok = s_ok != 0;
    const int f0 = freeze_lazy<Q>(lowfg[cur][0][32]);
    const int sc = ok ? inv_mod<Q>(f0) : 0;
    int16_t *o = out + (size_t)row * out_stride;
    for (int i = tid; i < P; i += NT) {
        const int v = freeze_lazy<Q>(half_value(st[cur][2][spos(OFF + P - 1 - i)]));
        o[i] = (int16_t)cmod<Q>(sc * v);
    }
    if (tid == 0) {
        if (okv) okv[e] = ok ? 1 : 0;
        if (!ok && err) atomicOr(err, err_bit);
    }
}

template <int P>
cudaError_t launch_rq_inv_jump(int n, const int16_t *in, long in_stride, int16_t *out,
                               long out_stride, int32_t *ok, int *err, int err_bit,
                               cudaStream_t st, const int *idx) {
    SNT_LAUNCH(k_rq_inv_jump<P>, n, JumpGeo<P>::NT, 0, st, n, in, in_stride, out, out_stride, ok,
        err, err_bit, idx);
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_r3_inv_jump(int n, const int16_t *in, long in_stride, int16_t *out,
                               long out_stride, int32_t *ok, int *err, int err_bit,
                               cudaStream_t st, const int *idx) {
    SNT_LAUNCH(k_rq_inv_jump<P, 3>, n, JumpGeo<P, 3>::NT, 0, st, n, in, in_stride, out, out_stride,
        ok, err, err_bit, idx);
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_rq_inv(int n, const int16_t *in, long in_stride, int16_t *out,
                          long out_stride, int32_t *ok, int *err, int err_bit, cudaStream_t st) {
    constexpr int NT = inv_threads<P>();
    SNT_LAUNCH(k_rq_inv<P, NT, int16_t>, n, NT, 0, st, n, in, in_stride, out, out_stride, ok, err,
        err_bit);
    return cudaGetLastError();
}

#define SNT_INV_INST(P)                                                                    \
    template cudaError_t launch_rq_inv<P>(int, const int16_t *, long, int16_t *, long,     \
                                          int32_t *, int *, int, cudaStream_t);            \
    template cudaError_t launch_rq_inv_jump<P>(int, const int16_t *, long, int16_t *, long, \
                                               int32_t *, int *, int, cudaStream_t, const int *); \
    template cudaError_t launch_r3_inv_jump<P>(int, const int16_t *, long, int16_t *, long, \
                                               int32_t *, int *, int, cudaStream_t, const int *);
SNT_INV_INST(653)
SNT_INV_INST(761)
SNT_INV_INST(857)

}  // namespace snt
