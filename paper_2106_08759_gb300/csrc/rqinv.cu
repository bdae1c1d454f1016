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
// apply chunk c, the leader computes the 32 low coefficients of F', G' itself
// and runs the divsteps of chunk c + 1, so a chunk costs about the larger of
// the two.  One barrier per chunk, ceil((2p-1)/31) chunks.
//
// Live extents.  A chunk's matrix entries have degree at most m, so F', G'
// are zero wherever F and G are (index i of F' reads F at i + m - k, k <= m),
// and V', R' reach at most m + 1 past V and R.  The block keeps the extent
// of each state (one past the highest nonzero coefficient of F or G, and of
// V or R, found by the appliers as they write) and computes only the live
// outputs, zeroing what the older state left above them in the target
// buffer.  F, G shrink while V, R grow, their extents summing to about
// p + 2, so a chunk applies the matrix to about p + 34 coefficients rather
// than to four full-length polynomials.  The live outputs are cut into
// items of NOUT consecutive coefficients of one pair ((F', G') or (V', R')),
// one item per applier thread in one code path for both pairs, so that a
// warp holding items of both pairs does not diverge.  Applier warps avoid
// the warp ids that share the leader's scheduler (warp w issues on
// scheduler w % 4), so the leader's serial chain keeps a scheduler to itself.
//
// Ranges: inside the leader's steps values are lazily reduced to [-q, 2q)
// (G(0) = 0 mod q iff G(0) is -q, 0 or q); the matrix and the state are
// centred between chunks, so a 64-term application sum stays below 2^31.
// ---------------------------------------------------------------------------
template <int P> struct JumpGeo {
    static constexpr int M = 31;                        // steps per chunk
    static constexpr int OFF = 32;                      // zero margin below index 0
    static constexpr int NWA = 6;                       // applier warps (ids 1-3, 5-7)
    static constexpr int NA = 32 * NWA;                 // applier threads
    // outputs per item: the fewest that keep the items of the widest chunk
    // (about p + 34 outputs, plus rounding of both pairs) within NA
    static constexpr int NOUT = (P + 34 + 3) / 4 + 2 <= NA ? 4 : 5;
    static constexpr int NW = 8;                        // leader, 6 appliers, 1 idle
    static constexpr int NT = 32 * NW;
    static constexpr int LEN = OFF + P + 1 + NOUT + 40; // slots per polynomial
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
__device__ __forceinline__ void leader_chunk(int m, int &delta, int fl, int gl, int &u, int &v,
                                             int &w, int &z) {
    const int lane = threadIdx.x & 31, from = (lane + 31) & 31;
    u = (lane == 0); v = 0; w = 0; z = (lane == 0);
    int f0 = __shfl_sync(0xffffffffu, fl, 0);
    int g0 = __shfl_sync(0xffffffffu, gl, 0);
    for (int s = 0; s < m; ++s) {
        // the chain: new G, then its shift and its coefficient 0 (read
        // straight from lane 1) issued first; the rest of the step runs in
        // the shuffles' shadow
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
    u = cmod<Q>(u); v = cmod<Q>(v); w = cmod<Q>(w); z = cmod<Q>(z);
}

// Eight consecutive matrix coefficients from a 16-byte aligned address.
__device__ __forceinline__ void load8(int (&c)[8], const int *p) {
    const int4 a = reinterpret_cast<const int4 *>(p)[0], b = reinterpret_cast<const int4 *>(p)[1];
    c[0] = a.x; c[1] = a.y; c[2] = a.z; c[3] = a.w;
    c[4] = b.x; c[5] = b.y; c[6] = b.z; c[7] = b.w;
}

// Lane k's coefficients of the chunk matrix into the six rows: coefficient k
// of u, v, w, z at 4 + k, v_k at 4 + (k - 1) of the v_{k+1} row and w_k at
// 4 + (k + 1) of the w_{k-1} row. The slots those rows leave unwritten (v_32
// and w_{-1}) stay zero from the block's start.
__device__ __forceinline__ void put_matrix(int (*An)[40], int lane, int u, int v, int w, int z) {
    An[0][4 + lane] = u; An[1][4 + lane] = v;
    An[2][4 + lane] = w; An[3][4 + lane] = z;
    An[4][3 + lane] = v; An[5][5 + lane] = w;
}

// Q: the coefficient modulus (q: R/q; 3: R/3, for the root inversions of
// the R/3 batch inversion).
template <int P, int Q = Geo<P>::q>
__global__ void __launch_bounds__(JumpGeo<P>::NT)
k_rq_inv_jump(int n, const int16_t *in, long in_stride, int16_t *out, long out_stride,
              int32_t *__restrict__ okv, int *__restrict__ err, int err_bit, const int *idx) {
    using JG = JumpGeo<P>;
    constexpr int LEN = JG::LEN, OFF = JG::OFF, NT = JG::NT, NOUT = JG::NOUT;
    constexpr int NCH = (2 * P - 1 + JG::M - 1) / JG::M;
    __shared__ int st[2][4][LEN];       // [buffer][F, G, V, R][index + OFF]
    // chunk matrix [buffer][row][4 + k]: rows u, v, w, z and the shifted
    // rows v_{k+1}, w_{k-1} used by (V', R'); 16-byte rows for vector loads,
    // zero outside k = 0..31
    __shared__ __align__(16) int mat[2][6][40];
    // extents of the state after chunk c - 1 in ext[c % 4]: [0] F, G and
    // [1] V, R (one past the highest nonzero coefficient)
    __shared__ int ext[4][2];
    __shared__ int s_ok;
    const int e = blockIdx.x;
    if (e >= n) return;
    const int tid = threadIdx.x, lane = tid & 31;
    const bool leader = tid < 32;
    const int row = idx ? idx[e] : e;
    const int16_t *a = in + (size_t)row * in_stride;
    for (int i = tid; i < 2 * 4 * LEN; i += NT) (&st[0][0][0])[i] = 0;
    for (int i = tid; i < 2 * 6 * 40; i += NT) (&mat[0][0][0])[i] = 0;
    if (tid < 8) (&ext[0][0])[tid] = 0;
    __syncthreads();
    for (int i = tid; i < P; i += NT) st[0][1][OFF + i] = (int)a[P - 1 - i];
    if (tid == 0) {
        st[0][0][OFF] = 1;
        st[0][0][OFF + P - 1] = -1;
        st[0][0][OFF + P] = -1;
        st[0][3][OFF] = 1;
        ext[0][0] = P + 1;
        ext[0][1] = 1;
    }
    __syncthreads();
    int delta = 1;  // leader only
    if (leader) {
        int u, v, w, z;
        leader_chunk<Q>(min(JG::M, 2 * P - 1), delta, st[0][0][OFF + lane], st[0][1][OFF + lane],
                        u, v, w, z);
        put_matrix(mat[0], lane, u, v, w, z);
    }
    __syncthreads();
    int cur = 0;
    for (int c = 0; c < NCH; ++c) {
        const int m = min(JG::M, 2 * P - 1 - c * JG::M);
        const int(*A)[40] = mat[c & 1];
        if (leader) {
            if (c + 1 < NCH) {
                // low 32 coefficients of F', G' (lane i), then chunk c + 1
                const int *F = st[cur][0], *G = st[cur][1];
                int af[2] = {0, 0}, ag[2] = {0, 0};
                const int hi = OFF + lane + m;
#pragma unroll
                for (int kb = 0; kb < 32; kb += 8) {
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
                const int m1 = min(JG::M, 2 * P - 1 - (c + 1) * JG::M);
                int u, v, w, z;
                leader_chunk<Q>(m1, delta, cmod<Q>(af[0] + af[1]), cmod<Q>(ag[0] + ag[1]), u, v, w,
                                z);
                put_matrix(mat[(c + 1) & 1], lane, u, v, w, z);
            } else if (lane == 0) {
                s_ok = (delta == 0);
            }
        } else if ((tid >> 5) & 3) {
            const int w = tid >> 5, ai = w - 1 - (w - 1) / 4;
            const int at = 32 * ai + lane;
            // live ranges of the outputs and what the target buffer held
            const int rfg = ext[c & 3][0], rvr = min(ext[c & 3][1] + m + 1, P + 1);
            const int ofg = ext[(c + 3) & 3][0], ovr = ext[(c + 3) & 3][1];
            int *T = &st[cur ^ 1][0][0];
            for (int i = rfg + at; i < ofg; i += JG::NA) { T[OFF + i] = 0; T[LEN + OFF + i] = 0; }
            for (int i = rvr + at; i < ovr; i += JG::NA) {
                T[2 * LEN + OFF + i] = 0; T[3 * LEN + OFF + i] = 0;
            }
            if (at == 0) { ext[(c + 2) & 3][0] = 0; ext[(c + 2) & 3][1] = 0; }
            const int nfg = (rfg + NOUT - 1) / NOUT, nit = nfg + (rvr + NOUT - 1) / NOUT;
            int top_fg = 0, top_vr = 0;
            for (int it = at; it < nit; it += JG::NA) {
                // pair 0: F' = (u F + v G) / x^m, G' = (w F + z G) / x^m, inputs at i + m - k
                // pair 1: V' = u V + (v/x) R, R' = (x w) V + z R, inputs at i - k
                const int pr = it >= nfg;
                const int i0 = NOUT * (pr ? it - nfg : it), r = pr ? rvr : rfg;
                const int *X = st[cur][2 * pr], *Y = st[cur][2 * pr + 1];
                const int *a0 = &A[0][4], *a1 = &A[pr ? 4 : 1][4], *a2 = &A[pr ? 5 : 2][4],
                          *a3 = &A[3][4];
                const int b = OFF + i0 + (pr ? 0 : m);
                int o1[NOUT], o2[NOUT], xh[NOUT], yh[NOUT];
#pragma unroll
                for (int t = 0; t < NOUT; ++t) {
                    o1[t] = 0; o2[t] = 0;
                    xh[t] = X[b + t]; yh[t] = Y[b + t];
                }
#pragma unroll 1
                for (int kb = 0; kb < 32; kb += 8) {
                    int xl[8], yl[8], c0[8], c1[8], c2[8], c3[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) { xl[j] = X[b - kb - 8 + j]; yl[j] = Y[b - kb - 8 + j]; }
                    load8(c0, a0 + kb); load8(c1, a1 + kb); load8(c2, a2 + kb); load8(c3, a3 + kb);
#pragma unroll
                    for (int kk = 0; kk < 8; ++kk)
#pragma unroll
                        for (int t = 0; t < NOUT; ++t) {
                            const int d = t - kk;
                            const int xv = d >= 0 ? xh[d] : xl[8 + d];
                            const int yv = d >= 0 ? yh[d] : yl[8 + d];
                            o1[t] += c0[kk] * xv + c1[kk] * yv;
                            o2[t] += c2[kk] * xv + c3[kk] * yv;
                        }
#pragma unroll
                    for (int t = 0; t < NOUT; ++t) { xh[t] = xl[t]; yh[t] = yl[t]; }
                }
                int *X2 = st[cur ^ 1][2 * pr], *Y2 = st[cur ^ 1][2 * pr + 1];
                int top = 0;
#pragma unroll
                for (int t = 0; t < NOUT; ++t)
                    if (i0 + t < r) {
                        const int v1 = cmod<Q>(o1[t]), v2 = cmod<Q>(o2[t]);
                        X2[OFF + i0 + t] = v1;
                        Y2[OFF + i0 + t] = v2;
                        if (v1 | v2) top = i0 + t + 1;
                    }
                if (pr) top_vr = max(top_vr, top); else top_fg = max(top_fg, top);
            }
            top_fg = __reduce_max_sync(0xffffffffu, top_fg);
            top_vr = __reduce_max_sync(0xffffffffu, top_vr);
            if (lane == 0) {
                atomicMax(&ext[(c + 1) & 3][0], top_fg);
                atomicMax(&ext[(c + 1) & 3][1], top_vr);
            }
        }
        __syncthreads();
        cur ^= 1;
    }
    const bool ok = s_ok != 0;
    const int f0 = freeze_lazy<Q>(st[cur][0][OFF]);
    const int sc = ok ? inv_mod<Q>(f0) : 0;
    int16_t *o = out + (size_t)row * out_stride;
    for (int i = tid; i < P; i += NT) {
        const int v = freeze_lazy<Q>(st[cur][2][OFF + P - 1 - i]);
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
    k_rq_inv_jump<P><<<n, JumpGeo<P>::NT, 0, st>>>(n, in, in_stride, out, out_stride, ok, err,
                                                   err_bit, idx);
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_r3_inv_jump(int n, const int16_t *in, long in_stride, int16_t *out,
                               long out_stride, int32_t *ok, int *err, int err_bit,
                               cudaStream_t st) {
    k_rq_inv_jump<P, 3><<<n, JumpGeo<P>::NT, 0, st>>>(n, in, in_stride, out, out_stride, ok, err,
                                                      err_bit, nullptr);
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_rq_inv(int n, const int16_t *in, long in_stride, int16_t *out,
                          long out_stride, int32_t *ok, int *err, int err_bit, cudaStream_t st) {
    constexpr int NT = inv_threads<P>();
    k_rq_inv<P, NT, int16_t><<<n, NT, 0, st>>>(n, in, in_stride, out, out_stride, ok, err, err_bit);
    return cudaGetLastError();
}

#define SNT_INV_INST(P)                                                                    \
    template cudaError_t launch_rq_inv<P>(int, const int16_t *, long, int16_t *, long,     \
                                          int32_t *, int *, int, cudaStream_t);            \
    template cudaError_t launch_rq_inv_jump<P>(int, const int16_t *, long, int16_t *, long, \
                                               int32_t *, int *, int, cudaStream_t, const int *); \
    template cudaError_t launch_r3_inv_jump<P>(int, const int16_t *, long, int16_t *, long, \
                                               int32_t *, int *, int, cudaStream_t);
SNT_INV_INST(653)
SNT_INV_INST(761)
SNT_INV_INST(857)

}  // namespace snt
