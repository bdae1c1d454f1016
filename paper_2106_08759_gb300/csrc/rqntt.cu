// rqntt.cu -- R/q products on the CUDA cores by the paper's own multiplier
// (Sec. 3.3): Schoenhage's trick manufactures the roots of unity, so the
// transforms need no multiplications in Z/q.
//
// A product of two elements of R/q = (Z/q)[x]/(x^p - x - 1) (degree < p) is
// first formed in (Z/q)[x] (degree < 2p - 1) and then folded by x^p = x + 1.
// The (Z/q)[x] product: cut each operand into NCH chunks of 32 coefficients,
// a = sum_j a_j(x) y^j with y = x^32, and view every chunk as an element of
// K = (Z/q)[x]/(x^64 + 1) (a chunk product has degree < 63, so nothing wraps
// in K).  The product in K[y] has degree < 2 NCH - 1 <= 32 + M, so it is
// recovered from its residues modulo y^32 + 1 and y^M - 1 (M = 16 for p <= 768,
// the paper's truncation to 48 points; M = 32 for sntrup857).  x is a 128th
// root of unity in K: y^32 + 1 = y^32 - x^64 splits by y^2m - c^2 =
// (y^m - c)(y^m + c) into 32 linear factors y - x^(2 odd), y^M - 1 into M
// factors y - x^(128 k / M); each split is a butterfly (u, v) -> (u + x^t v,
// u - x^t v), and multiplying by x^t in K is a negacyclic shift of the 64
// coefficients.  Then 32 + M pointwise products in K (64 x 64 negacyclic
// schoolbook on the IMAD pipe, int32 sums below 2^31), the inverse butterflies
// (Gentleman-Sande, x^-t = x^(128 - t)), the scalings 1/32 and 1/M, and the
// Chinese remainder step c = r1 + (y^32 + 1) s with s = (r2 - r1 mod (y^M - 1)) / 2.
// The paper multiplies in K by Nussbaumer's trick and Karatsuba; here the K
// products are register-tiled schoolbook sums (eight outputs per thread).
//
// One CTA computes NOUT products S * X_k that share the operand S (NOUT = 2:
// the down-sweep's T * y and T * x, with S's transform done once), with
// 2 + 2 NOUT warps:
//   1. transforms: one warp per (operand, part) holds coefficient L and L + 32
//      of every point in lane L (registers); the shifts x^t are shuffles
//      (t = 0, 32, 64, 96: in-lane), then residues mod q go to shared memory;
//   2. pointwise: 8 lanes per point, 8 outputs per lane, over all warps;
//   3. inverse transforms per (output, part), scaled;
//   4. per output, the warp of the negacyclic part combines the two parts,
//      overlaps the chunks and folds x^p = x + 1.
// Value bounds: inputs |x| <= (q-1)/2 < 2600; after 5 butterfly levels (and
// the cyclic fold of two chunks) |x| < 2^17; residues are re-centred before
// the pointwise sums (64 * 2583^2 < 2^29) and after them.
#include <atomic>

#include "common.cuh"
#include "kernels.h"
#include "pdl.cuh"

namespace snt {

template <int P> struct NttGeo {
    static constexpr int p = Geo<P>::p, q = Geo<P>::q;
    static constexpr int NCH = (p + 31) / 32;                  // 32-coefficient chunks
    static constexpr int M = (2 * NCH - 1 <= 48) ? 16 : 32;    // cyclic part
    static constexpr int NPT = 32 + M;                         // points
    static constexpr int SSTR = 65;                            // words per S point
    static constexpr int XSTR = 129;                           // words per extended X point
    static constexpr int DLEN = 32 * (NPT + 1);                // (Z/q)[x] product buffer
    static constexpr int inv2 = (q + 1) / 2;
    static_assert(2 * NCH - 1 <= NPT, "truncated transform too short");
    static_assert(NPT * SSTR >= 2 * M * 64, "cyclic results must fit the S area");
    static_assert(NPT * XSTR >= DLEN, "product buffer must fit an X area");
};

// a^-1 mod Q for small a (Fermat), at compile time.
template <int Q> __host__ __device__ constexpr int cinv(int a) {
    long long r = 1, b = a % Q;
    for (int e = Q - 2; e > 0; e >>= 1) {
        if (e & 1) r = r * b % Q;
        b = b * b % Q;
    }
    return (int)r;
}

// (x^T v) in K for the coefficient pair (lane, lane + 32) held by each lane;
// T a compile-time constant in [0, 128).  Coefficient i of x^t v is v[i - t]
// if i >= t, else -v[i - t + 64] (x^64 = -1).
template <int T>
__device__ __forceinline__ void kmulx(int &o0, int &o1, int r0, int r1, int lane) {
    constexpr int tt = T & 63;
    constexpr bool neg = T >= 64;
    int a, b;
    if constexpr (tt == 0) {
        a = r0; b = r1;
    } else if constexpr (tt == 32) {
        a = -r1; b = r0;
    } else {
        const int d = lane - tt;  // in [-63, 31]
        const int src = d & 31;
        const int lo = __shfl_sync(0xffffffffu, r0, src);
        const int hi = __shfl_sync(0xffffffffu, r1, src);
        // coefficient lane:      d >= 0: lo;  -32 <= d < 0: -hi;  d < -32: -lo
        // coefficient lane + 32: d >= 0: hi;  -32 <= d < 0:  lo;  d < -32: -hi
        a = d >= 0 ? lo : (d >= -32 ? -hi : -lo);
        b = d >= 0 ? hi : (d >= -32 ? lo : -hi);
    }
    o0 = neg ? -a : a;
    o1 = neg ? -b : b;
}

// Forward butterflies of the node v[S .. S + W) taken modulo y^W - x^E
// (Cooley-Tukey, children first split, then recursed).
template <int N, int S, int W, int E> struct NttFwd {
    static __device__ __forceinline__ void run(int (&v0)[N], int (&v1)[N], int lane) {
        if constexpr (W > 1) {
            constexpr int H = W / 2, T = E / 2;
#pragma unroll
            for (int j = 0; j < H; ++j) {
                int w0, w1;
                kmulx<T>(w0, w1, v0[S + j + H], v1[S + j + H], lane);
                const int u0 = v0[S + j], u1 = v1[S + j];
                v0[S + j] = u0 + w0;
                v1[S + j] = u1 + w1;
                v0[S + j + H] = u0 - w0;
                v1[S + j + H] = u1 - w1;
            }
            NttFwd<N, S, H, T>::run(v0, v1, lane);
            NttFwd<N, S + H, H, (T + 64) % 128>::run(v0, v1, lane);
        }
    }
};

// Inverse of NttFwd up to the factor W (Gentleman-Sande).
template <int N, int S, int W, int E> struct NttInv {
    static __device__ __forceinline__ void run(int (&v0)[N], int (&v1)[N], int lane) {
        if constexpr (W > 1) {
            constexpr int H = W / 2, T = E / 2;
            NttInv<N, S, H, T>::run(v0, v1, lane);
            NttInv<N, S + H, H, (T + 64) % 128>::run(v0, v1, lane);
#pragma unroll
            for (int j = 0; j < H; ++j) {
                const int g0 = v0[S + j], g1 = v1[S + j];
                const int h0 = v0[S + j + H], h1 = v1[S + j + H];
                v0[S + j] = g0 + h0;
                v1[S + j] = g1 + h1;
                kmulx<(128 - T) % 128>(v0[S + j + H], v1[S + j + H], g0 - h0, g1 - h1, lane);
            }
        }
    }
};

// Shared memory of one CTA: S points (plain, 65-word rows) and, per output,
// the X points in extended negacyclic form (row [j] = -X[j] for j < 64,
// X[j - 64] above), later the pointwise results, then the product buffer.
template <int P, int NOUT> struct NttSmem {
    using G = NttGeo<P>;
    int s[G::NPT * G::SSTR];
    int x[NOUT][G::NPT * G::XSTR];
};

// Forward transform of one part of an operand row (in: p coefficients),
// residues to shared memory.  part 0: the 32 chunks modulo y^32 + 1; part 1:
// the chunks folded modulo y^M - 1.  ext: write the extended form.
template <int P, int PART>
__device__ __forceinline__ void ntt_forward(const int16_t *__restrict__ in, int *dst, int stride,
                                            bool ext, int lane) {
    using G = NttGeo<P>;
    constexpr int N = PART == 0 ? 32 : G::M;
    int v0[N], v1[N];
#pragma unroll
    for (int j = 0; j < N; ++j) { v0[j] = 0; v1[j] = 0; }
#pragma unroll
    for (int c = 0; c < G::NCH; ++c) {
        const int i = 32 * c + lane;
        const int a = i < G::p ? (int)in[i] : 0;
        if (PART == 0) v0[c] = a;
        else v0[c % N] += a;
    }
    if (PART == 0) NttFwd<N, 0, N, 64>::run(v0, v1, lane);
    else NttFwd<N, 0, N, 0>::run(v0, v1, lane);
    const int base = PART == 0 ? 0 : 32;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const int a = cmod<G::q>(v0[j]), b = cmod<G::q>(v1[j]);
        int *row = dst + (base + j) * stride;
        if (ext) {
            row[lane] = -a; row[lane + 32] = -b;
            row[64 + lane] = a; row[96 + lane] = b;
        } else {
            row[lane] = a; row[lane + 32] = b;
        }
    }
}

// Pointwise products of points pt0 .. pt0 + 3 (8 lanes each): 64 x 64
// negacyclic schoolbook, outputs 8r .. 8r + 7 per lane, written (centred)
// over the X point rows.
template <int P>
__device__ __forceinline__ void ntt_pointwise(const int *__restrict__ s, int *x, int pt0,
                                              int lane) {
    using G = NttGeo<P>;
    const int pt = pt0 + (lane >> 3), r = lane & 7;
    const int *sp = s + pt * G::SSTR;
    int *xp = x + pt * G::XSTR;
    const int *xw = xp + 64 + 8 * r;  // Xext[8r + m] at xw[m]
    int acc[8], w[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) { acc[j] = 0; w[j] = xw[j]; }
#pragma unroll
    for (int i = 0; i < 64; ++i) {
        const int si = sp[i];
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j] += si * w[j];
        if (i < 63) {
#pragma unroll
            for (int j = 7; j > 0; --j) w[j] = w[j - 1];
            w[0] = xw[-i - 1];  // Xext[8r - i - 1]
        }
    }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 8; ++j) xp[8 * r + j] = cmod<G::q>(acc[j]);
}

// Inverse transform of one part of output k's pointwise results (rows at
// x, stride XSTR), scaled by 1/W and centred, into (v0, v1).
template <int P, int PART, int N>
__device__ __forceinline__ void ntt_inverse(const int *x, int (&v0)[N], int (&v1)[N], int lane) {
    using G = NttGeo<P>;
    const int base = PART == 0 ? 0 : 32;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        v0[j] = x[(base + j) * G::XSTR + lane];
        v1[j] = x[(base + j) * G::XSTR + lane + 32];
    }
    if (PART == 0) NttInv<N, 0, N, 64>::run(v0, v1, lane);
    else NttInv<N, 0, N, 0>::run(v0, v1, lane);
    constexpr int sc = cinv<G::q>(N);
#pragma unroll
    for (int j = 0; j < N; ++j) {
        v0[j] = cmod<G::q>(cmod<G::q>(v0[j]) * sc);
        v1[j] = cmod<G::q>(cmod<G::q>(v1[j]) * sc);
    }
}

// The CTA's work: out[k] = S * X[k] in R/q for k < NOUT.  Rows hold p
// coefficients (|x| <= (q-1)/2); outputs are centred, written over
// out_len coefficients (zeros from p on).  Every warp of the CTA calls it.
template <int P, int NOUT>
__device__ __forceinline__ void ntt_products(NttSmem<P, NOUT> &sm, const int16_t *S,
                                             const int16_t *const (&X)[NOUT],
                                             int16_t *const (&out)[NOUT], int out_len) {
    using G = NttGeo<P>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = 2 + 2 * NOUT;
    // 1. forward transforms
    if (warp == 0) ntt_forward<P, 0>(S, sm.s, G::SSTR, false, lane);
    else if (warp == 1) ntt_forward<P, 1>(S, sm.s, G::SSTR, false, lane);
    else {
        const int k = (warp - 2) >> 1;
        if ((warp & 1) == 0) ntt_forward<P, 0>(X[k], sm.x[k], G::XSTR, true, lane);
        else ntt_forward<P, 1>(X[k], sm.x[k], G::XSTR, true, lane);
    }
    __syncthreads();
    // 2. pointwise products, four points per warp pass
    constexpr int PASSES = NOUT * G::NPT / 4;
    for (int ps = warp; ps < PASSES; ps += NW) {
        const int k = (4 * ps) / G::NPT, pt0 = (4 * ps) % G::NPT;
        ntt_pointwise<P>(sm.s, sm.x[k], pt0, lane);
    }
    __syncthreads();
    // 3. inverse transforms: the cyclic parts to the S area, the negacyclic
    // parts stay in the registers of the warp that finishes the output
    int r0[32], r1[32];
    if (warp < 2 * NOUT) {
        const int k = warp >> 1;
        if (warp & 1) {
            int c0[G::M], c1[G::M];
            ntt_inverse<P, 1, G::M>(sm.x[k], c0, c1, lane);
            int *r2 = sm.s + k * G::M * 64;
#pragma unroll
            for (int j = 0; j < G::M; ++j) { r2[64 * j + lane] = c0[j]; r2[64 * j + 32 + lane] = c1[j]; }
        } else {
            ntt_inverse<P, 0, 32>(sm.x[k], r0, r1, lane);
        }
    }
    __syncthreads();
    // 4. combine the parts, overlap the chunks, fold by x^p = x + 1
    if (warp < 2 * NOUT && (warp & 1) == 0) {
        const int k = warp >> 1;
        const int *r2 = sm.s + k * G::M * 64;
        int *d = sm.x[k];
        // s_j = (r2_j - (r1 mod y^M - 1)_j) / 2; c_j = r1_j + s_j (j < M),
        // r1_j (M <= j < 32), s_(j-32) (32 <= j < 32 + M)
        int s0[G::M], s1[G::M];
#pragma unroll
        for (int j = 0; j < G::M; ++j) {
            int f0 = r0[j], f1 = r1[j];
#pragma unroll
            for (int jj = j + G::M; jj < 32; jj += G::M) { f0 += r0[jj]; f1 += r1[jj]; }
            s0[j] = cmod<G::q>((r2[64 * j + lane] - f0) * G::inv2);
            s1[j] = cmod<G::q>((r2[64 * j + 32 + lane] - f1) * G::inv2);
        }
        // d[32 j + lane] = c_j[lane] + c_(j-1)[lane + 32], j = 0 .. NPT
        int prev1 = 0;
#pragma unroll
        for (int j = 0; j <= G::NPT; ++j) {
            int c0 = 0, c1 = 0;
            if (j < 32) { c0 = r0[j]; c1 = r1[j]; }
            if (j < G::M) { c0 += s0[j]; c1 += s1[j]; }
            if (j >= 32 && j < G::NPT) { c0 = s0[j - 32]; c1 = s1[j - 32]; }
            d[32 * j + lane] = c0 + prev1;
            prev1 = c1;
        }
        __syncwarp();
        int16_t *o = out[k];
        for (int i = lane; i < out_len; i += 32) {
            int v = 0;
            if (i < G::p) {
                v = d[i];
                if (i <= G::p - 2) v += d[i + G::p];
                if (i >= 1) v += d[i + G::p - 1];
                v = cmod<G::q>(v);
            }
            o[i] = (int16_t)v;
        }
    }
}

template <int P, int NOUT>
constexpr int ntt_threads() { return 32 * (2 + 2 * NOUT); }

// c_i = a_i * b_i (rows of p coefficients, stride p).
template <int P>
__global__ void __launch_bounds__(ntt_threads<P, 1>())
k_mul_batch_ntt(const int16_t *__restrict__ a, const int16_t *__restrict__ b,
                int16_t *__restrict__ c) {
    extern __shared__ __align__(16) int ntt_dyn[];
    auto &sm = *reinterpret_cast<NttSmem<P, 1> *>(ntt_dyn);
    const size_t i = blockIdx.x;
    const int16_t *X[1] = {b + i * P};
    int16_t *const O[1] = {c + i * P};
    ntt_products<P, 1>(sm, a + i * P, X, O, P);
}

// Up-sweep level: node j = left * right of its two children (an unpaired
// child moves up unchanged).
template <int P>
__global__ void __launch_bounds__(ntt_threads<P, 1>())
k_tree_up_ntt(const int16_t *__restrict__ lin, LevelMap lm, int16_t *__restrict__ lout) {
    pdl_enter();
    using G = Geo<P>;
    extern __shared__ __align__(16) int ntt_dyn[];
    auto &sm = *reinterpret_cast<NttSmem<P, 1> *>(ntt_dyn);
    const int j = blockIdx.x;
    int idx, base, n_in;
    lm_node(lm, j, idx, base, n_in);
    const int16_t *a = lin + (size_t)(base + 2 * idx) * G::pad;
    int16_t *c = lout + (size_t)j * G::pad;
    if (2 * idx + 1 >= n_in) {
        for (int i = threadIdx.x; i < G::pad; i += blockDim.x) c[i] = a[i];
        return;
    }
    const int16_t *X[1] = {a + G::pad};
    int16_t *const O[1] = {c};
    ntt_products<P, 1>(sm, a, X, O, G::pad);
}

// Down-sweep level: with T = 1/parent, 1/x = T * y and 1/y = T * x over the
// two children in place (both are read into the transforms before the first
// output is written: the writes follow two CTA barriers).
template <int P>
__global__ void __launch_bounds__(ntt_threads<P, 2>())
k_tree_down_ntt(const int16_t *__restrict__ lpar, LevelMap lm, int16_t *__restrict__ lch) {
    pdl_enter();
    using G = Geo<P>;
    extern __shared__ __align__(16) int ntt_dyn[];
    auto &sm = *reinterpret_cast<NttSmem<P, 2> *>(ntt_dyn);
    const int j = blockIdx.x;
    int idx, base, n_ch;
    lm_node(lm, j, idx, base, n_ch);
    const int16_t *T = lpar + (size_t)j * G::pad;
    int16_t *x = lch + (size_t)(base + 2 * idx) * G::pad;
    if (2 * idx + 1 >= n_ch) {
        for (int i = threadIdx.x; i < G::pad; i += blockDim.x) x[i] = T[i];
        return;
    }
    int16_t *y = x + G::pad;
    const int16_t *X[2] = {y, x};
    int16_t *const O[2] = {x, y};
    ntt_products<P, 2>(sm, T, X, O, G::pad);
}

// The shared-memory opt-in above 48 KB, once per kernel and device (host
// state, not stream work).
template <int P, int NOUT, typename K>
static cudaError_t ntt_prepare(K kernel) {
    const int bytes = (int)sizeof(NttSmem<P, NOUT>);
    if (bytes <= 48 * 1024) return cudaSuccess;
    static std::atomic<uint64_t> opted{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = 1ull << (dev & 63);
    if (opted.load() & bit) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) opted.fetch_or(bit);
    return e;
}

template <int P>
cudaError_t launch_mul_batch_ntt(int n, const int16_t *a, const int16_t *b, int16_t *c,
                                 cudaStream_t st) {
    cudaError_t e = ntt_prepare<P, 1>(k_mul_batch_ntt<P>);
    if (e != cudaSuccess) return e;
    k_mul_batch_ntt<P><<<n, ntt_threads<P, 1>(), sizeof(NttSmem<P, 1>), st>>>(a, b, c);
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_tree_up_ntt(const int16_t *lin, const LevelMap &lm, int n_out, int16_t *lout,
                               cudaStream_t st) {
    cudaError_t e = ntt_prepare<P, 1>(k_tree_up_ntt<P>);
    if (e != cudaSuccess) return e;
    SNT_LAUNCH(k_tree_up_ntt<P>, n_out, ntt_threads<P, 1>(), sizeof(NttSmem<P, 1>), st, lin, lm,
        lout);
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_tree_down_ntt(const int16_t *lpar, const LevelMap &lm, int n_par, int16_t *lch,
                                 cudaStream_t st) {
    cudaError_t e = ntt_prepare<P, 2>(k_tree_down_ntt<P>);
    if (e != cudaSuccess) return e;
    SNT_LAUNCH(k_tree_down_ntt<P>, n_par, ntt_threads<P, 2>(), sizeof(NttSmem<P, 2>), st, lpar, lm,
        lch);
    return cudaGetLastError();
}

#define SNT_NTT_INST(P)                                                                        \
    template cudaError_t launch_mul_batch_ntt<P>(int, const int16_t *, const int16_t *,         \
                                                 int16_t *, cudaStream_t);                      \
    template cudaError_t launch_tree_up_ntt<P>(const int16_t *, const LevelMap &, int,          \
                                               int16_t *, cudaStream_t);                        \
    template cudaError_t launch_tree_down_ntt<P>(const int16_t *, const LevelMap &, int,        \
                                                 int16_t *, cudaStream_t);
SNT_NTT_INST(653)
SNT_NTT_INST(761)
SNT_NTT_INST(857)

}  // namespace snt
