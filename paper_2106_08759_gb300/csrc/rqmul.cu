// rqmul.cu -- R/q products of the batch-inversion product tree, and a batched
// product for the kernel microbenchmark.
//
// Montgomery's trick (Sec. 2.2) turns n inversions into 3n - 3
// multiplications and one inversion.  The paper runs it as a prefix chain;
// here the same multiplications are arranged as a binary product tree so
// that every level is one parallel launch:
//   up-sweep:   node(l, j) = node(l-1, 2j) * node(l-1, 2j+1)
//               (an unpaired last node moves up unchanged);
//   root:       one inversion (rqinv.cu);
//   down-sweep: with T = 1/node(l, j),
//               1/node(l-1, 2j) = T * node(l-1, 2j+1),
//               1/node(l-1, 2j+1) = T * node(l-1, 2j),
//               written over the two children in place.
// For B leaves that is B - 1 products up and 2(B - 1) down: 3B - 3 in total.
// Every polynomial is int16, centred, stride Geo<P>::pad.
#include "kernels.h"
#include "toeplitz.cuh"
#include "pdl.cuh"

namespace snt {

// Products per CTA are split K ways over the inner index (toeplitz_split):
// narrow tree levels (few products) use K = 8 to cut the latency of each
// product, wide levels K = 1 for throughput.
template <int P, int K>
__global__ void __launch_bounds__(Tp<P>::NT * K)
k_tree_up(const int16_t *__restrict__ lin, LevelMap lm, int16_t *__restrict__ lout) {
    pdl_enter();
    using G = Geo<P>;
    constexpr int NT = Tp<P>::NT;
    __shared__ __align__(16) int As[Tp<P>::p8];
    __shared__ __align__(16) int Es[Tp<P>::ESZ];
    __shared__ int part[K > 1 ? (K - 1) * Tp<P>::p8 : 1];
    const int j = blockIdx.x;
    int idx, base, n_in;  // this node's index in its tree, its children
    lm_node(lm, j, idx, base, n_in);
    const int16_t *a = lin + (size_t)(base + 2 * idx) * G::pad;
    int16_t *c = lout + (size_t)j * G::pad;
    if (2 * idx + 1 >= n_in) {  // unpaired: move up unchanged
        for (int i = threadIdx.x; i < G::pad; i += blockDim.x) c[i] = a[i];
        return;
    }
    const int16_t *b = a + G::pad;
    fill_A<P>(a, As);
    fill_E<P>(b, Es);
    __syncthreads();
    int acc[1][8];
    const int *const A1[1] = {As};
    toeplitz_split<P, 1, K>(A1, Es, part, acc);
    const int tloc = threadIdx.x % NT;
    const bool active = threadIdx.x < NT;
    const int bl[1] = {(int)b[P - 1]};
    toeplitz_finish<P, 1>(A1, bl, acc, tloc, active);
    if (active) store_tile<P>(c, acc[0], G::pad, tloc);
}

template <int P, int K>
__global__ void __launch_bounds__(Tp<P>::NT * K)
k_tree_down(const int16_t *__restrict__ lpar, LevelMap lm, int16_t *__restrict__ lch) {
    pdl_enter();
    using G = Geo<P>;
    constexpr int NT = Tp<P>::NT;
    __shared__ __align__(16) int Xs[Tp<P>::p8];
    __shared__ __align__(16) int Ys[Tp<P>::p8];
    __shared__ __align__(16) int Es[Tp<P>::ESZ];
    __shared__ int part[K > 1 ? (K - 1) * Tp<P>::p8 : 1];
    const int j = blockIdx.x;
    int idx, base, n_ch;
    lm_node(lm, j, idx, base, n_ch);
    const int16_t *T = lpar + (size_t)j * G::pad;
    int16_t *x = lch + (size_t)(base + 2 * idx) * G::pad;
    if (2 * idx + 1 >= n_ch) {  // unpaired child: its inverse is the parent's
        for (int i = threadIdx.x; i < G::pad; i += blockDim.x) x[i] = T[i];
        return;
    }
    int16_t *y = x + G::pad;
    fill_A<P>(x, Xs);
    fill_A<P>(y, Ys);
    fill_E<P>(T, Es);
    __syncthreads();  // both children are in shared memory before either is overwritten
    int acc[2][8];
    const int *const A2[2] = {Ys, Xs};
    toeplitz_split<P, 2, K>(A2, Es, part, acc);
    const int tloc = threadIdx.x % NT;
    const bool active = threadIdx.x < NT;
    const int tl = (int)T[P - 1];
    const int bl[2] = {tl, tl};
    toeplitz_finish<P, 2>(A2, bl, acc, tloc, active);
    if (active) {
        store_tile<P>(x, acc[0], G::pad, tloc);  // 1/x = T * y
        store_tile<P>(y, acc[1], G::pad, tloc);  // 1/y = T * x
    }
}

// Output-split forms of both sweeps for the narrow levels (toeplitz_seg):
// grid (nodes, S).  The down-sweep writes the children's inverses to a
// separate level buffer `lout` (same node indexing as lch), since the other
// segments of the same product still read the children.
template <int P, int S, int K>
__global__ void __launch_bounds__(SegGeo<P, S>::TS * K)
k_tree_up_seg(const int16_t *__restrict__ lin, LevelMap lm, int16_t *__restrict__ lout) {
    pdl_enter();
    using G = Geo<P>;
    __shared__ __align__(16) int As[Tp<P>::p8];
    __shared__ __align__(16) int Es[Tp<P>::ESZ];
    __shared__ int part[K > 1 ? (K - 1) * SegGeo<P, S>::TS * 8 : 1];
    const int j = blockIdx.x, seg = blockIdx.y;
    int idx, base, n_in;
    lm_node(lm, j, idx, base, n_in);
    const int16_t *a = lin + (size_t)(base + 2 * idx) * G::pad;
    int16_t *c = lout + (size_t)j * G::pad;
    if (2 * idx + 1 >= n_in) {  // unpaired: move up unchanged (segment 0 copies)
        if (seg == 0)
            for (int i = threadIdx.x; i < G::pad; i += blockDim.x) c[i] = a[i];
        return;
    }
    const int16_t *b = a + G::pad;
    fill_A<P>(a, As);
    fill_E<P>(b, Es);
    __syncthreads();
    int acc[1][8], tloc;
    bool active;
    const int *const A1[1] = {As};
    const int bl[1] = {(int)b[P - 1]};
    toeplitz_seg<P, 1, S, K>(A1, Es, bl, part, seg, acc, tloc, active);
    if (active) store_tile<P>(c, acc[0], G::pad, tloc);
}

template <int P, int S, int K>
__global__ void __launch_bounds__(SegGeo<P, S>::TS * K)
k_tree_down_seg(const int16_t *__restrict__ lpar, LevelMap lm, const int16_t *__restrict__ lch,
                int16_t *__restrict__ lout) {
    pdl_enter();
    using G = Geo<P>;
    __shared__ __align__(16) int Xs[Tp<P>::p8];
    __shared__ __align__(16) int Ys[Tp<P>::p8];
    __shared__ __align__(16) int Es[Tp<P>::ESZ];
    __shared__ int part[K > 1 ? (K - 1) * SegGeo<P, S>::TS * 8 : 1];
    const int j = blockIdx.x, seg = blockIdx.y;
    int idx, base, n_ch;
    lm_node(lm, j, idx, base, n_ch);
    const int16_t *T = lpar + (size_t)j * G::pad;
    const int16_t *x = lch + (size_t)(base + 2 * idx) * G::pad;
    int16_t *ox = lout + (size_t)(base + 2 * idx) * G::pad;
    if (2 * idx + 1 >= n_ch) {  // unpaired child: its inverse is the parent's
        if (seg == 0)
            for (int i = threadIdx.x; i < G::pad; i += blockDim.x) ox[i] = T[i];
        return;
    }
    const int16_t *y = x + G::pad;
    int16_t *oy = ox + G::pad;
    fill_A<P>(x, Xs);
    fill_A<P>(y, Ys);
    fill_E<P>(T, Es);
    __syncthreads();
    int acc[2][8], tloc;
    bool active;
    const int *const A2[2] = {Ys, Xs};
    const int tl = (int)T[P - 1];
    const int bl[2] = {tl, tl};
    toeplitz_seg<P, 2, S, K>(A2, Es, bl, part, seg, acc, tloc, active);
    if (active) {
        store_tile<P>(ox, acc[0], G::pad, tloc);  // 1/x = T * y
        store_tile<P>(oy, acc[1], G::pad, tloc);  // 1/y = T * x
    }
}

// Output split of a narrow level of n products: (S, K), S = 1 for a level
// wide enough to fill the GPU with one CTA per product.
inline void seg_plan(int n, int &S, int &K) {
    S = 1; K = 1;
    if (n <= 8)       { S = 12; K = 16; }
    else if (n <= 16) { S = 8;  K = 16; }
    else if (n <= 32) { S = 4;  K = 8; }
    else if (n <= kSegMaxNodes) { S = 2; K = 4; }
}

template <int P>
cudaError_t launch_tree_up_seg(const int16_t *lin, const LevelMap &lm, int n_out, int16_t *lout,
                               cudaStream_t st) {
    int S, K;
    seg_plan(n_out, S, K);
#define SNT_UP_SEG(SS, KK)                                                             \
    SNT_LAUNCH(k_tree_up_seg<P, SS, KK>, dim3(n_out, SS), SegGeo<P, SS>::TS * KK, 0, st, \
               lin, lm, lout)
    switch (S) {
        case 12: SNT_UP_SEG(12, 16); break;
        case 8: SNT_UP_SEG(8, 16); break;
        case 4: SNT_UP_SEG(4, 8); break;
        case 2: SNT_UP_SEG(2, 4); break;
        default: return cudaErrorInvalidValue;
    }
#undef SNT_UP_SEG
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_tree_down_seg(const int16_t *lpar, const LevelMap &lm, int n_par,
                                 const int16_t *lch, int16_t *lout, cudaStream_t st) {
    int S, K;
    seg_plan(n_par, S, K);
#define SNT_DOWN_SEG(SS, KK)                                                           \
    SNT_LAUNCH(k_tree_down_seg<P, SS, KK>, dim3(n_par, SS), SegGeo<P, SS>::TS * KK, 0, st, \
               lpar, lm, lch, lout)
    switch (S) {
        case 12: SNT_DOWN_SEG(12, 16); break;
        case 8: SNT_DOWN_SEG(8, 16); break;
        case 4: SNT_DOWN_SEG(4, 8); break;
        case 2: SNT_DOWN_SEG(2, 4); break;
        default: return cudaErrorInvalidValue;
    }
#undef SNT_DOWN_SEG
    return cudaGetLastError();
}

// c_e = a_e * b_e, n products, all operands stride p (microbenchmark layout).
template <int P>
__global__ void __launch_bounds__(Tp<P>::NT)
k_mul_batch(int n, const int16_t *__restrict__ a, const int16_t *__restrict__ b,
            int16_t *__restrict__ c) {
    __shared__ __align__(16) int As[Tp<P>::p8];
    __shared__ __align__(16) int Es[Tp<P>::ESZ];
    const int e = blockIdx.x;
    if (e >= n) return;
    const int16_t *ae = a + (size_t)e * P, *be = b + (size_t)e * P;
    fill_A<P>(ae, As);
    fill_E<P>(be, Es);
    __syncthreads();
    int acc[1][8];
    const int *const A1[1] = {As};
    toeplitz_tile<P, 1>(A1, Es, threadIdx.x, 0, Tp<P>::p8, acc);
    const int bl[1] = {(int)be[P - 1]};
    toeplitz_finish<P, 1>(A1, bl, acc, threadIdx.x, true);
    const int j0 = 8 * threadIdx.x;
#pragma unroll
    for (int t = 0; t < 8; ++t)
        if (j0 + t < P) c[(size_t)e * P + j0 + t] = (int16_t)acc[0][t];
}

// Split factor for a level of n products: enough threads to fill the GPU.
inline int split_for(int n, int max_split) {
    const int k = n <= 48 ? 8 : n <= 160 ? 4 : n <= 400 ? 2 : 1;
    return k < max_split ? k : max_split;
}

template <int P>
cudaError_t launch_tree_up(const int16_t *lin, const LevelMap &lm, int n_out, int16_t *lout,
                           cudaStream_t st, int max_split) {
    constexpr int NT = Tp<P>::NT;
    switch (split_for(n_out, max_split)) {
        case 8: SNT_LAUNCH(k_tree_up<P, 8>, n_out, NT * 8, 0, st, lin, lm, lout); break;
        case 4: SNT_LAUNCH(k_tree_up<P, 4>, n_out, NT * 4, 0, st, lin, lm, lout); break;
        case 2: SNT_LAUNCH(k_tree_up<P, 2>, n_out, NT * 2, 0, st, lin, lm, lout); break;
        default: SNT_LAUNCH(k_tree_up<P, 1>, n_out, NT, 0, st, lin, lm, lout); break;
    }
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_tree_down(const int16_t *lpar, const LevelMap &lm, int n_par, int16_t *lch,
                             cudaStream_t st, int max_split) {
    constexpr int NT = Tp<P>::NT;
    switch (split_for(n_par, max_split)) {
        case 8: SNT_LAUNCH(k_tree_down<P, 8>, n_par, NT * 8, 0, st, lpar, lm, lch); break;
        case 4: SNT_LAUNCH(k_tree_down<P, 4>, n_par, NT * 4, 0, st, lpar, lm, lch); break;
        case 2: SNT_LAUNCH(k_tree_down<P, 2>, n_par, NT * 2, 0, st, lpar, lm, lch); break;
        default: SNT_LAUNCH(k_tree_down<P, 1>, n_par, NT, 0, st, lpar, lm, lch); break;
    }
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_mul_batch(int n, const int16_t *a, const int16_t *b, int16_t *c,
                             cudaStream_t st) {
    k_mul_batch<P><<<n, Tp<P>::NT, 0, st>>>(n, a, b, c);
    return cudaGetLastError();
}

#define SNT_MUL_INST(P)                                                                        \
    template cudaError_t launch_tree_up<P>(const int16_t *, const LevelMap &, int, int16_t *,  \
                                           cudaStream_t, int);                                 \
    template cudaError_t launch_tree_down<P>(const int16_t *, const LevelMap &, int, int16_t *,\
                                             cudaStream_t, int);                               \
    template cudaError_t launch_mul_batch<P>(int, const int16_t *, const int16_t *, int16_t *, \
                                             cudaStream_t);                                    \
    template cudaError_t launch_tree_up_seg<P>(const int16_t *, const LevelMap &, int,         \
                                               int16_t *, cudaStream_t);                       \
    template cudaError_t launch_tree_down_seg<P>(const int16_t *, const LevelMap &, int,       \
                                                 const int16_t *, int16_t *, cudaStream_t);
SNT_MUL_INST(653)
SNT_MUL_INST(761)
SNT_MUL_INST(857)

}  // namespace snt
