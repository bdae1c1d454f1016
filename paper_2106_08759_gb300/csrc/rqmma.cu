// rqmma.cu -- the product tree and the batched product on the tensor cores
// (mma_mul.cuh): same products, same tree, same bytes as rqmul.cu.
//
// Work split.  A product is NTILE MMA tiles of 128 outputs; a CTA computes
// one product (up-sweep, batched product) or one parent's two children
// (down-sweep, sharing the parent's E table) with NW warps of NT tiles each.
// In the down-sweep the children are overwritten in place: every read of
// them happens before the CTA's first barrier and only this CTA touches them.
#include <cuda_fp16.h>

#include "kernels.h"
#include "mma_mul.cuh"

namespace snt {

namespace {

template <typename K> cudaError_t allow_smem(K kern, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Node mapping of a level (single tree or forest), as in rqmul.cu.
__device__ __forceinline__ void node_of(const LevelMap &lm, int j, int &idx, int &base, int &n_in) {
    idx = j; base = 0; n_in = lm.n_in;
    if (lm.nb > 0) {
        const int b = level_batch(lm.pre_out, lm.nb, j);
        idx = j - lm.pre_out[b];
        base = lm.pre_in[b];
        n_in = lm.pre_in[b + 1] - base;
    }
}

}  // namespace

template <int P, int NT, int MODE>
__global__ void __launch_bounds__(32 * MmaGeo<P, NT>::NW)
k_tree_up_mma(const int16_t *__restrict__ lin, LevelMap lm, int16_t *__restrict__ lout) {
    using G = Geo<P>;
    using M = MmaGeo<P, NT>;
    extern __shared__ __align__(16) uint8_t sm[];
    MmaE<P, NT> &E = *reinterpret_cast<MmaE<P, NT> *>(sm);
    MmaA<P, NT> &A = *reinterpret_cast<MmaA<P, NT> *>(sm + sizeof(MmaE<P, NT>));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nth = blockDim.x;
    const int j = blockIdx.x;
    int idx, base, n_in;
    node_of(lm, j, idx, base, n_in);
    const int16_t *a = lin + (size_t)(base + 2 * idx) * G::pad;
    int16_t *c = lout + (size_t)j * G::pad;
    if (2 * idx + 1 >= n_in) {  // unpaired: move up unchanged (uniform over the CTA)
        for (int i = threadIdx.x; i < G::pad; i += nth) c[i] = a[i];
        return;
    }
    mma_fill_a<P, NT, MODE>(a, A, threadIdx.x, nth);
    mma_fill_b<P, NT>(a + G::pad, E, threadIdx.x, nth);
    __syncthreads();
    mma_fill_pe<P, NT, MODE>(E, threadIdx.x, nth);
    __syncthreads();
    float acc[NT][1][3][4];
    const MmaA<P, NT> *const As[1] = {&A};
    mma_tiles<P, NT, 1, MODE>(E, As, warp * NT, lane, acc);
    __syncthreads();
    mma_stage<P, NT, 1, MODE>(A, warp * NT, lane, 0, acc);
    __syncthreads();
    mma_finish<P, NT>(A, (int)E.b[M::p - 1], c, G::pad, threadIdx.x, nth);
}

template <int P, int NT, int MODE>
__global__ void __launch_bounds__(32 * MmaGeo<P, NT>::NW)
k_tree_down_mma(const int16_t *__restrict__ lpar, LevelMap lm, int16_t *__restrict__ lch) {
    using G = Geo<P>;
    using M = MmaGeo<P, NT>;
    extern __shared__ __align__(16) uint8_t sm[];
    MmaE<P, NT> &E = *reinterpret_cast<MmaE<P, NT> *>(sm);
    MmaA<P, NT> *A = reinterpret_cast<MmaA<P, NT> *>(sm + sizeof(MmaE<P, NT>));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nth = blockDim.x;
    const int j = blockIdx.x;
    int idx, base, n_ch;
    node_of(lm, j, idx, base, n_ch);
    const int16_t *T = lpar + (size_t)j * G::pad;
    int16_t *x = lch + (size_t)(base + 2 * idx) * G::pad;
    int16_t *y = x + G::pad;
    if (2 * idx + 1 >= n_ch) {  // unpaired child: its inverse is the parent's
        for (int i = threadIdx.x; i < G::pad; i += nth) x[i] = T[i];
        return;
    }
    mma_fill_a<P, NT, MODE>(y, A[0], threadIdx.x, nth);  // 1/x = T * y
    mma_fill_a<P, NT, MODE>(x, A[1], threadIdx.x, nth);  // 1/y = T * x
    mma_fill_b<P, NT>(T, E, threadIdx.x, nth);
    __syncthreads();  // both children are in shared memory before either is overwritten
    mma_fill_pe<P, NT, MODE_GEN>(E, threadIdx.x, nth);  // T is never small
    __syncthreads();
    float acc[NT][2][3][4];
    const MmaA<P, NT> *const As[2] = {&A[0], &A[1]};
    mma_tiles<P, NT, 2, MODE>(E, As, warp * NT, lane, acc);
    __syncthreads();
    mma_stage<P, NT, 2, MODE>(A[0], warp * NT, lane, 0, acc);
    mma_stage<P, NT, 2, MODE>(A[1], warp * NT, lane, 1, acc);
    __syncthreads();
    const int tl = (int)E.b[M::p - 1];
    mma_finish<P, NT>(A[0], tl, x, G::pad, threadIdx.x, nth);
    mma_finish<P, NT>(A[1], tl, y, G::pad, threadIdx.x, nth);
}

// c_e = a_e * b_e, n products, all operands stride p (microbenchmark layout).
template <int P, int NT>
__global__ void __launch_bounds__(32 * MmaGeo<P, NT>::NW)
k_mul_batch_mma(const int16_t *__restrict__ a, const int16_t *__restrict__ b,
                int16_t *__restrict__ c) {
    using M = MmaGeo<P, NT>;
    extern __shared__ __align__(16) uint8_t sm[];
    MmaE<P, NT> &E = *reinterpret_cast<MmaE<P, NT> *>(sm);
    MmaA<P, NT> &A = *reinterpret_cast<MmaA<P, NT> *>(sm + sizeof(MmaE<P, NT>));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nth = blockDim.x;
    const size_t e = blockIdx.x;
    mma_fill_a<P, NT>(a + e * P, A, threadIdx.x, nth);
    mma_fill_b<P, NT>(b + e * P, E, threadIdx.x, nth);
    __syncthreads();
    mma_fill_pe<P, NT>(E, threadIdx.x, nth);
    __syncthreads();
    float acc[NT][1][3][4];
    const MmaA<P, NT> *const As[1] = {&A};
    mma_tiles<P, NT, 1>(E, As, warp * NT, lane, acc);
    __syncthreads();
    mma_stage<P, NT, 1>(A, warp * NT, lane, 0, acc);
    __syncthreads();
    mma_finish<P, NT>(A, (int)E.b[M::p - 1], c + e * P, P, threadIdx.x, nth);
}

namespace {
template <int P, int NT, int MODE>
cudaError_t up_nt(const int16_t *lin, const LevelMap &lm, int n_out, int16_t *lout, cudaStream_t st) {
    const size_t sm = sizeof(MmaE<P, NT>) + sizeof(MmaA<P, NT>);
    cudaError_t e = allow_smem(k_tree_up_mma<P, NT, MODE>, sm);
    if (e != cudaSuccess) return e;
    k_tree_up_mma<P, NT, MODE><<<n_out, 32 * MmaGeo<P, NT>::NW, sm, st>>>(lin, lm, lout);
    return cudaGetLastError();
}
template <int P, int NT, int MODE>
cudaError_t down_nt(const int16_t *lpar, const LevelMap &lm, int n_par, int16_t *lch, cudaStream_t st) {
    const size_t sm = sizeof(MmaE<P, NT>) + 2 * sizeof(MmaA<P, NT>);
    cudaError_t e = allow_smem(k_tree_down_mma<P, NT, MODE>, sm);
    if (e != cudaSuccess) return e;
    k_tree_down_mma<P, NT, MODE><<<n_par, 32 * MmaGeo<P, NT>::NW, sm, st>>>(lpar, lm, lch);
    return cudaGetLastError();
}
}  // namespace

template <int P>
cudaError_t launch_tree_up_mma(const int16_t *lin, const LevelMap &lm, int n_out, int16_t *lout,
                               cudaStream_t st, int tiles, bool leaves) {
    if (leaves) {  // leaf x leaf: both operands 3f, one MMA per tile
        switch (tiles) {
            case 2: return up_nt<P, 2, MODE_SAE>(lin, lm, n_out, lout, st);
            case 3: return up_nt<P, 3, MODE_SAE>(lin, lm, n_out, lout, st);
            default: return up_nt<P, 1, MODE_SAE>(lin, lm, n_out, lout, st);
        }
    }
    switch (tiles) {
        case 2: return up_nt<P, 2, MODE_GEN>(lin, lm, n_out, lout, st);
        case 3: return up_nt<P, 3, MODE_GEN>(lin, lm, n_out, lout, st);
        default: return up_nt<P, 1, MODE_GEN>(lin, lm, n_out, lout, st);
    }
}

template <int P>
cudaError_t launch_tree_down_mma(const int16_t *lpar, const LevelMap &lm, int n_par, int16_t *lch,
                                 cudaStream_t st, int tiles, bool leaves) {
    if (leaves) {  // parent inverse x leaf 3f: two MMAs per tile
        switch (tiles) {
            case 2: return down_nt<P, 2, MODE_SA>(lpar, lm, n_par, lch, st);
            case 3: return down_nt<P, 3, MODE_SA>(lpar, lm, n_par, lch, st);
            default: return down_nt<P, 1, MODE_SA>(lpar, lm, n_par, lch, st);
        }
    }
    switch (tiles) {
        case 2: return down_nt<P, 2, MODE_GEN>(lpar, lm, n_par, lch, st);
        case 3: return down_nt<P, 3, MODE_GEN>(lpar, lm, n_par, lch, st);
        default: return down_nt<P, 1, MODE_GEN>(lpar, lm, n_par, lch, st);
    }
}

template <int P>
cudaError_t launch_mul_batch_mma(int n, const int16_t *a, const int16_t *b, int16_t *c,
                                 cudaStream_t st) {
    constexpr int NT = 2;
    const size_t sm = sizeof(MmaE<P, NT>) + sizeof(MmaA<P, NT>);
    cudaError_t e = allow_smem(k_mul_batch_mma<P, NT>, sm);
    if (e != cudaSuccess) return e;
    k_mul_batch_mma<P, NT><<<n, 32 * MmaGeo<P, NT>::NW, sm, st>>>(a, b, c);
    return cudaGetLastError();
}

#define SNT_MMA_INST(P)                                                                         \
    template cudaError_t launch_tree_up_mma<P>(const int16_t *, const LevelMap &, int, int16_t *, \
                                               cudaStream_t, int, bool);                        \
    template cudaError_t launch_tree_down_mma<P>(const int16_t *, const LevelMap &, int,        \
                                                 int16_t *, cudaStream_t, int, bool);           \
    template cudaError_t launch_mul_batch_mma<P>(int, const int16_t *, const int16_t *,         \
                                                 int16_t *, cudaStream_t);
SNT_MMA_INST(653)
SNT_MMA_INST(761)
SNT_MMA_INST(857)

}  // namespace snt
