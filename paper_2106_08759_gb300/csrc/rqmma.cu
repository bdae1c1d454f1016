// rqmma.cu -- the product tree and the batched product on the tensor cores
// (mma_mul.cuh): same products, same tree, same bytes as rqmul.cu.
//
// Work split.  A product is NTILE MMA tiles of 128 outputs; a CTA computes
// one product (up-sweep, batched product) or one parent's two children
// (down-sweep, sharing the parent's E table) with NW warps of NT tiles each.
// In the down-sweep the children are overwritten in place: every read of
// them happens before the CTA's first barrier and only this CTA touches them.
// On narrow levels (few products: latency, not throughput) each tile's sum
// is also split over KS warps along D (K-split), cutting the serial MMA
// chain of a product KS-fold.
#include <cuda_fp16.h>

#include "kernels.h"
#include "mma_mul.cuh"
#include "pdl.cuh"

namespace snt {

namespace {

template <typename K> cudaError_t allow_smem(K kern, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}


}  // namespace

template <int P, int NT, int MODE, int KS, int Q = Prm<P>::q>
__global__ void __launch_bounds__(32 * MmaGeo<P, NT>::NW * KS)
k_tree_up_mma(const int16_t *__restrict__ lin, LevelMap lm, int16_t *__restrict__ lout) {
    pdl_enter();
    using G = Geo<P>;
    using M = MmaGeo<P, NT>;
    extern __shared__ __align__(16) uint8_t sm[];
    MmaE<P, NT> &E = *reinterpret_cast<MmaE<P, NT> *>(sm);
    MmaA<P, NT> &A = *reinterpret_cast<MmaA<P, NT> *>(sm + sizeof(MmaE<P, NT>));
    float *red = reinterpret_cast<float *>(sm + sizeof(MmaE<P, NT>) + sizeof(MmaA<P, NT>));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nth = blockDim.x;
    const int tw = warp % M::NW, ks = warp / M::NW;  // tile group, K-split part
    const int j = blockIdx.x;
    int idx, base, n_in;
    lm_node(lm, j, idx, base, n_in);
    const int16_t *a = lin + (size_t)(base + 2 * idx) * G::pad;
    int16_t *c = lout + (size_t)j * G::pad;
    if (2 * idx + 1 >= n_in) {  // unpaired: move up unchanged (uniform over the CTA)
        for (int i = threadIdx.x; i < G::pad; i += nth) c[i] = a[i];
        return;
    }
    mma_fill_a<P, NT, MODE>(a, A, threadIdx.x, nth);
    mma_fill_b<P, NT>(a + G::pad, E, threadIdx.x, nth);
    __syncthreads();
    mma_fill_pe<P, NT, MODE, Q>(E, threadIdx.x, nth);
    __syncthreads();
    const MmaA<P, NT> *const As[1] = {&A};
    if constexpr (MODE == MODE_GW) {
        int acc[NT][1][2][4];
        mma_tiles_gw<P, NT, 1>(E, As, tw * NT, lane, acc, ks, KS);
        if (KS > 1) mma_ksplit_reduce_gw<NT, 1>(acc, reinterpret_cast<int *>(red), ks, KS, tw, M::NW, lane);
        __syncthreads();
        if (ks == 0) mma_stage_gw<P, NT, 1>(A, tw * NT, lane, 0, acc);
    } else {
        float acc[NT][1][3][4];
        mma_tiles<P, NT, 1, MODE>(E, As, tw * NT, lane, acc, ks, KS);
        if (KS > 1) mma_ksplit_reduce<NT, 1>(acc, red, ks, KS, tw, M::NW, lane);
        __syncthreads();
        if (ks == 0) mma_stage<P, NT, 1, MODE, Q>(A, tw * NT, lane, 0, acc);
    }
    __syncthreads();
    mma_finish<P, NT, Q>(A, (int)E.b[M::p - 1], c, G::pad, threadIdx.x, nth);
}

template <int P, int NT, int MODE, int KS, int Q = Prm<P>::q>
__global__ void __launch_bounds__(32 * MmaGeo<P, NT>::NW * KS)
k_tree_down_mma(const int16_t *__restrict__ lpar, LevelMap lm, int16_t *__restrict__ lch) {
    using G = Geo<P>;
    using M = MmaGeo<P, NT>;
    extern __shared__ __align__(16) uint8_t sm[];
    MmaE<P, NT> &E = *reinterpret_cast<MmaE<P, NT> *>(sm);
    MmaA<P, NT> *A = reinterpret_cast<MmaA<P, NT> *>(sm + sizeof(MmaE<P, NT>));
    float *red = reinterpret_cast<float *>(sm + sizeof(MmaE<P, NT>) + 2 * sizeof(MmaA<P, NT>));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nth = blockDim.x;
    const int tw = warp % M::NW, ks = warp / M::NW;  // tile group, K-split part
    const int j = blockIdx.x;
    int idx, base, n_ch;
    lm_node(lm, j, idx, base, n_ch);
    const int16_t *T = lpar + (size_t)j * G::pad;
    int16_t *x = lch + (size_t)(base + 2 * idx) * G::pad;
    int16_t *y = x + G::pad;
    if (2 * idx + 1 >= n_ch) {  // unpaired child: its inverse is the parent's
        pdl_enter();
        for (int i = threadIdx.x; i < G::pad; i += nth) x[i] = T[i];
        return;
    }
    // the children were written by the up-sweep, several kernels back: their
    // tables are filled before the wait for the parent level
    mma_fill_a<P, NT, MODE>(y, A[0], threadIdx.x, nth);  // 1/x = T * y
    mma_fill_a<P, NT, MODE>(x, A[1], threadIdx.x, nth);  // 1/y = T * x
    pdl_enter();
    mma_fill_b<P, NT>(T, E, threadIdx.x, nth);
    __syncthreads();  // both children are in shared memory before either is overwritten
    // the parent T is small only in R/3 (MODE_SAE), never in R/q
    mma_fill_pe<P, NT, MODE == MODE_SAE ? MODE_SAE : MODE_GEN, Q>(E, threadIdx.x, nth);
    __syncthreads();
    const MmaA<P, NT> *const As[2] = {&A[0], &A[1]};
    if constexpr (MODE == MODE_GW) {
        int acc[NT][2][2][4];
        mma_tiles_gw<P, NT, 2>(E, As, tw * NT, lane, acc, ks, KS);
        if (KS > 1) mma_ksplit_reduce_gw<NT, 2>(acc, reinterpret_cast<int *>(red), ks, KS, tw, M::NW, lane);
        __syncthreads();
        if (ks == 0) {
            mma_stage_gw<P, NT, 2>(A[0], tw * NT, lane, 0, acc);
            mma_stage_gw<P, NT, 2>(A[1], tw * NT, lane, 1, acc);
        }
    } else {
        float acc[NT][2][3][4];
        mma_tiles<P, NT, 2, MODE>(E, As, tw * NT, lane, acc, ks, KS);
        if (KS > 1) mma_ksplit_reduce<NT, 2>(acc, red, ks, KS, tw, M::NW, lane);
        __syncthreads();
        if (ks == 0) {
            mma_stage<P, NT, 2, MODE, Q>(A[0], tw * NT, lane, 0, acc);
            mma_stage<P, NT, 2, MODE, Q>(A[1], tw * NT, lane, 1, acc);
        }
    }
    __syncthreads();
    const int tl = (int)E.b[M::p - 1];
    mma_finish<P, NT, Q>(A[0], tl, x, G::pad, threadIdx.x, nth);
    mma_finish<P, NT, Q>(A[1], tl, y, G::pad, threadIdx.x, nth);
}

// c_e = a_e * b_e, n products, all operands stride p (microbenchmark layout).
template <int P, int NT, int MODE = MODE_GEN>
__global__ void __launch_bounds__(32 * MmaGeo<P, NT>::NW)
k_mul_batch_mma(const int16_t *__restrict__ a, const int16_t *__restrict__ b,
                int16_t *__restrict__ c) {
    using M = MmaGeo<P, NT>;
    extern __shared__ __align__(16) uint8_t sm[];
    MmaE<P, NT> &E = *reinterpret_cast<MmaE<P, NT> *>(sm);
    MmaA<P, NT> &A = *reinterpret_cast<MmaA<P, NT> *>(sm + sizeof(MmaE<P, NT>));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nth = blockDim.x;
    const size_t e = blockIdx.x;
    mma_fill_a<P, NT, MODE>(a + e * P, A, threadIdx.x, nth);
    mma_fill_b<P, NT>(b + e * P, E, threadIdx.x, nth);
    __syncthreads();
    mma_fill_pe<P, NT>(E, threadIdx.x, nth);
    __syncthreads();
    const MmaA<P, NT> *const As[1] = {&A};
    if constexpr (MODE == MODE_GW) {
        int acc[NT][1][2][4];
        mma_tiles_gw<P, NT, 1>(E, As, warp * NT, lane, acc);
        __syncthreads();
        mma_stage_gw<P, NT, 1>(A, warp * NT, lane, 0, acc);
    } else {
        float acc[NT][1][3][4];
        mma_tiles<P, NT, 1>(E, As, warp * NT, lane, acc);
        __syncthreads();
        mma_stage<P, NT, 1>(A, warp * NT, lane, 0, acc);
    }
    __syncthreads();
    mma_finish<P, NT>(A, (int)E.b[M::p - 1], c + e * P, P, threadIdx.x, nth);
}

namespace {
template <int P, int NT, int MODE, int KS = 1, int Q = Prm<P>::q>
cudaError_t up_nt(const int16_t *lin, const LevelMap &lm, int n_out, int16_t *lout, cudaStream_t st) {
    using M = MmaGeo<P, NT>;
    const size_t sm = sizeof(MmaE<P, NT>) + sizeof(MmaA<P, NT>) +
                      (size_t)(KS - 1) * M::NW * 32 * NT * 12 * sizeof(float);
    cudaError_t e = allow_smem(k_tree_up_mma<P, NT, MODE, KS, Q>, sm);
    if (e != cudaSuccess) return e;
    SNT_LAUNCH(k_tree_up_mma<P, NT, MODE, KS, Q>, n_out, 32 * M::NW * KS, sm, st, lin, lm, lout);
    return cudaGetLastError();
}
template <int P, int NT, int MODE, int KS = 1, int Q = Prm<P>::q>
cudaError_t down_nt(const int16_t *lpar, const LevelMap &lm, int n_par, int16_t *lch, cudaStream_t st) {
    using M = MmaGeo<P, NT>;
    const size_t sm = sizeof(MmaE<P, NT>) + 2 * sizeof(MmaA<P, NT>) +
                      (size_t)(KS - 1) * M::NW * 32 * NT * 2 * 12 * sizeof(float);
    cudaError_t e = allow_smem(k_tree_down_mma<P, NT, MODE, KS, Q>, sm);
    if (e != cudaSuccess) return e;
    SNT_LAUNCH(k_tree_down_mma<P, NT, MODE, KS, Q>, n_par, 32 * M::NW * KS, sm, st, lpar, lm, lch);
    return cudaGetLastError();
}
// K-split of a level of n products (at most kmax): latency-bound levels only.
inline int ksplit_for(int n, int kmax) {
    const int k = n <= 64 ? 4 : n <= 256 ? 2 : 1;
    return k < kmax ? k : (kmax >= 4 ? 4 : kmax >= 2 ? 2 : 1);
}
}  // namespace

// General levels: four MMAs per step on two limbs a side (MODE_GEN), or
// (wide) two MMAs per step with one exact f16 limb on the vector side
// (MODE_GW).  Leaf levels use the small-operand forms either way.
template <int P, int GEN>
cudaError_t up_general(const int16_t *lin, const LevelMap &lm, int n_out, int16_t *lout,
                       cudaStream_t st, int tiles, int ks) {
    switch (ks) {
        case 4: return up_nt<P, 1, GEN, 4>(lin, lm, n_out, lout, st);
        case 2: return up_nt<P, 1, GEN, 2>(lin, lm, n_out, lout, st);
        default: break;
    }
    switch (tiles) {
        case 2: return up_nt<P, 2, GEN>(lin, lm, n_out, lout, st);
        case 3: return up_nt<P, 3, GEN>(lin, lm, n_out, lout, st);
        default: return up_nt<P, 1, GEN>(lin, lm, n_out, lout, st);
    }
}
template <int P, int GEN>
cudaError_t down_general(const int16_t *lpar, const LevelMap &lm, int n_par, int16_t *lch,
                         cudaStream_t st, int tiles, int ks) {
    switch (ks) {
        case 4: return down_nt<P, 1, GEN, 4>(lpar, lm, n_par, lch, st);
        case 2: return down_nt<P, 1, GEN, 2>(lpar, lm, n_par, lch, st);
        default: break;
    }
    switch (tiles) {
        case 2: return down_nt<P, 2, GEN>(lpar, lm, n_par, lch, st);
        case 3: return down_nt<P, 3, GEN>(lpar, lm, n_par, lch, st);
        default: return down_nt<P, 1, GEN>(lpar, lm, n_par, lch, st);
    }
}

template <int P>
cudaError_t launch_tree_up_mma(const int16_t *lin, const LevelMap &lm, int n_out, int16_t *lout,
                               cudaStream_t st, int tiles, bool leaves, int kmax, bool wide) {
    const int ks = ksplit_for(n_out, kmax);  // narrow level: one tile per warp, K-split
    if (leaves) {  // leaf x leaf: both operands 3f, one MMA per tile
        switch (ks) {
            case 4: return up_nt<P, 1, MODE_SAE, 4>(lin, lm, n_out, lout, st);
            case 2: return up_nt<P, 1, MODE_SAE, 2>(lin, lm, n_out, lout, st);
            default: break;
        }
        switch (tiles) {
            case 2: return up_nt<P, 2, MODE_SAE>(lin, lm, n_out, lout, st);
            case 3: return up_nt<P, 3, MODE_SAE>(lin, lm, n_out, lout, st);
            default: return up_nt<P, 1, MODE_SAE>(lin, lm, n_out, lout, st);
        }
    }
    return wide ? up_general<P, MODE_GW>(lin, lm, n_out, lout, st, tiles, ks)
                : up_general<P, MODE_GEN>(lin, lm, n_out, lout, st, tiles, ks);
}

template <int P>
cudaError_t launch_tree_down_mma(const int16_t *lpar, const LevelMap &lm, int n_par, int16_t *lch,
                                 cudaStream_t st, int tiles, bool leaves, int kmax, bool wide) {
    const int ks = ksplit_for(n_par, kmax);  // narrow level: one tile per warp, K-split
    if (leaves) {  // parent inverse x leaf 3f: two MMAs per tile
        switch (ks) {
            case 4: return down_nt<P, 1, MODE_SA, 4>(lpar, lm, n_par, lch, st);
            case 2: return down_nt<P, 1, MODE_SA, 2>(lpar, lm, n_par, lch, st);
            default: break;
        }
        switch (tiles) {
            case 2: return down_nt<P, 2, MODE_SA>(lpar, lm, n_par, lch, st);
            case 3: return down_nt<P, 3, MODE_SA>(lpar, lm, n_par, lch, st);
            default: return down_nt<P, 1, MODE_SA>(lpar, lm, n_par, lch, st);
        }
    }
    return wide ? down_general<P, MODE_GW>(lpar, lm, n_par, lch, st, tiles, ks)
                : down_general<P, MODE_GEN>(lpar, lm, n_par, lch, st, tiles, ks);
}

// The same trees in R/3 (coefficients mod 3, all operands small: one MMA
// per tile on every level), for the batch inversion of the g's.
template <int P>
cudaError_t launch_tree_up_mma3(const int16_t *lin, const LevelMap &lm, int n_out, int16_t *lout,
                                cudaStream_t st, int kmax) {
    switch (ksplit_for(n_out, kmax)) {
        case 4: return up_nt<P, 1, MODE_SAE, 4, 3>(lin, lm, n_out, lout, st);
        case 2: return up_nt<P, 1, MODE_SAE, 2, 3>(lin, lm, n_out, lout, st);
        default: return up_nt<P, 1, MODE_SAE, 1, 3>(lin, lm, n_out, lout, st);
    }
}
template <int P>
cudaError_t launch_tree_down_mma3(const int16_t *lpar, const LevelMap &lm, int n_par, int16_t *lch,
                                  cudaStream_t st, int kmax) {
    switch (ksplit_for(n_par, kmax)) {
        case 4: return down_nt<P, 1, MODE_SAE, 4, 3>(lpar, lm, n_par, lch, st);
        case 2: return down_nt<P, 1, MODE_SAE, 2, 3>(lpar, lm, n_par, lch, st);
        default: return down_nt<P, 1, MODE_SAE, 1, 3>(lpar, lm, n_par, lch, st);
    }
}

template <int P>
cudaError_t launch_mul_batch_mma(int n, const int16_t *a, const int16_t *b, int16_t *c,
                                 cudaStream_t st, bool wide) {
    constexpr int NT = 2;
    const size_t sm = sizeof(MmaE<P, NT>) + sizeof(MmaA<P, NT>);
    cudaError_t e = wide ? allow_smem(k_mul_batch_mma<P, NT, MODE_GW>, sm)
                         : allow_smem(k_mul_batch_mma<P, NT>, sm);
    if (e != cudaSuccess) return e;
    if (wide)
        k_mul_batch_mma<P, NT, MODE_GW><<<n, 32 * MmaGeo<P, NT>::NW, sm, st>>>(a, b, c);
    else
        k_mul_batch_mma<P, NT><<<n, 32 * MmaGeo<P, NT>::NW, sm, st>>>(a, b, c);
    return cudaGetLastError();
}

#define SNT_MMA_INST(P)                                                                         \
    template cudaError_t launch_tree_up_mma<P>(const int16_t *, const LevelMap &, int, int16_t *, \
                                               cudaStream_t, int, bool, int, bool);             \
    template cudaError_t launch_tree_down_mma<P>(const int16_t *, const LevelMap &, int,        \
                                                 int16_t *, cudaStream_t, int, bool, int, bool); \
    template cudaError_t launch_mul_batch_mma<P>(int, const int16_t *, const int16_t *,         \
                                                 int16_t *, cudaStream_t, bool);                \
    template cudaError_t launch_tree_up_mma3<P>(const int16_t *, const LevelMap &, int,         \
                                                int16_t *, cudaStream_t, int);                  \
    template cudaError_t launch_tree_down_mma3<P>(const int16_t *, const LevelMap &, int,       \
                                                  int16_t *, cudaStream_t, int);
SNT_MMA_INST(653)
SNT_MMA_INST(761)
SNT_MMA_INST(857)

}  // namespace snt
