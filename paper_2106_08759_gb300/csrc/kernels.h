// kernels.h -- host-side launchers of the sntrup GB300 kernels (internal).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace snt {

// One pass of the mixed-radix Rq_encode: n entries, all but the last of
// radix mu, the last of radix mlast; full pairs emit eu bytes each, a pair
// that contains the last entry emits elast; pair i writes at boff + i * eu.
struct EncLevel {
    int n;
    uint32_t mu, mlast;
    int eu, elast, boff;
};
struct EncSched {
    int nlev;
    EncLevel lev[16];
    int efinal, foff;  // bytes of the single remaining entry and their offset
    int total;         // encoded length
};

template <int P>
cudaError_t launch_sample_f(uint64_t seed, uint64_t first, int B, int16_t *leaves, uint8_t *sk,
                            int sk_bytes, int rho_off, cudaStream_t st);
template <int P>
cudaError_t launch_r3_keygen(uint64_t seed, uint64_t first, int B, int8_t *g_out, uint8_t *sk,
                             int sk_bytes, int sk_off, const uint64_t *inj_idx,
                             const int8_t *inj_g, int n_inj, int *err, cudaStream_t st,
                             int lanes);
template <int P>
cudaError_t launch_r3_inv(int n, const int8_t *g, int8_t *out, int32_t *ok, cudaStream_t st,
                          int lanes);
template <int P>
cudaError_t launch_tree_up(const int16_t *lin, int n_in, int16_t *lout, cudaStream_t st,
                           int max_split);
template <int P>
cudaError_t launch_tree_down(const int16_t *lpar, int16_t *lch, int n_ch, cudaStream_t st,
                             int max_split);
template <int P>
cudaError_t launch_mul_batch(int n, const int16_t *a, const int16_t *b, int16_t *c,
                             cudaStream_t st);
template <int P>
cudaError_t launch_rq_inv(int n, const int16_t *in, long in_stride, int16_t *out,
                          long out_stride, int32_t *ok, int *err, int err_bit, cudaStream_t st);
template <int P>
cudaError_t launch_rq_inv_jump(int n, const int16_t *in, long in_stride, int16_t *out,
                               long out_stride, int32_t *ok, int *err, int err_bit,
                               cudaStream_t st);
template <int P>
cudaError_t launch_finalize(int B, const int8_t *gbuf, const int16_t *ainv, uint8_t *pk,
                            int pk_bytes, uint8_t *sk, int sk_bytes, int sk_pk_off,
                            const EncSched &S, cudaStream_t st);
cudaError_t launch_sha512_pk(int B, const uint8_t *pk, int pk_bytes, uint8_t *sk, int sk_bytes,
                             int hash_off, cudaStream_t st);

}  // namespace snt
