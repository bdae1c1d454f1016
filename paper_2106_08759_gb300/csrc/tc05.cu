// tc05.cu -- throughput of the 5th-generation tensor-core MMA (tcgen05.mma,
// kind::f16: f16 operands from shared memory, f32 accumulator in tensor
// memory) at M = 128, K = 16 and N = 16 .. 256.  A measurement for choosing
// the R/q product engine, not part of key generation: the Toeplitz form of
// an R/q product gives an MMA only a few useful output columns per shared
// operand tile (one product's output blocks), so its rate at small N is the
// number that matters.
//
// k CTAs per SM (the dynamic shared memory request admits k; k = 1, 2 or 4,
// so that several issuing threads share one SM's tensor core), 128 threads
// each: thread 0 issues `iters` MMAs into one accumulator and commits
// them to an mbarrier; every thread waits for it (bounded by the SM clock),
// then each warp reads its 32 accumulator rows and checks them: with
// A[m][k] = (k == m mod 16) and B[n][k] = (n + 3 k) mod 8 (exact in f16),
// D[m][n] = iters * B[n][m mod 16].
#include <cuda_fp16.h>

#include "sntrup_gb300.h"

namespace {

constexpr int kM = 128, kK = 16;
// dynamic shared memory that admits k CTAs per SM
inline int dyn_smem_for(int k) { return k == 1 ? 200 * 1024 : k == 2 ? 100 * 1024 : 50 * 1024; }

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor of tcgen05: start address, leading
// (K-direction) and stride (M/N-direction) byte offsets between 8-row x
// 16-byte core matrices, each >> 4; the fixed 0b001 at bits 46-48; no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: D f32 (bits 4-5 = 1), A and B f16
// (bits 7-9, 10-12 = 0), both K-major (bits 15, 16 = 0), N >> 3 at bits
// 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_f16(int m, int n) {
    return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// Offset (in halves) of element (row r, k) of a K-major tile with 16 K
// columns: core matrix (r / 8, k / 8) at (2 (r / 8) + k / 8) * 128 bytes,
// rows of 16 bytes inside (leading offset 128 bytes, stride offset 256).
__device__ __forceinline__ int core_off(int r, int k) {
    return ((r >> 3) * 2 + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}

__device__ __forceinline__ bool mbar_done(uint32_t mbar) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(mbar)
        : "memory");
    return ok != 0;
}

// Waits for the mbarrier's first phase for at most `limit` SM cycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, long long limit) {
    const long long t0 = clock64();
    while (!mbar_done(mbar))
        if (clock64() - t0 > limit) return false;
    return true;
}

template <int N>
__global__ void __launch_bounds__(128, 1) k_tc05_rate(int iters, int *err) {
    constexpr int NCOLS = N < 32 ? 32 : N;  // tensor-memory columns (power of two >= 32)
    extern __shared__ __align__(1024) uint8_t dyn[];
    __half *A = reinterpret_cast<__half *>(dyn);
    __half *Bm = reinterpret_cast<__half *>(dyn + kM * kK * 2);
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int e = tid; e < kM * kK; e += 128) {
        const int m = e / kK, k = e % kK;
        A[core_off(m, k)] = __int2half_rn(k == (m & 15) ? 1 : 0);
    }
    for (int e = tid; e < N * kK; e += 128) {
        const int n = e / kK, k = e % kK;
        Bm[core_off(n, k)] = __int2half_rn((n + 3 * k) & 7);
    }
    const uint32_t mb = smem_u32(&mbar);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"(NCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // the operands were written by the generic proxy; the MMA reads them
    // through the async proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    if (tid == 0) {
        const uint64_t ad = smem_desc(smem_u32(A), 128, 256);
        const uint64_t bd = smem_desc(smem_u32(Bm), 128, 256);
        constexpr uint32_t id = idesc_f16(kM, N);
        for (int it = 0; it < iters; ++it)
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "setp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                "l"(ad), "l"(bd), "r"(id), "r"(it)
                : "memory");
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb)
            : "memory");
    }
    // about two seconds at 2 GHz; on time-out flag it and give the MMAs as
    // long again before the memory is read and released
    bool ok = mbar_wait_bounded(mb, 4000000000LL);
    if (!ok) {
        if (lane == 0) atomicOr(err, 1);
        ok = mbar_wait_bounded(mb, 4000000000LL);
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        const int m = 32 * warp + lane;  // accumulator row = tensor-memory lane
        const int cols[3] = {0, 1, N - 1};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            uint32_t v;
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];"
                         : "=r"(v)
                         : "r"(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)cols[c])
                         : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            const float want = (float)iters * (float)((cols[c] + 3 * (m & 15)) & 7);
            if (__uint_as_float(v) != want) atomicOr(err, 2);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(NCOLS)
                     : "memory");
}

template <int N>
cudaError_t run_tc05(int blocks, int dyn, int iters, int *err, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(k_tc05_rate<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         200 * 1024);
    if (e != cudaSuccess) return e;
    k_tc05_rate<N><<<blocks, 128, dyn, st>>>(iters, err);
    return cudaGetLastError();
}

}  // namespace

extern "C" snt_status snt_measure_tc05(int device, int n, int ctas_per_sm, double *macs_per_s,
                                       int *sms) {
    if (!macs_per_s || (n != 16 && n != 32 && n != 64 && n != 128 && n != 256)) return SNT_EINVAL;
    // k CTAs of max(32, n) tensor-memory columns each must fit the SM's 512
    if ((ctas_per_sm != 1 && ctas_per_sm != 2 && ctas_per_sm != 4) ||
        ctas_per_sm * (n < 32 ? 32 : n) > 512)
        return SNT_EINVAL;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) return SNT_ECUDA;
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, device);
    int *err = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    const int blocks = prop.multiProcessorCount * ctas_per_sm, dyn = dyn_smem_for(ctas_per_sm);
    const int iters = (1 << 19) / (n / 16);  // iters * 7 stays exact in f32
    float best = 1e30f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        cudaEventRecord(t0);
        switch (n) {
            case 16: e = run_tc05<16>(blocks, dyn, iters, err, nullptr); break;
            case 32: e = run_tc05<32>(blocks, dyn, iters, err, nullptr); break;
            case 64: e = run_tc05<64>(blocks, dyn, iters, err, nullptr); break;
            case 128: e = run_tc05<128>(blocks, dyn, iters, err, nullptr); break;
            default: e = run_tc05<256>(blocks, dyn, iters, err, nullptr); break;
        }
        if (e != cudaSuccess) break;
        cudaEventRecord(t1);
        e = cudaEventSynchronize(t1);
        float ms = 0;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
        if (rep > 0 && ms < best) best = ms;  // first launch is warm-up
    }
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) {
        *macs_per_s = (double)blocks * iters * (double)kM * n * kK / (best * 1e-3);
        if (sms) *sms = prop.multiProcessorCount;
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (err) cudaFree(err);
    cudaSetDevice(prev);
    if (e != cudaSuccess) return SNT_ECUDA;
    if (herr & 1) return SNT_ETIMEOUT;
    return herr ? SNT_EINTERNAL : SNT_OK;
}
