// noalloc.cu -- batch key generation that allocates no device memory.
//
// Some callers cannot call cudaMalloc: code that runs while a framework's
// caching allocator owns all free device memory, real-time or latency-bound
// paths where cudaMalloc/cudaFree would synchronise the device, and hosts
// whose memory policy forbids allocation after start-up.  snt_batch_keygen_static
// serves them: the caller still passes the pk/sk output buffers, and the
// scratch memory (product-tree nodes and the g of every key) is one
// file-scope __device__ array of fixed size that every GPU loading this
// library holds until the process exits.
//
// Host code must not pass the array's name to a kernel: on the host that
// name is only a stand-in, not a device address.  The first call on a device
// looks up the array's device address with cudaGetSymbolAddress (with that
// device current) and caches it; later calls reuse the cached address, which
// stays valid while the device's primary context lives (a cudaDeviceReset
// while the library is loaded is not supported).
#include <mutex>

#include "host_plan.h"

namespace {

// Largest batch of the allocation-free entry point, and the scratch it needs:
// 511 tree nodes of 864 int16 plus 256 g rows of 864 bytes for sntrup857
// (the largest parameter set) = 1,104,128 bytes, rounded up to 1152 KiB.
constexpr size_t kStaticMaxB = 256;
constexpr size_t kStaticScratchBytes = 1152 * 1024;
constexpr int kMaxDevices = 64;

__device__ __align__(256) uint8_t g_static_scratch[kStaticScratchBytes];
__device__ __align__(256) int g_static_err;

std::mutex g_setup_mutex;
uint8_t *g_scratch_addr[kMaxDevices] = {};
int *g_err_addr[kMaxDevices] = {};

#define SNT_CUDA_S(call)                                                                   \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return snt::set_error(SNT_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));     \
    } while (0)

// Device addresses of the static scratch and error word on `device` (which is
// current), looked up once per device.
snt_status static_addresses(int device, uint8_t **scratch, int **err) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[device]) {
        void *s = nullptr, *e = nullptr;
        SNT_CUDA_S(cudaGetSymbolAddress(&s, g_static_scratch));
        SNT_CUDA_S(cudaGetSymbolAddress(&e, g_static_err));
        g_err_addr[device] = static_cast<int *>(e);
        g_scratch_addr[device] = static_cast<uint8_t *>(s);
    }
    *scratch = g_scratch_addr[device];
    *err = g_err_addr[device];
    return SNT_OK;
}

template <int P>
snt_status run_static(const snt::ParamInfo &pi, uint64_t seed, uint64_t first, size_t B,
                      uint8_t *pk, uint8_t *sk, cudaStream_t st, uint8_t *scratch, int *err) {
    using namespace snt;
    const Tree t = make_tree(B);
    int16_t *nodes = reinterpret_cast<int16_t *>(scratch);
    int8_t *gbuf = reinterpret_cast<int8_t *>(scratch + align256(t.total * pi.pad * sizeof(int16_t)));
    const int Bi = (int)B, sb = pi.small_bytes;
    SNT_CUDA_S(cudaMemsetAsync(err, 0, sizeof(int), st));
    const KeyMap km = single_batch(seed, first, Bi, pk, sk);
    SNT_CUDA_S(launch_sample_f<P>(km, Bi, nodes, pi.sk_bytes, 2 * sb + pi.pk_bytes, st));
    SNT_CUDA_S(launch_r3_keygen<P>(km, Bi, gbuf, pi.sk_bytes, sb, nullptr, nullptr, 0, err, st,
                                   kDefaultR3Lanes));
    const int L = (int)t.n.size() - 1;
    for (int l = 1; l <= L; ++l)
        SNT_CUDA_S(launch_tree_up<P>(nodes + (size_t)t.off[l - 1] * pi.pad, single_tree(t.n[l - 1]),
                                     t.n[l], nodes + (size_t)t.off[l] * pi.pad, st, kDefaultTreeSplit));
    int16_t *root = nodes + (size_t)t.off[L] * pi.pad;
    SNT_CUDA_S(launch_rq_inv_jump<P>(1, root, pi.pad, root, pi.pad, nullptr, err, ERR_ROOT, st));
    for (int l = L; l >= 1; --l)
        SNT_CUDA_S(launch_tree_down<P>(nodes + (size_t)t.off[l] * pi.pad, single_tree(t.n[l - 1]),
                                       t.n[l], nodes + (size_t)t.off[l - 1] * pi.pad, st,
                                       kDefaultTreeSplit));
    SNT_CUDA_S(launch_finalize<P>(km, Bi, gbuf, nodes, pi.pk_bytes, pi.sk_bytes, 2 * sb, pi.sched,
                                  st));
    SNT_CUDA_S(launch_sha512_pk(km, Bi, pi.pk_bytes, pi.sk_bytes, 3 * sb + pi.pk_bytes, st));
    int herr = 0;
    SNT_CUDA_S(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    SNT_CUDA_S(cudaStreamSynchronize(st));
    if (herr)
        return snt::set_error(SNT_EINTERNAL, "device self-check failed (0x%x)", herr);
    return SNT_OK;
}

}  // namespace

extern "C" snt_status snt_batch_keygen_static(int device, int P, uint64_t seed,
                                              uint64_t first_key_index, size_t B,
                                              uint8_t *pk_dev, uint8_t *sk_dev,
                                              snt_stream stream) {
    using namespace snt;
    ParamInfo pi;
    if (!param_info(P, pi)) return set_error(SNT_EINVAL, "unknown parameter set %d", P);
    if (B == 0 || B > kStaticMaxB)
        return set_error(SNT_EINVAL,
                         "snt_batch_keygen_static takes 1 to %zu keys per call (got %zu); use "
                         "snt_batch_keygen with a context for larger batches",
                         kStaticMaxB, B);
    if (!pk_dev || !sk_dev) return set_error(SNT_EINVAL, "null output buffer");
    if (device < 0 || device >= kMaxDevices) return set_error(SNT_EINVAL, "device %d out of range", device);
    if (keygen_scratch(pi, B, false) > kStaticScratchBytes)
        return set_error(SNT_EINTERNAL, "static scratch too small for %zu keys", B);
    DeviceGuard dg(device);
    if (!dg.ok) return set_error(SNT_ECUDA, "cannot select device %d", device);
    uint8_t *scratch = nullptr;
    int *err = nullptr;
    const snt_status s = static_addresses(device, &scratch, &err);
    if (s != SNT_OK) return s;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    switch (P) {
        case 653: return run_static<653>(pi, seed, first_key_index, B, pk_dev, sk_dev, st, scratch, err);
        case 761: return run_static<761>(pi, seed, first_key_index, B, pk_dev, sk_dev, st, scratch, err);
        default:  return run_static<857>(pi, seed, first_key_index, B, pk_dev, sk_dev, st, scratch, err);
    }
}
