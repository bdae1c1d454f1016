// kem.cu -- encapsulation and decapsulation of Streamlined NTRU Prime on the
// device (the serving path): a CTA of 256 threads runs the ring arithmetic of
// up to 32 items in turn, then one warp hashes them, a lane per item.
//
// The paper measures these operations (Table 1) and relies on the NTRU Prime
// specification for their definition; reading (round-3 KEM):
//   Encap(pk; r Short from stream 3 of (seed, k)):
//     h = Rq_decode(pk); c = Round(h r) (each coefficient to the nearest
//     multiple of 3); C = Rounded_encode(c) (radix (q+2)/3 on (c+(q-1)/2)/3);
//     r_enc = Small_encode(r); h3 = Hash_prefix(3, r_enc);
//     ct = C | Hash_prefix(2, h3 | Hash_prefix(4, pk));
//     ss = Hash_prefix(1, h3 | ct).
//   Decap(ct, sk = f | v | pk | rho | Hash_prefix(4, pk)):
//     c = Rounded_decode(C); e = (3 f c in R/q, centred) mod 3;
//     r' = e v in R/3; r' = (1,..,1 (w), 0,..,0) unless weight(r') = w;
//     re-encrypt r' to ct'; ss = Hash_prefix(1, Hash_prefix(3, r'_enc) | ct)
//     if ct' = ct, else Hash_prefix(0, Hash_prefix(3, rho) | ct)
//     (the selections are branch-free).
// Decryption works because h 3f = g: 3f c = g r + 3 f (c - h r), whose
// coefficients stay below q/2, so e = g r mod 3 and e v = r.
#include "common.cuh"
#include "kernels.h"
#include "mixed.cuh"
#include "sha512.cuh"
#include "short.cuh"
#include "mma_mul.cuh"

namespace snt {

constexpr int KEM_THREADS = 256;

// Items per CTA: a CTA runs the arithmetic of its items one after another
// with all its threads, then warp 0 computes their hashes, one lane per item
// (SHA-512 is a serial chain per message, so a lone thread per item would
// leave the CTA waiting; 32 lanes hash 32 items for the instructions of one).
// Small launches keep one item per CTA for latency.
constexpr int KEM_MAX_IPC = 32;

// Bytes [0, n) of src (device memory) to dst (shared memory), n <= 256 K:
// every load is issued before the first store (a load / store loop would
// wait for each load in turn, the compiler not knowing that the two buffers
// never overlap).
template <int K>
__device__ __forceinline__ void g2s_bytes(uint8_t *dst, const uint8_t *src, int n, int tid) {
    uint32_t v[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int b = tid + k * KEM_THREADS;
        v[k] = b < n ? src[b] : 0u;
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int b = tid + k * KEM_THREADS;
        if (b < n) dst[b] = (uint8_t)v[k];
    }
}
// One ring product out = a * b in R/q (Q = q) or R/3 (Q = 3), Sec. 2.1's
// x^p = x + 1, on the tensor cores (mma_mul.cuh): a is small (coefficients of
// magnitude at most 3) and takes the vector side, b the Toeplitz side (any
// centred residue for R/q; -1, 0, 1 for R/3).  a, b and out are centred int16
// rows of Geo<P>::pad entries in shared memory; out may be a or b (both are
// copied into the product's tables first) and is written up to the pad with
// zeros beyond p.  Called by every thread of the CTA; the MMA warps are the
// first MmaGeo<P, 1>::NW of its 8.
template <int P, int Q>
__device__ __forceinline__ void kem_mul(const int16_t *a, const int16_t *b, int16_t *out,
                                        MmaE<P, 1> &E, MmaA<P, 1> &A) {
    using M = MmaGeo<P, 1>;
    static_assert(M::NW <= KEM_THREADS / 32, "one warp per MMA tile");
    constexpr int MA = Q == 3 ? MODE_SAE : MODE_SA;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    __syncthreads();  // a and b written
    mma_fill_a<P, 1, MA>(a, A, tid, KEM_THREADS);
    mma_fill_b<P, 1>(b, E, tid, KEM_THREADS);
    __syncthreads();
    mma_fill_pe<P, 1, MA, Q>(E, tid, KEM_THREADS);
    __syncthreads();
    const MmaA<P, 1> *const As[1] = {&A};
    float acc[1][1][3][4];
    if (warp < M::NW) mma_tiles<P, 1, 1, MA>(E, As, warp, lane, acc);
    __syncthreads();  // the vector records are read; the staging area overlays them
    if (warp < M::NW) mma_stage<P, 1, 1, MA, Q>(A, warp, lane, 0, acc);
    __syncthreads();
    mma_finish<P, 1, Q>(A, (int)E.b[M::p - 1], out, Geo<P>::pad, tid, KEM_THREADS);
    __syncthreads();  // out complete; the tables free
}

// The two product tables of a KEM CTA, in one shared buffer.
template <int P> struct KemMul {
    static constexpr size_t eoff = 0;
    static constexpr size_t aoff = (sizeof(MmaE<P, 1>) + 15) / 16 * 16;
    static constexpr size_t bytes = aoff + sizeof(MmaA<P, 1>);
};

inline int kem_items_per_cta(int n, int sms) {
    const int ipc = n / (8 * sms);
    return ipc < 1 ? 1 : (ipc > KEM_MAX_IPC ? KEM_MAX_IPC : ipc);
}

__device__ __forceinline__ EncItem enc_item(const EncMap &em, int it, int pk_bytes, int ct_bytes) {
    EncItem item;
    if (em.tab) {
        item = em.tab[it];
    } else {
        item.pk = em.pk + (size_t)it * pk_bytes;
        item.cache = nullptr;
        item.k = em.first + (uint64_t)it;
        item.ct = em.ct + (size_t)it * ct_bytes;
        item.ss = em.ss + (size_t)it * 32;
    }
    return item;
}

template <int P>
__global__ void __launch_bounds__(KEM_THREADS, 4)
k_encap(EncMap em, int n, int ipc, int pk_bytes, int ct_bytes, EncSched Spk, EncSched Sct) {
    using G = Geo<P>;
    __shared__ __align__(16) uint8_t pkb[1344];
    __shared__ __align__(16) uint8_t ctb[1216];
    __shared__ __align__(16) uint8_t mm[KemMul<P>::bytes];
    __shared__ uint32_t R[2][G::pad];
    __shared__ __align__(16) uint32_t xs[1024];
    __shared__ __align__(16) int16_t hv[G::pad];
    __shared__ __align__(16) int16_t rv[G::pad];
    __shared__ uint8_t renc[KEM_MAX_IPC][G::small_bytes];
    MmaE<P, 1> &mE = *reinterpret_cast<MmaE<P, 1> *>(mm + KemMul<P>::eoff);
    MmaA<P, 1> &mA = *reinterpret_cast<MmaA<P, 1> *>(mm + KemMul<P>::aoff);
    const int first = blockIdx.x * ipc;
    const int cnt = min(ipc, n - first);
    if (cnt <= 0) return;
    const int tid = threadIdx.x;
    const int rb = ct_bytes - 32;
    for (int r = 0; r < cnt; ++r) {
        const EncItem item = enc_item(em, first + r, pk_bytes, ct_bytes);
        g2s_bytes<(sizeof(pkb) + KEM_THREADS - 1) / KEM_THREADS>(pkb, item.pk, pk_bytes, tid);
        __syncthreads();
        const int cur = mixed_decode<G::pad>(pkb, Spk, R);
        for (int i = tid; i < G::pad; i += KEM_THREADS)
            hv[i] = (int16_t)((i < P) ? (int)R[cur][i] - G::half : 0);
        uint32_t v[4];
        short_sorted_words<P>(em.seed, item.k, STREAM_ENC, v, xs);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = 4 * tid + q;
            if (j < G::pad) rv[j] = (int16_t)((j < P) ? (int)(v[q] & 3u) - 1 : 0);
        }
        if (tid < G::small_bytes) {
            uint32_t byte = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (4 * tid + q < P) byte |= (v[q] & 3u) << (2 * q);
            renc[r][tid] = (uint8_t)byte;
        }
        // c = Round(h r)
        kem_mul<P, G::q>(rv, hv, hv, mE, mA);
        for (int j = tid; j < P; j += KEM_THREADS) {
            const int c = (int)hv[j] - cmod<3>((int)hv[j]);
            R[0][j] = (uint32_t)((c + G::half) / 3);
        }
        __syncthreads();
        mixed_encode<G::pad>(R, Sct, ctb);
        // the rounded encoding now; its confirmation hash below
        for (int b = tid; b < rb; b += KEM_THREADS) item.ct[b] = ctb[b];
        __syncthreads();  // buffers free for the next item; ct visible to warp 0
    }
    // hashes, lane r for item r:
    //   h3 = Hash_prefix(3, r_enc); h4 = Hash_prefix(4, pk) (or the cached copy);
    //   ct = C | Hash_prefix(2, h3 | h4); ss = Hash_prefix(1, h3 | ct)
    // (each lane reads back only its own item's ct, written before by the
    // CTA behind the barrier above or by the lane itself)
    if (tid >= cnt) return;
    const EncItem item = enc_item(em, first + tid, pk_bytes, ct_bytes);
    uint8_t h3[32], h4[32], conf[32], ss[32];
    if (item.cache) {
        for (int b = 0; b < 32; ++b) h4[b] = item.cache[b];
    } else {
        sha512_prefixed(4, item.pk, pk_bytes, nullptr, 0, h4);
    }
    sha512_prefixed(3, renc[tid], G::small_bytes, nullptr, 0, h3);
    sha512_prefixed(2, h3, 32, h4, 32, conf);
    for (int b = 0; b < 32; ++b) item.ct[rb + b] = conf[b];
    sha512_prefixed(1, h3, 32, item.ct, ct_bytes, ss);
    for (int b = 0; b < 32; ++b) item.ss[b] = ss[b];
}

__device__ __forceinline__ DecItem dec_item(const DecMap &dm, int it, int sk_bytes, int ct_bytes) {
    DecItem item;
    if (dm.tab) {
        item = dm.tab[it];
    } else {
        item.sk = dm.sk + (size_t)it * sk_bytes;
        item.ct = dm.ct + (size_t)it * ct_bytes;
        item.ss = dm.ss + (size_t)it * 32;
    }
    return item;
}

template <int P>
__global__ void __launch_bounds__(KEM_THREADS, 4)
k_decap(DecMap dm, int n, int ipc, int pk_bytes, int sk_bytes, int ct_bytes, EncSched Spk,
        EncSched Sct) {
    using G = Geo<P>;
    constexpr int SB = G::small_bytes;
    __shared__ __align__(16) uint8_t skb[2016];
    __shared__ __align__(16) uint8_t ctb[1216];
    __shared__ __align__(16) uint8_t ct2[1216];
    __shared__ __align__(16) uint8_t mm[KemMul<P>::bytes];
    __shared__ uint32_t R[2][G::pad];
    __shared__ __align__(16) int16_t va[G::pad];
    __shared__ __align__(16) int16_t vb[G::pad];
    __shared__ uint8_t renc[KEM_MAX_IPC][SB];
    __shared__ int cmatch[KEM_MAX_IPC];  // the re-encryption's rounded part equals ct's
    __shared__ int weight;
    MmaE<P, 1> &mE = *reinterpret_cast<MmaE<P, 1> *>(mm + KemMul<P>::eoff);
    MmaA<P, 1> &mA = *reinterpret_cast<MmaA<P, 1> *>(mm + KemMul<P>::aoff);
    const int first = blockIdx.x * ipc;
    const int cnt = min(ipc, n - first);
    if (cnt <= 0) return;
    const int tid = threadIdx.x;
    const int rb = ct_bytes - 32;
    for (int it_r = 0; it_r < cnt; ++it_r) {
        const DecItem item = dec_item(dm, first + it_r, sk_bytes, ct_bytes);
        g2s_bytes<(sizeof(skb) + KEM_THREADS - 1) / KEM_THREADS>(skb, item.sk, sk_bytes, tid);
        g2s_bytes<(sizeof(ctb) + KEM_THREADS - 1) / KEM_THREADS>(ctb, item.ct, ct_bytes, tid);
        if (tid == 0) weight = 0;
        __syncthreads();
        const uint8_t *pkb = skb + 2 * SB;
        // e = 3 f c in R/q (c = Rounded_decode(C)), then mod 3
        int cur = mixed_decode<G::pad>(ctb, Sct, R);
        for (int i = tid; i < G::pad; i += KEM_THREADS) {
            vb[i] = (int16_t)((i < P) ? 3 * (int)R[cur][i] - G::half : 0);
            va[i] = (int16_t)((i < P) ? 3 * ((int)((skb[i / 4] >> (2 * (i % 4))) & 3u) - 1) : 0);
        }
        kem_mul<P, G::q>(va, vb, va, mE, mA);
        for (int i = tid; i < G::pad; i += KEM_THREADS) {
            va[i] = (int16_t)cmod<3>((int)va[i]);
            vb[i] = (int16_t)((i < P) ? (int)((skb[SB + i / 4] >> (2 * (i % 4))) & 3u) - 1 : 0);
        }
        // r' = e v in R/3, and its weight
        kem_mul<P, 3>(va, vb, va, mE, mA);
        {
            int nz = 0;
            for (int j = tid; j < P; j += KEM_THREADS) nz += (va[j] != 0);
            nz = __reduce_add_sync(0xffffffffu, nz);
            if ((tid & 31) == 0) atomicAdd(&weight, nz);
        }
        __syncthreads();
        const bool wok = (weight == G::w);
        if (!wok)
            for (int j = tid; j < P; j += KEM_THREADS) va[j] = (int16_t)(j < G::w ? 1 : 0);
        __syncthreads();
        // re-encrypt r': h from pk, c' = Round(h r')
        cur = mixed_decode<G::pad>(pkb, Spk, R);
        for (int i = tid; i < G::pad; i += KEM_THREADS)
            vb[i] = (int16_t)((i < P) ? (int)R[cur][i] - G::half : 0);
        for (int b = tid; b < SB; b += KEM_THREADS) {
            uint32_t byte = 0;
            for (int r = 0; r < 4; ++r)
                if (4 * b + r < P) byte |= (uint32_t)(va[4 * b + r] + 1) << (2 * r);
            renc[it_r][b] = (uint8_t)byte;
        }
        kem_mul<P, G::q>(va, vb, vb, mE, mA);
        for (int j = tid; j < P; j += KEM_THREADS) {
            const int c = (int)vb[j] - cmod<3>((int)vb[j]);
            R[0][j] = (uint32_t)((c + G::half) / 3);
        }
        __syncthreads();
        mixed_encode<G::pad>(R, Sct, ct2);
        uint32_t diff = 0;
        for (int b = tid; b < rb; b += KEM_THREADS) diff |= (uint32_t)(ct2[b] ^ ctb[b]);
        const int same = __syncthreads_or(diff != 0) == 0;
        if (tid == 0) cmatch[it_r] = same;
        __syncthreads();  // buffers free for the next item
    }
    // hashes, lane r for item r: h3 = Hash_prefix(3, r'_enc), h3rho =
    // Hash_prefix(3, rho); the re-encryption's confirmation Hash_prefix(2, h3 |
    // Hash_prefix(4, pk)) against ct's; ss = Hash_prefix(1, h3 | ct) if the
    // re-encryption equals ct, else Hash_prefix(0, h3rho | ct) (selected
    // without branches)
    if (tid >= cnt) return;
    const DecItem item = dec_item(dm, first + tid, sk_bytes, ct_bytes);
    const uint8_t *rho = item.sk + 2 * SB + pk_bytes, *cache = item.sk + 3 * SB + pk_bytes;
    uint8_t h3[32], h3rho[32], conf[32], sel[32], ss[32];
    sha512_prefixed(3, renc[tid], SB, nullptr, 0, h3);
    sha512_prefixed(3, rho, SB, nullptr, 0, h3rho);
    sha512_prefixed(2, h3, 32, cache, 32, conf);
    uint32_t cd = 0;
    for (int b = 0; b < 32; ++b) cd |= (uint32_t)(conf[b] ^ item.ct[rb + b]);
    const uint32_t accept = (uint32_t)(cmatch[tid] != 0) & (uint32_t)(cd == 0);
    const uint32_t mask = 0u - accept;  // all ones if accepted
    for (int b = 0; b < 32; ++b) sel[b] = (uint8_t)((h3[b] & mask) | (h3rho[b] & ~mask));
    sha512_prefixed((uint8_t)accept, sel, 32, item.ct, ct_bytes, ss);
    for (int b = 0; b < 32; ++b) item.ss[b] = ss[b];
}

// SMs of the current device (host state, read once per device).
static int kem_sms() {
    static int cache[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    if (!cache[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
            v = 152;
        cache[dev] = v;
    }
    return cache[dev];
}

template <int P>
cudaError_t launch_encap(const EncMap &em, int n, int pk_bytes, int ct_bytes, const EncSched &Spk,
                         const EncSched &Sct, cudaStream_t st) {
    const int ipc = kem_items_per_cta(n, kem_sms());
    k_encap<P><<<(n + ipc - 1) / ipc, KEM_THREADS, 0, st>>>(em, n, ipc, pk_bytes, ct_bytes, Spk,
                                                           Sct);
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_decap(const DecMap &dm, int n, int pk_bytes, int sk_bytes, int ct_bytes,
                         const EncSched &Spk, const EncSched &Sct, cudaStream_t st) {
    const int ipc = kem_items_per_cta(n, kem_sms());
    k_decap<P><<<(n + ipc - 1) / ipc, KEM_THREADS, 0, st>>>(dm, n, ipc, pk_bytes, sk_bytes,
                                                           ct_bytes, Spk, Sct);
    return cudaGetLastError();
}

#define SNT_KEM_INST(P)                                                                     \
    template cudaError_t launch_encap<P>(const EncMap &, int, int, int, const EncSched &,  \
                                         const EncSched &, cudaStream_t);                   \
    template cudaError_t launch_decap<P>(const DecMap &, int, int, int, int,                \
                                         const EncSched &, const EncSched &, cudaStream_t);
SNT_KEM_INST(653)
SNT_KEM_INST(761)
SNT_KEM_INST(857)

}  // namespace snt
