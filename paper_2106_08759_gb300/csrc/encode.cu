// encode.cu -- public key h = g * (3f)^-1 in R/q (Sec. 3.1 KeyGen step 4,
// Algorithm 1 "H <- g * f-bar"), its Rq_encode, and the SHA-512 hash of the
// public key stored at the end of the secret key.
//
// Rq_encode (the paper relies on the NTRU Prime encoding; reading: the
// mixed-radix Encode with every radix q).  Entries (r_i, m_i), r_i in
// [0, m_i).  One pass merges neighbouring entries into (r_2i + m_2i r_2i+1,
// m_2i m_2i+1) and, while the merged radix is >= 2^14, emits the low byte and
// sets radix <- ceil(radix / 256); an unpaired last entry moves up as is.
// Within a pass every entry but the last has the same radix, so the number
// of bytes each pair emits and its output offset are fixed: the host
// computes that schedule once (EncSched) and each pair is one thread.
#include "common.cuh"
#include "kernels.h"
#include "toeplitz.cuh"
#include <atomic>

#include "sha512.cuh"
#include "mixed.cuh"
#include "mma_mul.cuh"
#include "pdl.cuh"

namespace snt {

template <int P>
__global__ void __launch_bounds__(Tp<P>::NT)
k_finalize(KeyMap km, const int8_t *__restrict__ gbuf, const int16_t *__restrict__ ainv,
           int pk_bytes, int sk_bytes, int sk_pk_off, EncSched S) {
    pdl_enter();
    using G = Geo<P>;
    __shared__ __align__(16) int As[Tp<P>::p8];
    __shared__ __align__(16) int Es[Tp<P>::ESZ];
    __shared__ uint32_t Rb[2][G::pad];
    __shared__ uint8_t ob[1344];
    const int key = blockIdx.x;
    const int8_t *g = gbuf + (size_t)key * G::pad;
    const int16_t *inv = ainv + (size_t)key * G::pad;
    fill_A<P>(g, As);
    fill_E<P>(inv, Es);
    __syncthreads();
    int acc[1][8];
    const int *const A1[1] = {As};
    toeplitz_tile<P, 1>(A1, Es, threadIdx.x, 0, Tp<P>::p8, acc);
    const int bl[1] = {(int)inv[P - 1]};
    toeplitz_finish<P, 1>(A1, bl, acc, threadIdx.x, true);
    const int j0 = 8 * threadIdx.x;
#pragma unroll
    for (int t = 0; t < 8; ++t)
        if (j0 + t < P) Rb[0][j0 + t] = (uint32_t)(acc[0][t] + G::half);
    __syncthreads();

    mixed_encode<G::pad>(Rb, S, ob);
    const BatchDesc d = key_batch(km, key);
    uint8_t *pkk = d.pk + (size_t)(key - d.key_base) * pk_bytes;
    uint8_t *skk = d.sk + (size_t)(key - d.key_base) * sk_bytes + sk_pk_off;
    for (int b = threadIdx.x; b < pk_bytes; b += blockDim.x) {
        pkk[b] = ob[b];
        skk[b] = ob[b];
    }
}

// The same with h on the tensor cores (mma_mul.cuh): E from (3f)^-1, the
// vector side g (small, MODE_SA), one warp per MMA tile; the encoding
// buffers reuse the E table's shared memory once the products are done.
template <int P>
__global__ void __launch_bounds__(32 * MmaGeo<P, 1>::NW)
k_finalize_mma(KeyMap km, const int8_t *__restrict__ gbuf, const int16_t *__restrict__ ainv,
               int pk_bytes, int sk_bytes, int sk_pk_off, EncSched S) {
    pdl_enter();
    using G = Geo<P>;
    using M = MmaGeo<P, 1>;
    static_assert(2 * G::pad * sizeof(uint32_t) + 1344 <= sizeof(MmaE<P, 1>), "encode buffers");
    extern __shared__ __align__(16) uint8_t sm[];
    MmaE<P, 1> &E = *reinterpret_cast<MmaE<P, 1> *>(sm);
    MmaA<P, 1> &A = *reinterpret_cast<MmaA<P, 1> *>(sm + sizeof(MmaE<P, 1>));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nth = blockDim.x;
    const int key = blockIdx.x;
    const int8_t *g = gbuf + (size_t)key * G::pad;
    const int16_t *inv = ainv + (size_t)key * G::pad;
    mma_fill_a<P, 1, MODE_SA>(g, A, threadIdx.x, nth);
    mma_fill_b<P, 1>(inv, E, threadIdx.x, nth);
    __syncthreads();
    mma_fill_pe<P, 1, MODE_GEN>(E, threadIdx.x, nth);
    __syncthreads();
    float acc[1][1][3][4];
    const MmaA<P, 1> *const As[1] = {&A};
    mma_tiles<P, 1, 1, MODE_SA>(E, As, warp, lane, acc);
    const int bl = (int)E.b[M::p - 1];
    __syncthreads();
    mma_stage<P, 1, 1, MODE_SA>(A, warp, lane, 0, acc);
    __syncthreads();
    uint32_t(*Rb)[G::pad] = reinterpret_cast<uint32_t(*)[G::pad]>(sm);  // over E
    uint8_t *ob = sm + 2 * G::pad * sizeof(uint32_t);
    for (int j = threadIdx.x; j < P; j += nth) {
        int v = (j == 0) ? A.u.stage[0] - A.u.stage[stage_slot(P - 1)] + (int)A.a[0] * bl
                         : A.u.stage[stage_slot(j)] + (int)A.a[j] * bl;
        Rb[0][j] = (uint32_t)(cmod<G::q>(v) + G::half);
    }
    __syncthreads();
    mixed_encode<G::pad>(Rb, S, ob);
    const BatchDesc d = key_batch(km, key);
    uint8_t *pkk = d.pk + (size_t)(key - d.key_base) * pk_bytes;
    uint8_t *skk = d.sk + (size_t)(key - d.key_base) * sk_bytes + sk_pk_off;
    for (int b = threadIdx.x; b < pk_bytes; b += nth) {
        pkk[b] = ob[b];
        skk[b] = ob[b];
    }
}

// s = g f for one key of a leaf pair: g's draw (int8 row) against f = (3f)/3
// of the other leaf, both small (one MMA per step); |s| <= 2w, so the row is
// exact without reduction.  Written to sv (any memory, pad entries) by the
// whole CTA; contains barriers.
template <int P>
__device__ __forceinline__ void leaf_pair_s(const int8_t *g, const int16_t *f3, MmaE<P, 1> &E,
                                            MmaA<P, 1> &A, int16_t *sv, int warp, int lane,
                                            int tid, int nth) {
    using G = Geo<P>;
    using M = MmaGeo<P, 1>;
    mma_fill_a<P, 1, MODE_SAE>(g, A, tid, nth);
    for (int k = tid; k < M::AN; k += nth) E.b[k] = k < M::p ? (int16_t)(f3[k] / 3) : 0;
    __syncthreads();
    mma_fill_pe<P, 1, MODE_SAE>(E, tid, nth);
    __syncthreads();
    float acc[1][1][3][4];
    const MmaA<P, 1> *const As[1] = {&A};
    mma_tiles<P, 1, 1, MODE_SAE>(E, As, warp, lane, acc);
    __syncthreads();
    mma_stage<P, 1, 1, MODE_SAE>(A, warp, lane, 0, acc);
    __syncthreads();
    const int bl = (int)E.b[M::p - 1];
    for (int k = tid; k < G::pad; k += nth) {
        int v = 0;
        if (k == 0) v = A.u.stage[0] - A.u.stage[stage_slot(M::p - 1)] + (int)A.a[0] * bl;
        else if (k < M::p) v = A.u.stage[stage_slot(k)] + (int)A.a[k] * bl;
        sv[k] = (int16_t)v;
    }
    __syncthreads();
}

// The leaf-pair products of every level-1 node into rows of sbuf (by key),
// ahead of the down-sweep (they need only g's draws and the leaves).
template <int P>
__global__ void __launch_bounds__(32 * MmaGeo<P, 1>::NW)
k_leaf_s(const int8_t *__restrict__ gbuf, const int16_t *__restrict__ leaves, LevelMap lm1,
         int16_t *__restrict__ sbuf) {
    pdl_enter();
    using G = Geo<P>;
    extern __shared__ __align__(16) uint8_t sm[];
    MmaE<P, 1> &E = *reinterpret_cast<MmaE<P, 1> *>(sm);
    MmaA<P, 1> &A = *reinterpret_cast<MmaA<P, 1> *>(sm + sizeof(MmaE<P, 1>));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nth = blockDim.x, tid = threadIdx.x;
    int idx, base, n_in;
    lm_node(lm1, blockIdx.x, idx, base, n_in);
    if (2 * idx + 1 >= n_in) return;  // unpaired leaf: h = g inv(node) needs no s
    const int kl = base + 2 * idx;
    for (int side = 0; side < 2; ++side) {
        const int kg = kl + side, kf = kl + 1 - side;
        leaf_pair_s<P>(gbuf + (size_t)kg * G::pad, leaves + (size_t)kf * G::pad, E, A,
                       sbuf + (size_t)kg * G::pad, warp, lane, tid, nth);
    }
}

// h for the two keys under a level-1 node j of the product forest, whose
// inverse inv(P_j) the down-sweep leaves at its row (the leaf level of the
// down-sweep is not run).  With P_j = (3 f_L)(3 f_R),
//     1/(3 f_L) = inv(P_j) 3 f_R,   so   h_L = g_L / (3 f_L) = 3 inv(P_j) (g_L f_R),
// and likewise for R (Sec. 2.2's Montgomery trick, the last level folded into
// h).  s_L = g_L f_R has both operands small (one MMA per step); each output
// coefficient of a product mod x^p - x - 1 is d_j + d_{p+j} + d_{p+j-1} with
// the first two over disjoint parts of f's support, so |s_L| <= 2w and s_L
// goes into the second product as one f16 limb: two MMAs per step against
// inv(P_j)'s pair table, which is built once for both keys (FuseLeaf<P>
// checks that the limb sums stay below 2^24).  An unpaired leaf (a subtree of
// odd size) is its own level-1 node: h = g inv(node) directly.
template <int P>
__global__ void __launch_bounds__(32 * MmaGeo<P, 1>::NW)
k_finalize_pair(KeyMap km, const int8_t *__restrict__ gbuf, const int16_t *__restrict__ leaves,
                const int16_t *__restrict__ inv1, LevelMap lm1, int pk_bytes, int sk_bytes,
                int sk_pk_off, EncSched S, const int16_t *__restrict__ sbuf) {
    pdl_enter();
    using G = Geo<P>;
    using M = MmaGeo<P, 1>;
    static_assert(FuseLeaf<P>::ok, "limb sums of the fused leaf level exceed 2^24");
    static_assert(2 * G::pad * sizeof(uint32_t) + 1344 <= sizeof(MmaE<P, 1>), "encode buffers");
    extern __shared__ __align__(16) uint8_t sm[];
    MmaE<P, 1> &E = *reinterpret_cast<MmaE<P, 1> *>(sm);
    MmaA<P, 1> *A = reinterpret_cast<MmaA<P, 1> *>(sm + sizeof(MmaE<P, 1>));
    int16_t(*sv)[G::pad] =
        reinterpret_cast<int16_t(*)[G::pad]>(sm + sizeof(MmaE<P, 1>) + 2 * sizeof(MmaA<P, 1>));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nth = blockDim.x, tid = threadIdx.x;
    const int j = blockIdx.x;
    int idx, base, n_in;
    lm_node(lm1, j, idx, base, n_in);
    const int kl = base + 2 * idx;  // leaf rows are key indices
    const bool paired = 2 * idx + 1 < n_in;
    const int16_t *ip = inv1 + (size_t)j * G::pad;
    if (paired) {
        const int16_t *s0 = sv[0], *s1 = sv[1];
        if (sbuf) {  // formed ahead by k_leaf_s
            s0 = sbuf + (size_t)kl * G::pad;
            s1 = sbuf + (size_t)(kl + 1) * G::pad;
        } else {
            for (int side = 0; side < 2; ++side)  // s = g_kg f_kf
                leaf_pair_s<P>(gbuf + (size_t)(kl + side) * G::pad,
                               leaves + (size_t)(kl + 1 - side) * G::pad, E, A[0], sv[side], warp,
                               lane, tid, nth);
        }
        // h' = inv(P_j) s for both keys, one pair table of inv(P_j)
        mma_fill_b<P, 1>(ip, E, tid, nth);
        mma_fill_a_wide<P, 1>(s0, A[0], tid, nth);
        mma_fill_a_wide<P, 1>(s1, A[1], tid, nth);
        __syncthreads();
        mma_fill_pe<P, 1, MODE_GEN>(E, tid, nth);
        __syncthreads();
        float acc[1][2][3][4];
        const MmaA<P, 1> *const As[2] = {&A[0], &A[1]};
        mma_tiles<P, 1, 2, MODE_SA>(E, As, warp, lane, acc);
        const int bl = (int)E.b[M::p - 1];
        __syncthreads();
        mma_stage<P, 1, 2, MODE_SA>(A[0], warp, lane, 0, acc);
        mma_stage<P, 1, 2, MODE_SA>(A[1], warp, lane, 1, acc);
        __syncthreads();
        // h for both keys: key L's encode buffers over E, key R's over the
        // vector records (written after every read of A, through registers)
        uint32_t(*Rb0)[G::pad] = reinterpret_cast<uint32_t(*)[G::pad]>(sm);
        uint8_t *ob0 = sm + 2 * G::pad * sizeof(uint32_t);
        uint32_t(*Rb1)[G::pad] = reinterpret_cast<uint32_t(*)[G::pad]>(sm + sizeof(MmaE<P, 1>));
        uint8_t *ob1 = sm + sizeof(MmaE<P, 1>) + 2 * G::pad * sizeof(uint32_t);
        static_assert(2 * G::pad * sizeof(uint32_t) + 1344 <= 2 * sizeof(MmaA<P, 1>) + 2 * G::pad * sizeof(int16_t),
                      "second encode buffer");
        constexpr int KPT = (P + 32 * MmaGeo<P, 1>::NW - 1) / (32 * MmaGeo<P, 1>::NW);
        uint32_t hr[KPT];
#pragma unroll
        for (int u = 0; u < KPT; ++u) {
            const int k = tid + u * nth;
            if (k < P) {
                int vl = (k == 0) ? A[0].u.stage[0] - A[0].u.stage[stage_slot(P - 1)] + (int)A[0].a[0] * bl
                                  : A[0].u.stage[stage_slot(k)] + (int)A[0].a[k] * bl;
                int vr = (k == 0) ? A[1].u.stage[0] - A[1].u.stage[stage_slot(P - 1)] + (int)A[1].a[0] * bl
                                  : A[1].u.stage[stage_slot(k)] + (int)A[1].a[k] * bl;
                Rb0[0][k] = (uint32_t)(cmod<G::q>(3 * cmod<G::q>(vl)) + G::half);
                hr[u] = (uint32_t)(cmod<G::q>(3 * cmod<G::q>(vr)) + G::half);
            }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < KPT; ++u) {
            const int k = tid + u * nth;
            if (k < P) Rb1[0][k] = hr[u];
        }
        __syncthreads();
        mixed_encode2<G::pad>(Rb0, Rb1, S, ob0, ob1);
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const int key = kl + side;
            const uint8_t *ob = side ? ob1 : ob0;
            const BatchDesc d = key_batch(km, key);
            uint8_t *pkk = d.pk + (size_t)(key - d.key_base) * pk_bytes;
            uint8_t *skk = d.sk + (size_t)(key - d.key_base) * sk_bytes + sk_pk_off;
            for (int b = tid; b < pk_bytes; b += nth) {
                pkk[b] = ob[b];
                skk[b] = ob[b];
            }
        }
        return;
    }
    // unpaired leaf: h = g * inv(node), as k_finalize_mma
    mma_fill_a<P, 1, MODE_SA>(gbuf + (size_t)kl * G::pad, A[0], tid, nth);
    mma_fill_b<P, 1>(ip, E, tid, nth);
    __syncthreads();
    mma_fill_pe<P, 1, MODE_GEN>(E, tid, nth);
    __syncthreads();
    float acc[1][1][3][4];
    const MmaA<P, 1> *const As[1] = {&A[0]};
    mma_tiles<P, 1, 1, MODE_SA>(E, As, warp, lane, acc);
    const int bl = (int)E.b[M::p - 1];
    __syncthreads();
    mma_stage<P, 1, 1, MODE_SA>(A[0], warp, lane, 0, acc);
    __syncthreads();
    uint32_t(*Rb)[G::pad] = reinterpret_cast<uint32_t(*)[G::pad]>(sm);
    uint8_t *ob = sm + 2 * G::pad * sizeof(uint32_t);
    for (int k = tid; k < P; k += nth) {
        int v = (k == 0) ? A[0].u.stage[0] - A[0].u.stage[stage_slot(P - 1)] + (int)A[0].a[0] * bl
                         : A[0].u.stage[stage_slot(k)] + (int)A[0].a[k] * bl;
        Rb[0][k] = (uint32_t)(cmod<G::q>(v) + G::half);
    }
    __syncthreads();
    mixed_encode<G::pad>(Rb, S, ob);
    const BatchDesc d = key_batch(km, kl);
    uint8_t *pkk = d.pk + (size_t)(kl - d.key_base) * pk_bytes;
    uint8_t *skk = d.sk + (size_t)(kl - d.key_base) * sk_bytes + sk_pk_off;
    for (int b = tid; b < pk_bytes; b += nth) {
        pkk[b] = ob[b];
        skk[b] = ob[b];
    }
}

// Fix-up of the keys whose g needed another attempt (deferred R/3 kernel):
// h = g * (3f)^-1 with the final g, Rq_encode into pk and sk, and the hash
// of the new pk into sk.  Runs after the h, hash and R/3 kernels of the call;
// CTAs take list entries in turn, so an empty list costs one read.  With
// leaves (the fused leaf level), ainv holds the level-1 inverses and
// (3f)^-1 = inv(node) * (3f of the sibling leaf) is formed here first.
template <int P>
__global__ void __launch_bounds__(Tp<P>::NT)
k_fixup(KeyMap km, const int *__restrict__ fix_count, const int *__restrict__ fix_keys,
        const int8_t *__restrict__ gfix, const int16_t *__restrict__ ainv, int pk_bytes,
        int sk_bytes, int sk_pk_off, int hash_off, EncSched S,
        const int16_t *__restrict__ leaves, LevelMap lm1, bool hash_here) {
    pdl_enter();
    using G = Geo<P>;
    __shared__ __align__(16) int As[Tp<P>::p8];
    __shared__ __align__(16) int Es[Tp<P>::ESZ];
    __shared__ uint32_t Rb[2][G::pad];
    __shared__ uint8_t ob[1344];
    __shared__ __align__(16) int16_t ik[G::pad];
    const int n = *fix_count;
    for (int f = blockIdx.x; f < n; f += gridDim.x) {
        const int key = fix_keys[f];
        const int16_t *inv = ainv + (size_t)key * G::pad;
        __syncthreads();  // shared buffers free from the previous entry
        if (leaves) {
            // leaf row key: tree b, index i in it; level-1 node (first node
            // of b) + i / 2; equal subtrees or (nb > 0) a forest of batches
            int b, i, first_leaf, n_leaf, first_node;
            if (lm1.nb > 0) {
                b = level_batch(lm1.pre_in, lm1.nb, key);
                first_leaf = lm1.pre_in[b];
                n_leaf = lm1.pre_in[b + 1] - first_leaf;
                first_node = lm1.pre_out[b];
            } else {
                b = key / lm1.n_in;
                first_leaf = b * lm1.n_in;
                n_leaf = lm1.n_in;
                first_node = b * lm1.sub_out;
            }
            i = key - first_leaf;
            const int16_t *node = ainv + (size_t)(first_node + i / 2) * G::pad;
            const int sib = i ^ 1;
            if (sib < n_leaf) {
                fill_A<P>(leaves + (size_t)(first_leaf + sib) * G::pad, As);
                fill_E<P>(node, Es);
                __syncthreads();
                int acc[1][8];
                const int *const A1[1] = {As};
                toeplitz_tile<P, 1>(A1, Es, threadIdx.x, 0, Tp<P>::p8, acc);
                const int bl[1] = {(int)node[P - 1]};
                toeplitz_finish<P, 1>(A1, bl, acc, threadIdx.x, true);
                const int j0 = 8 * threadIdx.x;
#pragma unroll
                for (int t = 0; t < 8; ++t)
                    if (j0 + t < G::pad) ik[j0 + t] = (int16_t)(j0 + t < P ? acc[0][t] : 0);
                inv = ik;
            } else {
                inv = node;  // unpaired: the node is the leaf
            }
            __syncthreads();
        }
        fill_A<P>(gfix + (size_t)f * G::pad, As);
        fill_E<P>(inv, Es);
        __syncthreads();
        int acc[1][8];
        const int *const A1[1] = {As};
        toeplitz_tile<P, 1>(A1, Es, threadIdx.x, 0, Tp<P>::p8, acc);
        const int bl[1] = {(int)inv[P - 1]};
        toeplitz_finish<P, 1>(A1, bl, acc, threadIdx.x, true);
        const int j0 = 8 * threadIdx.x;
#pragma unroll
        for (int t = 0; t < 8; ++t)
            if (j0 + t < P) Rb[0][j0 + t] = (uint32_t)(acc[0][t] + G::half);
        __syncthreads();
        mixed_encode<G::pad>(Rb, S, ob);
        const BatchDesc d = key_batch(km, key);
        uint8_t *pkk = d.pk + (size_t)(key - d.key_base) * pk_bytes;
        uint8_t *skk = d.sk + (size_t)(key - d.key_base) * sk_bytes;
        for (int b = threadIdx.x; b < pk_bytes; b += blockDim.x) {
            pkk[b] = ob[b];
            skk[sk_pk_off + b] = ob[b];
        }
        if (hash_here && threadIdx.x == 0) sha512_prefixed(4, ob, pk_bytes, nullptr, 0, skk + hash_off);
    }
}

// ---------------------------------------------------------------------------
// SHA-512 (FIPS 180-4) of 0x04 | pk, first 32 bytes into the secret key
// (Hash_prefix(4, pk) of the NTRU Prime secret key).
// ---------------------------------------------------------------------------



// Named barriers between the two warps of the pk-hash kernel.
__device__ __forceinline__ void nbar_sync(int id, int n) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void nbar_arrive(int id, int n) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// Two warps hash 32 keys, one key per lane, after copying the 32 public
// keys to shared memory (runs of contiguous rows, see below).
//
// A block's 80 rounds form one serial chain per key, and a single warp runs
// the whole compression at about three cycles per instruction, so the work
// is split by dependency: warp 1 (producer) reads the message 0x04 | pk_j of
// its lane byte by byte (the padding 0x80, zeros and 128-bit big-endian bit
// length generated), expands the schedule and writes W_t + K_t for the 80
// rounds into one of two table slots; warp 0 (consumer) runs the rounds from
// the table.  Named barriers 1, 2 mark slot 0, 1 full, 3, 4 mark it free
// again; each is used in a fixed order by both warps, once per block.
constexpr int kShaWkBytes = 2 * 80 * 32 * 8;
// rows of 32 public keys; a run starts at most 15 + 15 bytes after the
// previous run's end (rounding up to 16, then its source's phase)
constexpr int sha_blk_bytes(int pk_bytes) { return 32 * pk_bytes + 32 * 32; }
constexpr int kShaBlkMax = sha_blk_bytes(1322);  // the opt-in size: sntrup857's 1322-byte pk

// With list != null the CTA's keys are list[base .. base + 31] of the first
// *list_n entries (the fix-up's list): the list is another kernel's output,
// so the kernel waits for its predecessors first, and a CTA past the list's
// end does nothing.
//
// The kernel is compiled per public-key size: with the message length a
// constant the producer's per-block word assembly folds to a short
// instruction stream, and the producer, which sets the pace of the pair, keeps
// up with the rounds warp (a run-time length made both warps about 40%
// slower, measured on sntrup761).
template <int PKB>
__global__ void __launch_bounds__(64, 1)
k_sha512_pk(KeyMap km, int B, int sk_bytes, int hash_off, const int *__restrict__ list,
            const int *__restrict__ list_n) {
    constexpr int pk_bytes = PKB;
    extern __shared__ __align__(16) uint8_t sm[];
    uint64_t(*wk)[80][32] = reinterpret_cast<uint64_t(*)[80][32]>(sm);  // [slot][round][key]
    __shared__ uint64_t ks[80];  // the round constants
    for (int i = threadIdx.x; i < 80; i += 64) ks[i] = c_sha512_k[i];
    uint8_t *blk = sm + kShaWkBytes;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int base = blockIdx.x * 32;
    if (list) {
        pdl_enter();
        B = min(B, *list_n);
        if (base >= B) return;  // CTA-uniform
    }
    const int nkeys = min(32, B - base);
    // key of lane j of this CTA
    auto key_of = [&](int j) { return list ? list[base + j] : base + j; };
    // The keys form runs whose rows are contiguous in device memory (one run
    // for a single batch).  A run goes to a shared-memory offset congruent
    // to its source address mod 16, so that its middle moves in aligned
    // 16-byte words and only its two ends bytewise; rowoff[j] is the offset
    // of key base + j's row.  Warp 0 finds the runs, a lane per key.
    __shared__ int rowoff[32];
    __shared__ const uint8_t *run_src[32];
    __shared__ int run_dst[32], run_first[33];
    __shared__ int nruns;
    if (warp == 0) {
        uintptr_t row = 0;
        if (lane < nkeys) {
            const int key = key_of(lane);
            const BatchDesc d = key_batch(km, key);
            row = reinterpret_cast<uintptr_t>(d.pk + (size_t)(key - d.key_base) * pk_bytes);
        }
        const uintptr_t prev = __shfl_up_sync(0xffffffffu, (unsigned long long)row, 1);
        const bool start = lane < nkeys && (lane == 0 || row != prev + (uintptr_t)pk_bytes);
        const unsigned starts = __ballot_sync(0xffffffffu, start);
        const int r = __popc(starts & (0xffffffffu >> (31 - lane))) - 1;  // this lane's run
        if (start) {
            run_src[r] = reinterpret_cast<const uint8_t *>(row);
            run_first[r] = lane;
        }
        __syncwarp();
        if (lane == 0) {
            const int n = __popc(starts);
            run_first[n] = nkeys;
            int off = 0;
            for (int q = 0; q < n; ++q) {
                off = ((off + 15) & ~15) + (int)(reinterpret_cast<uintptr_t>(run_src[q]) & 15);
                run_dst[q] = off;
                off += (run_first[q + 1] - run_first[q]) * pk_bytes;
            }
            nruns = n;
        }
        __syncwarp();
        if (lane < nkeys) rowoff[lane] = run_dst[r] + (lane - run_first[r]) * pk_bytes;
    }
    // the row lookups above read only the batch table (and the list, after
    // the wait); the rows themselves are the previous kernel's output
    if (!list) pdl_enter();
    __syncthreads();
    for (int q = 0; q < nruns; ++q) {
        const uint8_t *src = run_src[q];
        uint8_t *dst = blk + run_dst[q];
        const int len = (run_first[q + 1] - run_first[q]) * pk_bytes;
        const int head = min(len, (int)((16 - (reinterpret_cast<uintptr_t>(src) & 15)) & 15));
        const int n16 = (len - head) / 16;
        // the middle as asynchronous 16-byte copies: all in flight at once
        // (a load / store loop through registers would wait for each load,
        // the compiler not knowing that the two buffers never overlap)
        const uint32_t d16 = (uint32_t)__cvta_generic_to_shared(dst + head);
        for (int i = tid; i < n16; i += 64)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d16 + 16u * (uint32_t)i),
                         "l"(src + head + 16 * (size_t)i)
                         : "memory");
        for (int i = tid; i < head; i += 64) dst[i] = src[i];
        for (int i = head + 16 * n16 + tid; i < len; i += 64) dst[i] = src[i];
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    constexpr int len = pk_bytes + 1;
    constexpr int nblk = (len + 1 + 16 + 127) / 128;
    if (warp == 1) {
        // lanes past the last key repeat it; their digests are not stored
        const uint8_t *row = blk + rowoff[min(lane, nkeys - 1)];  // byte pos (1..pk_bytes) at row[pos - 1]
        const uint64_t bitlen = (uint64_t)len * 8u;
        for (int b0 = 0; b0 < nblk; ++b0) {
            const int slot = b0 & 1;
            if (b0 >= 2) nbar_sync(3 + slot, 64);
            uint64_t W[16];
#pragma unroll
            for (int t = 0; t < 16; ++t) {
                const int pos = 128 * b0 + 8 * t;
                uint64_t v = 0;
                if (pos >= 1 && pos + 8 <= len) {
                    // message bytes pos .. pos + 7 = row bytes pos - 1 .. pos + 6,
                    // big-endian: three aligned words (at most 4 bytes past the
                    // row, inside the buffer's slack), funnel-shifted, reversed
                    const uintptr_t at = reinterpret_cast<uintptr_t>(row + pos - 1);
                    const uint32_t *a0 = reinterpret_cast<const uint32_t *>(at & ~(uintptr_t)3);
                    const uint32_t sh = 8u * (uint32_t)(at & 3u);
                    const uint32_t w0 = a0[0], w1 = a0[1], w2 = a0[2];
                    const uint32_t lo = __funnelshift_r(w0, w1, sh), hi = __funnelshift_r(w1, w2, sh);
                    v = ((uint64_t)__byte_perm(lo, 0, 0x0123) << 32) | __byte_perm(hi, 0, 0x0123);
                } else {
#pragma unroll
                    for (int b = 0; b < 8; ++b) {
                        const int q = pos + b;
                        uint32_t byte = 0;
                        if (q == 0) byte = 4u;
                        else if (q < len) byte = row[q - 1];
                        else if (q == len) byte = 0x80u;
                        else if (q >= nblk * 128 - 8) byte = (uint32_t)(bitlen >> (8 * (nblk * 128 - 1 - q))) & 255u;
                        v = (v << 8) | byte;
                    }
                }
                W[t] = v;
            }
#pragma unroll 1
            for (int r = 0; r < 80; r += 16) {
#pragma unroll
                for (int tt = 0; tt < 16; ++tt) {
                    if (r > 0) {
                        const uint64_t w15 = W[(tt + 1) & 15], w2 = W[(tt + 14) & 15];
                        const uint64_t s0 = rotr(w15, 1) ^ rotr(w15, 8) ^ (w15 >> 7);
                        const uint64_t s1 = rotr(w2, 19) ^ rotr(w2, 61) ^ (w2 >> 6);
                        W[tt] += s0 + W[(tt + 9) & 15] + s1;
                    }
                    wk[slot][r + tt][lane] = W[tt] + ks[r + tt];
                }
            }
            nbar_arrive(1 + slot, 64);
        }
        return;
    }
    uint64_t H[8] = {0x6a09e667f3bcc908ULL, 0xbb67ae8584caa73bULL, 0x3c6ef372fe94f82bULL,
                     0xa54ff53a5f1d36f1ULL, 0x510e527fade682d1ULL, 0x9b05688c2b3e6c1fULL,
                     0x1f83d9abfb41bd6bULL, 0x5be0cd19137e2179ULL};
    for (int b0 = 0; b0 < nblk; ++b0) {
        const int slot = b0 & 1;
        nbar_sync(1 + slot, 64);
        sha512_rounds_wk(H, wk[slot], lane);
        if (b0 + 2 < nblk) nbar_arrive(3 + slot, 64);
    }
    if (lane >= nkeys) return;
    const int key = key_of(lane);
    const BatchDesc dk = key_batch(km, key);
    uint8_t *out = dk.sk + (size_t)(key - dk.key_base) * sk_bytes + hash_off;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int b = 0; b < 8; ++b) out[8 * i + b] = (uint8_t)(H[i] >> (56 - 8 * b));
}

template <int P>
cudaError_t launch_finalize(const KeyMap &km, int nkeys, const int8_t *gbuf, const int16_t *ainv,
                            int pk_bytes, int sk_bytes, int sk_pk_off, const EncSched &S,
                            cudaStream_t st, bool mma) {
    if (mma) {
        const size_t sm = sizeof(MmaE<P, 1>) + sizeof(MmaA<P, 1>);
        if (sm > 48 * 1024) {
            const cudaError_t e = cudaFuncSetAttribute(
                k_finalize_mma<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e != cudaSuccess) return e;
        }
        SNT_LAUNCH(k_finalize_mma<P>, nkeys, 32 * MmaGeo<P, 1>::NW, sm, st, km, gbuf, ainv,
            pk_bytes, sk_bytes, sk_pk_off, S);
    } else {
        SNT_LAUNCH(k_finalize<P>, nkeys, Tp<P>::NT, 0, st, km, gbuf, ainv, pk_bytes, sk_bytes,
            sk_pk_off, S);
    }
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_fixup(const KeyMap &km, const int *fix_count, const int *fix_keys,
                         const int8_t *gfix, const int16_t *ainv, int pk_bytes, int sk_bytes,
                         int sk_pk_off, int hash_off, const EncSched &S, cudaStream_t st,
                         const int16_t *leaves, LevelMap lm1, int grid, int nkeys) {
    // sntrup653 redraws about one g in 27: its fix-up hashes the new public
    // keys afterwards a lane per key; for the others (a redraw about once in
    // 3^19 keys) each fix-up CTA hashes its key itself
    const bool hash_here = P != 653;
    SNT_LAUNCH(k_fixup<P>, grid, Tp<P>::NT, 0, st, km, fix_count, fix_keys, gfix, ainv, pk_bytes,
        sk_bytes, sk_pk_off, hash_off, S, leaves, lm1, hash_here);
    if (!hash_here) {
        const cudaError_t e = launch_sha512_pk(km, nkeys, pk_bytes, sk_bytes, hash_off, st,
                                               fix_keys, fix_count);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_finalize_pair(const KeyMap &km, int n1, const int8_t *gbuf,
                                 const int16_t *leaves, const int16_t *inv1, LevelMap lm1,
                                 int pk_bytes, int sk_bytes, int sk_pk_off, const EncSched &S,
                                 cudaStream_t st, const int16_t *sbuf) {
    if constexpr (!FuseLeaf<P>::ok) {
        return cudaErrorNotSupported;
    } else {
        const size_t sm = sizeof(MmaE<P, 1>) + 2 * sizeof(MmaA<P, 1>) + 2 * Geo<P>::pad * sizeof(int16_t);
        if (sm > 48 * 1024) {
            const cudaError_t e = cudaFuncSetAttribute(
                k_finalize_pair<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e != cudaSuccess) return e;
        }
        SNT_LAUNCH(k_finalize_pair<P>, n1, 32 * MmaGeo<P, 1>::NW, sm, st, km, gbuf, leaves, inv1,
            lm1, pk_bytes, sk_bytes, sk_pk_off, S, sbuf);
        return cudaGetLastError();
    }
}

template <int P>
cudaError_t launch_leaf_s(int n1, const int8_t *gbuf, const int16_t *leaves, LevelMap lm1,
                          int16_t *sbuf, cudaStream_t st) {
    if constexpr (!FuseLeaf<P>::ok) {
        return cudaErrorNotSupported;
    } else {
        const size_t sm = sizeof(MmaE<P, 1>) + sizeof(MmaA<P, 1>);
        SNT_LAUNCH(k_leaf_s<P>, n1, 32 * MmaGeo<P, 1>::NW, sm, st, gbuf, leaves, lm1, sbuf);
        return cudaGetLastError();
    }
}

template <int PKB>
static cudaError_t launch_sha512_pk_t(const KeyMap &km, int nkeys, int sk_bytes, int hash_off,
                                      cudaStream_t st, const int *list, const int *list_n) {
    constexpr int smem = kShaWkBytes + sha_blk_bytes(PKB);
    static_assert(smem <= kShaWkBytes + kShaBlkMax, "public key larger than the opt-in size");
    // the opt-in above 48 KB, once per device (host state, not stream work)
    static std::atomic<uint64_t> opted{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (!(opted.load() & (1ull << (dev & 63)))) {
        e = cudaFuncSetAttribute(k_sha512_pk<PKB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        opted.fetch_or(1ull << (dev & 63));
    }
    SNT_LAUNCH(k_sha512_pk<PKB>, (nkeys + 31) / 32, 64, smem, st, km, nkeys, sk_bytes, hash_off,
        list, list_n);
    return cudaGetLastError();
}

cudaError_t launch_sha512_pk(const KeyMap &km, int nkeys, int pk_bytes, int sk_bytes,
                             int hash_off, cudaStream_t st, const int *list, const int *list_n) {
    switch (pk_bytes) {  // Rq_encode sizes of sntrup653, sntrup761, sntrup857
    case 994: return launch_sha512_pk_t<994>(km, nkeys, sk_bytes, hash_off, st, list, list_n);
    case 1158: return launch_sha512_pk_t<1158>(km, nkeys, sk_bytes, hash_off, st, list, list_n);
    case 1322: return launch_sha512_pk_t<1322>(km, nkeys, sk_bytes, hash_off, st, list, list_n);
    default: return cudaErrorInvalidValue;
    }
}

#define SNT_FIN_INST(P)                                                                       \
    template cudaError_t launch_finalize<P>(const KeyMap &, int, const int8_t *, const int16_t *, \
                                            int, int, int, const EncSched &, cudaStream_t, bool); \
    template cudaError_t launch_fixup<P>(const KeyMap &, const int *, const int *, const int8_t *, \
                                         const int16_t *, int, int, int, int, const EncSched &,   \
                                         cudaStream_t, const int16_t *, LevelMap, int, int);      \
    template cudaError_t launch_finalize_pair<P>(const KeyMap &, int, const int8_t *,            \
                                                 const int16_t *, const int16_t *, LevelMap, int, \
                                                 int, int, const EncSched &, cudaStream_t,        \
                                                 const int16_t *);                                \
    template cudaError_t launch_leaf_s<P>(int, const int8_t *, const int16_t *, LevelMap,        \
                                          int16_t *, cudaStream_t);
SNT_FIN_INST(653)
SNT_FIN_INST(761)
SNT_FIN_INST(857)

}  // namespace snt
