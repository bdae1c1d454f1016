// host_plan.h -- host-side planning shared by the C-ABI entry points
// (internal): parameter sizes, the Rq_encode schedule, the product-tree
// layout, scratch sizes, device selection and the per-thread error string.
#pragma once
#include <cstdarg>
#include <cstdint>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "sntrup_gb300.h"

namespace snt {

// Defaults of the tuning options (snt_ctx_set_option).
constexpr int kDefaultR3Lanes = 4;     // lanes per element of the R/3 divstep kernel
constexpr int kDefaultTreeSplit = 8;   // largest split of one product over thread groups
constexpr int kDefaultR3Overlap = 1;   // R/3 on its own stream beside the tree
constexpr int kDefaultNarrowSeg = 1;   // output-split narrow tree levels
constexpr int kDefaultRqEngine = 1;    // R/q products on the tensor cores
constexpr int kDefaultMmaTiles = 1;    // MMA tiles per warp
constexpr int kDefaultR3Kpt = 1;       // R/3 elements per lane group
constexpr int kDefaultMmaKsplit = 4;   // K-split of narrow tensor-core levels
constexpr int kDefaultRoots = 1;       // subtrees (root inversions) per batch
constexpr int kDefaultR3Mode = 0;      // 0 per-key R/3 divsteps, 1 R/3 batch inversion

// Records a one-line error message (snt_last_error_string) and returns s.
snt_status set_error(snt_status s, const char *fmt, ...);

// Rq_encode schedule (see encode.cu) for p entries of radix m.
inline bool build_sched(int p, uint32_t m0, EncSched &S) {
    std::memset(&S, 0, sizeof(S));
    int n = p, off = 0;
    uint64_t mu = m0, ml = m0;
    while (n > 1) {
        if (S.nlev >= 16) return false;
        EncLevel &L = S.lev[S.nlev++];
        L.n = n;
        L.mu = (uint32_t)mu;
        L.mlast = (uint32_t)ml;
        L.boff = off;
        uint64_t m = mu * mu;
        int eu = 0;
        while (m >= 16384) { ++eu; m = (m + 255) >> 8; }
        const uint64_t mu2 = m;
        uint64_t ml2 = ml;
        int el = eu;
        const int npairs = n / 2;
        if (n % 2 == 0) {
            uint64_t m2 = mu * ml;
            el = 0;
            while (m2 >= 16384) { ++el; m2 = (m2 + 255) >> 8; }
            ml2 = m2;
            off += (npairs - 1) * eu + el;
        } else {
            off += npairs * eu;
        }
        L.eu = eu;
        L.elast = el;
        n = (n + 1) / 2;
        mu = mu2;
        ml = ml2;
    }
    int e = 0;
    for (uint64_t m = ml; m > 1; m = (m + 255) >> 8) ++e;
    S.efinal = e;
    S.mfinal = (uint32_t)ml;
    S.foff = off;
    S.total = off + e;
    return true;
}

struct ParamInfo {
    int P, p, q, w, pad;
    int small_bytes, pk_bytes, sk_bytes, ct_bytes;
    EncSched sched;   // Rq_encode (radix q)
    EncSched rsched;  // Rounded_encode (radix (q+2)/3)
};

inline bool param_info(int P, ParamInfo &pi) {
    int p, q, w, pad;
    switch (P) {
        case 653: p = Geo<653>::p; q = Geo<653>::q; w = Geo<653>::w; pad = Geo<653>::pad; break;
        case 761: p = Geo<761>::p; q = Geo<761>::q; w = Geo<761>::w; pad = Geo<761>::pad; break;
        case 857: p = Geo<857>::p; q = Geo<857>::q; w = Geo<857>::w; pad = Geo<857>::pad; break;
        default: return false;
    }
    pi.P = P; pi.p = p; pi.q = q; pi.w = w; pi.pad = pad;
    pi.small_bytes = (p + 3) / 4;
    if (!build_sched(p, (uint32_t)q, pi.sched)) return false;
    pi.pk_bytes = pi.sched.total;
    // sk = Small_encode(f) | Small_encode(1/g) | pk | rho | Hash_prefix(4, pk)
    pi.sk_bytes = 3 * pi.small_bytes + pi.pk_bytes + 32;
    // ct = Rounded encoding (radix (q+2)/3) | 32-byte confirmation hash
    if (!build_sched(p, (uint32_t)((q + 2) / 3), pi.rsched)) return false;
    pi.ct_bytes = pi.rsched.total + 32;
    return true;
}

// CTAs of the fix-up of redrawn keys for a call of n keys: the list is
// usually empty (a zero divisor among the first draws has probability
// 3^-19 per key for sntrup761), but x^653 - x - 1 has a factor of degree 3
// over F_3, so about one sntrup653 key in 27 is redrawn.  A CTA spends most
// of an entry's time in the single-thread hash of the new public key, so
// the grid (n / 16, up to 16 CTAs per SM) gives every expected entry a CTA
// of its own; CTAs without an entry exit after one read.
inline int fixup_grid(size_t n) {
    const size_t g = n / 16;
    return (int)(g < 8 ? 8 : g > 2432 ? 2432 : g);
}

// Product-tree levels over B leaves: level 0 = leaves, level l has
// ceil(n_(l-1) / 2) nodes, the last level has one.  Offsets in nodes.
struct Tree {
    std::vector<int> n, off;
    size_t total = 0;
};

inline Tree make_tree(size_t B) {
    Tree t;
    size_t n = B, off = 0;
    for (;;) {
        t.n.push_back((int)n);
        t.off.push_back((int)off);
        off += n;
        if (n == 1) break;
        n = (n + 1) / 2;
    }
    t.total = off;
    return t;
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// A batch as K equal subtrees side by side (Montgomery's trick per subtree,
// K root inversions in one launch): K is the largest power of two <= k_req
// that divides B and whose forest fits the single tree's node rows.  n[l]
// and off[l] count the whole level; sub[l] nodes of it belong to each
// subtree.  K = 1 is the single tree.
struct Forest {
    int K = 1;
    Tree t;
    std::vector<int> sub;
};

inline Forest make_forest(size_t B, int k_req) {
    const size_t single = make_tree(B).total;
    int K = 1;
    while (2 * K <= k_req && B % (size_t)(2 * K) == 0 &&
           (size_t)(2 * K) * make_tree(B / (2 * K)).total <= single)
        K *= 2;
    Forest f;
    f.K = K;
    const Tree s = make_tree(B / K);
    size_t off = 0;
    for (size_t l = 0; l < s.n.size(); ++l) {
        f.sub.push_back(s.n[l]);
        f.t.n.push_back(K * s.n[l]);
        f.t.off.push_back((int)off);
        off += (size_t)K * s.n[l];
    }
    f.t.total = off;
    return f;
}

// Scratch bytes for one keygen call: every tree node (int16, stride pad) and
// g (int8, stride pad) for each key; host_out adds device staging for pk/sk.
inline size_t keygen_scratch(const ParamInfo &pi, size_t B, bool host_out) {
    const Tree t = make_tree(B);
    size_t bytes = align256(t.total * pi.pad * sizeof(int16_t)) + align256(B * pi.pad);
    if (host_out) bytes += align256(B * pi.pk_bytes) + align256(B * pi.sk_bytes);
    return bytes;
}

// Arena bytes of a keygen call through a context: the scratch above plus two
// ping-pong level buffers for the output-split narrow levels of the
// down-sweep (at most 2 * kSegMaxNodes children per level), placed after it.
inline size_t narrow_scratch(const ParamInfo &pi) {
    return 2 * align256((size_t)2 * kSegMaxNodes * pi.pad * sizeof(int16_t));
}
// ... then the resampling list of the deferred R/3 kernel: a count, B key
// indices, B slot indices by key (the R/3 screen's, for the per-key
// fall-back) and B rows of g (int8, stride pad).
inline size_t fix_list_bytes(size_t B) { return align256(sizeof(int) * (1 + 2 * B)); }
inline size_t fix_scratch(const ParamInfo &pi, size_t B) {
    return fix_list_bytes(B) + align256(B * pi.pad);
}
// ... then the R/3 batch inversion's tree (int16 rows, like the R/q tree)
// and its subtree roots' invertibility flags.
constexpr size_t kR3OkBytes = 4 * 1024;
inline size_t r3_scratch(const ParamInfo &pi, size_t B) {
    return align256(make_tree(B).total * pi.pad * sizeof(int16_t)) + kR3OkBytes;
}
// ... then the leaf-pair products s = g_L f_R, g_R f_L of the fused leaf
// level (int16 rows, stride pad, one per key).
inline size_t s_scratch(const ParamInfo &pi, size_t B) {
    return align256(B * pi.pad * sizeof(int16_t));
}
inline size_t keygen_arena(const ParamInfo &pi, size_t B, bool host_out) {
    return keygen_scratch(pi, B, host_out) + narrow_scratch(pi) + fix_scratch(pi, B) +
           r3_scratch(pi, B) + s_scratch(pi, B);
}
// Arena layout of a context keygen call: tree nodes, g rows, the ping-pong
// buffers, the resampling list, then (host-buffer calls) the pk and sk
// staging at this offset.
inline size_t fix_offset(const ParamInfo &pi, size_t B) {
    return keygen_scratch(pi, B, false) + narrow_scratch(pi);
}
inline size_t r3_offset(const ParamInfo &pi, size_t B) {
    return fix_offset(pi, B) + fix_scratch(pi, B);
}
inline size_t s_offset(const ParamInfo &pi, size_t B) {
    return r3_offset(pi, B) + r3_scratch(pi, B);
}
inline size_t staging_offset(const ParamInfo &pi, size_t B) {
    return s_offset(pi, B) + s_scratch(pi, B);
}

struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && cudaSetDevice(dev) == cudaSuccess) ok = true;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// Batch keygen of B keys into pk / sk entirely on `stream` (no fork onto
// the context's own streams), for background refills of the serving pool.
snt_status keygen_into(snt_ctx *ctx, int P, uint64_t seed, uint64_t first, size_t B, uint8_t *pk,
                       uint8_t *sk, cudaStream_t stream);

}  // namespace snt
