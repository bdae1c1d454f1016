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
// One batch of a keygen launch: key i of the batch has key index first + i
// and randomness seed `seed`; its leaf / g rows are rows key_base + i of the
// launch's arrays and its outputs go to pk + i * pk_bytes, sk + i * sk_bytes.
struct BatchDesc {
    uint64_t seed, first;
    int key_base, nkeys;
    uint8_t *pk, *sk;
};

// The keys of one launch: a single batch passed by value (nb == 0), or a
// device table of nb >= 1 batches in increasing key_base order.
struct KeyMap {
    BatchDesc one;
    const BatchDesc *tab;
    int nb;
};

// Level of a product-tree forest: the nodes of every batch at this level are
// contiguous, batch b owning nodes [pre_out[b], pre_out[b+1]) of the level and
// its children [pre_in[b], pre_in[b+1]) of the level below.  nb == 0: one
// tree, n_in children (the arrays are unused).
// Irreducible factors of x^p - x - 1 over F_3 for the invertibility test:
// factor i has degree deg[i] and `words` 32-coefficient words per bit plane
// (m: nonzero, then s: coefficient -1) at w + off[i].
constexpr int kMaxR3Factors = 8;
struct R3Factors {
    int n = 0, total_words = 0;
    int deg[kMaxR3Factors] = {}, words[kMaxR3Factors] = {}, off[kMaxR3Factors] = {};
    const uint32_t *w = nullptr;
};
// Remainder tables of the factors of degree <= kScreenMaxDeg: for factor j
// and 0 <= i < p, t[2 (j p + i)] and t[2 (j p + i) + 1] are the bit planes
// (coefficient nonzero, coefficient -1) of x^i mod m_j.
constexpr int kScreenMaxDeg = 16;
constexpr int kMaxScreen = 2;
struct R3Screen {
    int n = 0;
    const uint32_t *t = nullptr;
};

// Nodes of one tree level.  nb > 0: a forest of batches with per-level node
// prefix sums (pre_in / pre_out, nb + 1 entries each).  Otherwise equal
// subtrees side by side: sub_out nodes of this level per subtree, each with
// n_in children (sub_out = 0 or the whole level: a single tree).
struct LevelMap {
    const int *pre_in = nullptr, *pre_out = nullptr;
    int nb = 0, n_in = 0;
    int sub_out = 0;
};

// Items of an encapsulation / decapsulation launch: a device table of items
// (tab != nullptr) or contiguous arrays (item i at base + i * size, key
// index first + i for the encapsulation randomness).
struct EncItem {
    const uint8_t *pk;
    const uint8_t *cache;  // Hash_prefix(4, pk) if already known (the sk tail), else nullptr
    uint64_t k;
    uint8_t *ct, *ss;
};
struct EncMap {
    const EncItem *tab;
    const uint8_t *pk;
    uint64_t first, seed;
    uint8_t *ct, *ss;
};
struct DecItem {
    const uint8_t *sk, *ct;
    uint8_t *ss;
};
struct DecMap {
    const DecItem *tab;
    const uint8_t *sk, *ct;
    uint8_t *ss;
};

struct EncSched {
    int nlev;
    EncLevel lev[16];
    int efinal, foff;  // bytes of the single remaining entry and their offset
    uint32_t mfinal;   // radix of that entry
    int total;         // encoded length
};

inline KeyMap single_batch(uint64_t seed, uint64_t first, int B, uint8_t *pk, uint8_t *sk) {
    KeyMap km;
    km.one.seed = seed; km.one.first = first; km.one.key_base = 0; km.one.nkeys = B;
    km.one.pk = pk; km.one.sk = sk;
    km.tab = nullptr;
    km.nb = 0;
    return km;
}

inline LevelMap single_tree(int n_in) {
    LevelMap lm;
    lm.pre_in = nullptr; lm.pre_out = nullptr; lm.nb = 0; lm.n_in = n_in; lm.sub_out = 0;
    return lm;
}
// Level of a forest of equal subtrees: n_in children and sub_out nodes each.
inline LevelMap equal_subtrees(int n_in, int sub_out) {
    LevelMap lm = single_tree(n_in);
    lm.sub_out = sub_out;
    return lm;
}

// g_out (optional): also g's attempt-0 draw per key (int8, stride pad), with
// the injected test draws, and *fix_count = 0 (the resampling list);
// g16_out (optional): the same draw as int16 rows (leaves of the R/3 forest).
template <int P>
cudaError_t launch_sample_f(const KeyMap &km, int nkeys, int16_t *leaves, int sk_bytes,
                            int rho_off, cudaStream_t st, int8_t *g_out = nullptr,
                            const uint64_t *inj_idx = nullptr, const int8_t *inj_g = nullptr,
                            int n_inj = 0, int *fix_count = nullptr,
                            int16_t *g16_out = nullptr);
// gfix != null: deferred form (attempt 0 read from g_out, g_out untouched,
// resampled keys appended to fix_keys / gfix rows, *fix_count of them).
// sub_ok != null: fall-back form, only warps holding a key of a subtree
// (sub_size keys each) whose flag is 0 do any work.  fix_slot (optional): a
// key with fix_slot[key] >= 0 reuses that slot of the list instead of
// appending one.
template <int P>
cudaError_t launch_r3_keygen(const KeyMap &km, int nkeys, int8_t *g_out, int sk_bytes,
                             int sk_off, const uint64_t *inj_idx, const int8_t *inj_g, int n_inj,
                             int *err, cudaStream_t st, int lanes, int kpt = 1,
                             int8_t *gfix = nullptr, int *fix_count = nullptr,
                             int *fix_keys = nullptr, const int *sub_ok = nullptr,
                             int sub_size = 0, const int *fix_slot = nullptr);
template <int P>
cudaError_t launch_r3_inv(int n, const int8_t *g, int8_t *out, int32_t *ok, cudaStream_t st,
                          int lanes, int kpt = 1);
template <int P>
cudaError_t launch_tree_up(const int16_t *lin, const LevelMap &lm, int n_out, int16_t *lout,
                           cudaStream_t st, int max_split);
template <int P>
cudaError_t launch_tree_down(const int16_t *lpar, const LevelMap &lm, int n_par, int16_t *lch,
                             cudaStream_t st, int max_split);
// Output-split narrow levels (at most kSegMaxNodes products per launch): the
// up-sweep as launch_tree_up; the down-sweep writes the children's inverses
// to lout (indexed like lch) instead of over the children.
constexpr int kSegMaxNodes = 64;
template <int P>
cudaError_t launch_tree_up_seg(const int16_t *lin, const LevelMap &lm, int n_out, int16_t *lout,
                               cudaStream_t st);
template <int P>
cudaError_t launch_tree_down_seg(const int16_t *lpar, const LevelMap &lm, int n_par,
                                 const int16_t *lch, int16_t *lout, cudaStream_t st);
template <int P>
cudaError_t launch_mul_batch(int n, const int16_t *a, const int16_t *b, int16_t *c,
                             cudaStream_t st);
// Tensor-core engine (rqmma.cu): same products and bytes; one CTA per
// product (per parent in the down-sweep), `tiles` MMA tiles per warp.  The
// down-sweep overwrites the children in place.
// `leaves`: the level's inputs (up) or children (down) are the leaves 3f,
// whose small coefficients need fewer limb products.  Levels of at most 256
// (64) products split each product's sum over 2 (4) warps, up to kmax.
template <int P>
cudaError_t launch_tree_up_mma(const int16_t *lin, const LevelMap &lm, int n_out, int16_t *lout,
                               cudaStream_t st, int tiles, bool leaves, int kmax = 4,
                               bool wide = false);
template <int P>
cudaError_t launch_tree_down_mma(const int16_t *lpar, const LevelMap &lm, int n_par, int16_t *lch,
                                 cudaStream_t st, int tiles, bool leaves, int kmax = 4,
                                 bool wide = false);
// R/3 trees for the batch inversion of the g's (coefficients mod 3).
template <int P>
cudaError_t launch_tree_up_mma3(const int16_t *lin, const LevelMap &lm, int n_out, int16_t *lout,
                                cudaStream_t st, int kmax);
template <int P>
cudaError_t launch_tree_down_mma3(const int16_t *lpar, const LevelMap &lm, int n_par, int16_t *lch,
                                  cudaStream_t st, int kmax);
template <int P>
cudaError_t launch_mul_batch_mma(int n, const int16_t *a, const int16_t *b, int16_t *c,
                                 cudaStream_t st, bool wide = false);
// R/q products by the paper's multiplier (Sec. 3.3): truncated transforms
// over K = (Z/q)[x]/(x^64 + 1) with x as the root of unity, pointwise products
// in K on the IMAD pipe (rqntt.cu).  Same layouts as the other engines.
template <int P>
cudaError_t launch_mul_batch_ntt(int n, const int16_t *a, const int16_t *b, int16_t *c,
                                 cudaStream_t st);
template <int P>
cudaError_t launch_tree_up_ntt(const int16_t *lin, const LevelMap &lm, int n_out, int16_t *lout,
                               cudaStream_t st);
template <int P>
cudaError_t launch_tree_down_ntt(const int16_t *lpar, const LevelMap &lm, int n_par, int16_t *lch,
                                 cudaStream_t st);
template <int P>
cudaError_t launch_rq_inv(int n, const int16_t *in, long in_stride, int16_t *out,
                          long out_stride, int32_t *ok, int *err, int err_bit, cudaStream_t st);
// idx (optional): element e is row idx[e] of in / out instead of row e.
template <int P>
cudaError_t launch_rq_inv_jump(int n, const int16_t *in, long in_stride, int16_t *out,
                               long out_stride, int32_t *ok, int *err, int err_bit,
                               cudaStream_t st, const int *idx = nullptr);
// R/3 batch path (r3batch.cu): invertibility test and resampling of g (warp
// per key; final g into the R/3 leaves, int16, and over a resampled gbuf
// row), and Small_encode(1/g) into sk from the inverted leaves.
template <int P>
cudaError_t launch_r3_check(const KeyMap &km, int B, int8_t *gbuf, int16_t *leaves3,
                            const R3Factors &fac, int *err, cudaStream_t st);
template <int P>
cudaError_t launch_r3_encode_v(const KeyMap &km, int B, const int16_t *v3, int sk_bytes,
                               int sk_off, cudaStream_t st, const int *sub_ok = nullptr,
                               int sub_size = 0);
// Screen of the first draws before the R/3 forest of mode 2 (warp per key):
// g is redrawn while a factor of degree <= kScreenMaxDeg divides it; a
// redrawn key gets its final-screen g in its R/3 leaf, a slot of the
// resampling list (fix_keys, gfix rows, *fix_count) and fix_slot[key] = the
// slot (-1 for a key kept), so that the per-key fall-back of a subtree whose
// root still fails can reuse the slot.
template <int P>
cudaError_t launch_r3_screen(const KeyMap &km, int B, const int8_t *gbuf, int16_t *leaves3,
                             const R3Screen &scr, int8_t *gfix, int *fix_count, int *fix_keys,
                             int *fix_slot, int *err, cudaStream_t st);
// Jump-divstep inversions in R/3 (entries mod 3, centred int16 rows); ok
// (optional) receives 1 per invertible element; err (optional) gets err_bit
// for a non-invertible one.
template <int P>
cudaError_t launch_r3_inv_jump(int n, const int16_t *in, long in_stride, int16_t *out,
                               long out_stride, int32_t *ok, int *err, int err_bit,
                               cudaStream_t st, const int *idx = nullptr);
// Keys on the resampling list: h with the final g, pk, sk's copy and hash;
// `grid` CTAs take list entries in turn (the list's length is on the device:
// size it by how many keys can be redrawn); nkeys: the call's key count, the
// list's largest possible length.
template <int P>
cudaError_t launch_fixup(const KeyMap &km, const int *fix_count, const int *fix_keys,
                         const int8_t *gfix, const int16_t *ainv, int pk_bytes, int sk_bytes,
                         int sk_pk_off, int hash_off, const EncSched &S, cudaStream_t st,
                         const int16_t *leaves, LevelMap lm1, int grid, int nkeys);
// sbuf (optional): the leaf-pair products s of launch_leaf_s, else formed here.
template <int P>
cudaError_t launch_finalize_pair(const KeyMap &km, int n1, const int8_t *gbuf,
                                 const int16_t *leaves, const int16_t *inv1, LevelMap lm1,
                                 int pk_bytes, int sk_bytes, int sk_pk_off, const EncSched &S,
                                 cudaStream_t st, const int16_t *sbuf = nullptr);
// s_L = g_L f_R and s_R = g_R f_L of every leaf pair (rows of sbuf by key),
// ahead of the down-sweep; needs only g's draws and the leaves.
template <int P>
cudaError_t launch_leaf_s(int n1, const int8_t *gbuf, const int16_t *leaves, LevelMap lm1,
                          int16_t *sbuf, cudaStream_t st);
// h = g * (3f)^-1, Rq_encode(h) into pk and sk; mma: h on the tensor cores.
template <int P>
cudaError_t launch_finalize(const KeyMap &km, int nkeys, const int8_t *gbuf, const int16_t *ainv,
                            int pk_bytes, int sk_bytes, int sk_pk_off, const EncSched &S,
                            cudaStream_t st, bool mma = false);
// list (optional): hash the keys list[0 .. *list_n) (at most nkeys) instead
// of keys 0 .. nkeys - 1.
cudaError_t launch_sha512_pk(const KeyMap &km, int nkeys, int pk_bytes, int sk_bytes,
                             int hash_off, cudaStream_t st, const int *list = nullptr,
                             const int *list_n = nullptr);
template <int P>
cudaError_t launch_encap(const EncMap &em, int n, int pk_bytes, int ct_bytes, const EncSched &Spk,
                         const EncSched &Sct, cudaStream_t st);
template <int P>
cudaError_t launch_decap(const DecMap &dm, int n, int pk_bytes, int sk_bytes, int ct_bytes,
                         const EncSched &Spk, const EncSched &Sct, cudaStream_t st);

}  // namespace snt
