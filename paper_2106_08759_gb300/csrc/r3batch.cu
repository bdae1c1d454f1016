// r3batch.cu -- batch inversion in R/3 (the paper's R/3 path, Sec. 3.1.1):
// every g of a batch is first checked invertible against the irreducible
// factors of x^p - x - 1 over F_3 (resampled until it is), then all g are
// inverted together with Montgomery's trick in R/3 (the product tree of
// rqmma.cu with coefficients mod 3, one jump-divstep inversion per subtree
// root), and Small_encode(1/g) goes into the secret key.
//
// isInvertible.  x^p - x - 1 is squarefree over F_3 and its distinct-degree
// factorization has exactly one irreducible factor of each degree that
// occurs (sntrup761: 19, 60, 682; sntrup653: 3, 16, 23, 77, 122, 124, 288;
// sntrup857: 25, 113, 719), so R/3 is a product of finite fields and g is
// invertible iff its remainder modulo every factor is nonzero.  The paper
// computes those remainders by Barrett reduction with AVX2 multiplications;
// here each remainder is a plain long division, one warp per key with one
// 32-trit word per lane (the same remainders).  The factors are computed once
// per parameter set on the host (distinct-degree factorization: Frobenius
// cubing and gcds) and kept in device memory.
#include <mutex>
#include <vector>

#include "ctx.h"
#include "pdl.cuh"

namespace snt {

namespace {

// ---- host: polynomials over F_3, coefficients in {0, 1, 2}, low degree first
using Poly = std::vector<uint8_t>;

void trim(Poly &a) {
    while (!a.empty() && a.back() == 0) a.pop_back();
}
int deg(const Poly &a) { return (int)a.size() - 1; }  // -1 for zero

// a mod m (m != 0)
Poly pmod(Poly a, const Poly &m) {
    trim(a);
    const int dm = deg(m);
    const uint8_t inv_lead = m[dm];  // 1^-1 = 1, 2^-1 = 2 in F_3
    while (deg(a) >= dm) {
        const int s = deg(a) - dm;
        const uint8_t c = (uint8_t)((a.back() * inv_lead) % 3);
        for (int i = 0; i <= dm; ++i) a[s + i] = (uint8_t)((a[s + i] + 3 * 3 - c * m[i]) % 3);
        trim(a);
    }
    return a;
}

// quotient of a by m when m divides a
Poly pdiv(Poly a, const Poly &m) {
    trim(a);
    const int dm = deg(m);
    const uint8_t inv_lead = m[dm];
    Poly q(deg(a) - dm + 1, 0);
    while (deg(a) >= dm) {
        const int s = deg(a) - dm;
        const uint8_t c = (uint8_t)((a.back() * inv_lead) % 3);
        q[s] = c;
        for (int i = 0; i <= dm; ++i) a[s + i] = (uint8_t)((a[s + i] + 3 * 3 - c * m[i]) % 3);
        trim(a);
    }
    trim(q);
    return q;
}

Poly pgcd(Poly a, Poly b) {
    trim(a);
    trim(b);
    while (!b.empty()) {
        Poly r = pmod(a, b);
        a = std::move(b);
        b = std::move(r);
    }
    if (!a.empty() && a.back() == 2)  // monic
        for (auto &c : a) c = (uint8_t)((c * 2) % 3);
    return a;
}

// h^3 mod m: in F_3 the Frobenius map is additive and fixes coefficients,
// so (sum h_i x^i)^3 = sum h_i x^(3i).
Poly cube_mod(const Poly &h, const Poly &m) {
    Poly c(3 * h.size() + 1, 0);
    for (size_t i = 0; i < h.size(); ++i) c[3 * i] = h[i];
    return pmod(c, m);
}

// Irreducible factors of x^p - x - 1 over F_3 by distinct-degree
// factorization; empty if some degree has more than one factor (the
// remainder test would then not decide invertibility).
std::vector<Poly> r3_factors(int p) {
    Poly m(p + 1, 0);
    m[0] = 2;  // -1
    m[1] = 2;  // -x
    m[p] = 1;
    std::vector<Poly> out;
    Poly M = m, h = {0, 1};
    for (int d = 1; deg(M) > 0; ++d) {
        if (deg(M) < 2 * d) {  // what is left is irreducible
            out.push_back(M);
            break;
        }
        h = cube_mod(h, M);
        Poly hx = h;
        if (hx.size() < 2) hx.resize(2, 0);
        hx[1] = (uint8_t)((hx[1] + 2) % 3);  // h - x
        const Poly g = pgcd(hx, M);
        if (deg(g) > 0) {
            if (deg(g) != d) return {};  // several factors of degree d
            out.push_back(g);
            M = pdiv(M, g);
            h = pmod(h, M);
        }
    }
    int total = 0;
    for (const Poly &f : out) total += deg(f);
    if (total != p) return {};
    return out;
}

struct HostFactors {
    bool done = false, ok = false;
    R3Factors f;             // host copy of the metadata (pointer filled per device)
    std::vector<uint32_t> w; // planes of all factors
    int screen_n = 0;        // factors of degree <= kScreenMaxDeg
    std::vector<uint32_t> screen;  // their remainder tables (R3Screen layout)
};

// Remainder table of factor m (degree d <= kScreenMaxDeg): the planes of
// x^i mod m for 0 <= i < p, appended to t.  x^(i+1) mod m is x (x^i mod m)
// with its degree-d term folded back (m monic: x^d = x^d - m).
void screen_table(const Poly &m, int p, std::vector<uint32_t> &t) {
    const int d = deg(m);
    Poly r(d, 0);
    r[0] = 1;  // x^0
    for (int i = 0; i < p; ++i) {
        uint32_t pm = 0, ps = 0;
        for (int k = 0; k < d; ++k) {
            pm |= (uint32_t)(r[k] != 0) << k;
            ps |= (uint32_t)(r[k] == 2) << k;
        }
        t.push_back(pm);
        t.push_back(ps);
        const uint8_t top = r[d - 1];
        for (int k = d - 1; k > 0; --k) r[k] = r[k - 1];
        r[0] = 0;
        for (int k = 0; k < d; ++k) r[k] = (uint8_t)((r[k] + 3 * 3 - top * m[k]) % 3);
    }
}

// Bit planes of the factors: per factor, its words of m (coefficient
// nonzero) then its words of s (coefficient is -1 = 2).
HostFactors build_factors(int p) {
    HostFactors H;
    H.done = true;
    const std::vector<Poly> fs = r3_factors(p);
    if (fs.empty() || (int)fs.size() > kMaxR3Factors) return H;
    H.f.n = (int)fs.size();
    int off = 0;
    for (int i = 0; i < H.f.n; ++i) {
        const int d = deg(fs[i]);
        const int words = (d + 1 + 31) / 32;
        H.f.deg[i] = d;
        H.f.words[i] = words;
        H.f.off[i] = off;
        for (int plane = 0; plane < 2; ++plane)
            for (int wd = 0; wd < words; ++wd) {
                uint32_t v = 0;
                for (int b = 0; b < 32; ++b) {
                    const int k = 32 * wd + b;
                    const uint8_t c = k <= d ? fs[i][k] : 0;
                    if (plane == 0 ? c != 0 : c == 2) v |= 1u << b;
                }
                H.w.push_back(v);
            }
        off += 2 * words;
        if (d <= kScreenMaxDeg && H.screen_n < kMaxScreen) {
            screen_table(fs[i], p, H.screen);
            ++H.screen_n;
        }
    }
    H.f.total_words = off;
    H.ok = true;
    return H;
}

std::mutex g_fac_mu;
HostFactors g_fac[3];

}  // namespace

// Device copy of the factors of parameter set P for this context (built on
// first use, kept until the context is destroyed).
snt_status r3_factors_for(snt_ctx *ctx, int P, R3Factors &out) {
    const int pi_ = pidx(P);
    {
        std::lock_guard<std::mutex> lk(g_fac_mu);
        if (!g_fac[pi_].done) g_fac[pi_] = build_factors(P);
        if (!g_fac[pi_].ok)
            return set_error(SNT_EINTERNAL, "x^%d - x - 1 has repeated factor degrees over F_3", P);
        out = g_fac[pi_].f;
    }
    if (!ctx->d_r3fac[pi_]) {
        const std::vector<uint32_t> &w = g_fac[pi_].w;
        cudaError_t e = cudaMalloc(&ctx->d_r3fac[pi_], w.size() * sizeof(uint32_t));
        if (e == cudaSuccess)
            e = cudaMemcpy(ctx->d_r3fac[pi_], w.data(), w.size() * sizeof(uint32_t),
                           cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            if (ctx->d_r3fac[pi_]) cudaFree(ctx->d_r3fac[pi_]);
            ctx->d_r3fac[pi_] = nullptr;
            return set_error(SNT_ECUDA, "R/3 factor table: %s", cudaGetErrorString(e));
        }
    }
    out.w = ctx->d_r3fac[pi_];
    return SNT_OK;
}

// Remainder tables of the small factors of parameter set P for this context
// (none for sntrup761 and sntrup857, whose smallest factors have degree 19
// and 25; sntrup653's of degree 3 and 16).
snt_status r3_screen_for(snt_ctx *ctx, int P, R3Screen &out) {
    const int pi_ = pidx(P);
    std::vector<uint32_t> t;
    {
        std::lock_guard<std::mutex> lk(g_fac_mu);
        if (!g_fac[pi_].done) g_fac[pi_] = build_factors(P);
        if (!g_fac[pi_].ok)
            return set_error(SNT_EINTERNAL, "x^%d - x - 1 has repeated factor degrees over F_3", P);
        out.n = g_fac[pi_].screen_n;
        t = g_fac[pi_].screen;
    }
    out.t = nullptr;
    if (out.n == 0) return SNT_OK;
    if (!ctx->d_r3screen[pi_]) {
        cudaError_t e = cudaMalloc(&ctx->d_r3screen[pi_], t.size() * sizeof(uint32_t));
        if (e == cudaSuccess)
            e = cudaMemcpy(ctx->d_r3screen[pi_], t.data(), t.size() * sizeof(uint32_t),
                           cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            if (ctx->d_r3screen[pi_]) cudaFree(ctx->d_r3screen[pi_]);
            ctx->d_r3screen[pi_] = nullptr;
            return set_error(SNT_ECUDA, "R/3 screen table: %s", cudaGetErrorString(e));
        }
    }
    out.t = ctx->d_r3screen[pi_];
    return SNT_OK;
}

// ---- device -----------------------------------------------------------------

constexpr unsigned kFull = 0xffffffffu;

// One warp per key, lane L = trits 32L .. 32L+31 of the polynomial (bit
// planes m: nonzero, s: the value is -1).  For attempt a = 0, 1, ...: g (a = 0
// from gbuf, sampled with f; otherwise stream 0 attempt a), then for every
// factor f of degree d the long division
//     for t = p-1 down to d:  r <- r - r_t x^(t-d) f
// (f monic); g is invertible iff no remainder is zero.  The first invertible
// g goes to the R/3 leaves (int16 rows) and, if it is not the first draw,
// over its gbuf row.
template <int P>
__global__ void __launch_bounds__(128)
k_r3_check(KeyMap km, int B, int8_t *__restrict__ gbuf, int16_t *__restrict__ leaves3,
           R3Factors fac, int *__restrict__ err) {
    pdl_enter();
    using G = Geo<P>;
    constexpr int W = (P + 31) / 32;  // words of a degree < p polynomial
    extern __shared__ uint32_t fw[];   // the factors' planes
    for (int i = threadIdx.x; i < fac.total_words; i += blockDim.x) fw[i] = fac.w[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int key = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (key >= B) return;  // whole warp
    const BatchDesc bd = key_batch(km, key);
    const uint64_t kidx = bd.first + (uint64_t)(key - bd.key_base);
    int8_t *grow = gbuf + (size_t)key * G::pad;
    bool ok = false;
    uint32_t gm = 0, gs = 0;
    int att = 0;
    for (; att < kMaxGAttempts && !ok; ++att) {
        // this lane's 32 trits of g
        gm = 0; gs = 0;
        if (lane < W) {
            if (att == 0) {
                for (int b = 0; b < 32; ++b) {
                    const int i = 32 * lane + b;
                    const int c = i < P ? grow[i] : 0;
                    gm |= (uint32_t)(c != 0) << b;
                    gs |= (uint32_t)(c < 0) << b;
                }
            } else {
                // g_i = floor(3 (u_i mod 2^30) / 2^30) - 1, word u_i of stream 0, attempt att
                for (int blk = 8 * lane; blk < 8 * lane + 8; ++blk) {
                    uint32_t r[4];
                    rand_block(bd.seed, kidx, STREAM_G, (uint32_t)att, (uint32_t)blk, r);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int i = 4 * blk + j;
                        if (i < P) {
                            const int c = (int)(((unsigned long long)(r[j] & 0x3fffffffu) * 3u) >> 30) - 1;
                            gm |= (uint32_t)(c != 0) << (i & 31);
                            gs |= (uint32_t)(c < 0) << (i & 31);
                        }
                    }
                }
            }
        }
        bool inv = true;
        for (int fi = 0; fi < fac.n && inv; ++fi) {
            const int d = fac.deg[fi], fwords = fac.words[fi];
            const uint32_t *fm = fw + fac.off[fi], *fs = fm + fwords;
            uint32_t rm = gm, rs = gs;
            for (int t = P - 1; t >= d; --t) {
                const uint32_t lead = __shfl_sync(kFull, ((rm >> (t & 31)) & 1u) | (((rs >> (t & 31)) & 1u) << 1), t >> 5);
                if (!(lead & 1u)) continue;  // warp-uniform
                // r <- r - c x^s f, c = +-1: add f shifted with sign (c == 1 ? -1 : +1)
                const int s = t - d, ws = s >> 5, bs = s & 31;
                const int k = lane - ws;  // word of f landing (its low part) in this lane
                const uint32_t hm = (k >= 0 && k < fwords) ? fm[k] : 0u;
                const uint32_t hs = (k >= 0 && k < fwords) ? fs[k] : 0u;
                const uint32_t lm = (k >= 1 && k - 1 < fwords) ? fm[k - 1] : 0u;
                const uint32_t ls = (k >= 1 && k - 1 < fwords) ? fs[k - 1] : 0u;
                const uint32_t sm = __funnelshift_l(lm, hm, bs), ss = __funnelshift_l(ls, hs, bs);
                const uint32_t bsgn = ss ^ ((lead & 2u) ? 0u : kFull);  // -c f
                // (rm, rs) + (sm, bsgn) in F_3 (signs only meaningful where m = 1)
                const uint32_t both = rm & sm;
                const uint32_t nm = (rm | sm) & ~(both & (rs ^ bsgn));
                const uint32_t ns = (rm & (rs ^ sm)) | (~rm & bsgn);
                rm = nm;
                rs = ns;
            }
            inv = __any_sync(kFull, rm != 0u);  // remainder (degree < d) nonzero
        }
        ok = inv;
    }
    if (!ok) {
        if (lane == 0) atomicOr(err, ERR_RESAMPLE);
        gm = 0; gs = 0;
    }
    // the R/3 leaf (int16, zero padded) and, for a later draw, the g row
    int16_t *leaf = leaves3 + (size_t)key * G::pad;
    for (int i = lane; i < G::pad; i += 32) {
        const int w = i >> 5, b = i & 31;
        const uint32_t m = __shfl_sync(kFull, gm, w & 31), s = __shfl_sync(kFull, gs, w & 31);
        const int c = (i < P && w < W) ? (((m >> b) & 1u) ? (((s >> b) & 1u) ? -1 : 1) : 0) : 0;
        leaf[i] = (int16_t)c;
        if (att > 1) grow[i] = (int8_t)c;
    }
}

// a + b in F_3 on 32 trits as bit planes (m: nonzero, s: -1, s within m).
__device__ __forceinline__ void f3_add(uint32_t &am, uint32_t &as, uint32_t bm, uint32_t bs) {
    const uint32_t both = am & bm;
    const uint32_t nm = (am | bm) & ~(both & (as ^ bs));
    const uint32_t ns = ((am & (as ^ bm)) | (~am & bs)) & nm;
    am = nm;
    as = ns;
}

// The screen before the R/3 forest of mode 2: one warp per key, lane L
// holding trits 32 L .. 32 L + 31 of g as bit planes.  For attempt a = 0, 1,
// ... (a = 0: the first draw from gbuf; otherwise stream 0 attempt a), the
// remainder of g modulo each small factor m_j is sum_i g_i (x^i mod m_j),
// each lane adding its own terms from the table and the warp adding the
// lanes' sums; g passes when no remainder is zero (about 1 - 1/27 per draw
// for sntrup653, whose cubic factor divides one draw in 27).
template <int P>
__global__ void __launch_bounds__(128)
k_r3_screen(KeyMap km, int B, const int8_t *__restrict__ gbuf, int16_t *__restrict__ leaves3,
            R3Screen scr, int8_t *__restrict__ gfix, int *__restrict__ fix_count,
            int *__restrict__ fix_keys, int *__restrict__ fix_slot, int *__restrict__ err) {
    pdl_enter();
    using G = Geo<P>;
    constexpr int W = (P + 31) / 32;
    extern __shared__ uint32_t tab[];  // scr.n tables of P plane pairs
    for (int i = threadIdx.x; i < 2 * P * scr.n; i += blockDim.x) tab[i] = scr.t[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int key = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (key >= B) return;  // whole warp
    const BatchDesc bd = key_batch(km, key);
    const uint64_t kidx = bd.first + (uint64_t)(key - bd.key_base);
    const int8_t *grow = gbuf + (size_t)key * G::pad;
    bool ok = false;
    uint32_t gm = 0, gs = 0;
    int att = 0;
    for (; att < kMaxGAttempts && !ok; ++att) {
        gm = 0; gs = 0;
        if (lane < W) {
            if (att == 0) {
                for (int b = 0; b < 32; ++b) {
                    const int i = 32 * lane + b;
                    const int c = i < P ? grow[i] : 0;
                    gm |= (uint32_t)(c != 0) << b;
                    gs |= (uint32_t)(c < 0) << b;
                }
            } else {
                // g_i = floor(3 (u_i mod 2^30) / 2^30) - 1, word u_i of stream 0, attempt att
                for (int blk = 8 * lane; blk < 8 * lane + 8; ++blk) {
                    uint32_t r[4];
                    rand_block(bd.seed, kidx, STREAM_G, (uint32_t)att, (uint32_t)blk, r);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int i = 4 * blk + j;
                        if (i < P) {
                            const int c = (int)(((unsigned long long)(r[j] & 0x3fffffffu) * 3u) >> 30) - 1;
                            gm |= (uint32_t)(c != 0) << (i & 31);
                            gs |= (uint32_t)(c < 0) << (i & 31);
                        }
                    }
                }
            }
        }
        ok = true;
        for (int j = 0; j < scr.n; ++j) {
            const uint32_t *tj = tab + 2 * P * j;
            uint32_t am = 0, as = 0;
            if (lane < W)
                for (int b = 0; b < 32; ++b) {
                    const int i = 32 * lane + b;
                    if (i < P && ((gm >> b) & 1u)) {
                        const uint32_t tm = tj[2 * i];
                        const uint32_t ts = tj[2 * i + 1] ^ (((gs >> b) & 1u) ? tm : 0u);
                        f3_add(am, as, tm, ts);
                    }
                }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const uint32_t om = __shfl_xor_sync(kFull, am, o), os = __shfl_xor_sync(kFull, as, o);
                f3_add(am, as, om, os);
            }
            ok = ok && am != 0u;  // the same sum in every lane
        }
    }
    if (!ok) {
        if (lane == 0) atomicOr(err, ERR_RESAMPLE);
        gm = 0; gs = 0;
    }
    const bool redrawn = att > 1;
    int slot = -1;
    if (redrawn && lane == 0) {
        slot = atomicAdd(fix_count, 1);
        fix_keys[slot] = key;
    }
    slot = __shfl_sync(kFull, slot, 0);
    if (lane == 0) fix_slot[key] = slot;
    if (!redrawn) return;
    // the final-screen g into the R/3 leaf and the resampling list
    int16_t *leaf = leaves3 + (size_t)key * G::pad;
    int8_t *fg = gfix + (size_t)slot * G::pad;
    for (int i = lane; i < G::pad; i += 32) {
        const int w = i >> 5, b = i & 31;
        const uint32_t m = __shfl_sync(kFull, gm, w & 31), s = __shfl_sync(kFull, gs, w & 31);
        const int c = (i < P && w < W) ? (((m >> b) & 1u) ? (((s >> b) & 1u) ? -1 : 1) : 0) : 0;
        leaf[i] = (int16_t)c;
        fg[i] = (int8_t)c;
    }
}

// Small_encode(1/g) into the secret key from the inverted R/3 leaves (keys of
// subtrees whose root did not invert skipped: sub_ok[key / sub_size] == 0, or
// with sub_size 0 the flag of the key's batch).
template <int P>
__global__ void __launch_bounds__(256)
k_r3_encode_v(KeyMap km, int B, const int16_t *__restrict__ v3, int sk_bytes, int sk_off,
              const int *__restrict__ sub_ok, int sub_size) {
    pdl_enter();
    using G = Geo<P>;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int key = idx / G::small_bytes, b = idx % G::small_bytes;
    if (key >= B) return;
    if (sub_ok && !sub_ok[key_subtree(km, key, sub_size)]) return;
    const int16_t *v = v3 + (size_t)key * G::pad;
    uint32_t byte = 0;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const int i = 4 * b + t;
        if (i < P) byte |= (uint32_t)(v[i] + 1) << (2 * t);
    }
    const BatchDesc d = key_batch(km, key);
    d.sk[(size_t)(key - d.key_base) * sk_bytes + sk_off + b] = (uint8_t)byte;
}

template <int P>
cudaError_t launch_r3_check(const KeyMap &km, int B, int8_t *gbuf, int16_t *leaves3,
                            const R3Factors &fac, int *err, cudaStream_t st) {
    SNT_LAUNCH(k_r3_check<P>, (B + 3) / 4, 128, fac.total_words * sizeof(uint32_t), st, km, B, gbuf,
        leaves3, fac, err);
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_r3_screen(const KeyMap &km, int B, const int8_t *gbuf, int16_t *leaves3,
                             const R3Screen &scr, int8_t *gfix, int *fix_count, int *fix_keys,
                             int *fix_slot, int *err, cudaStream_t st) {
    if (scr.n <= 0 || scr.n > kMaxScreen) return cudaErrorInvalidValue;
    SNT_LAUNCH(k_r3_screen<P>, (B + 3) / 4, 128, (size_t)2 * P * scr.n * sizeof(uint32_t), st, km,
        B, gbuf, leaves3, scr, gfix, fix_count, fix_keys, fix_slot, err);
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_r3_encode_v(const KeyMap &km, int B, const int16_t *v3, int sk_bytes,
                               int sk_off, cudaStream_t st, const int *sub_ok, int sub_size) {
    const long n = (long)B * Geo<P>::small_bytes;
    SNT_LAUNCH(k_r3_encode_v<P>, (unsigned)((n + 255) / 256), 256, 0, st, km, B, v3, sk_bytes,
        sk_off, sub_ok, sub_size);
    return cudaGetLastError();
}

#define SNT_R3B_INST(P)                                                                      \
    template cudaError_t launch_r3_check<P>(const KeyMap &, int, int8_t *, int16_t *,        \
                                            const R3Factors &, int *, cudaStream_t);         \
    template cudaError_t launch_r3_encode_v<P>(const KeyMap &, int, const int16_t *, int, int, \
                                               cudaStream_t, const int *, int);                \
    template cudaError_t launch_r3_screen<P>(const KeyMap &, int, const int8_t *, int16_t *,  \
                                             const R3Screen &, int8_t *, int *, int *, int *, \
                                             int *, cudaStream_t);
SNT_R3B_INST(653)
SNT_R3B_INST(761)
SNT_R3B_INST(857)

}  // namespace snt
