/*
 * sntrup_oracle.c -- plain, slow, CPU-only oracle for Streamlined NTRU Prime
 * key generation (sntrup653 / sntrup761 / sntrup857).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file; only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code, header, table or helper with the
 * CUDA library: every routine below is written out from its mathematical
 * definition, one key at a time, with 64-bit integer arithmetic and no
 * blocking, batching or reordering.
 *
 * What it follows (sections of arXiv 2106.08759, "OpenSSLNTRU"):
 *   - Sec. 2.1: R = Z[x]/(x^p - x - 1), R/3 and R/q; Short = ternary
 *     polynomials of weight exactly w; (p,q,w) = (653,4621,288),
 *     (761,4591,286), (857,5167,322).
 *   - Sec. 3.1 (KeyGen): sample small g until g is invertible in R/3,
 *     compute 1/g in R/3, sample f in Short, h = g/(3f) in R/q, output
 *     (h, (f, 1/g)).  Algorithm 1 (BatchKeyGen) computes exactly the same
 *     keys through Montgomery's trick; because R/q is a field the inverse
 *     of 3f is unique, so this per-key definition is the oracle for the
 *     batched path too.
 *   - Inversion here is the classical extended Euclidean algorithm over
 *     F_m[x] (m = 3 or q), NOT the divstep algorithm the GPU uses.
 *   - Multiplication is the schoolbook product followed by the reduction
 *     x^p = x + 1.
 *
 * Readings of points the paper leaves open (randomness, sampling, wire
 * formats, sk layout) are fixed in the repository's design notes and are
 * restated next to each routine.
 *
 * Parity status: every function here is pinned by the CPU test suite
 * (tests/test_oracle_*.py) against something other than itself, except the
 * byte-level wire format of Rq_encode / Small_encode / the sk layout, which
 * is pinned only by its lengths (Table 4 of the paper) and by round trips:
 * "parity unpinned" for byte compatibility with third-party encoders.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXP 2048

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as  */
/* easy as 1, 2, 3", SC'11).  Ten rounds of the Philox S-box on a 128-bit   */
/* counter with a 64-bit key bumped by the Weyl constants each round.       */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                       uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; round++) {
        uint64_t prod0 = (uint64_t)0xD2511F53u * c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/*
 * Reading of the paper's "uniform random" (Algorithm 1): the seed keys a
 * counter-based generator.  Word i of stream s, attempt a, key index k is
 * lane (i mod 4) of Philox4x32-10 with
 *     key     = (seed mod 2^32, seed >> 32)
 *     counter = ((s << 16) | (i / 4), a, k mod 2^32, k >> 32).
 * Streams: 0 = g, 1 = f, 2 = rho, 3 = encapsulation randomness.
 */
void orc_random_words(uint64_t seed, uint64_t k, uint32_t stream,
                      uint32_t attempt, int n, uint32_t *out)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int i = 0; i < n; i++) {
        uint32_t ctr[4] = {(stream << 16) | (uint32_t)(i / 4), attempt,
                           (uint32_t)k, (uint32_t)(k >> 32)};
        uint32_t blk[4];
        orc_philox4x32_10(ctr, key, blk);
        out[i] = blk[i % 4];
    }
}

/* Small g (Sec. 3.1 step 1): coefficient i = floor(3 * (u_i mod 2^30) / 2^30) - 1. */
void orc_sample_small(int p, uint64_t seed, uint64_t k, uint32_t attempt,
                      int8_t *g)
{
    uint32_t *u = (uint32_t *)malloc(sizeof(uint32_t) * p);
    orc_random_words(seed, k, 0, attempt, p, u);
    for (int i = 0; i < p; i++)
        g[i] = (int8_t)((int)(((uint64_t)(u[i] & 0x3fffffffu) * 3u) >> 30) - 1);
    free(u);
}

static int cmp_u32(const void *x, const void *y)
{
    uint32_t a = *(const uint32_t *)x, b = *(const uint32_t *)y;
    return (a > b) - (a < b);
}

/*
 * Short f (Sec. 2.1, Sec. 3.1 step 3): draw p words from stream 1; the first
 * w get low bits that decode to +-1 (bit 0 cleared, bit 1 random), the rest
 * get low bits 01 (decode to 0); sort the words as unsigned integers and
 * read coefficient j as (word_j mod 4) - 1.  Exactly w nonzero coefficients,
 * at uniformly random positions (ties in the upper 30 bits are broken by the
 * numeric order, deterministically).
 */
void orc_sample_short_stream(int p, int w, uint64_t seed, uint64_t k, uint32_t stream,
                             int8_t *f)
{
    uint32_t *u = (uint32_t *)malloc(sizeof(uint32_t) * p);
    orc_random_words(seed, k, stream, 0, p, u);
    for (int i = 0; i < p; i++) {
        if (i < w) u[i] = u[i] & ~1u;
        else       u[i] = (u[i] & ~3u) | 1u;
    }
    qsort(u, (size_t)p, sizeof(uint32_t), cmp_u32);
    for (int j = 0; j < p; j++) f[j] = (int8_t)((int)(u[j] & 3u) - 1);
    free(u);
}

void orc_sample_short(int p, int w, uint64_t seed, uint64_t k, int8_t *f)
{
    orc_sample_short_stream(p, w, seed, k, 1, f);
}

/* rho (part of the secret key, used for implicit rejection): nbytes bytes of
 * stream 2, byte j = byte (j mod 4) of word j/4, little-endian. */
void orc_rho(int nbytes, uint64_t seed, uint64_t k, uint8_t *rho)
{
    int nw = (nbytes + 3) / 4;
    uint32_t *u = (uint32_t *)malloc(sizeof(uint32_t) * nw);
    orc_random_words(seed, k, 2, 0, nw, u);
    for (int j = 0; j < nbytes; j++) rho[j] = (uint8_t)(u[j / 4] >> (8 * (j % 4)));
    free(u);
}

/* ------------------------------------------------------------------------ */
/* Arithmetic modulo a prime m                                              */
/* ------------------------------------------------------------------------ */
static int32_t md(int64_t x, int32_t m)
{
    int64_t r = x % m;
    if (r < 0) r += m;
    return (int32_t)r;
}

static int32_t centred(int64_t x, int32_t m)
{
    int32_t r = md(x, m);
    if (r > (m - 1) / 2) r -= m;
    return r;
}

static int32_t scalar_inv(int32_t a, int32_t m)
{
    /* a^(m-2) mod m (m prime, Fermat's little theorem) */
    int64_t base = md(a, m), acc = 1;
    int64_t e = m - 2;
    while (e > 0) {
        if (e & 1) acc = (acc * base) % m;
        base = (base * base) % m;
        e >>= 1;
    }
    return (int32_t)acc;
}

/* ------------------------------------------------------------------------ */
/* Ring multiplication in (Z/m)[x]/(x^p - x - 1) (Sec. 2.1).                */
/* Schoolbook product of two degree < p polynomials, then each coefficient  */
/* of x^k, k >= p, is folded down with x^k = x^(k-p+1) + x^(k-p), from the  */
/* top degree downwards.  Output centred in [-(m-1)/2, (m-1)/2].            */
/* ------------------------------------------------------------------------ */
void orc_ring_mul(int p, int32_t m, const int32_t *a, const int32_t *b,
                  int32_t *c)
{
    int64_t *t = (int64_t *)calloc((size_t)(2 * p - 1), sizeof(int64_t));
    for (int i = 0; i < p; i++)
        for (int j = 0; j < p; j++)
            t[i + j] += (int64_t)a[i] * b[j];
    for (int k = 2 * p - 2; k >= p; k--) {
        t[k - p + 1] += t[k];
        t[k - p] += t[k];
        t[k] = 0;
    }
    for (int i = 0; i < p; i++) c[i] = centred(t[i], m);
    free(t);
}

/* ------------------------------------------------------------------------ */
/* Generic polynomial helpers over F_m (m prime).  A polynomial is an array  */
/* of coefficients in [0, m), lowest degree first.                          */
/* ------------------------------------------------------------------------ */
static int pdeg(const int32_t *a, int n)
{
    for (int i = n - 1; i >= 0; i--)
        if (a[i] != 0) return i;
    return -1;
}

/* q, r such that a = q*b + r, deg r < deg b.  na, nb: array lengths;
 * quot has room for na entries, rem for na entries. */
static void pdivmod(const int32_t *a, int na, const int32_t *b, int nb,
                    int32_t m, int32_t *quot, int32_t *rem)
{
    int db = pdeg(b, nb);
    int32_t lead_inv = scalar_inv(b[db], m);
    memcpy(rem, a, sizeof(int32_t) * na);
    memset(quot, 0, sizeof(int32_t) * na);
    for (int d = pdeg(rem, na); d >= db; d = pdeg(rem, na)) {
        int32_t coef = (int32_t)(((int64_t)rem[d] * lead_inv) % m);
        int shift = d - db;
        quot[shift] = coef;
        for (int i = 0; i <= db; i++)
            rem[i + shift] = md((int64_t)rem[i + shift] - (int64_t)coef * b[i], m);
    }
}

/* c = a*b (plain product), arrays of length na, nb; c has na+nb-1 entries */
static void pmul(const int32_t *a, int na, const int32_t *b, int nb, int32_t m,
                 int32_t *c)
{
    int64_t *t = (int64_t *)calloc((size_t)(na + nb - 1), sizeof(int64_t));
    for (int i = 0; i < na; i++)
        if (a[i])
            for (int j = 0; j < nb; j++) t[i + j] += (int64_t)a[i] * b[j];
    for (int i = 0; i < na + nb - 1; i++) c[i] = md(t[i], m);
    free(t);
}

/* the modulus x^p - x - 1 over F_m, as an array of length p+1 */
static void modulus_poly(int p, int32_t m, int32_t *M)
{
    memset(M, 0, sizeof(int32_t) * (p + 1));
    M[p] = 1;
    M[1] = md(-1, m);
    M[0] = md(-1, m);
}

/* ------------------------------------------------------------------------ */
/* Inversion in (Z/m)[x]/(x^p - x - 1) by the extended Euclidean algorithm  */
/* (classical; deliberately not the divstep method of the GPU path).        */
/* Keeps r_i = s_i * a (mod x^p - x - 1) along the remainder sequence of     */
/* (x^p - x - 1, a).  When the gcd is a nonzero constant c, the inverse is   */
/* s / c.  Returns 1 if a is invertible (out = centred inverse), else 0      */
/* (out zeroed).                                                            */
/* ------------------------------------------------------------------------ */
int orc_ring_inv(int p, int32_t m, const int32_t *a, int32_t *out)
{
    int n = p + 1;
    int32_t *r0 = calloc(n, 4), *r1 = calloc(n, 4), *s0 = calloc(2 * n, 4),
            *s1 = calloc(2 * n, 4), *qt = calloc(n, 4), *rm = calloc(n, 4),
            *prod = calloc(3 * n, 4), *tmp = calloc(2 * n, 4);
    modulus_poly(p, m, r0);
    for (int i = 0; i < p; i++) r1[i] = md(a[i], m);
    s0[0] = 0;
    s1[0] = 1;
    while (pdeg(r1, n) >= 0) {
        pdivmod(r0, n, r1, n, m, qt, rm);
        /* s_new = s0 - qt * s1 (degrees stay below p + 1) */
        memset(prod, 0, sizeof(int32_t) * 3 * n);
        pmul(qt, n, s1, n, m, prod);
        for (int i = 0; i < n; i++) tmp[i] = md((int64_t)s0[i] - prod[i], m);
        memcpy(s0, s1, sizeof(int32_t) * n);
        memcpy(s1, tmp, sizeof(int32_t) * n);
        memcpy(r0, r1, sizeof(int32_t) * n);
        memcpy(r1, rm, sizeof(int32_t) * n);
    }
    int ok = (pdeg(r0, n) == 0);
    if (ok) {
        int32_t cinv = scalar_inv(r0[0], m);
        /* reduce s0 modulo x^p - x - 1 (its degree is already < p) */
        int32_t *M = calloc(n, 4), *qq = calloc(n, 4), *rr = calloc(n, 4);
        modulus_poly(p, m, M);
        pdivmod(s0, n, M, n, m, qq, rr);
        for (int i = 0; i < p; i++) out[i] = centred((int64_t)rr[i] * cinv, m);
        free(M); free(qq); free(rr);
    } else {
        memset(out, 0, sizeof(int32_t) * p);
    }
    free(r0); free(r1); free(s0); free(s1); free(qt); free(rm); free(prod);
    free(tmp);
    return ok;
}

/* a^e in (Z/m)[x]/(x^p - x - 1), e given little-endian in elen bytes
 * (left-to-right square and multiply with orc_ring_mul).  Test helper:
 * Fermat / Lagrange exponents give inverses independently of Euclid. */
void orc_ring_pow(int p, int32_t m, const int32_t *a, const uint8_t *e,
                  int elen, int32_t *out)
{
    int32_t *acc = calloc(p, 4), *t = calloc(p, 4);
    acc[0] = 1;
    for (int byte = elen - 1; byte >= 0; byte--)
        for (int bit = 7; bit >= 0; bit--) {
            orc_ring_mul(p, m, acc, acc, t);
            memcpy(acc, t, sizeof(int32_t) * p);
            if ((e[byte] >> bit) & 1) {
                orc_ring_mul(p, m, acc, a, t);
                memcpy(acc, t, sizeof(int32_t) * p);
            }
        }
    memcpy(out, acc, sizeof(int32_t) * p);
    free(acc); free(t);
}

/* ------------------------------------------------------------------------ */
/* Distinct-degree factorisation of x^p - x - 1 over F_m (test helper).     */
/* Sec. 3.1.1 states that x^761 - x - 1 splits mod 3 into irreducible       */
/* factors of degrees 19, 60 and 682.  For each d = 1, 2, ... the product   */
/* of all irreducible factors of degree d is gcd(x^(m^d) - x, f), where f is */
/* what remains after removing the lower-degree parts.                      */
/* Writes part_deg[i] (= d), part_total[i] (= degree of the product) and,    */
/* if parts != NULL, the monic product polynomial into parts + i*(p+1).     */
/* Returns the number of parts.                                             */
/* ------------------------------------------------------------------------ */
static void pmulmod(const int32_t *a, const int32_t *b, const int32_t *f,
                    int n, int32_t m, int32_t *out)
{
    int32_t *prod = calloc(2 * n, 4), *qq = calloc(2 * n, 4),
            *rr = calloc(2 * n, 4), *ff = calloc(2 * n, 4);
    pmul(a, n, b, n, m, prod);
    memcpy(ff, f, sizeof(int32_t) * n);
    pdivmod(prod, 2 * n - 1, ff, 2 * n - 1, m, qq, rr);
    memcpy(out, rr, sizeof(int32_t) * n);
    free(prod); free(qq); free(rr); free(ff);
}

static void pgcd_monic(const int32_t *a, const int32_t *b, int n, int32_t m,
                       int32_t *g)
{
    int32_t *x = calloc(n, 4), *y = calloc(n, 4), *qq = calloc(n, 4),
            *rr = calloc(n, 4);
    memcpy(x, a, sizeof(int32_t) * n);
    memcpy(y, b, sizeof(int32_t) * n);
    while (pdeg(y, n) >= 0) {
        pdivmod(x, n, y, n, m, qq, rr);
        memcpy(x, y, sizeof(int32_t) * n);
        memcpy(y, rr, sizeof(int32_t) * n);
    }
    int d = pdeg(x, n);
    int32_t li = scalar_inv(x[d], m);
    for (int i = 0; i < n; i++) g[i] = (int32_t)(((int64_t)x[i] * li) % m);
    free(x); free(y); free(qq); free(rr);
}

int orc_ddf(int p, int32_t m, int *part_deg, int *part_total, int32_t *parts,
            int maxparts)
{
    int n = p + 1, np = 0;
    int32_t *f = calloc(n, 4), *h = calloc(n, 4), *t = calloc(n, 4),
            *g = calloc(n, 4), *qq = calloc(n, 4), *rr = calloc(n, 4),
            *hh = calloc(n, 4);
    modulus_poly(p, m, f);
    h[1] = 1; /* h = x */
    for (int d = 1; 2 * d <= pdeg(f, n); d++) {
        /* h <- h^m mod f (right-to-left square and multiply) */
        memcpy(hh, h, sizeof(int32_t) * n);
        int32_t *acc = calloc(n, 4);
        acc[0] = 1;
        for (int32_t e = m; e > 0; e >>= 1) {
            if (e & 1) {
                pmulmod(acc, hh, f, n, m, t);
                memcpy(acc, t, sizeof(int32_t) * n);
            }
            if (e > 1) {
                pmulmod(hh, hh, f, n, m, t);
                memcpy(hh, t, sizeof(int32_t) * n);
            }
        }
        memcpy(h, acc, sizeof(int32_t) * n);
        free(acc);
        memcpy(t, h, sizeof(int32_t) * n);
        t[1] = md((int64_t)t[1] - 1, m); /* h - x */
        if (pdeg(t, n) < 0) continue;
        pgcd_monic(t, f, n, m, g);
        if (pdeg(g, n) > 0) {
            if (np < maxparts) {
                part_deg[np] = d;
                part_total[np] = pdeg(g, n);
                if (parts) memcpy(parts + (size_t)np * n, g, sizeof(int32_t) * n);
            }
            np++;
            pdivmod(f, n, g, n, m, qq, rr);
            memcpy(f, qq, sizeof(int32_t) * n);
            pdivmod(h, n, f, n, m, qq, rr);
            memcpy(h, rr, sizeof(int32_t) * n);
        }
    }
    if (pdeg(f, n) > 0) {
        if (np < maxparts) {
            part_deg[np] = pdeg(f, n);
            part_total[np] = pdeg(f, n);
            if (parts) {
                int32_t li = scalar_inv(f[pdeg(f, n)], m);
                for (int i = 0; i < n; i++)
                    parts[(size_t)np * n + i] = (int32_t)(((int64_t)f[i] * li) % m);
            }
        }
        np++;
    }
    free(f); free(h); free(t); free(g); free(qq); free(rr); free(hh);
    return np;
}

/* ------------------------------------------------------------------------ */
/* Encodings.                                                               */
/* Rq_encode (reading of the NTRU Prime mixed-radix Encode with every radix  */
/* equal to q): entries (r_i, m_i) with 0 <= r_i < m_i.  One pass merges     */
/* neighbouring entries into (r_i + m_i r_(i+1), m_i m_(i+1)) and, while the */
/* merged radix is at least 2^14, emits the low byte of the value and       */
/* replaces the radix by ceil(radix / 256); an unpaired last entry moves up  */
/* unchanged.  The pass's bytes precede those of the next pass.  A single    */
/* remaining entry is emitted byte by byte while its radix exceeds 1.       */
/* ------------------------------------------------------------------------ */
static size_t enc_rec(uint8_t *out, const uint64_t *R, const uint64_t *M,
                      size_t n)
{
    size_t len = 0;
    if (n == 0) return 0;
    if (n == 1) {
        uint64_t r = R[0], mm = M[0];
        while (mm > 1) {
            if (out) out[len] = (uint8_t)(r & 255);
            len++;
            r >>= 8;
            mm = (mm + 255) >> 8;
        }
        return len;
    }
    size_t n2 = (n + 1) / 2;
    uint64_t *R2 = malloc(8 * n2), *M2 = malloc(8 * n2);
    for (size_t i = 0; i + 1 < n; i += 2) {
        uint64_t mm = M[i] * M[i + 1];
        uint64_t r = R[i] + M[i] * R[i + 1];
        while (mm >= 16384) {
            if (out) out[len] = (uint8_t)(r & 255);
            len++;
            r >>= 8;
            mm = (mm + 255) >> 8;
        }
        R2[i / 2] = r;
        M2[i / 2] = mm;
    }
    if (n & 1) {
        R2[n2 - 1] = R[n - 1];
        M2[n2 - 1] = M[n - 1];
    }
    len += enc_rec(out ? out + len : NULL, R2, M2, n2);
    free(R2); free(M2);
    return len;
}

static void dec_rec(const uint8_t *in, uint64_t *R, const uint64_t *M, size_t n)
{
    if (n == 0) return;
    if (n == 1) {
        uint64_t mm = M[0], r = 0;
        int nb = 0;
        while (mm > 1) { nb++; mm = (mm + 255) >> 8; }
        for (int b = nb - 1; b >= 0; b--) r = (r << 8) | in[b];
        R[0] = M[0] ? r % M[0] : 0;
        return;
    }
    size_t n2 = (n + 1) / 2, npairs = n / 2, total = 0;
    uint64_t *R2 = malloc(8 * n2), *M2 = malloc(8 * n2);
    int *nbytes = malloc(sizeof(int) * (npairs + 1));
    for (size_t i = 0; i + 1 < n; i += 2) {
        uint64_t mm = M[i] * M[i + 1];
        int e = 0;
        while (mm >= 16384) { e++; mm = (mm + 255) >> 8; }
        M2[i / 2] = mm;
        nbytes[i / 2] = e;
        total += (size_t)e;
    }
    if (n & 1) M2[n2 - 1] = M[n - 1];
    dec_rec(in + total, R2, M2, n2);
    size_t off = 0;
    for (size_t i = 0; i + 1 < n; i += 2) {
        uint64_t r = R2[i / 2];
        int e = nbytes[i / 2];
        for (int b = e - 1; b >= 0; b--) r = (r << 8) | in[off + (size_t)b];
        off += (size_t)e;
        R[i] = r % M[i];
        R[i + 1] = (r / M[i]) % M[i + 1];
    }
    if (n & 1) R[n - 1] = R2[n2 - 1];
    free(R2); free(M2); free(nbytes);
}

/* h: p centred coefficients in [-(q-1)/2, (q-1)/2]; returns bytes written */
size_t orc_rq_encode(int p, int32_t q, const int16_t *h, uint8_t *out)
{
    uint64_t *R = malloc(8 * (size_t)p), *M = malloc(8 * (size_t)p);
    for (int i = 0; i < p; i++) {
        R[i] = (uint64_t)(h[i] + (q - 1) / 2);
        M[i] = (uint64_t)q;
    }
    size_t len = enc_rec(out, R, M, (size_t)p);
    free(R); free(M);
    return len;
}

size_t orc_rq_encoded_bytes(int p, int32_t q)
{
    uint64_t *R = calloc((size_t)p, 8), *M = malloc(8 * (size_t)p);
    for (int i = 0; i < p; i++) M[i] = (uint64_t)q;
    size_t len = enc_rec(NULL, R, M, (size_t)p);
    free(R); free(M);
    return len;
}

void orc_rq_decode(int p, int32_t q, const uint8_t *in, int16_t *h)
{
    uint64_t *R = calloc((size_t)p, 8), *M = calloc((size_t)p, 8);
    for (int i = 0; i < p; i++) M[i] = (uint64_t)q;
    dec_rec(in, R, M, (size_t)p);
    for (int i = 0; i < p; i++) h[i] = (int16_t)((int64_t)R[i] - (q - 1) / 2);
    free(R); free(M);
}

/* Small_encode: four coefficients per byte, coefficient c stored as c + 1 in
 * two bits, lowest index in the lowest bits; ceil(p/4) bytes. */
void orc_small_encode(int p, const int8_t *c, uint8_t *out)
{
    for (int j = 0; j < (p + 3) / 4; j++) {
        unsigned byte = 0;
        for (int t = 0; t < 4; t++) {
            int i = 4 * j + t;
            if (i < p) byte |= (unsigned)(c[i] + 1) << (2 * t);
        }
        out[j] = (uint8_t)byte;
    }
}

void orc_small_decode(int p, const uint8_t *in, int8_t *c)
{
    for (int i = 0; i < p; i++)
        c[i] = (int8_t)((int)((in[i / 4] >> (2 * (i % 4))) & 3) - 1);
}

/* ------------------------------------------------------------------------ */
/* SHA-512 (FIPS 180-4, Sec. 6.4).                                          */
/* ------------------------------------------------------------------------ */
static const uint64_t SHA512_K[80] = {
    0x428a2f98d728ae22ULL, 0x7137449123ef65cdULL, 0xb5c0fbcfec4d3b2fULL, 0xe9b5dba58189dbbcULL,
    0x3956c25bf348b538ULL, 0x59f111f1b605d019ULL, 0x923f82a4af194f9bULL, 0xab1c5ed5da6d8118ULL,
    0xd807aa98a3030242ULL, 0x12835b0145706fbeULL, 0x243185be4ee4b28cULL, 0x550c7dc3d5ffb4e2ULL,
    0x72be5d74f27b896fULL, 0x80deb1fe3b1696b1ULL, 0x9bdc06a725c71235ULL, 0xc19bf174cf692694ULL,
    0xe49b69c19ef14ad2ULL, 0xefbe4786384f25e3ULL, 0x0fc19dc68b8cd5b5ULL, 0x240ca1cc77ac9c65ULL,
    0x2de92c6f592b0275ULL, 0x4a7484aa6ea6e483ULL, 0x5cb0a9dcbd41fbd4ULL, 0x76f988da831153b5ULL,
    0x983e5152ee66dfabULL, 0xa831c66d2db43210ULL, 0xb00327c898fb213fULL, 0xbf597fc7beef0ee4ULL,
    0xc6e00bf33da88fc2ULL, 0xd5a79147930aa725ULL, 0x06ca6351e003826fULL, 0x142929670a0e6e70ULL,
    0x27b70a8546d22ffcULL, 0x2e1b21385c26c926ULL, 0x4d2c6dfc5ac42aedULL, 0x53380d139d95b3dfULL,
    0x650a73548baf63deULL, 0x766a0abb3c77b2a8ULL, 0x81c2c92e47edaee6ULL, 0x92722c851482353bULL,
    0xa2bfe8a14cf10364ULL, 0xa81a664bbc423001ULL, 0xc24b8b70d0f89791ULL, 0xc76c51a30654be30ULL,
    0xd192e819d6ef5218ULL, 0xd69906245565a910ULL, 0xf40e35855771202aULL, 0x106aa07032bbd1b8ULL,
    0x19a4c116b8d2d0c8ULL, 0x1e376c085141ab53ULL, 0x2748774cdf8eeb99ULL, 0x34b0bcb5e19b48a8ULL,
    0x391c0cb3c5c95a63ULL, 0x4ed8aa4ae3418acbULL, 0x5b9cca4f7763e373ULL, 0x682e6ff3d6b2b8a3ULL,
    0x748f82ee5defb2fcULL, 0x78a5636f43172f60ULL, 0x84c87814a1f0ab72ULL, 0x8cc702081a6439ecULL,
    0x90befffa23631e28ULL, 0xa4506cebde82bde9ULL, 0xbef9a3f7b2c67915ULL, 0xc67178f2e372532bULL,
    0xca273eceea26619cULL, 0xd186b8c721c0c207ULL, 0xeada7dd6cde0eb1eULL, 0xf57d4f7fee6ed178ULL,
    0x06f067aa72176fbaULL, 0x0a637dc5a2c898a6ULL, 0x113f9804bef90daeULL, 0x1b710b35131c471bULL,
    0x28db77f523047d84ULL, 0x32caab7b40c72493ULL, 0x3c9ebe0a15c9bebcULL, 0x431d67c49c100d4cULL,
    0x4cc5d4becb3e42b6ULL, 0x597f299cfc657e2aULL, 0x5fcb6fab3ad6faecULL, 0x6c44198c4a475817ULL,
};

static const uint64_t SHA512_H0[8] = {
    0x6a09e667f3bcc908ULL, 0xbb67ae8584caa73bULL, 0x3c6ef372fe94f82bULL, 0xa54ff53a5f1d36f1ULL,
    0x510e527fade682d1ULL, 0x9b05688c2b3e6c1fULL, 0x1f83d9abfb41bd6bULL, 0x5be0cd19137e2179ULL,
};

static uint64_t rotr64(uint64_t x, int n) { return (x >> n) | (x << (64 - n)); }

static void sha512_block(uint64_t H[8], const uint8_t blk[128])
{
    uint64_t W[80];
    for (int t = 0; t < 16; t++) {
        uint64_t v = 0;
        for (int b = 0; b < 8; b++) v = (v << 8) | blk[8 * t + b];
        W[t] = v;
    }
    for (int t = 16; t < 80; t++) {
        uint64_t s0 = rotr64(W[t - 15], 1) ^ rotr64(W[t - 15], 8) ^ (W[t - 15] >> 7);
        uint64_t s1 = rotr64(W[t - 2], 19) ^ rotr64(W[t - 2], 61) ^ (W[t - 2] >> 6);
        W[t] = W[t - 16] + s0 + W[t - 7] + s1;
    }
    uint64_t a = H[0], b = H[1], c = H[2], d = H[3], e = H[4], f = H[5],
             g = H[6], h = H[7];
    for (int t = 0; t < 80; t++) {
        uint64_t S1 = rotr64(e, 14) ^ rotr64(e, 18) ^ rotr64(e, 41);
        uint64_t ch = (e & f) ^ (~e & g);
        uint64_t T1 = h + S1 + ch + SHA512_K[t] + W[t];
        uint64_t S0 = rotr64(a, 28) ^ rotr64(a, 34) ^ rotr64(a, 39);
        uint64_t maj = (a & b) ^ (a & c) ^ (b & c);
        uint64_t T2 = S0 + maj;
        h = g; g = f; f = e; e = d + T1;
        d = c; c = b; b = a; a = T1 + T2;
    }
    H[0] += a; H[1] += b; H[2] += c; H[3] += d;
    H[4] += e; H[5] += f; H[6] += g; H[7] += h;
}

void orc_sha512(const uint8_t *msg, size_t len, uint8_t out[64])
{
    uint64_t H[8];
    memcpy(H, SHA512_H0, sizeof(H));
    size_t full = len / 128;
    for (size_t i = 0; i < full; i++) sha512_block(H, msg + 128 * i);
    uint8_t tail[256];
    memset(tail, 0, sizeof(tail));
    size_t rem = len - 128 * full;
    memcpy(tail, msg + 128 * full, rem);
    tail[rem] = 0x80;
    size_t tl = (rem + 1 + 16 <= 128) ? 128 : 256;
    uint64_t bits = (uint64_t)len * 8u; /* messages here are < 2^61 bytes */
    for (int b = 0; b < 8; b++) tail[tl - 1 - b] = (uint8_t)(bits >> (8 * b));
    sha512_block(H, tail);
    if (tl == 256) sha512_block(H, tail + 128);
    for (int i = 0; i < 8; i++)
        for (int b = 0; b < 8; b++) out[8 * i + b] = (uint8_t)(H[i] >> (56 - 8 * b));
}

/* ------------------------------------------------------------------------ */
/* Sizes and key generation                                                 */
/* ------------------------------------------------------------------------ */
/* sk = Small_encode(f) | Small_encode(1/g) | pk | rho | Hash_prefix(4, pk),
 * rho has Small_encode's length, the hash prefix is 32 bytes. */
void orc_sizes(int p, int32_t q, size_t *pk_bytes, size_t *sk_bytes,
               size_t *small_bytes)
{
    size_t sb = (size_t)(p + 3) / 4;
    size_t pkb = orc_rq_encoded_bytes(p, q);
    if (small_bytes) *small_bytes = sb;
    if (pk_bytes) *pk_bytes = pkb;
    if (sk_bytes) *sk_bytes = 3 * sb + pkb + 32;
}

/*
 * One key pair, index k (Sec. 3.1 KeyGen, with the randomness reading above).
 *   g: attempt a = 0, 1, ... of stream 0 until invertible in R/3
 *      (g_attempt0, if not NULL, replaces the attempt-0 draw: test hook for
 *      the resampling path);
 *   f: stream 1 (independent of how many g attempts were needed);
 *   v = 1/g in R/3, a = 3f, ainv = 1/a in R/q, h = g * ainv in R/q.
 * Returns the number of g attempts used (>= 1), or -1 if max_attempts ran
 * out.  Optional intermediates (f, g, v, h) are written when non-NULL.
 */
int orc_keygen(int p, int32_t q, int w, uint64_t seed, uint64_t k,
               const int8_t *g_attempt0, int max_attempts, uint8_t *pk,
               uint8_t *sk, int8_t *f_out, int8_t *g_out, int8_t *v_out,
               int16_t *h_out)
{
    int8_t *g = malloc((size_t)p), *f = malloc((size_t)p), *v = malloc((size_t)p);
    int32_t *g32 = malloc(4 * (size_t)p), *v32 = malloc(4 * (size_t)p),
            *a32 = malloc(4 * (size_t)p), *ai32 = malloc(4 * (size_t)p),
            *h32 = malloc(4 * (size_t)p);
    int16_t *h = malloc(2 * (size_t)p);
    int attempts = -1;
    for (int att = 0; att < max_attempts; att++) {
        if (att == 0 && g_attempt0) memcpy(g, g_attempt0, (size_t)p);
        else orc_sample_small(p, seed, k, (uint32_t)att, g);
        for (int i = 0; i < p; i++) g32[i] = g[i];
        if (orc_ring_inv(p, 3, g32, v32)) {
            attempts = att + 1;
            break;
        }
    }
    if (attempts < 0) goto done;
    for (int i = 0; i < p; i++) v[i] = (int8_t)v32[i];
    orc_sample_short(p, w, seed, k, f);
    for (int i = 0; i < p; i++) a32[i] = 3 * f[i];
    if (!orc_ring_inv(p, q, a32, ai32)) { attempts = -2; goto done; } /* cannot happen: R/q is a field */
    orc_ring_mul(p, q, g32, ai32, h32);
    for (int i = 0; i < p; i++) h[i] = (int16_t)h32[i];

    size_t sb, pkb, skb;
    orc_sizes(p, q, &pkb, &skb, &sb);
    if (pk) orc_rq_encode(p, q, h, pk);
    if (sk) {
        uint8_t *pkbuf = malloc(pkb), *hin = malloc(pkb + 1), digest[64];
        orc_rq_encode(p, q, h, pkbuf);
        orc_small_encode(p, f, sk);
        orc_small_encode(p, v, sk + sb);
        memcpy(sk + 2 * sb, pkbuf, pkb);
        orc_rho((int)sb, seed, k, sk + 2 * sb + pkb);
        hin[0] = 4;
        memcpy(hin + 1, pkbuf, pkb);
        orc_sha512(hin, pkb + 1, digest);
        memcpy(sk + 3 * sb + pkb, digest, 32);
        free(pkbuf); free(hin);
    }
    if (f_out) memcpy(f_out, f, (size_t)p);
    if (g_out) memcpy(g_out, g, (size_t)p);
    if (v_out) memcpy(v_out, v, (size_t)p);
    if (h_out) memcpy(h_out, h, 2 * (size_t)p);
done:
    free(g); free(f); free(v); free(g32); free(v32); free(a32); free(ai32);
    free(h32); free(h);
    return attempts;
}

/* ------------------------------------------------------------------------ */
/* Encapsulation and decapsulation (the serving path).  The paper measures   */
/* them (Table 1) and defers their definition to the NTRU Prime             */
/* specification; reading (round-3 Streamlined NTRU Prime KEM):             */
/*   Round(a): each coefficient to the nearest multiple of 3 (centred).      */
/*   Rounded_encode: Encode of (c_i + (q-1)/2) / 3 with radix (q+2)/3.       */
/*   Hash_prefix(b, x) = SHA-512(b | x)[0:32].                              */
/*   Encap(pk; r Short from stream 3):                                      */
/*     c = Round(h r), C = Rounded_encode(c), r_enc = Small_encode(r),       */
/*     confirm = Hash_prefix(2, Hash_prefix(3, r_enc) | Hash_prefix(4, pk)), */
/*     ct = C | confirm, ss = Hash_prefix(1, Hash_prefix(3, r_enc) | ct).    */
/*   Decap(ct, sk):                                                         */
/*     e = (3 f c mod q, centred) mod 3, r' = e v in R/3 (v = 1/g);           */
/*     if weight(r') != w: r' = (1, ..., 1 (w times), 0, ..., 0);            */
/*     re-encrypt r' to ct'; ss = Hash_prefix(1, Hash_prefix(3, r'_enc) | ct)*/
/*     if ct' == ct, else Hash_prefix(0, Hash_prefix(3, rho) | ct).          */
/* ------------------------------------------------------------------------ */
static void hash_prefix(uint8_t b, const uint8_t *x, size_t len, uint8_t out[32])
{
    uint8_t *m = malloc(len + 1), d[64];
    m[0] = b;
    memcpy(m + 1, x, len);
    orc_sha512(m, len + 1, d);
    memcpy(out, d, 32);
    free(m);
}

size_t orc_rounded_bytes(int p, int32_t q)
{
    uint64_t *R = calloc((size_t)p, 8), *M = malloc(8 * (size_t)p);
    for (int i = 0; i < p; i++) M[i] = (uint64_t)((q + 2) / 3);
    size_t len = enc_rec(NULL, R, M, (size_t)p);
    free(R); free(M);
    return len;
}

/* c: centred multiples of 3 */
void rounded_encode(int p, int32_t q, const int32_t *c, uint8_t *out)
{
    uint64_t *R = malloc(8 * (size_t)p), *M = malloc(8 * (size_t)p);
    for (int i = 0; i < p; i++) {
        R[i] = (uint64_t)((c[i] + (q - 1) / 2) / 3);
        M[i] = (uint64_t)((q + 2) / 3);
    }
    enc_rec(out, R, M, (size_t)p);
    free(R); free(M);
}

void rounded_decode(int p, int32_t q, const uint8_t *in, int32_t *c)
{
    uint64_t *R = calloc((size_t)p, 8), *M = malloc(8 * (size_t)p);
    for (int i = 0; i < p; i++) M[i] = (uint64_t)((q + 2) / 3);
    dec_rec(in, R, M, (size_t)p);
    for (int i = 0; i < p; i++) c[i] = (int32_t)(3 * (int64_t)R[i] - (q - 1) / 2);
    free(R); free(M);
}

/* Round(h r) for the centred product */
static void round3(int p, int32_t q, const int32_t *hr, int32_t *c)
{
    for (int i = 0; i < p; i++) c[i] = hr[i] - centred(hr[i], 3);
    (void)q;
}

/* ct = Rounded_encode(Round(h r)) | confirm; returns via ct (length
 * rounded_bytes + 32); h3_out = Hash_prefix(3, Small_encode(r)). */
static void encrypt_confirm(int p, int32_t q, const int32_t *h, const int8_t *r,
                            const uint8_t cache[32], uint8_t *ct, uint8_t h3_out[32])
{
    size_t rb = orc_rounded_bytes(p, q), sb = (size_t)(p + 3) / 4;
    int32_t *r32 = malloc(4 * (size_t)p), *hr = malloc(4 * (size_t)p), *c = malloc(4 * (size_t)p);
    for (int i = 0; i < p; i++) r32[i] = r[i];
    orc_ring_mul(p, q, h, r32, hr);
    round3(p, q, hr, c);
    rounded_encode(p, q, c, ct);
    uint8_t *renc = malloc(sb), buf[64];
    orc_small_encode(p, r, renc);
    hash_prefix(3, renc, sb, h3_out);
    memcpy(buf, h3_out, 32);
    memcpy(buf + 32, cache, 32);
    hash_prefix(2, buf, 64, ct + rb);
    free(r32); free(hr); free(c); free(renc);
}

/* Encapsulation for key index k of the request stream (r from stream 3). */
void orc_encap(int p, int32_t q, int w, const uint8_t *pk, uint64_t seed, uint64_t k,
               uint8_t *ct, uint8_t ss[32])
{
    size_t pkb = orc_rq_encoded_bytes(p, q), rb = orc_rounded_bytes(p, q);
    int16_t *h16 = malloc(2 * (size_t)p);
    int32_t *h = malloc(4 * (size_t)p);
    int8_t *r = malloc((size_t)p);
    orc_rq_decode(p, q, pk, h16);
    for (int i = 0; i < p; i++) h[i] = h16[i];
    orc_sample_short_stream(p, w, seed, k, 3, r);
    uint8_t cache[32], h3[32];
    hash_prefix(4, pk, pkb, cache);
    encrypt_confirm(p, q, h, r, cache, ct, h3);
    uint8_t *buf = malloc(32 + rb + 32);
    memcpy(buf, h3, 32);
    memcpy(buf + 32, ct, rb + 32);
    hash_prefix(1, buf, 32 + rb + 32, ss);
    free(buf); free(h16); free(h); free(r);
}

/* Decapsulation; returns 1 if the ciphertext was accepted (re-encryption
 * matched), 0 if the implicit-rejection key was produced. */
int orc_decap(int p, int32_t q, int w, const uint8_t *sk, const uint8_t *ct, uint8_t ss[32])
{
    size_t sb = (size_t)(p + 3) / 4, pkb = orc_rq_encoded_bytes(p, q), rb = orc_rounded_bytes(p, q);
    const uint8_t *pk = sk + 2 * sb, *rho = sk + 2 * sb + pkb, *cache = sk + 3 * sb + pkb;
    int8_t *f = malloc((size_t)p), *v = malloc((size_t)p), *rr = malloc((size_t)p);
    int32_t *c = malloc(4 * (size_t)p), *f3 = malloc(4 * (size_t)p), *e = malloc(4 * (size_t)p),
            *e3 = malloc(4 * (size_t)p), *v32 = malloc(4 * (size_t)p), *r32 = malloc(4 * (size_t)p),
            *h = malloc(4 * (size_t)p);
    int16_t *h16 = malloc(2 * (size_t)p);
    orc_small_decode(p, sk, f);
    orc_small_decode(p, sk + sb, v);
    rounded_decode(p, q, ct, c);
    for (int i = 0; i < p; i++) f3[i] = 3 * f[i];
    orc_ring_mul(p, q, c, f3, e);                      /* 3 f c, centred */
    for (int i = 0; i < p; i++) { e3[i] = centred(e[i], 3); v32[i] = v[i]; }
    orc_ring_mul(p, 3, e3, v32, r32);                  /* r' = e v in R/3 */
    int weight = 0;
    for (int i = 0; i < p; i++) weight += (r32[i] != 0);
    for (int i = 0; i < p; i++) rr[i] = (int8_t)(weight == w ? r32[i] : (i < w ? 1 : 0));
    orc_rq_decode(p, q, pk, h16);
    for (int i = 0; i < p; i++) h[i] = h16[i];
    uint8_t *ct2 = malloc(rb + 32), h3[32];
    encrypt_confirm(p, q, h, rr, cache, ct2, h3);
    int ok = (memcmp(ct2, ct, rb + 32) == 0);
    uint8_t *buf = malloc(32 + rb + 32);
    if (ok) {
        memcpy(buf, h3, 32);
    } else {
        hash_prefix(3, rho, sb, buf);
    }
    memcpy(buf + 32, ct, rb + 32);
    hash_prefix(ok ? 1 : 0, buf, 32 + rb + 32, ss);
    free(buf); free(ct2); free(f); free(v); free(rr); free(c); free(f3); free(e); free(e3);
    free(v32); free(r32); free(h); free(h16);
    return ok;
}
