"""Pins of the CPU oracle against things other than itself (no GPU).

Each test ties one oracle routine to a fact fixed by the paper (arXiv
2106.08759) or by mathematics: printed parameters and sizes, the factor
degrees of x^761 - x - 1 mod 3 (Sec. 3.1.1), field-theoretic closed forms
(Fermat / Lagrange exponents), brute force over toy rings, big-integer
(Kronecker) products, hashlib's SHA-512 and the Philox known answers.
"""
import hashlib
import random

import numpy as np
import pytest

import oracle
from conftest import read_golden

PARAMS = {int(r[0]): (int(r[0]), int(r[1]), int(r[2])) for r in read_golden("params.txt")}


def test_params_match_paper():
    assert PARAMS == oracle.PARAMS


# ---------------------------------------------------------------- randomness
def test_philox_known_answers():
    for row in read_golden("philox4x32_10_kat.txt"):
        vals = [int(x, 16) for x in row]
        out = oracle.philox4x32_10(vals[0:4], vals[4:6])
        assert list(out) == vals[6:10]


def test_random_words_counter_layout():
    # word i of (stream, attempt, k) is lane i%4 of one Philox block
    seed, k = 0x0123456789ABCDEF, (7 << 32) | 5
    w = oracle.random_words(seed, k, 1, 3, 10)
    for i in range(10):
        blk = oracle.philox4x32_10([(1 << 16) | (i // 4), 3, k & 0xffffffff, k >> 32],
                                   [seed & 0xffffffff, seed >> 32])
        assert w[i] == blk[i % 4]


def _philox_words(seed, k, stream, attempt, n):
    """n words of the randomness reading, built here from single Philox
    blocks (pinned by the known answers above): word j is lane j mod 4 of the
    block with counter ((stream << 16) | (j / 4), attempt, k mod 2^32, k >> 32)."""
    key = [seed & 0xffffffff, seed >> 32]
    return [int(oracle.philox4x32_10([(stream << 16) | (j // 4), attempt, k & 0xffffffff, k >> 32],
                                     key)[j % 4]) for j in range(n)]


@pytest.mark.parametrize("p", [653, 761, 857])
def test_rho_is_stream_2_little_endian(p):
    # rho (the implicit-rejection part of sk): byte j is byte j mod 4 of word
    # j / 4 of stream 2, least significant byte first; pinned against Philox
    # blocks and an explicit byte split, and in the oracle's own keys
    sb = (p + 3) // 4
    pkb, _, _ = oracle.sizes(p)
    for seed, k in [(0x0123456789ABCDEF, 0), (1, (3 << 32) | 77), (0xFFFFFFFFFFFFFFFF, 4095)]:
        words = _philox_words(seed, k, 2, 0, (sb + 3) // 4)
        want = b"".join(w.to_bytes(4, "little") for w in words)[:sb]
        assert oracle.rho(sb, seed, k).tobytes() == want
        if k < 5000:
            _, sk, _ = oracle.keygen(p, seed, k)
            assert sk[2 * sb + pkb:3 * sb + pkb].tobytes() == want


@pytest.mark.parametrize("p", [653, 761, 857])
def test_small_g_is_scaled_stream_0_words(p):
    # g coefficient i at attempt a: floor(3 (u mod 2^30) / 2^30) - 1 for word
    # i of stream 0, attempt a (integer arithmetic in Python)
    for seed, k, a in [(99, 3, 0), (5, 1 << 33, 2)]:
        words = _philox_words(seed, k, 0, a, p)
        want = [((u & (2**30 - 1)) * 3 >> 30) - 1 for u in words]
        assert oracle.sample_small(p, seed, k, a).tolist() == want


@pytest.mark.parametrize("p", [653, 761, 857])
def test_short_f_is_sorted_forced_stream_1_words(p):
    # Short f: p words of stream 1, the first w with bit 0 cleared (low bits
    # 00 or 10: coefficient -1 or +1), the rest with low bits 01 (zero),
    # sorted as unsigned integers (Python's sort), coefficient = low 2 bits - 1
    w = PARAMS[p][2]
    for seed, k in [(99, 3), (0xDEADBEEF, 1 << 40)]:
        words = _philox_words(seed, k, 1, 0, p)
        forced = [u & ~1 & 0xffffffff if i < w else (u & ~3 & 0xffffffff) | 1
                  for i, u in enumerate(words)]
        want = [(u & 3) - 1 for u in sorted(forced)]
        assert oracle.sample_short(p, w, seed, k).tolist() == want


# ------------------------------------------------------------------ sampling
@pytest.mark.parametrize("p", [653, 761, 857])
def test_short_and_small_invariants(p):
    _, q, w = PARAMS[p]
    for k in range(20):
        f = oracle.sample_short(p, w, 99, k)
        assert np.count_nonzero(f) == w
        assert set(np.unique(f)) <= {-1, 0, 1}
        g = oracle.sample_small(p, 99, k, 0)
        assert set(np.unique(g)) <= {-1, 0, 1}


def test_sampling_distributions():
    # g coefficients uniform over {-1,0,1}; Short positions uniform; signs balanced
    p, q, w = PARAMS[761]
    gs = np.concatenate([oracle.sample_small(p, 5, k, 0) for k in range(200)])
    counts = np.array([(gs == v).sum() for v in (-1, 0, 1)])
    exp = gs.size / 3
    assert ((counts - exp) ** 2 / exp).sum() < 20  # chi^2, 2 dof
    fs = np.stack([oracle.sample_short(p, w, 6, k) for k in range(400)])
    pos = (fs != 0).mean(axis=0)  # each position nonzero w.p. w/p
    assert abs(pos.mean() - w / p) < 1e-9
    assert np.abs(pos - w / p).max() < 0.12
    signs = fs[fs != 0]
    assert abs((signs == 1).mean() - 0.5) < 0.01


# ------------------------------------------------------------ multiplication
def kron_mul_reduce(a, b, p, m):
    """Independent product: Kronecker substitution with Python integers,
    then long division by the monic x^p - x - 1."""
    base = 1 << 64
    off = 1 << 40
    A = sum((int(x) + m) << (64 * i) for i, x in enumerate(a))
    B = sum((int(x) + m) << (64 * i) for i, x in enumerate(b))
    C = A * B
    # unpack (a_i+m)(b_j+m) sums: subtract the known offset terms
    raw = []
    for i in range(2 * p - 1):
        raw.append((C >> (64 * i)) & (base - 1))
    sa = sum(int(x) + m for x in a)
    sb = sum(int(x) + m for x in b)
    del sa, sb
    # c_k = sum (a_i+m)(b_j+m) - m*sum_{i+j=k} a_i - m*sum b_j - m^2 * #terms
    Aa = [int(x) for x in a]
    Bb = [int(x) for x in b]
    pa = [0] + list(np.cumsum(Aa))
    pb = [0] + list(np.cumsum(Bb))
    c = []
    for k in range(2 * p - 1):
        lo, hi = max(0, k - p + 1), min(k, p - 1)
        n = hi - lo + 1
        s_a = pa[hi + 1] - pa[lo]
        s_b = pb[k - lo + 1] - pb[k - hi]
        c.append(int(raw[k]) - m * s_a - m * s_b - m * m * n)
    # long division by x^p - x - 1 (monic): top coefficient t of x^d, d >= p,
    # subtract t*x^(d-p)*(x^p - x - 1)
    for d in range(2 * p - 2, p - 1, -1):
        t = c[d]
        c[d] = 0
        c[d - p + 1] += t
        c[d - p] += t
    out = [x % m for x in c[:p]]
    return np.array([x - m if x > (m - 1) // 2 else x for x in out], np.int64)


@pytest.mark.parametrize("p", [653, 761, 857])
def test_ring_mul_vs_kronecker(p):
    _, q, _ = PARAMS[p]
    rng = np.random.default_rng(p)
    half = (q - 1) // 2
    cases = [
        (rng.integers(-half, half + 1, p), rng.integers(-half, half + 1, p)),
        (np.full(p, half), np.full(p, half)),
        (np.full(p, -half), np.full(p, half)),
        (rng.integers(-1, 2, p), rng.integers(-half, half + 1, p)),
    ]
    for a, b in cases:
        got = oracle.ring_mul(p, q, a, b)
        assert np.array_equal(got, kron_mul_reduce(a, b, p, q))
    # R/3 arithmetic through the same routine
    a, b = rng.integers(-1, 2, p), rng.integers(-1, 2, p)
    assert np.array_equal(oracle.ring_mul(p, 3, a, b), kron_mul_reduce(a, b, p, 3))


def test_ring_mul_monomials():
    # x^i * x^j = x^(i+j) with x^p = x + 1 applied once
    p, q, _ = PARAMS[761]
    for i, j in [(0, 0), (1, p - 1), (p - 1, p - 1), (300, 500)]:
        a = np.zeros(p, np.int64); a[i] = 1
        b = np.zeros(p, np.int64); b[j] = 1
        exp = np.zeros(p, np.int64)
        k = i + j
        if k < p:
            exp[k] = 1
        else:
            exp[k - p] += 1
            exp[k - p + 1] += 1
        assert np.array_equal(oracle.ring_mul(p, q, a, b), exp)


# ----------------------------------------------------------------- inversion
def test_factor_degrees_mod3_match_paper():
    # Sec. 3.1.1: x^761 - x - 1 splits mod 3 into irreducibles of degree 19, 60, 682.
    row = read_golden("factor_degrees_mod3.txt")[0]
    p, degs = int(row[0]), sorted(int(x) for x in row[1:])
    parts = oracle.ddf(p, 3)
    # each distinct-degree part is a single irreducible here (total == d)
    assert sorted(d for d, tot, _ in parts) == degs
    assert all(d == tot for d, tot, _ in parts)
    # and the parts multiply back to x^p - x - 1
    prod = np.zeros(1, np.int64); prod[0] = 1
    for _, _, poly in parts:
        prod = np.convolve(prod, poly[: int(np.nonzero(poly)[0].max()) + 1]) % 3
    exp = np.zeros(p + 1, np.int64); exp[p] = 1; exp[1] = 2; exp[0] = 2
    assert np.array_equal(prod, exp)


def test_rq_inverse_matches_fermat():
    # In the field F_{q^p}, a^-1 = a^(q^p - 2) (no Euclid involved).
    p, q, _ = PARAMS[761]
    rng = np.random.default_rng(1)
    a = rng.integers(-(q - 1) // 2, (q - 1) // 2 + 1, p)
    ok, inv = oracle.ring_inv(p, q, a)
    assert ok
    assert np.array_equal(inv, oracle.ring_pow(p, q, a, q ** p - 2))


def test_r3_inverse_matches_lagrange():
    # R/3 = F_3[x]/(f1 f2 f3) with deg 19, 60, 682 (Sec. 3.1.1); its unit group
    # has order N = prod(3^d - 1), so a^-1 = a^(N-1) for every unit a.
    p = 761
    N = 1
    for d in (19, 60, 682):
        N *= 3 ** d - 1
    rng = np.random.default_rng(2)
    for _ in range(2):
        a = rng.integers(-1, 2, p)
        ok, inv = oracle.ring_inv(p, 3, a)
        assert ok
        assert np.array_equal(inv, oracle.ring_pow(p, 3, a, N - 1))
        assert np.array_equal(oracle.ring_mul(p, 3, a, inv), np.eye(1, p, 0, dtype=np.int64)[0])


def _all_elements(p, m):
    idx = np.arange(m ** p)
    digits = np.stack([(idx // m ** i) % m for i in range(p)], axis=1)
    return digits


def _toy_mul_all(a, B, p, m):
    """a times every row of B in (Z/m)[x]/(x^p - x - 1), vectorised."""
    n = B.shape[0]
    c = np.zeros((n, 2 * p - 1), np.int64)
    for i in range(p):
        c[:, i:i + p] += int(a[i]) * B
    for k in range(2 * p - 2, p - 1, -1):
        c[:, k - p + 1] += c[:, k]
        c[:, k - p] += c[:, k]
    return c[:, :p] % m


@pytest.mark.parametrize("p0,m", [(7, 3), (5, 3), (3, 13)])
def test_inverse_brute_force_toy(p0, m):
    """Exhaustive search of inverses in (Z/m)[x]/(x^p0 - x - 1)."""
    if m != 3:
        # the R/q analogue must be a field: the oracle checks irreducibility itself
        assert [(d, t) for d, t, _ in oracle.ddf(p0, m)] == [(p0, p0)]
    E = _all_elements(p0, m)
    one = np.zeros(p0, np.int64); one[0] = 1
    n_inv = 0
    for a in E:
        prods = _toy_mul_all(a, E, p0, m)
        hits = np.nonzero((prods == one).all(axis=1))[0]
        ok, inv = oracle.ring_inv(p0, m, a)
        assert ok == (hits.size == 1)
        if ok:
            n_inv += 1
            assert np.array_equal(inv % m, E[hits[0]])
        else:
            assert hits.size == 0
    if m == 3:
        # units of prod F_3[x]/(f_i) number prod(3^deg - 1)
        N = 1
        for d, tot, _ in oracle.ddf(p0, 3):
            assert d == tot or tot % d == 0
            for _ in range(tot // d):
                N *= 3 ** d - 1
        assert n_inv == N
    else:
        assert n_inv == m ** p0 - 1


def test_non_invertible_g_from_factor():
    # g = f1 * r with f1 the degree-19 factor (Sec. 3.1.1) is a zero divisor in R/3
    p = 761
    parts = oracle.ddf(p, 3)
    f1 = [poly for d, _, poly in parts if d == 19][0][:20]
    rng = np.random.default_rng(3)
    r = rng.integers(0, 3, p - 19)
    g = np.convolve(f1, r) % 3
    g = np.where(g == 2, -1, g)
    assert g.size == p
    ok, _ = oracle.ring_inv(p, 3, g)
    assert not ok


# ----------------------------------------------------------------- encodings
@pytest.mark.parametrize("p", [653, 761, 857])
def test_sizes_match_table4(p):
    storage = {int(r[0]): int(r[1]) for r in read_golden("table4_keypair_storage.txt")}
    pkb, skb, sb = oracle.sizes(p)
    assert sb == (p + 3) // 4
    assert pkb + skb == storage[p]


@pytest.mark.parametrize("p", [653, 761, 857])
def test_rq_encode_roundtrip(p):
    _, q, _ = PARAMS[p]
    half = (q - 1) // 2
    rng = np.random.default_rng(p + 1)
    cases = [rng.integers(-half, half + 1, p), np.full(p, half), np.full(p, -half),
             np.zeros(p, np.int64)]
    for h in cases:
        enc = oracle.rq_encode(p, q, h)
        assert np.array_equal(oracle.rq_decode(p, q, enc), h)
    # injective on a sample: distinct inputs -> distinct encodings
    encs = {bytes(oracle.rq_encode(p, q, rng.integers(-half, half + 1, p))) for _ in range(50)}
    assert len(encs) == 50


def test_rq_encode_is_mixed_radix_bijection_small():
    # For tiny inputs the encoding is the base-q number sum r_i q^i written in
    # little-endian bytes whenever no intermediate radix reaches 2^14.
    q = 7
    for p in (1, 2, 3, 4):
        for trial in range(20):
            rng = np.random.default_rng(trial)
            h = rng.integers(-3, 4, p)
            enc = oracle.rq_encode(p, q, h)
            val = sum(int(x + 3) * q ** i for i, x in enumerate(h))
            assert int.from_bytes(bytes(enc), "little") == val
            nbytes, m = 0, q ** p
            while m > 1:
                nbytes, m = nbytes + 1, (m + 255) // 256
            assert len(enc) == nbytes


@pytest.mark.parametrize("p", [653, 761, 857])
def test_small_encode_roundtrip(p):
    rng = np.random.default_rng(p + 2)
    c = rng.integers(-1, 2, p).astype(np.int8)
    enc = oracle.small_encode(p, c)
    assert enc.size == (p + 3) // 4
    assert np.array_equal(oracle.small_decode(p, enc), c)


def test_sha512_vs_hashlib():
    rng = random.Random(5)
    for n in [0, 1, 3, 111, 112, 113, 127, 128, 129, 255, 256, 995, 1159, 1323, 4000]:
        msg = bytes(rng.randrange(256) for _ in range(n))
        assert oracle.sha512(msg) == hashlib.sha512(msg).digest()


# --------------------------------------------------------------------- keygen
@pytest.mark.parametrize("p", [653, 761, 857])
def test_keygen_identities(p):
    _, q, w = PARAMS[p]
    pkb, skb, sb = oracle.sizes(p)
    for k in range(3):
        r = oracle.keygen(p, 0x0123456789ABCDEF, k, intermediates=True)
        f, g, v, h = (r[x].astype(np.int64) for x in "fgvh")
        # g * (1/g) = 1 in R/3
        assert np.array_equal(oracle.ring_mul(p, 3, g, v), np.eye(1, p, 0, dtype=np.int64)[0])
        # h * 3f = g in R/q
        assert np.array_equal(oracle.ring_mul(p, q, h, 3 * f), g)
        # f * (1/f) = 1 in R/q
        ok, finv = oracle.ring_inv(p, q, f)
        assert ok and np.array_equal(oracle.ring_mul(p, q, f, finv), np.eye(1, p, 0, dtype=np.int64)[0])
        assert np.abs(h).max() <= (q - 1) // 2
        assert np.count_nonzero(f) == w
        pk, sk = r["pk"], r["sk"]
        assert pk.size == pkb and sk.size == skb
        assert np.array_equal(oracle.rq_decode(p, q, pk), h)
        assert np.array_equal(oracle.small_decode(p, sk[:sb]), f)
        assert np.array_equal(oracle.small_decode(p, sk[sb:2 * sb]), v)
        assert np.array_equal(sk[2 * sb:2 * sb + pkb], pk)
        assert np.array_equal(sk[2 * sb + pkb:3 * sb + pkb], oracle.rho(sb, 0x0123456789ABCDEF, k))
        assert bytes(sk[3 * sb + pkb:]) == hashlib.sha512(b"\x04" + bytes(pk)).digest()[:32]
        assert np.array_equal(r["g"], oracle.sample_small(p, 0x0123456789ABCDEF, k, r["attempts"] - 1))
        assert np.array_equal(r["f"], oracle.sample_short(p, w, 0x0123456789ABCDEF, k))


def test_keygen_resamples_non_invertible_g():
    p = 761
    parts = oracle.ddf(p, 3)
    f1 = [poly for d, _, poly in parts if d == 19][0][:20]
    r = np.random.default_rng(4).integers(0, 3, p - 19)
    bad = np.convolve(f1, r) % 3
    bad = np.where(bad == 2, -1, bad).astype(np.int8)
    seed, k = 11, 42
    out = oracle.keygen(p, seed, k, g_attempt0=bad, intermediates=True)
    assert out["attempts"] == 2
    assert np.array_equal(out["g"], oracle.sample_small(p, seed, k, 1))
    # f does not depend on how many g attempts were needed
    assert np.array_equal(out["f"], oracle.keygen(p, seed, k, intermediates=True)["f"])


# ------------------------------------------------------------ encap / decap
def test_ct_size_matches_table1():
    # Table 1: sntrup761 public key + ciphertext = 2197 bytes
    row = read_golden("table1_sizes.txt")[0]
    pkb, _, _ = oracle.sizes(761)
    assert pkb + oracle.ct_bytes(761) == int(row[1])


@pytest.mark.parametrize("p", [653, 761, 857])
def test_decap_of_encap_gives_the_session_key(p):
    _, q, w = PARAMS[p]
    for k in range(4):
        pk, sk, _ = oracle.keygen(p, 77, k)
        ct, ss = oracle.encap(p, pk, 123, k)
        ss2, ok = oracle.decap(p, sk, ct)
        assert ok and ss2.tobytes() == ss.tobytes()
        # the ciphertext body is Round(h r): decode it and check it is a
        # multiple of 3 in every coefficient, close to h r
        r = oracle.sample_short_stream(p, w, 123, k, 3)
        h = oracle.rq_decode(p, q, pk).astype(np.int64)
        hr = oracle.ring_mul(p, q, h, r.astype(np.int64))
        assert np.count_nonzero(r) == w
        c = oracle.rounded_decode(p, ct[:-32]).astype(np.int64)
        assert np.all(c % 3 == 0) and np.abs(c - hr).max() <= 1   # Round(h r)
        assert np.array_equal(oracle.rounded_encode(p, c), ct[:-32])


def test_session_key_definition_vs_hashlib():
    p = 761
    pkb, skb, sb = oracle.sizes(p)
    pk, sk, _ = oracle.keygen(p, 5, 1)
    ct, ss = oracle.encap(p, pk, 9, 2)
    r = oracle.sample_short_stream(p, 286, 9, 2, 3)
    renc = oracle.small_encode(p, r).tobytes()
    h3 = hashlib.sha512(b"\x03" + renc).digest()[:32]
    cache = hashlib.sha512(b"\x04" + pk.tobytes()).digest()[:32]
    confirm = hashlib.sha512(b"\x02" + h3 + cache).digest()[:32]
    assert ct.tobytes()[-32:] == confirm
    assert ss.tobytes() == hashlib.sha512(b"\x01" + h3 + ct.tobytes()).digest()[:32]


def test_tampered_ciphertext_gets_implicit_rejection():
    p = 761
    pkb, skb, sb = oracle.sizes(p)
    pk, sk, _ = oracle.keygen(p, 5, 3)
    ct, ss = oracle.encap(p, pk, 9, 4)
    bad = ct.copy()
    bad[10] ^= 1
    ss2, ok = oracle.decap(p, sk, bad)
    assert not ok and ss2.tobytes() != ss.tobytes()
    rho = sk[2 * sb + pkb:3 * sb + pkb].tobytes()
    h3r = hashlib.sha512(b"\x03" + rho).digest()[:32]
    assert ss2.tobytes() == hashlib.sha512(b"\x00" + h3r + bad.tobytes()).digest()[:32]
