"""ctypes driver for the C oracle in ``sntrup_oracle.c``.

Test infrastructure only (see the package docstring).  Every function takes
and returns numpy arrays; none of them does arithmetic of its own beyond
marshalling.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sntrup_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD_DIR, "liboracle.so")

# (p, q, w) of the three parameter sets, Sec. 2.1 of the paper.
PARAMS = {653: (653, 4621, 288), 761: (761, 4591, 286), 857: (857, 5167, 322)}

_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile the oracle with gcc into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + ".tmp.%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC",
                           "-o", tmp, _SRC])
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            P = ctypes.c_void_p
            i32, u32, u64, sz = (ctypes.c_int32, ctypes.c_uint32,
                                 ctypes.c_uint64, ctypes.c_size_t)
            sig = {
                "orc_philox4x32_10": (None, [P, P, P]),
                "orc_random_words": (None, [u64, u64, u32, u32, ctypes.c_int, P]),
                "orc_sample_small": (None, [ctypes.c_int, u64, u64, u32, P]),
                "orc_sample_short": (None, [ctypes.c_int, ctypes.c_int, u64, u64, P]),
                "orc_rho": (None, [ctypes.c_int, u64, u64, P]),
                "orc_ring_mul": (None, [ctypes.c_int, i32, P, P, P]),
                "orc_ring_inv": (ctypes.c_int, [ctypes.c_int, i32, P, P]),
                "orc_ring_pow": (None, [ctypes.c_int, i32, P, P, ctypes.c_int, P]),
                "orc_ddf": (ctypes.c_int, [ctypes.c_int, i32, P, P, P, ctypes.c_int]),
                "orc_rq_encode": (sz, [ctypes.c_int, i32, P, P]),
                "orc_rq_encoded_bytes": (sz, [ctypes.c_int, i32]),
                "orc_rq_decode": (None, [ctypes.c_int, i32, P, P]),
                "orc_small_encode": (None, [ctypes.c_int, P, P]),
                "orc_small_decode": (None, [ctypes.c_int, P, P]),
                "orc_sha512": (None, [P, sz, P]),
                "orc_sizes": (None, [ctypes.c_int, i32, P, P, P]),
                "orc_keygen": (ctypes.c_int, [ctypes.c_int, i32, ctypes.c_int, u64, u64,
                                              P, ctypes.c_int, P, P, P, P, P, P]),
                "orc_sample_short_stream": (None, [ctypes.c_int, ctypes.c_int, u64, u64, u32, P]),
                "orc_rounded_bytes": (sz, [ctypes.c_int, i32]),
                "rounded_encode": (None, [ctypes.c_int, i32, P, P]),
                "rounded_decode": (None, [ctypes.c_int, i32, P, P]),
                "orc_encap": (None, [ctypes.c_int, i32, ctypes.c_int, P, u64, u64, P, P]),
                "orc_decap": (ctypes.c_int, [ctypes.c_int, i32, ctypes.c_int, P, P, P]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def random_words(seed, k, stream, attempt, n):
    out = np.zeros(n, np.uint32)
    lib().orc_random_words(seed, k, stream, attempt, n, _ptr(out))
    return out


def sample_small(p, seed, k, attempt=0):
    g = np.zeros(p, np.int8)
    lib().orc_sample_small(p, seed, k, attempt, _ptr(g))
    return g


def sample_short(p, w, seed, k):
    f = np.zeros(p, np.int8)
    lib().orc_sample_short(p, w, seed, k, _ptr(f))
    return f


def rho(nbytes, seed, k):
    out = np.zeros(nbytes, np.uint8)
    lib().orc_rho(nbytes, seed, k, _ptr(out))
    return out


def ring_mul(p, m, a, b):
    """a*b in (Z/m)[x]/(x^p - x - 1), centred output (int32)."""
    a = np.ascontiguousarray(a, dtype=np.int32)
    b = np.ascontiguousarray(b, dtype=np.int32)
    assert a.shape == (p,) and b.shape == (p,)
    c = np.zeros(p, np.int32)
    lib().orc_ring_mul(p, m, _ptr(a), _ptr(b), _ptr(c))
    return c


def ring_inv(p, m, a):
    """(ok, 1/a) in (Z/m)[x]/(x^p - x - 1) by extended Euclid."""
    a = np.ascontiguousarray(a, dtype=np.int32)
    out = np.zeros(p, np.int32)
    ok = lib().orc_ring_inv(p, m, _ptr(a), _ptr(out))
    return bool(ok), out


def ring_pow(p, m, a, e):
    """a^e for a Python integer e >= 0."""
    a = np.ascontiguousarray(a, dtype=np.int32)
    nbytes = max(1, (int(e).bit_length() + 7) // 8)
    eb = np.frombuffer(int(e).to_bytes(nbytes, "little"), np.uint8).copy()
    out = np.zeros(p, np.int32)
    lib().orc_ring_pow(p, m, _ptr(a), _ptr(eb), nbytes, _ptr(out))
    return out


def ddf(p, m, maxparts=64):
    """Distinct-degree factorisation of x^p - x - 1 over F_m.

    Returns a list of (d, total_degree, monic_product_poly) with the
    product of all irreducible factors of degree d."""
    degs = np.zeros(maxparts, np.int32)
    tot = np.zeros(maxparts, np.int32)
    parts = np.zeros((maxparts, p + 1), np.int32)
    n = lib().orc_ddf(p, m, _ptr(degs), _ptr(tot), _ptr(parts), maxparts)
    assert n <= maxparts
    return [(int(degs[i]), int(tot[i]), parts[i].copy()) for i in range(n)]


def rq_encode(p, q, h):
    h = np.ascontiguousarray(h, dtype=np.int16)
    out = np.zeros(rq_encoded_bytes(p, q), np.uint8)
    n = lib().orc_rq_encode(p, q, _ptr(h), _ptr(out))
    assert n == out.size
    return out


def rq_encoded_bytes(p, q):
    return int(lib().orc_rq_encoded_bytes(p, q))


def rq_decode(p, q, data):
    data = np.ascontiguousarray(data, dtype=np.uint8)
    h = np.zeros(p, np.int16)
    lib().orc_rq_decode(p, q, _ptr(data), _ptr(h))
    return h


def small_encode(p, c):
    c = np.ascontiguousarray(c, dtype=np.int8)
    out = np.zeros((p + 3) // 4, np.uint8)
    lib().orc_small_encode(p, _ptr(c), _ptr(out))
    return out


def small_decode(p, data):
    data = np.ascontiguousarray(data, dtype=np.uint8)
    c = np.zeros(p, np.int8)
    lib().orc_small_decode(p, _ptr(data), _ptr(c))
    return c


def sha512(msg):
    m = np.frombuffer(bytes(msg), np.uint8).copy() if not isinstance(msg, np.ndarray) else np.ascontiguousarray(msg, np.uint8)
    out = np.zeros(64, np.uint8)
    lib().orc_sha512(_ptr(m) if m.size else None, m.size, _ptr(out))
    return bytes(out)


def sizes(p):
    """(pk_bytes, sk_bytes, small_bytes) for parameter set p."""
    q = PARAMS[p][1]
    pk = ctypes.c_size_t()
    sk = ctypes.c_size_t()
    sb = ctypes.c_size_t()
    lib().orc_sizes(p, q, ctypes.byref(pk), ctypes.byref(sk), ctypes.byref(sb))
    return pk.value, sk.value, sb.value


def keygen(p, seed, k, g_attempt0=None, max_attempts=64, intermediates=False):
    """One key pair (Sec. 3.1 KeyGen) for key index k.

    Returns (pk, sk, attempts) or, with intermediates=True, a dict that also
    holds f, g, v = 1/g in R/3 and h."""
    _, q, w = PARAMS[p]
    pkb, skb, _ = sizes(p)
    pk = np.zeros(pkb, np.uint8)
    sk = np.zeros(skb, np.uint8)
    f = np.zeros(p, np.int8)
    g = np.zeros(p, np.int8)
    v = np.zeros(p, np.int8)
    h = np.zeros(p, np.int16)
    g0 = None
    if g_attempt0 is not None:
        g0 = np.ascontiguousarray(g_attempt0, dtype=np.int8)
        assert g0.shape == (p,)
    att = lib().orc_keygen(p, q, w, seed, k, _ptr(g0), max_attempts, _ptr(pk),
                           _ptr(sk), _ptr(f), _ptr(g), _ptr(v), _ptr(h))
    if att < 0:
        raise RuntimeError("oracle keygen failed (status %d)" % att)
    if intermediates:
        return dict(pk=pk, sk=sk, attempts=att, f=f, g=g, v=v, h=h)
    return pk, sk, att


def keygen_batch(p, seed, first, B, g_inject=None):
    """B consecutive keys; returns (pk[B, pkb], sk[B, skb]).

    g_inject: optional dict {key_offset: g} replacing attempt 0 of those keys."""
    pkb, skb, _ = sizes(p)
    pks = np.zeros((B, pkb), np.uint8)
    sks = np.zeros((B, skb), np.uint8)
    for i in range(B):
        g0 = None if g_inject is None else g_inject.get(i)
        pk, sk, _ = keygen(p, seed, first + i, g_attempt0=g0)
        pks[i] = pk
        sks[i] = sk
    return pks, sks


def ct_bytes(p):
    _, q, _ = PARAMS[p]
    return int(lib().orc_rounded_bytes(p, q)) + 32


def sample_short_stream(p, w, seed, k, stream):
    f = np.zeros(p, np.int8)
    lib().orc_sample_short_stream(p, w, seed, k, stream, _ptr(f))
    return f


def encap(p, pk, seed, k):
    """(ct, ss) for public key pk; r is Short from stream 3 of (seed, k)."""
    _, q, w = PARAMS[p]
    pk = np.ascontiguousarray(pk, dtype=np.uint8)
    ct = np.zeros(ct_bytes(p), np.uint8)
    ss = np.zeros(32, np.uint8)
    lib().orc_encap(p, q, w, _ptr(pk), seed, k, _ptr(ct), _ptr(ss))
    return ct, ss


def decap(p, sk, ct):
    """(ss, accepted) for secret key sk and ciphertext ct."""
    _, q, w = PARAMS[p]
    sk = np.ascontiguousarray(sk, dtype=np.uint8)
    ct = np.ascontiguousarray(ct, dtype=np.uint8)
    ss = np.zeros(32, np.uint8)
    ok = lib().orc_decap(p, q, w, _ptr(sk), _ptr(ct), _ptr(ss))
    return ss, bool(ok)


def rounded_decode(p, data):
    _, q, _ = PARAMS[p]
    data = np.ascontiguousarray(data, dtype=np.uint8)
    c = np.zeros(p, np.int32)
    lib().rounded_decode(p, q, _ptr(data), _ptr(c))
    return c


def rounded_encode(p, c):
    _, q, _ = PARAMS[p]
    c = np.ascontiguousarray(c, dtype=np.int32)
    out = np.zeros(ct_bytes(p) - 32, np.uint8)
    lib().rounded_encode(p, q, _ptr(c), _ptr(out))
    return out
