"""Python binding of libsntrup_gb300 (sntrup batch key generation on GB300).

Argument marshalling only: every step of key generation runs in the CUDA
kernels behind the C ABI declared in include/sntrup_gb300.h.  PyTorch is used
for device memory and streams.  The functions keep the C names; device
buffers are torch CUDA tensors (contiguous, of the dtype the C call expects),
host buffers are numpy arrays.

There is no fallback: if the shared library has not been built, importing
the functions raises with instructions to build it.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libsntrup_gb300.so")

SNTRUP653, SNTRUP761, SNTRUP857 = 653, 761, 857
PARAMS = {653: (653, 4621, 288), 761: (761, 4591, 286), 857: (857, 5167, 322)}

# tuning options (snt_option)
SNT_OPT_R3_LANES, SNT_OPT_TREE_SPLIT, SNT_OPT_R3_OVERLAP, SNT_OPT_NARROW_SEG = 1, 2, 3, 4
SNT_OPT_RQ_ENGINE, SNT_OPT_MMA_TILES, SNT_OPT_R3_KPT, SNT_OPT_MMA_KSPLIT = 5, 6, 7, 8
SNT_OPT_ROOTS, SNT_OPT_R3_MODE, SNT_OPT_FUSE_LEAF, SNT_OPT_PERKEY_INV = 9, 10, 11, 12
SNT_OPT_PARTS = 13
SNT_OPT_PDL = 14
SNT_OPT_R3_ROOTS = 15

# phase names of snt_ctx_phase_times (SNT_NPHASES entries)
PHASES = ("sample_f", "r3_inv", "tree_up", "root_inv", "tree_down", "h_encode", "sha512",
          "total", "r3_join_fixup")
NPHASES = len(PHASES)

STATUS = {0: "SNT_OK", -1: "SNT_EINVAL", -2: "SNT_ENOMEM", -3: "SNT_ECUDA",
          -4: "SNT_ETIMEOUT", -5: "SNT_EINTERNAL"}


class ServeConfig(ctypes.Structure):
    _fields_ = [("P", ctypes.c_int), ("rate", ctypes.c_double), ("duration_s", ctypes.c_double),
                ("max_items", ctypes.c_int), ("dec_fraction", ctypes.c_double),
                ("pool_keys", ctypes.c_size_t), ("refill_batch", ctypes.c_size_t),
                ("mem_budget", ctypes.c_size_t), ("max_inflight", ctypes.c_int),
                ("max_launch_items", ctypes.c_int), ("seed", ctypes.c_uint64)]


class ServeStats(ctypes.Structure):
    _fields_ = [("requests", ctypes.c_size_t), ("items_enc", ctypes.c_size_t),
                ("items_dec", ctypes.c_size_t), ("keys_generated", ctypes.c_size_t),
                ("mismatches", ctypes.c_size_t), ("memory_waits", ctypes.c_size_t),
                ("max_queue", ctypes.c_size_t), ("wall_s", ctypes.c_double),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("mean_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("items_per_s", ctypes.c_double), ("requests_per_s", ctypes.c_double)]


class ServeAudit(ctypes.Structure):
    _fields_ = [("cap", ctypes.c_size_t), ("count", ctypes.c_size_t),
                ("k", ctypes.POINTER(ctypes.c_uint64)), ("pk", ctypes.POINTER(ctypes.c_uint8)),
                ("ct", ctypes.POINTER(ctypes.c_uint8)), ("ss", ctypes.POINTER(ctypes.c_uint8))]


class SntError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (%d): %s" % (STATUS.get(status, "?"), status, msg))
        self.status = status


_lib = None


def load():
    """Load the CUDA library (built by __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libsntrup_gb300.so is not built (expected at %s); run "
                          "`python -c 'import __graft_entry__ as g; g.build()'`" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    P, sz, u64, i32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint64, ctypes.c_int
    szp = ctypes.POINTER(ctypes.c_size_t)
    sigs = {
        "snt_param_sizes": [i32, szp, szp, szp, szp],
        "snt_ctx_create": [i32, sz, ctypes.POINTER(ctypes.c_void_p)],
        "snt_ctx_destroy": [P],
        "snt_ctx_max_batch": [P, i32, szp],
        "snt_ctx_sync": [P, P],
        "snt_batch_keygen": [P, i32, u64, u64, sz, P, P, P],
        "snt_keygen_perkey": [P, i32, u64, u64, sz, P, P, P],
        "snt_batch_keygen_host": [P, i32, u64, u64, sz, P, P],
        "snt_batch_keygen_host_async": [P, i32, u64, u64, sz, P, P, P],
        "snt_batch_keygen_static": [i32, i32, u64, u64, sz, P, P, P],
        "snt_batch_keygen_ragged": [P, sz, P, P, P, P, P, P, P],
        "snt_rq_mul": [P, i32, sz, P, P, P, P],
        "snt_enc": [P, i32, sz, P, u64, u64, P, P, P],
        "snt_serve_run": [P, P, P, P, sz, P],
        "snt_dec": [P, i32, sz, P, P, P, P],
        "snt_rq_inv": [P, i32, sz, P, P, P, P],
        "snt_rq_inv_latency": [P, i32, sz, P, P, P, P],
        "snt_r3_inv": [P, i32, sz, P, P, P, P],
        "snt_debug_inject_g": [P, i32, sz, P, P],
        "snt_ctx_set_timing": [P, i32],
        "snt_ctx_set_option": [P, i32, i32],
        "snt_autotune": [P, i32, sz, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                         ctypes.POINTER(ctypes.c_int)],
        "snt_autotune_ex": [P, i32, sz, ctypes.POINTER(ctypes.c_int)],
        "snt_ctx_tuned": [P, i32, sz, ctypes.POINTER(ctypes.c_int), i32],
        "snt_ctx_get_option": [P, i32, ctypes.POINTER(ctypes.c_int)],
        "snt_ctx_phase_times": [P, P, i32],
        "snt_measure_int_peak": [i32, i32, ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(ctypes.c_int)],
        "snt_measure_tc05": [i32, i32, i32, ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(ctypes.c_int)],
    }
    for name, args in sigs.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    L.snt_last_error_string.argtypes = []
    L.snt_last_error_string.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(status):
    if status != 0:
        raise SntError(status, load().snt_last_error_string().decode())
    return status


def _dptr(t, dtype=None):
    """Device pointer of a contiguous torch CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError("expected dtype %s, got %s" % (dtype, t.dtype))
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(getattr(stream, "cuda_stream", stream))


def snt_param_sizes(P):
    """(pk_bytes, sk_bytes, ct_bytes, ss_bytes) of parameter set P."""
    v = [ctypes.c_size_t() for _ in range(4)]
    _check(load().snt_param_sizes(P, *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


class Context:
    """Owns an snt_ctx (device scratch within a memory budget)."""

    def __init__(self, device=0, mem_budget=0):
        h = ctypes.c_void_p()
        _check(load().snt_ctx_create(device, mem_budget, ctypes.byref(h)))
        self.handle = h
        self.device = device

    def close(self):
        if self.handle:
            _check(load().snt_ctx_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def max_batch(self, P):
        v = ctypes.c_size_t()
        _check(load().snt_ctx_max_batch(self.handle, P, ctypes.byref(v)))
        return v.value

    def sync(self, stream=None):
        _check(load().snt_ctx_sync(self.handle, _stream(stream)))

    def set_option(self, option, value):
        _check(load().snt_ctx_set_option(self.handle, option, value))

    def get_option(self, option):
        v = ctypes.c_int()
        _check(load().snt_ctx_get_option(self.handle, option, ctypes.byref(v)))
        return v.value

    def autotune(self, P, B):
        """Pick the fastest kernel layouts for (P, B) on this GPU; returns them."""
        c = (ctypes.c_int * 8)()
        _check(load().snt_autotune_ex(self.handle, P, B, c))
        return self.tuned(P, B)

    def tuned(self, P, B):
        """The layouts the autotuner kept for (P, B) on this context."""
        c = (ctypes.c_int * 10)()
        _check(load().snt_ctx_tuned(self.handle, P, B, c, 10))
        return {"r3_lanes": c[0], "tree_split": c[1], "r3_overlap": c[2], "rq_engine": c[3],
                "mma_tiles": c[4], "r3_kpt": c[5], "roots": c[6], "r3_mode": c[7],
                "parts": c[8], "r3_roots": c[9]}

    def set_timing(self, on=True):
        _check(load().snt_ctx_set_timing(self.handle, 1 if on else 0))

    def phase_times(self):
        """Phase durations (ms) of the last keygen call issued with timing on."""
        out = (ctypes.c_float * NPHASES)()
        _check(load().snt_ctx_phase_times(self.handle, out, NPHASES))
        return dict(zip(PHASES, [float(x) for x in out]))


def snt_ctx_create(device=0, mem_budget=0):
    return Context(device, mem_budget)


def snt_ctx_sync(ctx, stream=None):
    ctx.sync(stream)


def _check_room(P, B, pk, sk):
    """Raise ValueError if pk / sk cannot hold B keys of parameter set P (the
    kernels write B * pk_bytes and B * sk_bytes).  An unknown P or B = 0 is
    left to the C call, which rejects it with SNT_EINVAL."""
    if P not in PARAMS or B <= 0:
        return
    pkb, skb, _, _ = snt_param_sizes(P)
    for t, need, name in ((pk, B * pkb, "pk"), (sk, B * skb, "sk")):
        if t is not None and t.numel() * t.element_size() < need:
            raise ValueError("%s holds %d bytes, %d keys of sntrup%d need %d"
                             % (name, t.numel() * t.element_size(), B, P, need))


def snt_batch_keygen(ctx, P, seed, first_key_index, B, pk, sk, stream=None):
    import torch
    _check_room(P, B, pk, sk)
    _check(load().snt_batch_keygen(ctx.handle, P, seed, first_key_index, B,
                                   _dptr(pk, torch.uint8), _dptr(sk, torch.uint8),
                                   _stream(stream)))


def snt_keygen_perkey(ctx, P, seed, first_key_index, B, pk, sk, stream=None):
    import torch
    _check_room(P, B, pk, sk)
    _check(load().snt_keygen_perkey(ctx.handle, P, seed, first_key_index, B,
                                    _dptr(pk, torch.uint8), _dptr(sk, torch.uint8),
                                    _stream(stream)))


def snt_batch_keygen_ragged(ctx, Ps, Bs, seeds, firsts, pks, sks, stream=None):
    """Many batches (mixed sizes and parameter sets) in one graph launch.

    pks / sks: lists of uint8 CUDA tensors, one per batch."""
    import torch
    n = len(Ps)
    assert len(Bs) == n and len(seeds) == n and len(firsts) == n and len(pks) == n and len(sks) == n
    P_arr = (ctypes.c_int * n)(*[int(x) for x in Ps])
    B_arr = (ctypes.c_size_t * n)(*[int(x) for x in Bs])
    S_arr = (ctypes.c_uint64 * n)(*[int(x) for x in seeds])
    F_arr = (ctypes.c_uint64 * n)(*[int(x) for x in firsts])
    PK = (ctypes.c_void_p * n)(*[_dptr(t, torch.uint8).value for t in pks])
    SK = (ctypes.c_void_p * n)(*[_dptr(t, torch.uint8).value for t in sks])
    _check(load().snt_batch_keygen_ragged(ctx.handle, n, P_arr, B_arr, S_arr, F_arr, PK, SK,
                                          _stream(stream)))


def snt_batch_keygen_static(device, P, seed, first_key_index, B, pk, sk, stream=None):
    """Keygen without any device allocation (fixed static scratch, B <= 256).

    For callers that cannot allocate device memory; returns when the keys are
    written.  See include/sntrup_gb300.h for the sharing rules."""
    import torch
    _check_room(P, B, pk, sk)
    _check(load().snt_batch_keygen_static(device, P, seed, first_key_index, B,
                                          _dptr(pk, torch.uint8), _dptr(sk, torch.uint8),
                                          _stream(stream)))


def snt_batch_keygen_host(ctx, P, seed, first_key_index, B, pk_host=None, sk_host=None):
    """Generates B keys into host numpy buffers (allocated if not given)."""
    pkb, skb, _, _ = snt_param_sizes(P)
    if pk_host is None:
        pk_host = np.empty((B, pkb), np.uint8)
    if sk_host is None:
        sk_host = np.empty((B, skb), np.uint8)
    assert pk_host.flags.c_contiguous and pk_host.nbytes >= B * pkb
    assert sk_host.flags.c_contiguous and sk_host.nbytes >= B * skb
    _check(load().snt_batch_keygen_host(ctx.handle, P, seed, first_key_index, B,
                                        pk_host.ctypes.data_as(ctypes.c_void_p),
                                        sk_host.ctypes.data_as(ctypes.c_void_p)))
    return pk_host, sk_host


def snt_batch_keygen_host_async(ctx, P, seed, first_key_index, B, pk_host, sk_host, stream=None):
    """Enqueues the generation of B keys into host numpy buffers and returns;
    the keys are there once ctx.sync(stream) has returned.  The buffers
    should be page-locked (e.g. a pinned torch tensor's numpy view) and must
    stay alive and untouched until the sync."""
    pkb, skb, _, _ = snt_param_sizes(P)
    if not (pk_host.flags.c_contiguous and pk_host.nbytes >= B * pkb):
        raise ValueError("pk_host must be contiguous with room for %d keys" % B)
    if not (sk_host.flags.c_contiguous and sk_host.nbytes >= B * skb):
        raise ValueError("sk_host must be contiguous with room for %d keys" % B)
    _check(load().snt_batch_keygen_host_async(ctx.handle, P, seed, first_key_index, B,
                                              pk_host.ctypes.data_as(ctypes.c_void_p),
                                              sk_host.ctypes.data_as(ctypes.c_void_p),
                                              _stream(stream)))
    return pk_host, sk_host


def snt_enc(ctx, P, n, pk, seed, first_idx, ct, ss, stream=None):
    import torch
    _check(load().snt_enc(ctx.handle, P, n, _dptr(pk, torch.uint8), seed, first_idx,
                          _dptr(ct, torch.uint8), _dptr(ss, torch.uint8), _stream(stream)))


def snt_dec(ctx, P, n, sk, ct, ss, stream=None):
    import torch
    _check(load().snt_dec(ctx.handle, P, n, _dptr(sk, torch.uint8), _dptr(ct, torch.uint8),
                          _dptr(ss, torch.uint8), _stream(stream)))


def snt_serve_run(ctx, P=761, rate=1e4, duration_s=1.0, max_items=64, dec_fraction=1.0,
                  pool_keys=16384, refill_batch=8192, mem_budget=16 << 30, max_inflight=4,
                  max_launch_items=4096, seed=1, audit=0):
    """Serving loop (Poisson handshakes: encapsulation requests, each followed
    with probability dec_fraction by the decapsulation of its items; continuous
    batching; device key pool).  Returns (stats dict, per-request latencies in
    ms, audit dict)."""
    cfg = ServeConfig(P, rate, duration_s, max_items, dec_fraction, pool_keys, refill_batch,
                      mem_budget, max_inflight, max_launch_items, seed)
    st = ServeStats()
    cap = int(rate * duration_s * 2) + 1024
    lat = np.zeros(cap, np.float64)
    pkb, _, ctb, _ = snt_param_sizes(P)
    aud = None
    bufs = None
    if audit:
        bufs = dict(k=np.zeros(audit, np.uint64), pk=np.zeros((audit, pkb), np.uint8),
                    ct=np.zeros((audit, ctb), np.uint8), ss=np.zeros((audit, 32), np.uint8))
        aud = ServeAudit(audit, 0,
                         bufs["k"].ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                         bufs["pk"].ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                         bufs["ct"].ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                         bufs["ss"].ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    _check(load().snt_serve_run(ctx.handle, ctypes.byref(cfg), ctypes.byref(st),
                                lat.ctypes.data_as(ctypes.c_void_p), cap,
                                ctypes.byref(aud) if aud is not None else None))
    stats = {name: getattr(st, name) for name, _ in ServeStats._fields_}
    n = min(stats["requests"], cap)
    audit_out = None
    if aud is not None:
        c = aud.count
        audit_out = {key: v[:c] for key, v in bufs.items()}
    return stats, lat[:n], audit_out


def snt_rq_mul(ctx, P, n, a, b, c, stream=None):
    import torch
    _check(load().snt_rq_mul(ctx.handle, P, n, _dptr(a, torch.int16), _dptr(b, torch.int16),
                             _dptr(c, torch.int16), _stream(stream)))


def snt_rq_inv(ctx, P, n, a, out, ok, stream=None):
    import torch
    _check(load().snt_rq_inv(ctx.handle, P, n, _dptr(a, torch.int16), _dptr(out, torch.int16),
                             _dptr(ok, torch.int32), _stream(stream)))


def snt_rq_inv_latency(ctx, P, n, a, out, ok, stream=None):
    import torch
    _check(load().snt_rq_inv_latency(ctx.handle, P, n, _dptr(a, torch.int16),
                                     _dptr(out, torch.int16), _dptr(ok, torch.int32),
                                     _stream(stream)))


def snt_r3_inv(ctx, P, n, g, out, ok, stream=None):
    import torch
    _check(load().snt_r3_inv(ctx.handle, P, n, _dptr(g, torch.int8), _dptr(out, torch.int8),
                             _dptr(ok, torch.int32), _stream(stream)))


def snt_measure_int_peak(device=0, kind=0):
    """(instructions/s, SM count) of an instruction stream: 0 LOP3, 1 IMAD,
    2 DP4A, 3 IMAD+LOP3, 4 PRMT, 5 SHF, 6 DP4A+PRMT; 7 and 8 are warp MMA
    streams (f16 m16n8k16, s8 m16n8k32) in multiply-adds per second."""
    v = ctypes.c_double()
    n = ctypes.c_int()
    _check(load().snt_measure_int_peak(device, kind, ctypes.byref(v), ctypes.byref(n)))
    return v.value, n.value


def snt_measure_tc05(device=0, n=16, ctas_per_sm=1):
    """(multiply-adds/s, SM count) of back-to-back tcgen05.mma kind::f16 at
    M = 128, K = 16, N = n, operands in shared memory, ctas_per_sm issuing
    CTAs per SM (result checked)."""
    v = ctypes.c_double()
    k = ctypes.c_int()
    _check(load().snt_measure_tc05(device, n, ctas_per_sm, ctypes.byref(v), ctypes.byref(k)))
    return v.value, k.value


def snt_debug_inject_g(ctx, P, key_indices, gs):
    """Replace attempt 0 of the given key indices by the given g (test hook)."""
    idx = np.ascontiguousarray(key_indices, dtype=np.uint64)
    g = np.ascontiguousarray(gs, dtype=np.int8)
    n = idx.size
    _check(load().snt_debug_inject_g(ctx.handle, P, n,
                                     idx.ctypes.data_as(ctypes.c_void_p) if n else None,
                                     g.ctypes.data_as(ctypes.c_void_p) if n else None))
