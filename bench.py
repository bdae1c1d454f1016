#!/usr/bin/env python3
"""Benchmark: sntrup761 batch key generation (B = 4096 keys per step) on GB300.

One step = one snt_batch_keygen call: B fresh key pairs from a 64-bit seed
(sampling, per-key R/3 inversions, the R/q product tree with its root
inversion, h, Rq_encode, sk assembly and SHA-512), all on the device.  The
line also reports the per-key GPU path (snt_keygen_perkey) on the same
workload, the end-to-end rate through the host-buffer call, the ALU roofline
of the dominant kernel against measured integer-pipe peaks, the CPU oracle
timed on the host cores, and the serving loop (p50/p99 latency and
throughput of encapsulation/decapsulation handshakes over the device key
pool at 10^4, 10^5 and 10^6 requests/s).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun as independent replicas (one tree per GPU, no
data-path collective); value = keys of all ranks / max time over ranks.
"""
import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sntrup761 keygens/s on 1 GB300, batched vs per-key GPU path; p50/p99 serve ms"
P, Q, W = 761, 4591, 286
WORDS = (P + 1 + 31) // 32
L2_FLUSH_BYTES = 256 << 20   # > 129 MB L2
def fused_leaf(tuned, p=None):
    """Whether the library forms h from the level-1 inverses (its default on
    the tensor-core engine for p = 653, 761: the leaf level of the down-sweep
    folded into the h kernel)."""
    return tuned.get("rq_engine") in (1, 2, 3) and (p or P) in (653, 761)


def launches_per_call(B, tuned):
    """Library kernel launches of one batch keygen call under the tuned layouts.

    R/q: sampling, up-sweep (one per level), roots, down-sweep (without its
    leaf level when fused), h, SHA-512, and with the fused leaf level (unless
    g is redrawn before h) the leaf-pair products s on the side stream; R/3 per key: its kernel and the
    fix-up; R/3 check-first batch: the check, its forest (2 per level + roots)
    and the encoding; R/3 first-draw batch: the forest, the encoding, the
    fall-back kernel and the fix-up."""
    K = forest_roots(B, tuned.get("roots", 1))
    K3 = forest_roots(B, tuned.get("r3_roots") or tuned.get("roots", 1))
    L, L3 = tree_levels(B // K), tree_levels(B // K3)
    fused = fused_leaf(tuned) and L >= 1
    down = L - 1 if fused else L
    side = 1 if (fused and tuned.get("r3_mode", 0) != 1) else 0  # leaf-pair products s
    rq = 1 + L + 1 + down + 1 + 1 + side
    r3 = {0: 2, 1: 1 + 2 * L3 + 1 + 1, 2: 2 * L3 + 1 + 1 + 1 + 1}[tuned.get("r3_mode", 0)]
    return rq + r3


def tree_levels(n):
    """Product levels above the leaves of a subtree of n leaves."""
    L = 0
    while n > 1:
        n = (n + 1) // 2
        L += 1
    return L

# DRAM bytes (read + write) per call of a phase's kernels at B = 4096,
# summed over the phase's launches of one call, from the committed ncu
# launch-list capture of one keygen call (caches flushed by ncu before each
# launch), keyed by kernel; a kernel is absent until a capture of its current
# code exists.  Writes stay in L2.  Engine 3: 16 subtrees, the R/3 forest 4
# (the layout of the capture); engine 1: 64 subtrees; the R/q root inversion:
# 32 roots (its inputs, 32 rows).
NCU_TRAFFIC_BYTES = {
    "k_tree_up_mma": 12532992,
    "k_tree_down_mma": 9324544,
    "k_tree_up_mma (one wide limb)": 12721152,
    "k_tree_down_mma (one wide limb)": 9627904,
    "k_rq_inv_jump<761, 4591>": 115456,
    "k_finalize_pair<761>": 9503232,
    "k_tree_up_mma / k_tree_down_mma (mod 3) + k_rq_inv_jump<761, 3>": 38448384,
}


def kernel_of(phase, tuned):
    """Kernel instantiation that runs a phase under the tuned layouts."""
    if phase == "r3_inv":
        if tuned.get("r3_mode", 0) == 0:
            return "k_r3_keygen<761, %d>" % tuned.get("r3_lanes", 4)
        return "k_tree_up_mma / k_tree_down_mma (mod 3) + k_rq_inv_jump<761, 3>"
    eng = tuned.get("rq_engine")
    mma = eng in (1, 2, 3)
    tree = {1: "%s_mma", 2: "%s_ntt + %s_mma (leaf level)", 3: "%s_mma (one wide limb)"}
    name = lambda k: (tree[eng].replace("%s", k) if mma else k)
    return {"tree_up": name("k_tree_up"),
            "tree_down": name("k_tree_down"),
            "h_encode": ("k_finalize_pair<761>" if fused_leaf(tuned) else "k_finalize_mma<761>")
                        if mma else "k_finalize<761>",
            "root_inv": "k_rq_inv_jump<761, 4591>"}[phase]


# ---- replicas (N > 1): one process per GPU, independent batches ----------------
def replica_key_base(rank):
    """First key index of a rank: disjoint 2^40-key ranges, so replicas never
    generate the same key (key i of a call uses (seed, first + i) only)."""
    return rank << 40


def max_over_ranks(x, dist, device):
    """Max of a per-rank number over all ranks (the job's wall time)."""
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, B, steps, seconds):
    """Keys of all ranks per second of the slowest rank."""
    return world * B * steps / seconds


def tree_nodes(n):
    t = 0
    while True:
        t += n
        if n == 1:
            return t
        n = (n + 1) // 2


def forest_roots(B, roots):
    """Subtrees the library uses for a batch (its forest rule)."""
    k = 1
    while 2 * k <= roots and B % (2 * k) == 0 and 2 * k * tree_nodes(B // (2 * k)) <= tree_nodes(B):
        k *= 2
    return k


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--seed", type=lambda s: int(s, 0), default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--perkey-steps", type=int, default=None)
    ap.add_argument("--serve-rates", default="1e4,1e5,1e6",
                    help="request rates of the serving runs (empty: none)")
    ap.add_argument("--serve-duration", type=float, default=0.5)
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the B=32, ragged and building-block measurements")
    return ap.parse_args()


# ------------------------------------------------------------------ CPU side
def _oracle_keys(args):
    seed, first, n = args
    import oracle
    for k in range(first, first + n):
        oracle.keygen(P, seed, k)
    return n


def cpu_pool():
    cores = os.cpu_count() or 1
    return mp.get_context("spawn").Pool(cores), cores


def oracle_rate(pool, cores, seed, first, keys_per_core):
    """Keys/s of the CPU oracle with keys split across all host cores."""
    jobs = [(seed, first + i * keys_per_core, keys_per_core) for i in range(cores)]
    t0 = time.perf_counter()
    n = sum(pool.map(_oracle_keys, jobs))
    return n / (time.perf_counter() - t0), n


# ------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.device)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in getattr(self, "lines", []):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------- algorithmic ops
def _measured_peaks():
    """The measured copy and GEMM peaks of this GPU model (MEASURED_PEAKS.json),
    if the file is present."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def ops_per_call(B, K=1, r3_mode=0, p=P, fused=False, s_side=False, K3=None):
    """Algorithmic integer operations of each phase for one call of B keys in
    K subtrees.

    Products count p^2 multiply-adds (the Toeplitz/schoolbook form every
    product kernel computes; a forest of K subtrees has B - K products up and
    2(B - K) down, h one per key); with the fused leaf level the down-sweep
    stops at level 1 (2 products per pair above it) and h costs, per leaf
    pair, g_L f_R, g_R f_L and inv(P) s for both keys (an unpaired leaf one),
    of which the two s products are counted as "leaf_s" when they run on the
    side stream beside the root inversions (no phase time of their own);
    the per-key R/3 divsteps count 6 word operations per 32-trit word for each
    of the two polynomial updates per step (bit-sliced F_3 multiply-add), the
    R/3 batch paths their 3(B - K3) products mod 3 (K3 subtrees, default K);
    a root inversion counts 2 multiply-reduce updates of p + 1 coefficients
    per step."""
    K3 = K if K3 is None else K3
    steps = 2 * p - 1
    mac = p * p
    n0 = B // K
    pairs, n = [], n0
    while n > 1:
        pairs.append(n // 2)
        n = (n + 1) // 2
    side = 0
    if fused and pairs:
        down = 2 * (n0 - 1 - pairs[0]) * K
        h = (4 * pairs[0] + (n0 - 2 * pairs[0])) * K
        if s_side:
            side = 2 * pairs[0] * K
            h -= side
    else:
        down, h = 2 * (B - K), B
    ops = {
        "r3_inv": B * steps * 2 * WORDS * 6 if r3_mode == 0 else 3 * (B - K3) * mac,
        "tree_up": (B - K) * mac,
        "tree_down": down * mac,
        "h_encode": h * mac,
        "root_inv": K * steps * 2 * (p + 1),
    }
    if side:
        ops["leaf_s"] = side * mac
    return ops


PIPE_OF = {"r3_inv": "lop3", "tree_up": "imad", "tree_down": "imad", "h_encode": "imad",
           "root_inv": "imad"}
# with the tensor-core engine the products are f16 MMAs
TENSOR_PHASES = ("tree_up", "tree_down", "h_encode")


# ----------------------------------------------- the other configurations
def micro_inputs(torch, n, seed, dev, short=False):
    """n seeded synthetic sntrup761 operands on the device: R/q elements
    uniform in [-(q-1)/2, (q-1)/2], or Short rows (w positions uniform among
    p, random signs), generated in chunks by a seeded torch generator (the
    same distributions as the test inputs)."""
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    h = (Q - 1) // 2
    out = torch.empty((n, P), dtype=torch.int16, device=dev)
    step = 1 << 16
    for i in range(0, n, step):
        m = min(step, n - i)
        if short:
            pos = torch.rand((m, P), generator=g, device=dev).topk(W, dim=1).indices
            sgn = torch.randint(0, 2, (m, W), generator=g, device=dev, dtype=torch.int16) * 2 - 1
            blk = torch.zeros((m, P), dtype=torch.int16, device=dev)
            blk.scatter_(1, pos, sgn)
            out[i:i + m] = blk
        else:
            out[i:i + m] = torch.randint(-h, h + 1, (m, P), generator=g, device=dev,
                                         dtype=torch.int16)
    return out


def event_ms(torch, stream, flush, fn, reps):
    """Median device time of fn over reps launches (CUDA events on the
    launching stream, L2 flushed before each), after one warm-up."""
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def measure_b32(snt, torch, dev, stream, flush, seed, steps):
    """Configuration 1: B = 32 keys per call (the paper's BatchKeyGen size),
    batched and per key, autotuned for (761, 32)."""
    B = 32
    pkb, skb, _, _ = snt.snt_param_sizes(P)
    out = {}
    with snt.Context(dev.index or 0, 64 << 20) as c:
        tuned = c.autotune(P, B)
        pk = torch.empty(B * pkb, dtype=torch.uint8, device=dev)
        sk = torch.empty(B * skb, dtype=torch.uint8, device=dev)
        it = [0]

        def call(fn):
            def f():
                it[0] += 1
                fn(c, P, seed, (7 << 40) + it[0] * B, B, pk, sk, stream)
            return f
        for name, fn in (("batched", snt.snt_batch_keygen), ("perkey", snt.snt_keygen_perkey)):
            ms = event_ms(torch, stream, flush, call(fn), steps)
            out[name] = {"keys_per_s": round(B / ms * 1e3, 1), "ms_per_call": round(ms, 4)}
        c.set_option(snt.SNT_OPT_PDL, 0)
        ms = event_ms(torch, stream, flush, call(snt.snt_batch_keygen), steps)
        out["batched_plain_launch"] = {"keys_per_s": round(B / ms * 1e3, 1),
                                       "ms_per_call": round(ms, 4)}
        c.set_option(snt.SNT_OPT_PDL, 1)
        c.sync()
    out["roots"] = tuned["roots"]
    out["r3_mode"] = tuned["r3_mode"]
    return out


def measure_ragged(snt, torch, np, dev, stream, flush, reps):
    """Configuration 3: 256 batches, sizes floor(exp(U[0, ln 2048])), a
    shuffled equal mix of sntrup653/761/857 (seed 42), one graph launch."""
    from synth import ragged_batches
    sizes, ps = ragged_batches(256, 2048, 42)
    pks, sks = [], []
    for P_, B_ in zip(ps, sizes):
        pkb_, skb_, _, _ = snt.snt_param_sizes(int(P_))
        pks.append(torch.empty(int(B_) * pkb_, dtype=torch.uint8, device=dev))
        sks.append(torch.empty(int(B_) * skb_, dtype=torch.uint8, device=dev))
    firsts = [int(x) for x in np.cumsum([0] + list(sizes[:-1]))]
    it = [0]
    with snt.Context(dev.index or 0, 1 << 30) as c:
        # layouts per (p, bucket of the largest batch), as a user would tune
        tuned = {str(x): c.autotune(x, 2048) for x in (653, 761, 857)}

        def ragged():
            it[0] += 1
            snt.snt_batch_keygen_ragged(c, [int(x) for x in ps], [int(x) for x in sizes],
                                        [it[0] * 1000 + i for i in range(256)], firsts, pks,
                                        sks, stream)
        ms = event_ms(torch, stream, flush, ragged, reps)
        c.sync()
    nkeys = int(sizes.sum())
    return {"batches": 256, "keys": nkeys, "ms_per_launch": round(ms, 4),
            "keys_per_s": round(nkeys / ms * 1e3, 1),
            "keys_by_p": {str(x): int(sizes[ps == x].sum()) for x in (653, 761, 857)},
            "r3_batched": {k: v["r3_mode"] != 0 for k, v in tuned.items()}}


def measure_micro(snt, torch, ctx, dev, stream, flush, reps):
    """Configuration 4 (p = 761): 2^20 general x general and 2^20 general x
    Short R/q products, 2^16 R/3 inversions, 2^10 R/q inversions (jump
    divsteps and the step-at-a-time kernel)."""
    n = 1 << 20
    a = micro_inputs(torch, n, 1, dev)
    b = micro_inputs(torch, n, 2, dev)
    s = micro_inputs(torch, n, 3, dev, short=True)
    c = torch.empty_like(a)
    out = {}
    ms = event_ms(torch, stream, flush, lambda: snt.snt_rq_mul(ctx, P, n, a, b, c, stream), reps)
    out["rq_mul_general"] = {"n": n, "ms": round(ms, 3), "products_per_s": round(n / ms * 1e3),
                             "gop_per_s": round(2 * n * P * P / ms / 1e6, 1)}
    ms = event_ms(torch, stream, flush, lambda: snt.snt_rq_mul(ctx, P, n, a, s, c, stream), reps)
    out["rq_mul_short"] = {"n": n, "ms": round(ms, 3), "products_per_s": round(n / ms * 1e3),
                           "gop_per_s": round(n * P * W / ms / 1e6, 1)}
    # the same general products on each engine: 0 CUDA-core Toeplitz (IMAD),
    # 1 tensor-core Toeplitz (f16 limbs), 2 the transform multiplier (IMAD),
    # 3 tensor-core Toeplitz with one wide limb on the vector side
    eng = ctx.get_option(snt.SNT_OPT_RQ_ENGINE)
    by_engine = {}
    for e in (0, 1, 2, 3):
        ctx.set_option(snt.SNT_OPT_RQ_ENGINE, e)
        ms = event_ms(torch, stream, flush, lambda: snt.snt_rq_mul(ctx, P, n, a, b, c, stream),
                      reps)
        by_engine[str(e)] = round(n / ms * 1e3)
    ctx.set_option(snt.SNT_OPT_RQ_ENGINE, eng)
    out["rq_mul_general_products_per_s_by_engine"] = by_engine
    del a, b, s, c
    m = 1 << 16
    g = torch.randint(-1, 2, (m, P), generator=torch.Generator(device=dev).manual_seed(5),
                      device=dev, dtype=torch.int8)
    o = torch.empty_like(g)
    ok = torch.empty(m, dtype=torch.int32, device=dev)
    ms = event_ms(torch, stream, flush, lambda: snt.snt_r3_inv(ctx, P, m, g, o, ok, stream), reps)
    out["r3_inv"] = {"n": m, "ms": round(ms, 3), "inv_per_s": round(m / ms * 1e3)}
    k = 1 << 10
    x = micro_inputs(torch, k, 6, dev)
    xo = torch.empty_like(x)
    xk = torch.empty(k, dtype=torch.int32, device=dev)
    ms = event_ms(torch, stream, flush,
                  lambda: snt.snt_rq_inv_latency(ctx, P, k, x, xo, xk, stream), reps)
    out["rq_inv_jump"] = {"n": k, "ms": round(ms, 3), "inv_per_s": round(k / ms * 1e3)}
    ms = event_ms(torch, stream, flush, lambda: snt.snt_rq_inv(ctx, P, k, x, xo, xk, stream), reps)
    out["rq_inv_step"] = {"n": k, "ms": round(ms, 3), "inv_per_s": round(k / ms * 1e3)}
    out["ops"] = "general: 2 p^2 per product (multiply-adds); Short: p w add/sub per product"
    # the serving path's kernels alone: 65536 encapsulations and decapsulations
    # (one CTA per item) on keys from batch keygen
    nk = 1 << 16
    pkb, skb, ctb, _ = snt.snt_param_sizes(P)
    kpk = torch.empty(nk * pkb, dtype=torch.uint8, device=dev)
    ksk = torch.empty(nk * skb, dtype=torch.uint8, device=dev)
    for i in range(0, nk, 4096):
        snt.snt_batch_keygen(ctx, P, 77, i, 4096, kpk[i * pkb:(i + 4096) * pkb],
                             ksk[i * skb:(i + 4096) * skb], stream)
    ct = torch.empty(nk * ctb, dtype=torch.uint8, device=dev)
    ss = torch.empty(nk * 32, dtype=torch.uint8, device=dev)
    ss2 = torch.empty(nk * 32, dtype=torch.uint8, device=dev)
    ms_e = event_ms(torch, stream, flush, lambda: snt.snt_enc(ctx, P, nk, kpk, 5, 0, ct, ss, stream),
                    reps)
    ms_d = event_ms(torch, stream, flush, lambda: snt.snt_dec(ctx, P, nk, ksk, ct, ss2, stream),
                    reps)
    ctx.sync()
    out["kem"] = {"n": nk, "enc_per_s": round(nk / ms_e * 1e3), "dec_per_s": round(nk / ms_d * 1e3),
                  "dec_matches_enc": bool(torch.equal(ss, ss2))}
    return out


# ------------------------------------------------------------------ our arm
def run_ours(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    do_cpu = (rank == 0 and world == 1 and not args.no_cpu_baseline)
    pool = None
    if do_cpu:
        pool, cores = cpu_pool()  # spawned before the first GPU call
        pool.map(_oracle_keys, [(1, 0, 1)] * cores)  # import + build in workers

    import numpy as np
    import torch
    import paper_2106_08759_gb300 as snt

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    B = args.batch
    pkb, skb, _, _ = snt.snt_param_sizes(P)
    ctx = snt.Context(local, 256 << 20)
    pk = torch.empty(B * pkb, dtype=torch.uint8, device=dev)
    sk = torch.empty(B * skb, dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    base = replica_key_base(rank)

    lop3_peak, sms = snt.snt_measure_int_peak(local, 0)
    imad_peak, _ = snt.snt_measure_int_peak(local, 1)
    mma_peak, _ = snt.snt_measure_int_peak(local, 7)  # warp-MMA f16 multiply-adds per second
    peaks = _measured_peaks()
    tuned = ctx.autotune(P, B)  # kernel layouts for this GPU, before any timed step

    launches_per_step = launches_per_call(B, tuned)

    def timed(fn, steps, warmup, phases=False):
        ctx.set_timing(phases)
        for i in range(warmup):
            fn(base + (10**9) + i * B)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        acc = {}
        total_ms = 0.0
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        for i in range(steps):
            flush.zero_()  # evict L2 between steps (not timed)
            evs[i][0].record(stream)
            fn(base + i * B)
            evs[i][1].record(stream)
            if phases:
                for k, v in ctx.phase_times().items():
                    acc[k] = acc.get(k, 0.0) + v
        torch.cuda.synchronize()
        ctx.sync()
        total_ms = sum(a.elapsed_time(b) for a, b in evs)
        if dist:
            total_ms = max_over_ranks(total_ms, dist, dev)
        return total_ms, {k: v / steps for k, v in acc.items()}

    def batched(first):
        snt.snt_batch_keygen(ctx, P, args.seed, first, B, pk, sk, stream)

    def perkey(first):
        snt.snt_keygen_perkey(ctx, P, args.seed, first, B, pk, sk, stream)

    # the timed steps run back to back (the phase events, which wait for
    # every step, are taken in a separate run below)
    with ClockSampler(local) as clk:
        total_ms, _ = timed(batched, args.steps, max(3, args.warmup))
    clocks = clk.summary()
    ms_per_step = total_ms / args.steps
    value = whole_job_rate(world, B, args.steps, total_ms * 1e-3)
    ph_steps = max(3, min(args.steps, 10))
    _, phase = timed(batched, ph_steps, 3, phases=True)
    # the same steps with every kernel launched plainly (no programmatic
    # dependent launch): what the launch mode is worth
    ctx.set_option(snt.SNT_OPT_PDL, 0)
    plain_ms, _ = timed(batched, ph_steps, 3)
    ctx.set_option(snt.SNT_OPT_PDL, 1)
    launch_modes = {"pdl_ms_per_step": round(ms_per_step, 4),
                    "plain_ms_per_step": round(plain_ms / ph_steps, 4)}

    pk_steps = args.perkey_steps or max(3, args.steps // 10)
    pk_ms, _ = timed(perkey, pk_steps, 3)
    perkey_rate = whole_job_rate(world, B, pk_steps, pk_ms * 1e-3)

    # end to end through the host-buffer entry point (device->host copy of
    # every key pair inside the timed region; the only inputs are the seed and
    # key index, passed by value)
    # Two ways: the synchronous call (returns when the keys are in host
    # memory), and the calls that do not wait, each step into its own pair
    # of pinned buffers, synced once at the end (the headline: a caller
    # producing many batches overlaps one batch's copies with the next
    # batch's generation).
    hbuf = [(torch.empty(B * pkb, dtype=torch.uint8, pin_memory=True).numpy().reshape(B, pkb),
             torch.empty(B * skb, dtype=torch.uint8, pin_memory=True).numpy().reshape(B, skb))
            for _ in range(2)]
    hpk, hsk = hbuf[0]
    ctx.set_timing(False)
    for i in range(3):
        snt.snt_batch_keygen_host(ctx, P, args.seed, base + (2 * 10**9) + i * B, B, hpk, hsk)
    e2e_steps = max(3, args.steps // 5)
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        snt.snt_batch_keygen_host(ctx, P, args.seed, base + (3 * 10**9) + i * B, B, hpk, hsk)
    e2e_sync_s = time.perf_counter() - t0
    if dist:
        e2e_sync_s = max_over_ranks(e2e_sync_s, dist, dev)
    e2e_sync_rate = whole_job_rate(world, B, e2e_steps, e2e_sync_s)
    async_steps = max(3, args.steps)
    for i in range(3):
        snt.snt_batch_keygen_host_async(ctx, P, args.seed, base + (4 * 10**9) + i * B, B,
                                        *hbuf[i & 1], stream=stream)
    ctx.sync(stream)
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for i in range(async_steps):
        snt.snt_batch_keygen_host_async(ctx, P, args.seed, base + (5 * 10**9) + i * B, B,
                                        *hbuf[i & 1], stream=stream)
    ctx.sync(stream)
    e2e_s = time.perf_counter() - t0
    if dist:
        e2e_s = max_over_ranks(e2e_s, dist, dev)
    e2e_rate = whole_job_rate(world, B, async_steps, e2e_s)

    # roofline of every counted phase (phase time from the library's events,
    # algorithmic work per call): the integer-pipe bound for the divsteps and
    # the CUDA-core products, the tensor bound for products on the tensor
    # cores.  "roofline" is the longest phase on the critical path; the R/3
    # phase runs beside the tree (auxiliary stream) unless its overlap is 0.
    K = forest_roots(B, tuned.get("roots", 1))
    K3 = forest_roots(B, tuned.get("r3_roots") or tuned.get("roots", 1))
    r3m = tuned.get("r3_mode", 0)
    fused = fused_leaf(tuned)
    ops = ops_per_call(B, K, r3m, fused=fused, s_side=fused and r3m != 1, K3=K3)
    Lk = tree_levels(B // K)
    launches_of = {"r3_inv": 1 if r3m == 0 else 2 * tree_levels(B // K3) + 3, "tree_up": Lk,
                   "tree_down": Lk - 1 if (fused and Lk >= 1) else Lk,
                   "h_encode": 1, "root_inv": 1, "leaf_s": 1}
    tensor_phases = TENSOR_PHASES + (("r3_inv",) if r3m else ())

    def roofline_of(ph):
        ms = phase.get(ph, 0.0)
        if ms <= 0:
            return None
        if tuned.get("rq_engine") in (1, 3) and ph in tensor_phases:
            achieved = 2.0 * ops[ph] / (ms * 1e-3) / 1e12  # TFLOP/s of the p^2 products
            peak = peaks.get("bf16_tflops") or 1900.0
            return {
                "bound": "tensor", "kernel": kernel_of(ph, tuned), "phase": ph,
                "pipe": "tensor (mma.sync f16, f32 accumulate)",
                "achieved": round(achieved, 3), "peak": round(peak, 1), "unit": "TFLOP/s",
                "frac": round(achieved / peak, 4),
                "peak_source": ("of measured: dense bf16 GEMM burst in MEASURED_PEAKS.json (f16 "
                                "has the same nominal rate)" if peaks.get("bf16_tflops") else
                                "of fallback: 1.9 PFLOP/s bf16 burst"),
                "warp_mma_f16_peak_tflops": round(2.0 * mma_peak / 1e12, 1),
                "flops_per_call": 2 * ops[ph], "launches_per_call": launches_of[ph],
                "ms_per_call": round(ms, 4),
                "traffic": NCU_TRAFFIC_BYTES.get(kernel_of(ph, tuned)),
            }
        achieved = ops[ph] / (ms * 1e-3) / 1e12
        peak = (lop3_peak if PIPE_OF[ph] == "lop3" else imad_peak) / 1e12
        return {
            "bound": "alu", "kernel": kernel_of(ph, tuned), "phase": ph, "pipe": PIPE_OF[ph],
            "achieved": round(achieved, 3), "peak": round(peak, 3), "unit": "Tops/s",
            "frac": round(achieved / peak, 4),
            "peak_source": "measured on this GPU by snt_measure_int_peak (%s stream, %d SMs)"
                           % (PIPE_OF[ph].upper(), sms),
            "ops_per_call": ops[ph], "launches_per_call": launches_of[ph],
            "ms_per_call": round(ms, 4),
            "traffic": NCU_TRAFFIC_BYTES.get(kernel_of(ph, tuned)),
        }

    phase_roofline = {ph: roofline_of(ph) for ph in ops if ph in phase}
    # the whole path's algorithmic operations per key (the formula of each
    # phase above, summed) at the measured key rate, against the measured
    # integer multiply-add stream
    ops_key = sum(ops.values()) / B
    path_rate = value * ops_key
    path_ops = {
        "formula": ("per call: R/q products (up B-K, down and h as counted with the fused "
                    "leaf level) x p^2 multiply-adds, root inversions K x (2p-1) x 2(p+1) "
                    "multiply-reduces, R/3 " + ("per-key bit-sliced divsteps (word ops)"
                                                if r3m == 0 else "batch products 3(B-K) x p^2 "
                                                "multiply-adds mod 3") + "; divided by B"),
        "ops_per_key": round(ops_key),
        "rate_tops": round(path_rate / 1e12, 3),
        "int32_peak_tops": round(imad_peak / 1e12, 3),
        "frac_of_int32_peak": round(path_rate / imad_peak, 3),
        "note": "the products run on the tensor cores (f16 warp MMA with exact limbs), so the "
                "path can exceed the integer multiply-add peak",
    }
    critical = [ph for ph in ops if ph != "r3_inv" or tuned.get("r3_overlap", 1) == 0]
    dom = max(critical, key=lambda ph: phase.get(ph, 0.0))
    roofline = dict(phase_roofline[dom])
    roofline["roots"] = K

    # serving loop: Poisson handshakes (encapsulation, then decapsulation of
    # the same items), log-uniform sizes in [1, 64], key pool refilled in
    # batches of 8192, 16 GiB device budget; latency from arrival to completion
    serve = []
    for r in [float(x) for x in args.serve_rates.split(",") if x.strip()]:
        st, _, _ = snt.snt_serve_run(ctx, P=P, rate=r, duration_s=args.serve_duration,
                                     max_items=64, dec_fraction=1.0, pool_keys=16384,
                                     refill_batch=8192, mem_budget=16 << 30, max_inflight=4,
                                     max_launch_items=4096, seed=args.seed + 17)
        serve.append({"rate": r, "requests": st["requests"],
                      "p50_ms": round(st["p50_ms"], 4), "p99_ms": round(st["p99_ms"], 4),
                      "max_ms": round(st["max_ms"], 3),
                      "served_requests_per_s": round(st["requests_per_s"], 1),
                      "items_per_s": round(st["items_per_s"], 1),
                      "items_enc": st["items_enc"], "items_dec": st["items_dec"],
                      "keys_generated": st["keys_generated"], "mismatches": st["mismatches"],
                      "max_queue": st["max_queue"], "wall_s": round(st["wall_s"], 3),
                      # items of the requests that arrived, per second of the arrival window
                      "offered_items_per_s": round((st["items_enc"] + st["items_dec"])
                                                   / args.serve_duration, 1)})

    extra = {}
    if not args.no_extra and rank == 0:
        extra["b32"] = measure_b32(snt, torch, dev, stream, flush, args.seed, 50)
        extra["ragged"] = measure_ragged(snt, torch, np, dev, stream, flush, 5)
        extra["micro"] = measure_micro(snt, torch, ctx, dev, stream, flush, 3)

    cpu = None
    if do_cpu:
        rate, nkeys = oracle_rate(pool, cores, args.seed, 5 * 10**9, 24)
        cpu = {"value": round(rate, 2), "unit": "keys/s", "cores": cores, "kind": "oracle",
               "sample": "%d sntrup761 keys (24 per core), plain C oracle: schoolbook products, "
                         "extended-Euclid inversions, per key" % nkeys}
        pool.close()

    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "keys/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": "sntrup761 batch keygen, B=%d keys per launch, seeded "
                               "(seed %d), fresh key indices every step" % (B, args.seed),
                   "p": P, "q": Q, "w": W, "B": B, "parallelism": "replicas" if world > 1 else "1gpu",
                   "l2": "flushed between steps (256 MiB write)"},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": round(e2e_rate, 1), "unit": "keys/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": B * (pkb + skb),
                "api": "snt_batch_keygen_host_async per step into pinned host buffers, "
                       "snt_ctx_sync once after the %d steps (host wall clock)" % async_steps,
                "synchronous_call_keys_per_s": round(e2e_sync_rate, 1)},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
        "int_peaks_tops": {"lop3": round(lop3_peak / 1e12, 3), "imad": round(imad_peak / 1e12, 3),
                           "warp_mma_f16_macs": round(mma_peak / 1e12, 3),
                           "sms": sms},
        "phase_roofline": phase_roofline,
        "path_ops": path_ops,
        "paper_context": "156317 Haswell cycles/key at n=32 (E3-1275 v3, 3.5 GHz: ~22.4k keys/s/core)",
        "serve": {"workload": "sntrup761 handshakes for %.2f s per rate: Poisson encapsulation "
                              "requests of log-uniform size in [1, 64], each followed by the "
                              "decapsulation of its items; 16384-key device pool refilled by "
                              "8192-key batch keygen; 16 GiB budget; 4 launch streams"
                              % args.serve_duration,
                  "runs": serve,
                  # the loop's saturation throughput: the served rate of the
                  # most loaded run whose offered load exceeded what it served
                  "capacity_items_per_s": max([r["items_per_s"] for r in serve
                                               if r["offered_items_per_s"] > 1.2 * r["items_per_s"]]
                                              or [None])},
        # last, so that a reader of the line's tail sees them
        "perkey_gpu": {"value": round(perkey_rate, 1), "unit": "keys/s",
                       "ms_per_step": round(pk_ms / pk_steps, 4),
                       "batched_speedup": round(value / perkey_rate, 3)},
    }
    line.update(extra)
    line["launch_modes"] = launch_modes
    line["phases_ms"] = {k: round(v, 4) for k, v in phase.items()}
    line["tuned"] = tuned
    ctx.close()
    if dist:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


# ------------------------------------------------------------ reference arm
def run_reference(args):
    """The oracle (the deliberately slow CPU definition) on the host cores,
    same metric and workload, each step a bounded sample of keys."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    pool, cores = cpu_pool()
    pool.map(_oracle_keys, [(1, 0, 1)] * cores)
    per_core = 2
    for i in range(max(3, args.warmup) if args.warmup else 0):
        oracle_rate(pool, cores, args.seed, 7 * 10**9 + i * cores * per_core, per_core)
    total_keys, t0 = 0, time.perf_counter()
    for i in range(args.steps):
        _, n = oracle_rate(pool, cores, args.seed, i * cores * per_core, per_core)
        total_keys += n
    el = time.perf_counter() - t0
    pool.close()
    value = total_keys / el
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 2), "unit": "keys/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * el / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": "sntrup761 batch keygen, B=%d keys per launch, seeded "
                               "(seed %d)" % (args.batch, args.seed),
                   "p": P, "q": Q, "w": W, "B": args.batch},
        "cpu_baseline": {"value": round(value, 2), "unit": "keys/s", "cores": cores,
                         "kind": "oracle",
                         "sample": "each step %d keys (%d per core) of the workload" % (
                             cores * per_core, per_core)},
        "e2e": {"value": round(value, 2), "unit": "keys/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
