"""Kernel microbenchmark (sntrup761 building blocks) on one GPU.

    python -m paper_2106_08759_gb300.microbench [--quick] [--sweep] [--keygen-only B]

Times each building block alone (CUDA events on the launching stream, L2
flushed before every timed launch) on seeded synthetic inputs:
  - R/q products, general x general and general x Short (2^20 each),
  - R/3 inversions by bit-sliced divsteps (2^16),
  - R/q inversions by per-step divsteps (2^10) and by jump divsteps (2^10,
    and one element alone: the latency of the tree's root inversion),
  - batch keygen phases at B = 4096 with the auxiliary-stream overlap.
Prints one JSON line.  Inputs come from synth (numpy); outputs are not
checked here (the parity tests do that).
"""
import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--quick", action="store_true", help="smaller counts")
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--sweep", action="store_true",
                    help="also time the layout options of the R/3 kernel and of keygen")
    ap.add_argument("--keygen-only", type=int, default=0, metavar="B",
                    help="only run batch keygen of B keys --reps times with the default "
                         "options (a small, fixed target for a profiler)")
    ap.add_argument("--opt", action="append", default=[], metavar="NAME=VALUE",
                    help="context option for --keygen-only / --ragged-only, e.g. R3_MODE=1 "
                         "(SNT_OPT_ prefix implied)")
    ap.add_argument("--ragged-only", type=int, default=0, metavar="N",
                    help="only run the 256-batch ragged workload N times with the given options "
                         "(a small, fixed target for a profiler)")
    ap.add_argument("--tuned", action="store_true",
                    help="with --ragged-only: autotune each parameter set for batches of up to "
                         "2048 keys first, as the bench does; with --keygen-only: autotune "
                         "(761, B) first.  The last call is bracketed by cudaProfilerStart/Stop "
                         "(ncu --profile-from-start off captures it alone).  Under a profiler "
                         "the autotuner times serialised kernels and picks other layouts: pin "
                         "the layouts with --opt for a profile")
    ap.add_argument("--kem-only", type=int, default=0, metavar="N",
                    help="only run N encapsulations and decapsulations of sntrup761 keys, twice")
    ap.add_argument("--mul-only", type=int, default=0, metavar="N",
                    help="only run N general R/q products twice with the given options "
                         "(e.g. RQ_ENGINE=2)")
    ap.add_argument("--tc05-only", type=int, default=0, metavar="NCOLS",
                    help="only run the tcgen05.mma rate measurement at N = NCOLS")
    args = ap.parse_args()

    import numpy as np
    import torch

    import paper_2106_08759_gb300 as snt
    from synth import rq_uniform, short_batch, ternary_batch

    P, p = 761, 761
    dev = torch.device("cuda", 0)
    ctx = snt.Context(0, 512 << 20)
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream()

    def timeit(fn):
        fn()
        torch.cuda.synchronize()
        best = None
        for _ in range(args.reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            fn()
            b.record(st)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            best = ms if best is None else min(best, ms)
        return best

    def t(x, dt):
        return torch.from_numpy(np.ascontiguousarray(x)).to(dtype=dt, device=dev)

    if args.ragged_only:
        from synth import ragged_batches
        sizes, ps = ragged_batches(256, 2048, 42)
        pks, sks = [], []
        for P_, B_ in zip(ps, sizes):
            pkb_, skb_, _, _ = snt.snt_param_sizes(int(P_))
            pks.append(torch.empty(int(B_) * pkb_, dtype=torch.uint8, device=dev))
            sks.append(torch.empty(int(B_) * skb_, dtype=torch.uint8, device=dev))
        firsts = [int(x) for x in np.cumsum([0] + list(sizes[:-1]))]
        with snt.Context(0, 1 << 30) as rc:
            for o in args.opt:
                name, val = o.split("=")
                rc.set_option(getattr(snt, "SNT_OPT_" + name), int(val))
            if args.tuned:
                for x in (653, 761, 857):
                    rc.autotune(x, 2048)
            rc.sync()
            for it in range(args.ragged_only):
                last = it == args.ragged_only - 1
                if last:
                    torch.cuda.profiler.start()
                snt.snt_batch_keygen_ragged(rc, [int(x) for x in ps], [int(x) for x in sizes],
                                            [it * 1000 + i for i in range(256)], firsts, pks, sks)
                rc.sync()
                if last:
                    torch.cuda.profiler.stop()
        print(json.dumps({"ragged_only": args.ragged_only, "keys": int(sizes.sum())}))
        ctx.close()
        return
    if args.tc05_only:
        rate, sms = snt.snt_measure_tc05(0, args.tc05_only, 1)
        print(json.dumps({"tc05_n": args.tc05_only, "tmacs": rate / 1e12, "sms": sms}))
        ctx.close()
        return
    if args.mul_only:
        for o in args.opt:
            name, val = o.split("=")
            ctx.set_option(getattr(snt, "SNT_OPT_" + name), int(val))
        n = args.mul_only
        A = t(rq_uniform(P, n, 1).ravel(), torch.int16)
        Bm = t(rq_uniform(P, n, 2).ravel(), torch.int16)
        C = torch.empty(n * p, dtype=torch.int16, device=dev)
        for _ in range(2):
            snt.snt_rq_mul(ctx, P, n, A, Bm, C)
        torch.cuda.synchronize()
        print(json.dumps({"mul_only": n}))
        ctx.close()
        return
    if args.kem_only:
        n = args.kem_only
        pkb, skb, ctb, _ = snt.snt_param_sizes(P)
        pk = torch.empty(n * pkb, dtype=torch.uint8, device=dev)
        sk = torch.empty(n * skb, dtype=torch.uint8, device=dev)
        for i in range(0, n, 4096):
            m = min(4096, n - i)
            snt.snt_batch_keygen(ctx, P, 3, i, m, pk[i * pkb:(i + m) * pkb],
                                 sk[i * skb:(i + m) * skb])
        ct = torch.empty(n * ctb, dtype=torch.uint8, device=dev)
        ss = torch.empty(n * 32, dtype=torch.uint8, device=dev)
        ss2 = torch.empty(n * 32, dtype=torch.uint8, device=dev)
        for _ in range(2):
            snt.snt_enc(ctx, P, n, pk, 5, 0, ct, ss)
            snt.snt_dec(ctx, P, n, sk, ct, ss2)
        ctx.sync()
        print(json.dumps({"kem_only": n, "dec_matches_enc": bool(torch.equal(ss, ss2))}))
        ctx.close()
        return
    if args.keygen_only:
        for o in args.opt:
            name, val = o.split("=")
            ctx.set_option(getattr(snt, "SNT_OPT_" + name), int(val))
        B = args.keygen_only
        tuned = ctx.autotune(P, B) if args.tuned else None
        pkb, skb, _, _ = snt.snt_param_sizes(P)
        pk = torch.empty(B * pkb, dtype=torch.uint8, device=dev)
        sk = torch.empty(B * skb, dtype=torch.uint8, device=dev)
        for i in range(args.reps):
            flush.zero_()
            last = i == args.reps - 1
            if last:
                torch.cuda.synchronize()
                torch.cuda.profiler.start()
            snt.snt_batch_keygen(ctx, P, 1, i * B, B, pk, sk, st)
            if last:
                torch.cuda.synchronize()
                ctx.sync()
                torch.cuda.profiler.stop()
        torch.cuda.synchronize()
        ctx.sync()
        print(json.dumps({"keygen_only": B, "reps": args.reps, "tuned": tuned}))
        ctx.close()
        return

    out = {"p": p}
    n = (1 << 16) if args.quick else (1 << 20)
    A = t(rq_uniform(P, n, 1).ravel(), torch.int16)
    Bm = t(rq_uniform(P, n, 2).ravel(), torch.int16)
    S = t(short_batch(P, n, 3).ravel(), torch.int16)
    C = torch.empty(n * p, dtype=torch.int16, device=dev)
    ms = timeit(lambda: snt.snt_rq_mul(ctx, P, n, A, Bm, C))
    out["rq_mul_gen"] = {"n": n, "ms": ms, "products_per_s": n / ms * 1e3,
                         "gmac_per_s": n * p * p / ms / 1e6}
    ms = timeit(lambda: snt.snt_rq_mul(ctx, P, n, A, S, C))
    out["rq_mul_short"] = {"n": n, "ms": ms, "products_per_s": n / ms * 1e3}
    eng = ctx.get_option(snt.SNT_OPT_RQ_ENGINE)
    for e in (0, 1):
        ctx.set_option(snt.SNT_OPT_RQ_ENGINE, e)
        ms = timeit(lambda: snt.snt_rq_mul(ctx, P, n, A, Bm, C))
        out["rq_mul_gen_engine%d" % e] = {"n": n, "ms": ms, "products_per_s": n / ms * 1e3,
                                          "gmac_per_s": n * p * p / ms / 1e6}
    ctx.set_option(snt.SNT_OPT_RQ_ENGINE, eng)
    del A, Bm, S, C

    m = (1 << 12) if args.quick else (1 << 16)
    G = t(ternary_batch(P, m, 5).ravel(), torch.int8)
    O = torch.empty(m * p, dtype=torch.int8, device=dev)
    OK = torch.empty(m, dtype=torch.int32, device=dev)
    ms = timeit(lambda: snt.snt_r3_inv(ctx, P, m, G, O, OK))
    out["r3_inv"] = {"n": m, "ms": ms, "inv_per_s": m / ms * 1e3}
    G4 = G[: 4096 * p]
    ms = timeit(lambda: snt.snt_r3_inv(ctx, P, 4096, G4, O, OK))
    out["r3_inv_4096"] = {"n": 4096, "ms": ms}
    if args.sweep:
        default_lanes = ctx.get_option(snt.SNT_OPT_R3_LANES)
        for lanes in (4, 8, 32):
            for kpt in (1, 2):
                ctx.set_option(snt.SNT_OPT_R3_LANES, lanes)
                ctx.set_option(snt.SNT_OPT_R3_KPT, kpt)
                out["r3_inv_4096_lanes%d_kpt%d_ms" % (lanes, kpt)] = timeit(
                    lambda: snt.snt_r3_inv(ctx, P, 4096, G4, O, OK))
                out["r3_inv_%d_lanes%d_kpt%d_ms" % (m, lanes, kpt)] = timeit(
                    lambda: snt.snt_r3_inv(ctx, P, m, G, O, OK))
        ctx.set_option(snt.SNT_OPT_R3_LANES, default_lanes)
        ctx.set_option(snt.SNT_OPT_R3_KPT, 1)

    k = 1 << 10
    X = t(rq_uniform(P, k, 6).ravel(), torch.int16)
    XO = torch.empty(k * p, dtype=torch.int16, device=dev)
    XK = torch.empty(k, dtype=torch.int32, device=dev)
    ms = timeit(lambda: snt.snt_rq_inv(ctx, P, k, X, XO, XK))
    out["rq_inv_perstep"] = {"n": k, "ms": ms, "inv_per_s": k / ms * 1e3}
    ms = timeit(lambda: snt.snt_rq_inv_latency(ctx, P, k, X, XO, XK))
    out["rq_inv_jump"] = {"n": k, "ms": ms, "inv_per_s": k / ms * 1e3}
    ms = timeit(lambda: snt.snt_rq_inv_latency(ctx, P, 1, X, XO, XK))
    out["rq_inv_jump_single_ms"] = ms
    ms = timeit(lambda: snt.snt_rq_inv(ctx, P, 1, X, XO, XK))
    out["rq_inv_perstep_single_ms"] = ms

    Bk = 4096
    pkb, skb, _, _ = snt.snt_param_sizes(P)
    pk = torch.empty(Bk * pkb, dtype=torch.uint8, device=dev)
    sk = torch.empty(Bk * skb, dtype=torch.uint8, device=dev)
    ctx.set_timing(True)
    snt.snt_batch_keygen(ctx, P, 1, 0, Bk, pk, sk)
    ph = ctx.phase_times()
    tot = 0.0
    for i in range(args.reps):
        flush.zero_()
        snt.snt_batch_keygen(ctx, P, 1, (i + 1) * Bk, Bk, pk, sk)
        ph = ctx.phase_times()
        tot += ph["total"]
    out["keygen_4096_phases_ms"] = ph
    out["keygen_4096_ms"] = tot / args.reps
    if args.sweep:
        sweep = {}
        def run_keygen_avg():
            snt.snt_batch_keygen(ctx, P, 1, 0, Bk, pk, sk)
            ctx.phase_times()
            tot = 0.0
            for i in range(args.reps):
                flush.zero_()
                snt.snt_batch_keygen(ctx, P, 1, (i + 1) * Bk, Bk, pk, sk)
                ph = ctx.phase_times()
                tot += ph["total"]
            return {"ms": round(tot / args.reps, 4), "phases": {k: round(v, 4) for k, v in ph.items()}}
        ctx.set_option(snt.SNT_OPT_R3_LANES, 4)
        ctx.set_option(snt.SNT_OPT_TREE_SPLIT, 8)
        for overlap in (0, 1, 2, 3):
            ctx.set_option(snt.SNT_OPT_R3_OVERLAP, overlap)
            for roots in (1, 4, 16, 64):
                for r3mode in (0, 1, 2):
                    ctx.set_option(snt.SNT_OPT_RQ_ENGINE, 1)
                    ctx.set_option(snt.SNT_OPT_ROOTS, roots)
                    ctx.set_option(snt.SNT_OPT_R3_MODE, r3mode)
                    sweep["mma_roots%d_overlap%d_r3mode%d" % (roots, overlap, r3mode)] = \
                        run_keygen_avg()
        ctx.set_option(snt.SNT_OPT_ROOTS, 1)
        ctx.set_option(snt.SNT_OPT_R3_MODE, 0)
        ctx.set_option(snt.SNT_OPT_RQ_ENGINE, 0)
        for narrow in (0, 1):
            for overlap in (0, 1, 2, 3):
                for lanes in (4, 8):
                    for split in (4, 8):
                        ctx.set_option(snt.SNT_OPT_NARROW_SEG, narrow)
                        ctx.set_option(snt.SNT_OPT_R3_OVERLAP, overlap)
                        ctx.set_option(snt.SNT_OPT_R3_LANES, lanes)
                        ctx.set_option(snt.SNT_OPT_TREE_SPLIT, split)
                        snt.snt_batch_keygen(ctx, P, 1, 0, Bk, pk, sk)
                        ctx.phase_times()
                        tot = 0.0
                        for i in range(args.reps):
                            flush.zero_()
                            snt.snt_batch_keygen(ctx, P, 1, (i + 1) * Bk, Bk, pk, sk)
                            ph = ctx.phase_times()
                            tot += ph["total"]
                        key = "narrow%d_overlap%d_lanes%d_split%d" % (narrow, overlap, lanes, split)
                        sweep[key] = {"ms": round(tot / args.reps, 4),
                                      "phases": {k: round(v, 4) for k, v in ph.items()}}
        ctx.set_option(snt.SNT_OPT_RQ_ENGINE, 1)
        out["keygen_4096_sweep"] = sweep
    ctx.close()

    # ragged workload: 256 batches, log-uniform sizes in [1, 2048], mixed
    # parameter sets, one graph launch (timed after the graph is built)
    from synth import ragged_batches
    sizes, ps = ragged_batches(256, 2048, 42)
    rctx = snt.Context(0, 1 << 30)
    pks, sks = [], []
    for P_, B_ in zip(ps, sizes):
        pkb_, skb_, _, _ = snt.snt_param_sizes(int(P_))
        pks.append(torch.empty(int(B_) * pkb_, dtype=torch.uint8, device=dev))
        sks.append(torch.empty(int(B_) * skb_, dtype=torch.uint8, device=dev))
    firsts = [int(x) for x in np.cumsum([0] + list(sizes[:-1]))]
    it = [0]

    def ragged():
        it[0] += 1
        snt.snt_batch_keygen_ragged(rctx, [int(x) for x in ps], [int(x) for x in sizes],
                                    [it[0] * 1000 + i for i in range(256)], firsts, pks, sks)

    ms = timeit(ragged)
    nkeys = int(sizes.sum())
    out["ragged_256"] = {"batches": 256, "keys": nkeys, "ms": ms, "keys_per_s": nkeys / ms * 1e3,
                         "keys_by_p": {int(P_): int(sizes[ps == P_].sum()) for P_ in (653, 761, 857)}}
    rctx.close()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
