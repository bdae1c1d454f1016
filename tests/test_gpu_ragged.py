"""Ragged keygen (many batches, mixed sizes and parameter sets, one graph
launch): every batch must equal snt_batch_keygen of that batch alone, which
the other tests tie to the oracle; a few keys are also checked against the
oracle directly."""
import numpy as np
import pytest

import oracle
from gpu_util import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def snt():
    require_gpu()
    import paper_2106_08759_gb300 as m
    m.load()
    return m


def _run_ragged(snt, ctx, Ps, Bs, seeds, firsts):
    import torch
    pks, sks = [], []
    for P, B in zip(Ps, Bs):
        pkb, skb, _, _ = snt.snt_param_sizes(P)
        pks.append(torch.full((B * pkb,), 0xAA, dtype=torch.uint8, device="cuda"))
        sks.append(torch.full((B * skb,), 0xAA, dtype=torch.uint8, device="cuda"))
    snt.snt_batch_keygen_ragged(ctx, Ps, Bs, seeds, firsts, pks, sks)
    ctx.sync()
    return [(pk.cpu().numpy().reshape(B, -1), sk.cpu().numpy().reshape(B, -1))
            for pk, sk, B in zip(pks, sks, Bs)]


def _single(snt, ctx, P, B, seed, first):
    import torch
    pkb, skb, _, _ = snt.snt_param_sizes(P)
    pk = torch.empty(B * pkb, dtype=torch.uint8, device="cuda")
    sk = torch.empty(B * skb, dtype=torch.uint8, device="cuda")
    snt.snt_batch_keygen(ctx, P, seed, first, B, pk, sk)
    ctx.sync()
    return pk.cpu().numpy().reshape(B, -1), sk.cpu().numpy().reshape(B, -1)


@pytest.mark.parametrize("r3_mode", [0, 1, 2])
def test_ragged_small_mixed(snt, r3_mode):
    # R/3 per key (0), batched after the invertibility test (1), or batched on
    # the first draws with the per-batch fall-back (2)
    Ps = [761, 653, 857, 761, 761, 653, 857]
    Bs = [5, 1, 33, 2, 64, 17, 1]
    firsts = [0, 10, 20, 100, 200, 300, 400]
    with snt.Context(0, 128 << 20) as ctx:
        ctx.set_option(snt.SNT_OPT_R3_MODE, r3_mode)
        for rnd, seeds in enumerate([[11, 12, 13, 14, 15, 16, 17], [21, 22, 23, 24, 25, 26, 27]]):
            # the second round replays the cached graph with new seeds
            got = _run_ragged(snt, ctx, Ps, Bs, seeds, firsts)
            for (pk, sk), P, B, s, f in zip(got, Ps, Bs, seeds, firsts):
                rpk, rsk = _single(snt, ctx, P, B, s, f)
                assert np.array_equal(pk, rpk) and np.array_equal(sk, rsk), (rnd, P, B)
        # oracle spot checks (second round's seeds)
        for i in (1, 2, 6):
            opk, osk, _ = oracle.keygen(Ps[i], seeds[i], firsts[i] + Bs[i] - 1)
            assert np.array_equal(got[i][0][-1], opk) and np.array_equal(got[i][1][-1], osk)


@pytest.mark.parametrize("layout", ["options", "autotuned"])
def test_ragged_full_workload_256_batches(snt, layout):
    """The ragged workload: 256 batches of log-uniform size in [1, 2048]
    (seed 42), equal shares of sntrup653/761/857 after a seeded shuffle; with
    the context's default options, and with the layouts the autotuner picks
    for (p, 2048), the configuration the benchmark times."""
    from synth import ragged_batches
    sizes, ps = ragged_batches(256, 2048, 42)
    seeds = [1000 + i for i in range(256)]
    firsts = list(np.cumsum([0] + list(sizes[:-1])))
    with snt.Context(0, 1 << 30) as ctx:
        if layout == "autotuned":
            for P in (653, 761, 857):
                ctx.autotune(P, 2048)
        got = _run_ragged(snt, ctx, list(ps), list(sizes), seeds, firsts)
        for i in range(256):
            rpk, rsk = _single(snt, ctx, int(ps[i]), int(sizes[i]), seeds[i], int(firsts[i]))
            assert np.array_equal(got[i][0], rpk) and np.array_equal(got[i][1], rsk), i
    rng = np.random.default_rng(3)
    for i in rng.integers(0, 256, 6):
        j = int(rng.integers(0, sizes[i]))
        opk, osk, _ = oracle.keygen(int(ps[i]), seeds[i], int(firsts[i]) + j)
        assert np.array_equal(got[i][0][j], opk) and np.array_equal(got[i][1][j], osk)


@pytest.mark.parametrize("r3_mode", [0, 1, 2])
def test_ragged_redraws_injected_zero_divisors(snt, r3_mode):
    # first draws of g that are zero divisors in R/3 (one per irreducible
    # factor of x^761 - x - 1 over F_3) in two batches: the invertibility test
    # (mode 1), the failing batch roots with the per-key fall-back and the
    # fix-up of h, pk and its hash (mode 2), or the per-key kernel (mode 0)
    # must redraw them exactly as the oracle does
    rng = np.random.default_rng(11)
    bads = []
    for d, _, poly in oracle.ddf(761, 3):
        f = np.asarray(poly[: d + 1]) % 3
        g = np.convolve(f, rng.integers(0, 3, 761 - d))[:761] % 3
        bads.append(np.where(g == 2, -1, g).astype(np.int8))
    Ps = [761, 653, 761, 857, 761]
    Bs = [40, 7, 1, 9, 33]
    firsts = [0, 1000, 2000, 3000, 4000]
    seeds = [5, 6, 7, 8, 9]
    keys = [3, 2000, 4031]  # batch 0 key 3, the one-key batch, batch 4 key 31
    with snt.Context(0, 128 << 20) as ctx:
        snt.snt_debug_inject_g(ctx, 761, keys, np.stack(bads))
        ctx.set_option(snt.SNT_OPT_R3_MODE, r3_mode)
        got = _run_ragged(snt, ctx, Ps, Bs, seeds, firsts)
    for (pk, sk), P, B, s, f in zip(got, Ps, Bs, seeds, firsts):
        inj = {k - f: b for k, b in zip(keys, bads) if P == 761 and f <= k < f + B}
        rpk, rsk = oracle.keygen_batch(P, s, f, B, g_inject=inj)
        assert np.array_equal(pk, rpk) and np.array_equal(sk, rsk), (P, B)


def test_ragged_with_and_without_programmatic_launch(snt):
    # the graph is captured again when the launch mode changes; same bytes
    Ps = [653, 761, 857, 761, 653]
    Bs = [40, 129, 7, 1, 300]
    seeds = [31, 32, 33, 34, 35]
    firsts = [0, 50, 200, 300, 400]
    with snt.Context(0, 256 << 20) as ctx:
        ctx.set_option(snt.SNT_OPT_R3_MODE, 2)
        on = _run_ragged(snt, ctx, Ps, Bs, seeds, firsts)
        ctx.set_option(snt.SNT_OPT_PDL, 0)
        off = _run_ragged(snt, ctx, Ps, Bs, seeds, firsts)
        for (a, b), (c, d) in zip(on, off):
            assert np.array_equal(a, c) and np.array_equal(b, d)
        for i in (0, 2, 4):
            opk, osk, _ = oracle.keygen(Ps[i], seeds[i], firsts[i] + Bs[i] - 1)
            assert np.array_equal(on[i][0][-1], opk) and np.array_equal(on[i][1][-1], osk)


def test_ragged_batches_in_one_buffer_at_odd_offsets(snt):
    # every batch's rows inside one buffer, some batches adjacent (their rows
    # form one contiguous run for the hash kernel), some separated by an odd
    # gap; each batch must equal its single-batch call
    import torch
    Ps = [761, 761, 761, 653, 653, 857, 761]
    Bs = [3, 40, 1, 20, 17, 9, 33]
    gaps = [5, 0, 0, 3, 0, 1, 7]
    seeds = [41, 42, 43, 44, 45, 46, 47]
    firsts = [0, 10, 60, 70, 100, 130, 150]
    pk_all = torch.zeros(1 << 18, dtype=torch.uint8, device="cuda")
    sk_all = torch.zeros(1 << 18, dtype=torch.uint8, device="cuda")
    pks, sks, offs = [], [], []
    o_pk = o_sk = 0
    for P, B, gap in zip(Ps, Bs, gaps):
        pkb, skb, _, _ = snt.snt_param_sizes(P)
        o_pk += gap
        o_sk += gap
        pks.append(pk_all[o_pk:o_pk + B * pkb])
        sks.append(sk_all[o_sk:o_sk + B * skb])
        offs.append((o_pk, o_sk, pkb, skb))
        o_pk += B * pkb
        o_sk += B * skb
    with snt.Context(0, 256 << 20) as ctx:
        snt.snt_batch_keygen_ragged(ctx, Ps, Bs, seeds, firsts, pks, sks)
        ctx.sync()
        hp, hs = pk_all.cpu().numpy(), sk_all.cpu().numpy()
        for i, (P, B) in enumerate(zip(Ps, Bs)):
            a, b, pkb, skb = offs[i]
            rpk, rsk = _single(snt, ctx, P, B, seeds[i], firsts[i])
            assert np.array_equal(hp[a:a + B * pkb].reshape(B, pkb), rpk), i
            assert np.array_equal(hs[b:b + B * skb].reshape(B, skb), rsk), i
