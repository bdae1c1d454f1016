"""Building-block kernels (R/q product, R/q and R/3 inversion) vs the oracle,
on small cases and on the full-size microbenchmark workload (sampled)."""
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


@pytest.fixture(scope="module")
def ctx(snt):
    c = snt.Context(0, 64 << 20)
    yield c
    c.close()


def _t(x, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to(dtype=dtype, device="cuda")


def _rq_cases(p, q, rng, n):
    h = (q - 1) // 2
    a = rng.integers(-h, h + 1, (n, p))
    b = rng.integers(-h, h + 1, (n, p))
    a[0], b[0] = h, h            # all-max coefficients
    a[1], b[1] = -h, h
    a[2], b[2] = 0, rng.integers(-h, h + 1, p)
    a[3] = 0; a[3, p - 1] = 1    # x^(p-1) * x^(p-1)
    b[3] = 0; b[3, p - 1] = 1
    a[4] = rng.integers(-1, 2, p)  # ternary operand
    return a, b


@pytest.mark.parametrize("engine", [0, 1, 2, 3])
@pytest.mark.parametrize("P", [653, 761, 857])
def test_rq_mul_matches_oracle(snt, ctx, P, engine):
    # engine 0: CUDA-core Toeplitz products; 1: the same products as warp MMAs
    # on exact f16 limbs (extreme operands exercise the limb and sum bounds);
    # 2: the transform multiplier over K = (Z/q)[x]/(x^64 + 1) (extreme
    # operands exercise the growth bounds of the butterflies); 3: warp MMAs
    # with one wide f16 limb on the vector side (all-max operands reach the
    # int32 sums' bound; odd residues above 2048 take the moved representative)
    import torch
    p, q, _ = oracle.PARAMS[P]
    rng = np.random.default_rng(P)
    n = 41  # ragged last CTA of the 4-products-per-CTA tensor-core kernel
    a, b = _rq_cases(p, q, rng, n)
    c = torch.empty(n * p, dtype=torch.int16, device="cuda")
    ctx.set_option(snt.SNT_OPT_RQ_ENGINE, engine)
    try:
        snt.snt_rq_mul(ctx, P, n, _t(a.ravel(), torch.int16), _t(b.ravel(), torch.int16), c)
    finally:
        ctx.set_option(snt.SNT_OPT_RQ_ENGINE, 1)
    got = c.cpu().numpy().reshape(n, p)
    for i in range(n):
        assert np.array_equal(got[i], oracle.ring_mul(p, q, a[i], b[i])), i


@pytest.mark.parametrize("latency", [False, True])
@pytest.mark.parametrize("P", [653, 761, 857])
def test_rq_inv_matches_oracle(snt, ctx, P, latency):
    import torch
    p, q, _ = oracle.PARAMS[P]
    rng = np.random.default_rng(P + 1)
    n = 12
    h = (q - 1) // 2
    a = rng.integers(-h, h + 1, (n, p))
    a[0] = 0                      # not invertible
    a[1] = 0; a[1, 0] = 1         # 1
    a[2] = 3 * rng.integers(-1, 2, p)
    out = torch.empty(n * p, dtype=torch.int16, device="cuda")
    ok = torch.empty(n, dtype=torch.int32, device="cuda")
    fn = snt.snt_rq_inv_latency if latency else snt.snt_rq_inv
    fn(ctx, P, n, _t(a.ravel(), torch.int16), out, ok)
    got = out.cpu().numpy().reshape(n, p)
    okh = ok.cpu().numpy()
    for i in range(n):
        rok, ref = oracle.ring_inv(p, q, a[i])
        assert bool(okh[i]) == rok, i
        assert np.array_equal(got[i], ref), i


def _non_invertible(p, rng):
    parts = oracle.ddf(p, 3)
    d, _, f1 = min(parts, key=lambda t: t[0])
    f1 = f1[: d + 1]
    r = rng.integers(0, 3, p - d)
    g = np.convolve(f1, r) % 3
    return np.where(g == 2, -1, g)


@pytest.mark.parametrize("lanes,kpt", [(4, 1), (8, 1), (32, 1), (4, 2), (8, 2), (32, 2)])
@pytest.mark.parametrize("P", [653, 761, 857])
def test_r3_inv_matches_oracle(snt, ctx, P, lanes, kpt):
    import torch
    p = P
    rng = np.random.default_rng(P + 2)
    n = 37  # ragged: not a multiple of the elements per CTA
    g = rng.integers(-1, 2, (n, p))
    g[0] = 0
    g[1] = 0; g[1, 0] = 1
    g[2] = _non_invertible(p, rng)
    g[3] = 1
    out = torch.empty(n * p, dtype=torch.int8, device="cuda")
    ok = torch.empty(n, dtype=torch.int32, device="cuda")
    ctx.set_option(snt.SNT_OPT_R3_LANES, lanes)
    ctx.set_option(snt.SNT_OPT_R3_KPT, kpt)  # 2: two elements per lane group, interleaved
    try:
        snt.snt_r3_inv(ctx, P, n, _t(g.ravel(), torch.int8), out, ok)
    finally:
        ctx.set_option(snt.SNT_OPT_R3_LANES, 4)
        ctx.set_option(snt.SNT_OPT_R3_KPT, 1)
    got = out.cpu().numpy().reshape(n, p)
    okh = ok.cpu().numpy()
    assert okh[2] == 0 and okh[0] == 0
    for i in range(n):
        rok, ref = oracle.ring_inv(p, 3, g[i])
        assert bool(okh[i]) == rok, i
        assert np.array_equal(got[i], ref), i


@pytest.fixture(scope="module")
def pool():
    from oracle_pool import OraclePool
    p = OraclePool()
    yield p
    p.close()


def test_microbench_products_vs_oracle(snt, ctx, pool):
    """Kernel microbenchmark workload at full size (p = 761): 2^20 general x
    general and 2^20 general x Short products, 4096 sampled products of each
    kind (the first, the last and the boundaries of the 4-products-per-CTA
    groups among them) checked against the oracle's schoolbook product."""
    import torch
    p, q, w = oracle.PARAMS[761]
    from synth import rq_uniform, short_batch
    n = 1 << 20
    a = rq_uniform(761, n, seed=1)
    b = rq_uniform(761, n, seed=2)
    s = short_batch(761, n, seed=3)
    assert (np.count_nonzero(s, axis=1) == w).all()
    da, db, ds = _t(a.ravel(), torch.int16), _t(b.ravel(), torch.int16), _t(s.ravel(), torch.int16)
    c = torch.empty(n * p, dtype=torch.int16, device="cuda")
    c2 = torch.empty(n * p, dtype=torch.int16, device="cuda")
    snt.snt_rq_mul(ctx, 761, n, da, db, c)
    snt.snt_rq_mul(ctx, 761, n, da, ds, c2)
    # the transform multiplier and the one-wide-limb tensor-core form give
    # every one of the 2^20 + 2^20 products the tensor-core engine gives (which
    # is checked against the oracle below)
    c3 = torch.empty_like(c)
    try:
        for engine in (2, 3):
            ctx.set_option(snt.SNT_OPT_RQ_ENGINE, engine)
            snt.snt_rq_mul(ctx, 761, n, da, db, c3)
            assert torch.equal(c, c3), engine
            snt.snt_rq_mul(ctx, 761, n, da, ds, c3)
            assert torch.equal(c2, c3), engine
    finally:
        ctx.set_option(snt.SNT_OPT_RQ_ENGINE, 1)
    del c3
    torch.cuda.synchronize()
    rng = np.random.default_rng(4)
    idx = np.unique(np.concatenate([[0, 1, 2, 3, 4, n - 5, n - 4, n - 1],
                                    rng.choice(n, 4096, replace=False)]))
    assert idx.size >= 4096
    ti = torch.from_numpy(idx).cuda()
    got = c.view(n, p)[ti].cpu().numpy()
    got2 = c2.view(n, p)[ti].cpu().numpy()
    assert pool.bad_products(p, q, a[idx], b[idx], got) == []
    assert pool.bad_products(p, q, a[idx], s[idx], got2) == []


def test_microbench_all_r3_inversions(snt, ctx, pool):
    """All 2^16 R/3 inversions of the microbenchmark workload: every output
    with its flag set satisfies g * v = 1 in R/3 (the inverse is unique, so
    this pins v), every flagged failure is a zero divisor per the oracle."""
    import torch
    from synth import ternary_batch
    p = 761
    m = 1 << 16
    g = ternary_batch(761, m, seed=5)
    out = torch.empty(m * p, dtype=torch.int8, device="cuda")
    ok = torch.empty(m, dtype=torch.int32, device="cuda")
    snt.snt_r3_inv(ctx, 761, m, _t(g.ravel(), torch.int8), out, ok)
    outh = out.cpu().numpy().reshape(m, p)
    okh = ok.cpu().numpy()
    assert pool.bad_identities(p, 3, g, outh, okh) == []


@pytest.mark.parametrize("latency", [False, True])
def test_microbench_all_rq_inversions(snt, ctx, pool, latency):
    """All 2^10 R/q inversions of the microbenchmark workload, by the
    step-at-a-time kernel and by jump divsteps, equal to the oracle's
    extended-Euclid inverses."""
    import torch
    from synth import rq_uniform
    p, q, _ = oracle.PARAMS[761]
    k = 1 << 10
    x = rq_uniform(761, k, seed=6)
    out = torch.empty(k * p, dtype=torch.int16, device="cuda")
    ok = torch.empty(k, dtype=torch.int32, device="cuda")
    fn = snt.snt_rq_inv_latency if latency else snt.snt_rq_inv
    fn(ctx, 761, k, _t(x.ravel(), torch.int16), out, ok)
    outh = out.cpu().numpy().reshape(k, p)
    okh = ok.cpu().numpy()
    assert okh.all()
    assert pool.bad_inverses(p, q, x, outh, okh) == []


@pytest.mark.parametrize("n,k", [(16, 1), (64, 1), (256, 1), (16, 4), (128, 4), (256, 2)])
def test_tcgen05_measurement_checks_its_accumulator(snt, n, k):
    # the tcgen05.mma rate measurement (engine choice; not on the keygen path)
    # verifies D = A B^T against its closed form before reporting a rate;
    # k CTAs per SM share the tensor core (k * max(32, n) <= 512 columns)
    rate, sms = snt.snt_measure_tc05(0, n, k)
    assert rate > 0 and sms > 0
    with pytest.raises(snt.SntError):
        snt.snt_measure_tc05(0, 256, 4)  # 1024 tensor-memory columns: refused
