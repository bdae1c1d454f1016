"""Key generation on the GPU, byte for byte against the CPU oracle.

Batched path (Algorithm 1 with a product tree for batchInv, Sec. 2.2) and
per-key path (Sec. 3.1 KeyGen) must both reproduce the oracle's keys exactly:
inverses in the field R/q are unique, so batching cannot change any byte.
"""
import numpy as np
import pytest

import oracle
from gpu_util import first_mismatch, gpu_keygen, require_gpu

pytestmark = pytest.mark.gpu

SEED = 0x0123456789ABCDEF


@pytest.fixture(scope="module")
def snt():
    require_gpu()
    import paper_2106_08759_gb300 as m
    m.load()
    return m


@pytest.fixture(scope="module")
def ctx(snt):
    c = snt.Context(0, 256 << 20)
    yield c
    c.close()


@pytest.mark.parametrize("path", ["batched", "perkey_jump", "perkey_step"])
def test_b32_every_key_matches_oracle(snt, ctx, path):
    # 32 keys of sntrup761 from a fixed 64-bit seed, key indices 0..31; the
    # per-key path with either R/q inversion kernel
    ctx.set_option(snt.SNT_OPT_PERKEY_INV, 0 if path == "perkey_step" else 1)
    try:
        pk, sk = gpu_keygen(snt, ctx, 761, SEED, 0, 32, perkey=path != "batched")
    finally:
        ctx.set_option(snt.SNT_OPT_PERKEY_INV, 1)
    rpk, rsk = oracle.keygen_batch(761, SEED, 0, 32)
    assert first_mismatch(pk, rpk) is None
    assert first_mismatch(sk, rsk) is None


@pytest.mark.parametrize("P", [653, 857])
def test_other_parameter_sets(snt, ctx, P):
    pk, sk = gpu_keygen(snt, ctx, P, 77, 1000, 9)
    rpk, rsk = oracle.keygen_batch(P, 77, 1000, 9)
    assert first_mismatch(pk, rpk) is None
    assert first_mismatch(sk, rsk) is None


@pytest.mark.parametrize("B", [1, 2, 3, 5, 31, 33])
def test_ragged_tree_shapes(snt, ctx, B):
    # non-power-of-two B: unpaired nodes move up unchanged
    pk, sk = gpu_keygen(snt, ctx, 761, 5, 40, B)
    rpk, rsk = oracle.keygen_batch(761, 5, 40, B)
    assert first_mismatch(pk, rpk) is None
    assert first_mismatch(sk, rsk) is None


@pytest.mark.parametrize("opts", [(4, 8, 1), (8, 1, 0), (32, 2, 2), (4, 4, 0), (8, 8, 2),
                                  (8, 8, 3), (4, 2, 3)])
def test_tuning_options_do_not_change_keys(snt, ctx, opts):
    # R/3 lanes per element, tree split, R/3 overlap: layouts only
    lanes, split, overlap = opts
    ref = gpu_keygen(snt, ctx, 761, 21, 300, 45)
    ctx.set_option(snt.SNT_OPT_R3_LANES, lanes)
    ctx.set_option(snt.SNT_OPT_TREE_SPLIT, split)
    ctx.set_option(snt.SNT_OPT_R3_OVERLAP, overlap)
    try:
        got = gpu_keygen(snt, ctx, 761, 21, 300, 45)
        got857 = gpu_keygen(snt, ctx, 857, 22, 0, 19)
    finally:
        ctx.set_option(snt.SNT_OPT_R3_LANES, 4)
        ctx.set_option(snt.SNT_OPT_TREE_SPLIT, 8)
        ctx.set_option(snt.SNT_OPT_R3_OVERLAP, 1)
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    rpk, rsk = oracle.keygen_batch(857, 22, 0, 19)
    assert first_mismatch(got857[0], rpk) is None and first_mismatch(got857[1], rsk) is None


@pytest.mark.parametrize("B", [2, 3, 9, 17, 33, 65, 130, 257])
def test_output_split_narrow_levels_give_the_same_keys(snt, ctx, B):
    # CUDA-core engine: narrow tree levels split by output segments over
    # several CTAs (up and down, with the ping-pong inverse buffers) against
    # one CTA per product; B spans every segment plan and unpaired nodes
    ctx.set_option(snt.SNT_OPT_RQ_ENGINE, 0)
    ctx.set_option(snt.SNT_OPT_NARROW_SEG, 0)
    try:
        ref = gpu_keygen(snt, ctx, 761, 77, 1000, B)
        ctx.set_option(snt.SNT_OPT_NARROW_SEG, 1)
        got = gpu_keygen(snt, ctx, 761, 77, 1000, B)
    finally:
        ctx.set_option(snt.SNT_OPT_NARROW_SEG, 1)
        ctx.set_option(snt.SNT_OPT_RQ_ENGINE, 1)
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])


@pytest.mark.parametrize("lanes,kpt", [(4, 2), (8, 2), (32, 2)])
def test_r3_two_elements_per_lane_group_give_the_same_keys(snt, ctx, lanes, kpt):
    # R/3 kernel with two interleaved elements per lane group (ragged B, an
    # injected zero divisor that forces a second attempt for one element of
    # a pair while the other is done)
    bad = _non_invertible_g()
    ref = gpu_keygen(snt, ctx, 761, 12, 100, 45)
    ctx.set_option(snt.SNT_OPT_R3_LANES, lanes)
    ctx.set_option(snt.SNT_OPT_R3_KPT, kpt)
    try:
        got = gpu_keygen(snt, ctx, 761, 12, 100, 45)
        snt.snt_debug_inject_g(ctx, 761, [107], np.stack([bad]))
        inj = gpu_keygen(snt, ctx, 761, 12, 100, 45)
    finally:
        snt.snt_debug_inject_g(ctx, 761, [], np.zeros((0, 761), np.int8))
        ctx.set_option(snt.SNT_OPT_R3_LANES, 4)
        ctx.set_option(snt.SNT_OPT_R3_KPT, 1)
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    rpk, rsk = oracle.keygen_batch(761, 12, 100, 45, g_inject={7: bad})
    assert first_mismatch(inj[0], rpk) is None and first_mismatch(inj[1], rsk) is None


@pytest.mark.parametrize("engine", [2, 3])
@pytest.mark.parametrize("P,B", [(761, 300), (653, 77), (857, 130), (761, 2), (761, 5)])
def test_transform_engine_gives_the_same_keys(snt, ctx, P, B, engine):
    # general x general tree levels by the transform multiplier (engine 2) or
    # by warp MMAs with one wide limb on the vector side (engine 3, narrow
    # levels K-split too) against the CUDA-core Toeplitz engine; B = 2 and 5
    # have few or no general levels (the leaf levels stay small-operand forms)
    ctx.set_option(snt.SNT_OPT_RQ_ENGINE, 0)
    try:
        ref = gpu_keygen(snt, ctx, P, 5, 40, B)
        ctx.set_option(snt.SNT_OPT_RQ_ENGINE, engine)
        got = gpu_keygen(snt, ctx, P, 5, 40, B)
    finally:
        ctx.set_option(snt.SNT_OPT_RQ_ENGINE, 1)
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    if B <= 5:
        rpk, rsk = oracle.keygen_batch(P, 5, 40, B)
        assert first_mismatch(got[0], rpk) is None and first_mismatch(got[1], rsk) is None


@pytest.mark.parametrize("tiles", [1, 2, 3])
@pytest.mark.parametrize("P,B", [(761, 300), (653, 77), (857, 130)])
@pytest.mark.parametrize("wide", [False, True])
def test_tensor_core_engine_gives_the_same_keys(snt, ctx, P, B, tiles, wide):
    # tree products as warp MMAs on exact f16 limbs, 1, 2 or 3 tiles of 128
    # outputs per warp (ragged last warp for 653 and 857); wide: one f16 limb
    # on the vector side of the general levels (engine 3)
    ctx.set_option(snt.SNT_OPT_RQ_ENGINE, 0)
    try:
        ref = gpu_keygen(snt, ctx, P, 5, 40, B)
    finally:
        ctx.set_option(snt.SNT_OPT_RQ_ENGINE, 1)
    ctx.set_option(snt.SNT_OPT_MMA_TILES, tiles)
    ctx.set_option(snt.SNT_OPT_RQ_ENGINE, 3 if wide else 1)
    try:
        got = gpu_keygen(snt, ctx, P, 5, 40, B)
    finally:
        ctx.set_option(snt.SNT_OPT_MMA_TILES, 1)
        ctx.set_option(snt.SNT_OPT_RQ_ENGINE, 1)
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])


@pytest.mark.parametrize("engine", [1, 0, 2, 3])
@pytest.mark.parametrize("roots,B", [(2, 96), (32, 96), (1024, 96), (4, 300), (8, 7), (64, 4096)])
def test_forest_of_subtrees_gives_the_same_keys(snt, ctx, engine, roots, B):
    # Montgomery's trick over K equal subtrees with K root inversions in one
    # launch (K = the largest power of two <= roots dividing B: 300 -> 4,
    # 7 -> 1); inverses are unique, so the bytes equal the single tree's
    ctx.set_option(snt.SNT_OPT_RQ_ENGINE, engine)
    try:
        ref = gpu_keygen(snt, ctx, 761, 8, 500, B)
        ctx.set_option(snt.SNT_OPT_ROOTS, roots)
        got = gpu_keygen(snt, ctx, 761, 8, 500, B)
    finally:
        ctx.set_option(snt.SNT_OPT_ROOTS, 1)
        ctx.set_option(snt.SNT_OPT_RQ_ENGINE, 1)
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    if B <= 96:
        rpk, rsk = oracle.keygen_batch(761, 8, 500, B)
        assert first_mismatch(got[0], rpk) is None and first_mismatch(got[1], rsk) is None


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("roots", [1, 16])
@pytest.mark.parametrize("P,B", [(761, 64), (653, 45), (857, 33), (761, 2)])
def test_r3_batch_inversion_matches_oracle(snt, ctx, P, B, roots, mode):
    # mode 1: isInvertible by remainders modulo the F_3 factors, then
    # Montgomery's trick in R/3 (tensor-core forest, jump-divstep roots mod 3);
    # mode 2: the forest on the first draws, invertibility from the roots
    ctx.set_option(snt.SNT_OPT_R3_MODE, mode)
    ctx.set_option(snt.SNT_OPT_ROOTS, roots)
    try:
        pk, sk = gpu_keygen(snt, ctx, P, 21, 9, B)
    finally:
        ctx.set_option(snt.SNT_OPT_R3_MODE, 0)
        ctx.set_option(snt.SNT_OPT_ROOTS, 1)
    rpk, rsk = oracle.keygen_batch(P, 21, 9, B)
    assert first_mismatch(pk, rpk) is None and first_mismatch(sk, rsk) is None


def _zero_divisors(p, rng):
    """g = f_i * r for every irreducible factor f_i of x^p - x - 1 over F_3."""
    out = []
    for d, _, poly in oracle.ddf(p, 3):
        f = np.asarray(poly[: d + 1]) % 3
        r = rng.integers(0, 3, p - d)
        g = np.convolve(f, r)[:p] % 3
        out.append(np.where(g == 2, -1, g).astype(np.int8))
    return out


@pytest.mark.parametrize("mode,roots", [(1, 1), (2, 1), (2, 8)])
@pytest.mark.parametrize("P", [653, 761, 857])
def test_r3_batch_redraws_every_kind_of_zero_divisor(snt, ctx, P, mode, roots):
    # one injected non-invertible first draw per factor of x^p - x - 1: the
    # remainder test (mode 1) or the failing subtree root (mode 2, then the
    # per-key fall-back and the fix-up of h, pk and its hash) must reject each,
    # and the redraw must match the oracle
    p = oracle.PARAMS[P][0]
    bads = _zero_divisors(p, np.random.default_rng(P))
    B = 40
    offs = [3 + 5 * i for i in range(len(bads))]
    snt.snt_debug_inject_g(ctx, P, [200 + o for o in offs], np.stack(bads))
    ctx.set_option(snt.SNT_OPT_R3_MODE, mode)
    ctx.set_option(snt.SNT_OPT_ROOTS, roots)
    try:
        pk, sk = gpu_keygen(snt, ctx, P, 4, 200, B)
    finally:
        ctx.set_option(snt.SNT_OPT_R3_MODE, 0)
        ctx.set_option(snt.SNT_OPT_ROOTS, 1)
        snt.snt_debug_inject_g(ctx, P, [], np.zeros((0, p), np.int8))
    rpk, rsk = oracle.keygen_batch(P, 4, 200, B, g_inject=dict(zip(offs, bads)))
    assert first_mismatch(pk, rpk) is None and first_mismatch(sk, rsk) is None
    for o, g in zip(offs, bads):  # each was really redrawn
        assert oracle.keygen(P, 4, 200 + o, g_attempt0=g)[2] >= 2


@pytest.mark.parametrize("mode", [1, 2])
def test_r3_batch_equals_per_key_at_b4096(snt, ctx, mode):
    ref = gpu_keygen(snt, ctx, 761, 33, 0, 4096)
    ctx.set_option(snt.SNT_OPT_R3_MODE, mode)
    ctx.set_option(snt.SNT_OPT_ROOTS, 64)
    try:
        got = gpu_keygen(snt, ctx, 761, 33, 0, 4096)
    finally:
        ctx.set_option(snt.SNT_OPT_R3_MODE, 0)
        ctx.set_option(snt.SNT_OPT_ROOTS, 1)
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])


@pytest.mark.parametrize("ksplit", [1, 2, 4])
@pytest.mark.parametrize("P,B", [(761, 600), (653, 5), (857, 200)])
def test_tensor_core_ksplit_gives_the_same_keys(snt, ctx, P, B, ksplit):
    # narrow levels with each tile's sum split over 1, 2 or 4 warps; B = 5
    # and 200 make the leaf levels narrow too (the small-operand forms)
    ctx.set_option(snt.SNT_OPT_RQ_ENGINE, 0)
    try:
        ref = gpu_keygen(snt, ctx, P, 6, 77, B)
    finally:
        ctx.set_option(snt.SNT_OPT_RQ_ENGINE, 1)
    ctx.set_option(snt.SNT_OPT_MMA_KSPLIT, ksplit)
    try:
        got = gpu_keygen(snt, ctx, P, 6, 77, B)
    finally:
        ctx.set_option(snt.SNT_OPT_MMA_KSPLIT, 4)
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])


@pytest.mark.parametrize("P,B", [(653, 9), (857, 33)])
def test_output_split_narrow_levels_vs_oracle(snt, ctx, P, B):
    assert ctx.get_option(snt.SNT_OPT_NARROW_SEG) == 1
    ctx.set_option(snt.SNT_OPT_RQ_ENGINE, 0)
    try:
        pk, sk = gpu_keygen(snt, ctx, P, 78, 3, B)
    finally:
        ctx.set_option(snt.SNT_OPT_RQ_ENGINE, 1)
    rpk, rsk = oracle.keygen_batch(P, 78, 3, B)
    assert first_mismatch(pk, rpk) is None and first_mismatch(sk, rsk) is None


def test_autotuned_layouts_give_the_same_keys(snt):
    with snt.Context(0, 64 << 20) as c:
        choice = c.autotune(761, 48)
        assert choice["r3_lanes"] in (4, 8, 32) and choice["r3_overlap"] in (0, 1, 2, 3)
        pk, sk = gpu_keygen(snt, c, 761, 31, 7, 48)
    rpk, rsk = oracle.keygen_batch(761, 31, 7, 48)
    assert first_mismatch(pk, rpk) is None and first_mismatch(sk, rsk) is None


def test_split_batches_give_identical_bytes(snt, ctx):
    pk, sk = gpu_keygen(snt, ctx, 761, 9, 100, 37)
    pk1, sk1 = gpu_keygen(snt, ctx, 761, 9, 100, 20)
    pk2, sk2 = gpu_keygen(snt, ctx, 761, 9, 120, 17)
    assert np.array_equal(pk, np.concatenate([pk1, pk2]))
    assert np.array_equal(sk, np.concatenate([sk1, sk2]))


def _non_invertible_g(p=761):
    parts = oracle.ddf(p, 3)
    f1 = [poly for d, _, poly in parts if d == 19][0][:20]
    r = np.random.default_rng(12).integers(0, 3, p - 19)
    bad = np.convolve(f1, r) % 3
    return np.where(bad == 2, -1, bad).astype(np.int8)


def test_resampling_of_non_invertible_g(snt, ctx):
    bad = _non_invertible_g()
    snt.snt_debug_inject_g(ctx, 761, [7, 9], np.stack([bad, bad]))
    try:
        pk, sk = gpu_keygen(snt, ctx, 761, 3, 5, 8)  # key indices 5..12
    finally:
        snt.snt_debug_inject_g(ctx, 761, [], np.zeros((0, 761), np.int8))
    rpk, rsk = oracle.keygen_batch(761, 3, 5, 8, g_inject={2: bad, 4: bad})
    assert first_mismatch(pk, rpk) is None
    assert first_mismatch(sk, rsk) is None
    # the injected keys really took the second attempt
    assert oracle.keygen(761, 3, 7, g_attempt0=bad)[2] == 2


def test_b4096_sampled_keys_and_batched_equals_perkey(snt, ctx):
    B, seed = 4096, 1
    pk, sk = gpu_keygen(snt, ctx, 761, seed, 0, B)
    pk2, sk2 = gpu_keygen(snt, ctx, 761, seed, 0, B, perkey=True)
    assert np.array_equal(pk, pk2) and np.array_equal(sk, sk2)
    rng = np.random.default_rng(2)
    idx = sorted(set([0, 1, 2047, 2048, 4094, 4095] + list(rng.integers(0, B, 26))))
    for i in idx:
        rpk, rsk, _ = oracle.keygen(761, seed, i)
        assert np.array_equal(pk[i], rpk), i
        assert np.array_equal(sk[i], rsk), i


def test_invalid_arguments(snt, ctx):
    torch = require_gpu()
    pk = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(snt.SntError) as e:
        snt.snt_batch_keygen(ctx, 761, 0, 0, 0, pk, pk)
    assert e.value.status == -1
    with pytest.raises(snt.SntError) as e:
        snt.snt_batch_keygen(ctx, 760, 0, 0, 1, pk, pk)
    assert e.value.status == -1
    small = snt.Context(0, 1 << 20)
    big = torch.empty(4096 * 1763, dtype=torch.uint8, device="cuda")
    with pytest.raises(snt.SntError) as e:
        snt.snt_batch_keygen(small, 761, 0, 0, 4096, big, big)
    assert e.value.status == -2
    with pytest.raises(ValueError):  # the binding checks the output room
        snt.snt_batch_keygen(ctx, 761, 0, 0, 2, pk, pk)
    assert small.max_batch(761) >= 1
    small.close()


def test_host_buffer_entry_point(snt, ctx):
    pk, sk = snt.snt_batch_keygen_host(ctx, 761, SEED, 3, 6)
    rpk, rsk = oracle.keygen_batch(761, SEED, 3, 6)
    assert np.array_equal(pk, rpk) and np.array_equal(sk, rsk)


@pytest.mark.parametrize("P,roots,B", [(761, 1, 1), (761, 1, 2), (761, 1, 3), (653, 1, 7),
                                       (761, 32, 96), (761, 4, 300), (653, 8, 40),
                                       (761, 64, 4096), (857, 1, 9)])
def test_fused_leaf_level_gives_the_same_keys(snt, ctx, P, roots, B):
    # h = 3 inv(P) (g_L f_R) from the level-1 inverses (the leaf level of the
    # down-sweep skipped) against the leaf level plus h = g (3f)^-1: the same
    # bytes; B = 2 has the root as its level-1 node, B = 3 and the 32-root
    # forest of 3-key subtrees have unpaired leaves, 857 keeps the leaf level
    ctx.set_option(snt.SNT_OPT_ROOTS, roots)
    try:
        ctx.set_option(snt.SNT_OPT_FUSE_LEAF, 0)
        ref = gpu_keygen(snt, ctx, P, 12, 70, B)
        ctx.set_option(snt.SNT_OPT_FUSE_LEAF, 1)
        got = gpu_keygen(snt, ctx, P, 12, 70, B)
    finally:
        ctx.set_option(snt.SNT_OPT_FUSE_LEAF, 1)
        ctx.set_option(snt.SNT_OPT_ROOTS, 1)
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    if B <= 96:
        rpk, rsk = oracle.keygen_batch(P, 12, 70, B)
        assert first_mismatch(got[0], rpk) is None and first_mismatch(got[1], rsk) is None


@pytest.fixture(scope="module")
def pool():
    from oracle_pool import OraclePool
    p = OraclePool()
    yield p
    p.close()


def test_benchmarked_layout_b4096_vs_perkey_and_oracle(snt, pool):
    """The configuration the benchmark times: a 256 MiB context autotuned for
    (761, 4096), seed 1, B = 4096.  All keys equal the per-key path's (both
    R/q inversion kernels), and at least 256 keys equal the oracle's: the
    first and last key, both ends of every subtree of the tuned forest and
    random ones."""
    B, seed = 4096, 1
    with snt.Context(0, 256 << 20) as c:
        tuned = c.autotune(761, B)
        pk, sk = gpu_keygen(snt, c, 761, seed, 0, B)
        pk2, sk2 = gpu_keygen(snt, c, 761, seed, 0, B, perkey=True)
        c.set_option(snt.SNT_OPT_PERKEY_INV, 0)
        pk3, sk3 = gpu_keygen(snt, c, 761, seed, 0, B, perkey=True)
    assert first_mismatch(pk, pk2) is None and first_mismatch(sk, sk2) is None
    assert first_mismatch(pk, pk3) is None and first_mismatch(sk, sk3) is None
    # forest rule of the library: for B = 4096 every power of two up to 256
    # divides B and fits the node rows, so K = the tuned root count
    K = tuned["roots"]
    assert K in (1, 4, 8, 16, 32, 64, 128, 256)
    sub = B // K
    ends = [x for j in range(K) for x in (j * sub, j * sub + sub - 1)]
    rng = np.random.default_rng(3)
    idx = set(ends) | {0, B - 1}
    while len(idx) < 256 + len(ends) // 2:
        idx.add(int(rng.integers(0, B)))
    idx = np.array(sorted(idx))
    assert idx.size >= 256
    assert pool.bad_keys(761, seed, idx, pk[idx], sk[idx]) == []


@pytest.mark.parametrize("parts,roots,B,engine,r3mode,fuse", [
    (2, 64, 4096, 1, 2, 1), (4, 64, 4096, 1, 2, 1), (4, 128, 4096, 1, 0, 1),
    (2, 16, 96, 1, 0, 1), (4, 32, 96, 1, 1, 1), (4, 8, 96, 1, 2, 0), (2, 8, 96, 2, 0, 1),
    (2, 2, 6, 1, 0, 1), (4, 2, 96, 1, 0, 1)])
def test_pipelined_parts_give_the_same_keys(snt, ctx, parts, roots, B, engine, r3mode, fuse):
    # the forest's subtrees split into groups of consecutive keys on their own
    # streams (96 keys in 32 subtrees: 3-key subtrees with unpaired leaves);
    # (4, 2, 96): the forest has 2 subtrees, not a multiple of 4, so the call
    # runs in one part
    ctx.set_option(snt.SNT_OPT_ROOTS, roots)
    ctx.set_option(snt.SNT_OPT_RQ_ENGINE, engine)
    ctx.set_option(snt.SNT_OPT_R3_MODE, r3mode)
    ctx.set_option(snt.SNT_OPT_FUSE_LEAF, fuse)
    try:
        ref = gpu_keygen(snt, ctx, 761, 14, 90, B)
        ctx.set_option(snt.SNT_OPT_PARTS, parts)
        got = gpu_keygen(snt, ctx, 761, 14, 90, B)
    finally:
        ctx.set_option(snt.SNT_OPT_PARTS, 1)
        ctx.set_option(snt.SNT_OPT_ROOTS, 1)
        ctx.set_option(snt.SNT_OPT_RQ_ENGINE, 1)
        ctx.set_option(snt.SNT_OPT_R3_MODE, 0)
        ctx.set_option(snt.SNT_OPT_FUSE_LEAF, 1)
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    if B <= 96:
        rpk, rsk = oracle.keygen_batch(761, 14, 90, B)
        assert first_mismatch(got[0], rpk) is None and first_mismatch(got[1], rsk) is None


def test_pipelined_parts_redraw_injected_zero_divisors(snt, ctx):
    # keys of both parts whose first g is a zero divisor: the per-key R/3
    # fall-back and the fix-up run after the parts join
    bads = _zero_divisors(761, np.random.default_rng(9))
    offs = [5, 60]
    snt.snt_debug_inject_g(ctx, 761, [300 + o for o in offs], np.stack(bads[:2]))
    ctx.set_option(snt.SNT_OPT_ROOTS, 8)
    ctx.set_option(snt.SNT_OPT_PARTS, 2)
    ctx.set_option(snt.SNT_OPT_R3_MODE, 2)
    try:
        pk, sk = gpu_keygen(snt, ctx, 761, 4, 300, 96)
    finally:
        ctx.set_option(snt.SNT_OPT_PARTS, 1)
        ctx.set_option(snt.SNT_OPT_ROOTS, 1)
        ctx.set_option(snt.SNT_OPT_R3_MODE, 0)
        snt.snt_debug_inject_g(ctx, 761, [], np.zeros((0, 761), np.int8))
    rpk, rsk = oracle.keygen_batch(761, 4, 300, 96, g_inject=dict(zip(offs, bads[:2])))
    assert first_mismatch(pk, rpk) is None and first_mismatch(sk, rsk) is None


def test_sntrup653_first_draw_batch_with_many_redraws(snt, ctx, pool):
    # x^653 - x - 1 has a factor of degree 3 over F_3, so about one first draw
    # of g in 27 is a zero divisor: the screen against the factors of degree 3
    # and 16 redraws those before the R/3 forest (without it most 32-key
    # subtrees would fail) and dozens of keys go to the fix-up; all keys equal
    # the per-key path's, and the redrawn ones (and others) the oracle's
    B, seed = 2048, 17
    ctx.set_option(snt.SNT_OPT_R3_MODE, 2)
    ctx.set_option(snt.SNT_OPT_ROOTS, 64)
    try:
        pk, sk = gpu_keygen(snt, ctx, 653, seed, 0, B)
    finally:
        ctx.set_option(snt.SNT_OPT_R3_MODE, 0)
        ctx.set_option(snt.SNT_OPT_ROOTS, 1)
    pk2, sk2 = gpu_keygen(snt, ctx, 653, seed, 0, B, perkey=True)
    assert first_mismatch(pk, pk2) is None and first_mismatch(sk, sk2) is None
    # keys among the first 600 whose first draw is not invertible (about 22)
    redrawn = [k for k in range(600)
               if not oracle.ring_inv(653, 3, oracle.sample_small(653, seed, k, 0))[0]]
    assert len(redrawn) > 10  # the fix-up had real work
    idx = np.array(sorted(set(redrawn) | {0, 1, B - 1}))
    assert pool.bad_keys(653, seed, idx, pk[idx], sk[idx]) == []


@pytest.mark.parametrize("B,roots,r3mode,engine", [
    (4096, 64, 2, 3), (4096, 64, 1, 1), (96, 8, 0, 1), (33, 1, 1, 0), (5, 1, 2, 2), (1, 1, 0, 3)])
def test_programmatic_dependent_launch_gives_the_same_keys(snt, ctx, B, roots, r3mode, engine):
    # the chain kernels launched with programmatic stream serialization (the
    # default) and plainly: same bytes, and the oracle's on a few keys
    assert ctx.get_option(snt.SNT_OPT_PDL) == 1
    ctx.set_option(snt.SNT_OPT_ROOTS, roots)
    ctx.set_option(snt.SNT_OPT_R3_MODE, r3mode)
    ctx.set_option(snt.SNT_OPT_RQ_ENGINE, engine)
    try:
        on = gpu_keygen(snt, ctx, 761, 21, 7, B)
        ctx.set_option(snt.SNT_OPT_PDL, 0)
        off = gpu_keygen(snt, ctx, 761, 21, 7, B)
    finally:
        ctx.set_option(snt.SNT_OPT_PDL, 1)
        ctx.set_option(snt.SNT_OPT_ROOTS, 1)
        ctx.set_option(snt.SNT_OPT_R3_MODE, 0)
        ctx.set_option(snt.SNT_OPT_RQ_ENGINE, 1)
    assert np.array_equal(on[0], off[0]) and np.array_equal(on[1], off[1])
    for j in sorted({0, B // 2, B - 1}):
        opk, osk, _ = oracle.keygen(761, 21, 7 + j)
        assert np.array_equal(on[0][j], opk) and np.array_equal(on[1][j], osk), j


@pytest.mark.parametrize("shift", [1, 6, 13])
def test_unaligned_output_buffers(snt, ctx, shift):
    # pk / sk at an odd or unaligned device address: the hash kernel copies
    # the public keys with 16-byte words in phase with the source address
    import torch
    B = 70
    pkb, skb, _, _ = snt.snt_param_sizes(761)
    ref = gpu_keygen(snt, ctx, 761, 8, 123, B)
    pk = torch.zeros(B * pkb + 64, dtype=torch.uint8, device="cuda")
    sk = torch.zeros(B * skb + 64, dtype=torch.uint8, device="cuda")
    snt.snt_batch_keygen(ctx, 761, 8, 123, B, pk[shift:shift + B * pkb], sk[shift:shift + B * skb])
    ctx.sync()
    got_pk = pk.cpu().numpy()[shift:shift + B * pkb].reshape(B, pkb)
    got_sk = sk.cpu().numpy()[shift:shift + B * skb].reshape(B, skb)
    assert np.array_equal(got_pk, ref[0]) and np.array_equal(got_sk, ref[1])


@pytest.mark.parametrize("r3mode,roots,B", [(2, 16, 4096), (1, 16, 300), (0, 4, 300), (2, 1, 33)])
def test_r3_from_the_end_of_the_up_sweep(snt, ctx, r3mode, roots, B):
    # R/3 overlap 3: the R/3 work forked when the R/q up-sweep ends
    ctx.set_option(snt.SNT_OPT_ROOTS, roots)
    ctx.set_option(snt.SNT_OPT_R3_MODE, r3mode)
    try:
        ref = gpu_keygen(snt, ctx, 761, 33, 1000, B)
        ctx.set_option(snt.SNT_OPT_R3_OVERLAP, 3)
        got = gpu_keygen(snt, ctx, 761, 33, 1000, B)
    finally:
        ctx.set_option(snt.SNT_OPT_R3_OVERLAP, 1)
        ctx.set_option(snt.SNT_OPT_ROOTS, 1)
        ctx.set_option(snt.SNT_OPT_R3_MODE, 0)
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    for j in sorted({0, B // 3, B - 1}):
        opk, osk, _ = oracle.keygen(761, 33, 1000 + j)
        assert np.array_equal(got[0][j], opk) and np.array_equal(got[1][j], osk), j


@pytest.mark.parametrize("P,roots,r3roots,mode,B", [
    (761, 64, 4, 2, 4096), (761, 32, 4, 2, 4096), (761, 128, 16, 1, 1024), (653, 64, 1, 2, 300),
    (857, 4, 16, 2, 96)])
def test_r3_forest_with_its_own_root_count(snt, ctx, P, roots, r3roots, mode, B):
    # the R/3 forest with another number of subtrees than the R/q forest, with
    # one injected zero divisor per factor (the screen, the failing R/3
    # subtree and its per-key fall-back): same bytes as the per-key R/3 path
    p = oracle.PARAMS[P][0]
    bads = _zero_divisors(p, np.random.default_rng(P + r3roots))
    offs = [1 + 7 * i for i in range(len(bads))]
    snt.snt_debug_inject_g(ctx, P, [50 + o for o in offs], np.stack(bads))
    try:
        ref = gpu_keygen(snt, ctx, P, 6, 50, B)
        ctx.set_option(snt.SNT_OPT_ROOTS, roots)
        ctx.set_option(snt.SNT_OPT_R3_ROOTS, r3roots)
        ctx.set_option(snt.SNT_OPT_R3_MODE, mode)
        got = gpu_keygen(snt, ctx, P, 6, 50, B)
    finally:
        ctx.set_option(snt.SNT_OPT_R3_ROOTS, 0)
        ctx.set_option(snt.SNT_OPT_ROOTS, 1)
        ctx.set_option(snt.SNT_OPT_R3_MODE, 0)
        snt.snt_debug_inject_g(ctx, P, [], np.zeros((0, p), np.int8))
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    rpk, rsk = oracle.keygen_batch(P, 6, 50, min(B, 64), g_inject=dict(zip(offs, bads)))
    assert first_mismatch(got[0][:64], rpk) is None and first_mismatch(got[1][:64], rsk) is None


def test_option_values_are_checked(snt, ctx):
    # every option rejects values outside its documented range and keeps the
    # old value
    bad = [(snt.SNT_OPT_PDL, 2), (snt.SNT_OPT_PDL, -1), (snt.SNT_OPT_R3_ROOTS, 3),
           (snt.SNT_OPT_R3_ROOTS, 2048), (snt.SNT_OPT_R3_OVERLAP, 4), (snt.SNT_OPT_ROOTS, 6),
           (snt.SNT_OPT_PARTS, 3), (snt.SNT_OPT_R3_MODE, 3)]
    for opt, val in bad:
        before = ctx.get_option(opt)
        with pytest.raises(snt.SntError) as e:
            ctx.set_option(opt, val)
        assert e.value.status == -1, (opt, val)
        assert ctx.get_option(opt) == before
    for opt, val in [(snt.SNT_OPT_PDL, 0), (snt.SNT_OPT_R3_ROOTS, 4), (snt.SNT_OPT_R3_OVERLAP, 3)]:
        before = ctx.get_option(opt)
        ctx.set_option(opt, val)
        assert ctx.get_option(opt) == val
        ctx.set_option(opt, before)


def test_host_async_calls_overlap_and_match(snt):
    # several calls that do not wait, into pinned host buffers, alternating
    # staging slots, then a change of batch size (every pending copy first)
    # and a device-buffer call in between; every batch equals the device
    # call's keys once the context is synced
    import torch
    calls = [(761, 300, 11, 0), (761, 300, 12, 300), (761, 300, 13, 600), (653, 64, 14, 0),
             (761, 300, 15, 900)]
    with snt.Context(0, 256 << 20) as c:
        outs = []
        for P, B, seed, first in calls:
            pkb, skb, _, _ = snt.snt_param_sizes(P)
            hpk = torch.zeros(B * pkb, dtype=torch.uint8).pin_memory().numpy().reshape(B, pkb)
            hsk = torch.zeros(B * skb, dtype=torch.uint8).pin_memory().numpy().reshape(B, skb)
            snt.snt_batch_keygen_host_async(c, P, seed, first, B, hpk, hsk)
            outs.append((hpk, hsk))
            if seed == 12:  # a device call while copies may be pending
                ref_mid = gpu_keygen(snt, c, 857, 3, 0, 5)
        c.sync()
        for (P, B, seed, first), (hpk, hsk) in zip(calls, outs):
            rpk, rsk = gpu_keygen(snt, c, P, seed, first, B)
            assert np.array_equal(hpk, rpk) and np.array_equal(hsk, rsk), (P, B, seed)
        opk, osk = oracle.keygen_batch(857, 3, 0, 5)
        assert first_mismatch(ref_mid[0], opk) is None and first_mismatch(ref_mid[1], osk) is None
    opk, osk, _ = oracle.keygen(761, 15, 900 + 299)
    assert np.array_equal(outs[-1][0][-1], opk) and np.array_equal(outs[-1][1][-1], osk)
