"""The benchmark's algorithmic-work and launch accounting (host logic), checked
against a direct simulation of the product forest the library builds: K equal
subtrees of B/K leaves, each level pairing neighbours (an odd node moves up
unchanged), every pair one product up and two down; with the fused leaf level
the down-sweep stops above the leaves and each leaf pair costs four products
(g_L f_R, g_R f_L, inv(P) s for both keys; the first two on the side stream
when they are formed ahead), an unpaired leaf one."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _simulate(B, K, fused, s_side=False):
    n0 = B // K
    levels = []
    n = n0
    while n > 1:
        levels.append(n // 2)  # pairs at this level
        n = (n + 1) // 2
    up = K * sum(levels)
    down_levels = levels[1:] if (fused and levels) else levels
    down = K * 2 * sum(down_levels)
    side = 0
    if fused and levels:
        h = K * (4 * levels[0] + (n0 - 2 * levels[0]))
        if s_side:  # g_L f_R and g_R f_L of every leaf pair move out of the h kernel
            side = K * 2 * levels[0]
            h -= side
    else:
        h = B
    return up, down, h, len(levels), side


@pytest.mark.parametrize("B,roots", [(4096, 64), (4096, 1), (300, 4), (96, 32), (7, 8),
                                     (33, 1), (2, 1), (1, 1), (4096, 256)])
@pytest.mark.parametrize("fused,s_side", [(False, False), (True, False), (True, True)])
def test_product_counts_match_the_forest(B, roots, fused, s_side):
    K = bench.forest_roots(B, roots)
    mac = bench.P * bench.P
    ops = bench.ops_per_call(B, K, r3_mode=2, fused=fused, s_side=s_side)
    up, down, h, L, side = _simulate(B, K, fused, s_side)
    assert ops["tree_up"] == up * mac
    assert ops["tree_down"] == down * mac
    assert ops["h_encode"] == h * mac
    assert ops.get("leaf_s", 0) == side * mac
    assert ops["root_inv"] == K * (2 * bench.P - 1) * 2 * (bench.P + 1)
    if not fused:
        assert up == B - K and down == 2 * (B - K)


@pytest.mark.parametrize("B,roots", [(4096, 64), (4096, 1), (300, 4), (2, 1)])
def test_launch_counts(B, roots):
    K = bench.forest_roots(B, roots)
    _, _, _, L, _ = _simulate(B, K, False)
    for engine, fused in ((1, True), (0, False)):
        tuned = {"roots": roots, "r3_mode": 2, "rq_engine": engine}
        assert bench.fused_leaf(tuned) == fused
        down = L - 1 if (fused and L >= 1) else L
        side = 1 if (fused and L >= 1) else 0
        # sample, up levels, roots, down levels, h, hash, the leaf-pair
        # products on the side stream; R/3 first-draw forest: 2 launches per
        # level, roots, encoding, fall-back, fix-up
        assert bench.launches_per_call(B, tuned) == (1 + L + 1 + down + 1 + 1 + side) + (2 * L + 4)


def test_bench_line_at_the_headline_config():
    # 4096 keys in 64 subtrees with the fused leaf level: 4032 products up,
    # 3968 down, 4096 leaf-pair products s beside the roots, 4096 in the h
    # kernel (inv(P) s for both keys of a pair)
    ops = bench.ops_per_call(4096, 64, 2, fused=True, s_side=True)
    mac = bench.P * bench.P
    assert (ops["tree_up"] // mac, ops["tree_down"] // mac, ops["leaf_s"] // mac,
            ops["h_encode"] // mac) == (4032, 3968, 4096, 4096)
    assert bench.launches_per_call(4096, {"roots": 64, "r3_mode": 2, "rq_engine": 1}) == 32


def test_r3_forest_with_its_own_root_count():
    # R/q forest of 16 subtrees of 256 keys (8 levels), R/3 forest of 4
    # subtrees of 1024 (10 levels): 20 R/q launches (sample, 8 up, roots, 7
    # down, h, hash, leaf-pair products) and 24 R/3 ones (2 per level, roots,
    # encoding, fall-back, fix-up); the R/3 products are 3 (4096 - 4)
    tuned = {"roots": 16, "r3_roots": 4, "r3_mode": 2, "rq_engine": 3}
    assert bench.launches_per_call(4096, tuned) == 20 + 24
    ops = bench.ops_per_call(4096, 16, 2, fused=True, s_side=True, K3=4)
    assert ops["r3_inv"] == 3 * (4096 - 4) * bench.P * bench.P
    assert bench.launches_per_call(4096, dict(tuned, r3_roots=0)) == 20 + 2 * 8 + 4
