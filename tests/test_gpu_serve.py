"""Serving loop: continuous batching of encapsulation / decapsulation requests
over a device key pool.  dec(enc(pk)) = ss on every served item; every audited
item is byte-identical to the same item computed alone (snt_enc) and to the
oracle."""
import numpy as np
import pytest

import oracle
from gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def test_serving_loop_results_alone_and_in_the_mix():
    torch = require_gpu()
    import paper_2106_08759_gb300 as snt
    seed = 4242
    with snt.Context(0, 128 << 20) as ctx:
        stats, lat, audit = snt.snt_serve_run(ctx, P=761, rate=3000.0, duration_s=0.6,
                                              max_items=64, pool_keys=4096, refill_batch=1024,
                                              max_inflight=3, max_launch_items=1024, seed=seed,
                                              audit=48)
        assert stats["requests"] > 100
        assert stats["mismatches"] == 0          # dec(enc(pk)) = ss on every item
        assert stats["items_dec"] > 0 and stats["items_enc"] > 0
        assert np.all(lat >= 0) and stats["p99_ms"] >= stats["p50_ms"] > 0
        assert stats["keys_generated"] > 0        # the pool was refilled while serving
        n = len(audit["k"])
        assert n == 48
        # the same items alone, through the plain entry point
        pkb, _, ctb, _ = snt.snt_param_sizes(761)
        for i in range(n):
            dpk = torch.from_numpy(audit["pk"][i].copy()).cuda()
            ct = torch.empty(ctb, dtype=torch.uint8, device="cuda")
            ss = torch.empty(32, dtype=torch.uint8, device="cuda")
            snt.snt_enc(ctx, 761, 1, dpk, seed, int(audit["k"][i]), ct, ss)
            torch.cuda.synchronize()
            assert np.array_equal(ct.cpu().numpy(), audit["ct"][i]), i
            assert np.array_equal(ss.cpu().numpy(), audit["ss"][i]), i
    for i in (0, 17, 47):
        rct, rss = oracle.encap(761, audit["pk"][i], seed, int(audit["k"][i]))
        assert np.array_equal(rct, audit["ct"][i]) and np.array_equal(rss, audit["ss"][i])


@pytest.mark.parametrize("dec_fraction", [0.0, 0.5])
def test_serving_tiny_pool_splits_requests_and_drains(dec_fraction):
    """A pool of two 64-key chunks is smaller than the work in flight: requests
    are split across launches, chunks are refilled as soon as all their keys
    are used up, and every request still completes."""
    require_gpu()
    import paper_2106_08759_gb300 as snt
    with snt.Context(0, 64 << 20) as ctx:
        stats, lat, _ = snt.snt_serve_run(ctx, P=653, rate=4000.0, duration_s=0.25, max_items=64,
                                          dec_fraction=dec_fraction, pool_keys=128,
                                          refill_batch=64, max_inflight=2, max_launch_items=64,
                                          seed=9)
    assert stats["mismatches"] == 0
    assert len(lat) == stats["requests"] and np.all(lat >= 0)
    assert stats["keys_generated"] + 128 >= stats["items_enc"] > 128
    if dec_fraction == 0.0:
        assert stats["items_dec"] == 0
    else:
        assert 0 < stats["items_dec"] < stats["items_enc"]
