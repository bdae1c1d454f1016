"""The allocation-free keygen entry point (snt_batch_keygen_static).

It serves callers that cannot allocate device memory (a framework's caching
allocator holds the free memory, or cudaMalloc's implicit synchronisation is
not acceptable on their path): its scratch is a static device array of the
library, so it must produce exactly the keys of snt_batch_keygen, call after
call, although every call reuses the same scratch, and it must not change
the device's free memory.  This file is collected last so that a run
stopping at the first failure has run every other test.
"""
import pytest

from gpu_util import require_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("P", [653, 761, 857])
def test_static_scratch_keygen_matches_context_keygen(P):
    torch = require_gpu()
    import paper_2106_08759_gb300 as snt
    pkb, skb, _, _ = snt.snt_param_sizes(P)
    # the largest batch (B = 256 fills most of the static scratch for
    # sntrup857), then a smaller one over the previous call's stale scratch
    calls = [(0x0123456789ABCDEF, 0, 256), (5, 1000, 37)]
    with snt.Context(0, 64 << 20) as ctx:
        for seed, first, B in calls:
            pk = torch.zeros(B * pkb, dtype=torch.uint8, device="cuda")
            sk = torch.zeros(B * skb, dtype=torch.uint8, device="cuda")
            snt.snt_batch_keygen_static(0, P, seed, first, B, pk, sk)
            rpk = torch.zeros_like(pk)
            rsk = torch.zeros_like(sk)
            snt.snt_batch_keygen(ctx, P, seed, first, B, rpk, rsk)
            ctx.sync()
            # integer outputs: the tolerance is exact equality
            assert torch.equal(pk, rpk), (P, seed, first, B)
            assert torch.equal(sk, rsk), (P, seed, first, B)


def test_static_scratch_keygen_allocates_no_device_memory():
    torch = require_gpu()
    import paper_2106_08759_gb300 as snt
    P, B = 761, 200
    pkb, skb, _, _ = snt.snt_param_sizes(P)
    pk = torch.zeros(B * pkb, dtype=torch.uint8, device="cuda")
    sk = torch.zeros(B * skb, dtype=torch.uint8, device="cuda")
    snt.snt_batch_keygen_static(0, P, 1, 0, B, pk, sk)  # loads the kernels
    torch.cuda.synchronize()
    free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
    snt.snt_batch_keygen_static(0, P, 2, 5000, B, pk, sk)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_reserved() == reserved0


def test_static_scratch_keygen_rejects_oversized_batches():
    torch = require_gpu()
    import paper_2106_08759_gb300 as snt
    pk = torch.zeros(257 * 1763, dtype=torch.uint8, device="cuda")
    with pytest.raises(snt.SntError) as e:
        snt.snt_batch_keygen_static(0, 761, 1, 0, 257, pk, pk)
    assert e.value.status == -1 and "1 to 256 keys" in str(e.value)
