"""Encapsulation / decapsulation on the GPU vs the oracle (byte for byte),
dec(enc(pk)) = ss on every key, and implicit rejection of tampered
ciphertexts."""
import numpy as np
import pytest

import oracle
from gpu_util import gpu_keygen, require_gpu

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


def _enc(snt, ctx, P, pk, seed, first):
    import torch
    n = pk.shape[0]
    _, _, ctb, _ = snt.snt_param_sizes(P)
    dpk = torch.from_numpy(np.ascontiguousarray(pk).ravel()).cuda()
    ct = torch.full((n * ctb,), 0xAA, dtype=torch.uint8, device="cuda")
    ss = torch.full((n * 32,), 0xAA, dtype=torch.uint8, device="cuda")
    snt.snt_enc(ctx, P, n, dpk, seed, first, ct, ss)
    torch.cuda.synchronize()
    return ct.cpu().numpy().reshape(n, ctb), ss.cpu().numpy().reshape(n, 32)


def _dec(snt, ctx, P, sk, ct):
    import torch
    n = sk.shape[0]
    dsk = torch.from_numpy(np.ascontiguousarray(sk).ravel()).cuda()
    dct = torch.from_numpy(np.ascontiguousarray(ct).ravel()).cuda()
    ss = torch.full((n * 32,), 0xAA, dtype=torch.uint8, device="cuda")
    snt.snt_dec(ctx, P, n, dsk, dct, ss)
    torch.cuda.synchronize()
    return ss.cpu().numpy().reshape(n, 32)


@pytest.mark.parametrize("P", [653, 761, 857])
def test_enc_dec_match_oracle(snt, ctx, P):
    n = 9
    pk, sk = gpu_keygen(snt, ctx, P, 404, 0, n)
    ct, ss = _enc(snt, ctx, P, pk, 77, 1000)
    for i in range(n):
        rct, rss = oracle.encap(P, pk[i], 77, 1000 + i)
        assert np.array_equal(ct[i], rct) and np.array_equal(ss[i], rss), i
    ss2 = _dec(snt, ctx, P, sk, ct)
    assert np.array_equal(ss2, ss)  # dec(enc(pk)) = ss on every key
    # tampered ciphertexts: implicit rejection, equal to the oracle's value
    bad = ct.copy()
    bad[:, 5] ^= 0x10
    bad[3, -1] ^= 1
    ss3 = _dec(snt, ctx, P, sk, bad)
    for i in range(n):
        rss, ok = oracle.decap(P, sk[i], bad[i])
        assert not ok and np.array_equal(ss3[i], rss), i


def test_dec_of_enc_on_many_keys(snt, ctx):
    n = 2048
    pk, sk = gpu_keygen(snt, ctx, 761, 5, 0, n)
    ct, ss = _enc(snt, ctx, 761, pk, 6, 0)
    assert np.array_equal(_dec(snt, ctx, 761, sk, ct), ss)
    for i in (0, 777, 2047):
        rct, rss = oracle.encap(761, pk[i], 6, i)
        assert np.array_equal(ct[i], rct) and np.array_equal(ss[i], rss)
