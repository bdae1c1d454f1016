"""Shared fixtures for the GPU parity tests (CUDA path vs the CPU oracle)."""
import numpy as np
import pytest


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def gpu_keygen(snt, ctx, P, seed, first, B, perkey=False):
    torch = require_gpu()
    pkb, skb, _, _ = snt.snt_param_sizes(P)
    pk = torch.full((B * pkb,), 0xAA, dtype=torch.uint8, device="cuda")
    sk = torch.full((B * skb,), 0xAA, dtype=torch.uint8, device="cuda")
    fn = snt.snt_keygen_perkey if perkey else snt.snt_batch_keygen
    fn(ctx, P, seed, first, B, pk, sk)
    ctx.sync()
    return pk.cpu().numpy().reshape(B, pkb), sk.cpu().numpy().reshape(B, skb)


def first_mismatch(got, ref):
    bad = np.nonzero((got != ref).any(axis=1))[0]
    return None if bad.size == 0 else int(bad[0])
