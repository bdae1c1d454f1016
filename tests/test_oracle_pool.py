"""The parallel oracle checks used by the full-size GPU parity tests (no GPU):
they accept the oracle's own results and flag planted mistakes."""
import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module")
def pool():
    from oracle_pool import OraclePool
    p = OraclePool(2)
    yield p
    p.close()


def test_pool_checks_accept_oracle_results_and_flag_planted_mistakes(pool):
    p, q, _ = oracle.PARAMS[761]
    rng = np.random.default_rng(0)
    a = rng.integers(-2295, 2296, (6, p)).astype(np.int16)
    b = rng.integers(-2295, 2296, (6, p)).astype(np.int16)
    c = np.stack([oracle.ring_mul(p, q, a[i], b[i]) for i in range(6)]).astype(np.int16)
    assert pool.bad_products(p, q, a, b, c) == []
    c[4, 100] += 1  # planted mistake
    assert pool.bad_products(p, q, a, b, c) == [4]

    g = rng.integers(-1, 2, (5, p)).astype(np.int8)
    g[3] = 0  # not invertible
    inv = np.stack([oracle.ring_inv(p, 3, g[i])[1] for i in range(5)]).astype(np.int8)
    ok = np.array([oracle.ring_inv(p, 3, g[i])[0] for i in range(5)], np.int32)
    assert ok.tolist() == [1, 1, 1, 0, 1]
    assert pool.bad_identities(p, 3, g, inv, ok) == []
    assert pool.bad_inverses(p, 3, g, inv, ok) == []
    inv2 = inv.copy()
    inv2[1, 7] = -inv2[1, 7] if inv2[1, 7] else 1  # wrong inverse
    ok2 = ok.copy()
    ok2[3] = 1  # a zero divisor claimed invertible
    assert pool.bad_identities(p, 3, g, inv2, ok2) == [1, 3]
    assert pool.bad_inverses(p, 3, g, inv2, ok2) == [1, 3]


def test_pool_key_check_flags_a_wrong_key(pool):
    idx = np.array([0, 5, 9])
    keys = [oracle.keygen(761, 3, int(k)) for k in idx]
    pk = np.stack([k[0] for k in keys])
    sk = np.stack([k[1] for k in keys])
    assert pool.bad_keys(761, 3, idx, pk, sk) == []
    sk[2, -1] ^= 1
    assert pool.bad_keys(761, 3, idx, pk, sk) == [9]
