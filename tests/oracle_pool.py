"""A spawned process pool that checks many GPU results against the CPU oracle.

The oracle is per element and single-threaded; the full-size checks (every
inversion of the microbenchmark workload, hundreds of B = 4096 keys) split
their elements over all host cores.  The pool is started with the "spawn"
method, so it is safe in a process that already initialised CUDA.  Each
worker returns the indices of the elements that do NOT match, so a failing
test can name them.
"""
import multiprocessing as mp
import os

import numpy as np


def _chunks(n, parts):
    step = max(1, -(-n // parts))
    return [(i, min(n, i + step)) for i in range(0, n, step)]


def _bad_products(args):
    p, m, a, b, got = args
    import oracle
    return [i for i in range(len(a)) if not np.array_equal(oracle.ring_mul(p, m, a[i], b[i]), got[i])]


def _bad_inverses(args):
    """Rows whose claimed inverse or invertibility flag disagrees with the
    oracle's extended Euclid."""
    p, m, a, got, ok = args
    import oracle
    bad = []
    for i in range(len(a)):
        rok, ref = oracle.ring_inv(p, m, a[i])
        if bool(ok[i]) != rok or not np.array_equal(ref, got[i]):
            bad.append(i)
    return bad


def _bad_identities(args):
    """Rows with ok set whose a * v is not 1 in (Z/m)[x]/(x^p - x - 1) (the
    inverse is unique, so a * v = 1 pins v), and rows without ok that the
    oracle finds invertible or whose output is not zero."""
    p, m, a, got, ok = args
    import oracle
    one = np.zeros(p, np.int32)
    one[0] = 1
    bad = []
    for i in range(len(a)):
        if ok[i]:
            if not np.array_equal(oracle.ring_mul(p, m, a[i], got[i]), one):
                bad.append(i)
        elif oracle.ring_inv(p, m, a[i])[0] or np.any(got[i]):
            bad.append(i)
    return bad


def _bad_keys(args):
    p, seed, idx, pk, sk = args
    import oracle
    bad = []
    for j, k in enumerate(idx):
        rpk, rsk, _ = oracle.keygen(p, seed, int(k))
        if not (np.array_equal(rpk, pk[j]) and np.array_equal(rsk, sk[j])):
            bad.append(int(k))
    return bad


class OraclePool:
    def __init__(self, workers=None):
        self.n = workers or os.cpu_count() or 1
        self.pool = mp.get_context("spawn").Pool(self.n)

    def close(self):
        self.pool.close()
        self.pool.join()

    def _run(self, fn, n, make):
        parts = _chunks(n, 4 * self.n)
        out = self.pool.map(fn, [make(lo, hi) for lo, hi in parts])
        return [lo + i for (lo, _), bad in zip(parts, out) for i in bad]

    def bad_products(self, p, m, a, b, got):
        return self._run(_bad_products, len(a),
                         lambda lo, hi: (p, m, a[lo:hi], b[lo:hi], got[lo:hi]))

    def bad_inverses(self, p, m, a, got, ok):
        return self._run(_bad_inverses, len(a),
                         lambda lo, hi: (p, m, a[lo:hi], got[lo:hi], ok[lo:hi]))

    def bad_identities(self, p, m, a, got, ok):
        return self._run(_bad_identities, len(a),
                         lambda lo, hi: (p, m, a[lo:hi], got[lo:hi], ok[lo:hi]))

    def bad_keys(self, p, seed, idx, pk, sk):
        """Key indices idx[j] whose (pk[j], sk[j]) differ from the oracle's."""
        idx = np.asarray(idx)
        parts = _chunks(len(idx), 4 * self.n)
        out = self.pool.map(_bad_keys, [(p, seed, idx[lo:hi], pk[lo:hi], sk[lo:hi])
                                        for lo, hi in parts])
        return [k for bad in out for k in bad]
