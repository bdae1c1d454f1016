"""Seeded synthetic inputs shared by the tests and the benchmark.

Only input generation lives here (numpy's PCG64 streams); none of the
method's arithmetic does.  Shapes and distributions follow the kernel
microbenchmark workload: R/q elements uniform in [-(q-1)/2, (q-1)/2], Short
elements (weight w, +-1 at uniform positions), uniform ternary elements, and
the log-uniform batch sizes / parameter-set mix of the ragged workload.
"""
import numpy as np

PARAMS = {653: (653, 4621, 288), 761: (761, 4591, 286), 857: (857, 5167, 322)}


def rq_uniform(P, n, seed):
    p, q, _ = PARAMS[P]
    h = (q - 1) // 2
    return np.random.default_rng(seed).integers(-h, h + 1, (n, p), dtype=np.int16)


def ternary_batch(P, n, seed):
    p = PARAMS[P][0]
    return np.random.default_rng(seed).integers(-1, 2, (n, p), dtype=np.int8)


def short_batch(P, n, seed):
    """n weight-w ternary rows: w positions chosen uniformly, random signs."""
    p, _, w = PARAMS[P]
    rng = np.random.default_rng(seed)
    keys = rng.random((n, p))
    pos = np.argpartition(keys, w, axis=1)[:, :w]
    out = np.zeros((n, p), np.int8)
    signs = rng.integers(0, 2, (n, w), dtype=np.int8) * 2 - 1
    np.put_along_axis(out, pos, signs, axis=1)
    return out


def ragged_batches(n_batches=256, max_b=2048, seed=42):
    """Batch sizes floor(exp(U[0, ln max_b])) clamped to [1, max_b], and a
    parameter set per batch: equal shares of 653/761/857 after a seeded shuffle."""
    rng = np.random.default_rng(seed)
    sizes = np.floor(np.exp(rng.uniform(0.0, np.log(max_b), n_batches))).astype(np.int64)
    sizes = np.clip(sizes, 1, max_b)
    ps = np.array([(653, 761, 857)[i % 3] for i in range(n_batches)])
    rng.shuffle(ps)
    return sizes, ps


def poisson_arrivals(rate_per_s, duration_s, seed):
    rng = np.random.default_rng(seed)
    n = rng.poisson(rate_per_s * duration_s)
    return np.sort(rng.uniform(0.0, duration_s, n))
