"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds none of the method's arithmetic: only random draws.  It is
the one module both the product (bench, serving driver) and the tests use to
make inputs; the oracle itself never imports it (tests pass the arrays in).
"""
import numpy as np


def complex_gaussian(N, m, seed=0, dtype=np.complex128):
    """F[N, m] with Re, Im i.i.d. N(0, 1) (numpy PCG64, ``seed``)."""
    rng = np.random.default_rng(seed)
    F = np.empty((N, m), dtype=np.complex128)
    F.real = rng.standard_normal((N, m))
    F.imag = rng.standard_normal((N, m))
    return F.astype(dtype, copy=False)


def sample_rows(N, k, seed=0):
    """k distinct sorted row indices in [0, N) (the sampled set S of Sec. 5)."""
    rng = np.random.default_rng(seed + 7919)
    return np.sort(rng.choice(N, min(k, N), replace=False)).astype(np.int64)


def uneven_batch(n_ops=32, log2n_lo=12, log2n_hi=18, m_lo=1, m_hi=128, seed=0):
    """(N_i, m_i) for a batch of operators: N = 2^floor(U(lo, hi + 1)), m ~ U{m_lo..m_hi}."""
    rng = np.random.default_rng(seed)
    e = np.floor(rng.uniform(log2n_lo, log2n_hi + 1, size=n_ops)).astype(int)
    e = np.minimum(e, log2n_hi)
    m = rng.integers(m_lo, m_hi + 1, size=n_ops)
    return [(int(2 ** a), int(b)) for a, b in zip(e, m)]


def poisson_requests(rate_per_s, duration_s, n_ops, m_choices=(1, 4, 16, 64), seed=0):
    """Arrival times (s), operator index and RHS count of a Poisson request stream."""
    rng = np.random.default_rng(seed)
    n = int(rate_per_s * duration_s * 1.5) + 16
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))
    t = t[t < duration_s]
    ops = rng.integers(0, n_ops, size=t.size)
    ms = rng.choice(np.asarray(m_choices), size=t.size)
    return t, ops, ms
