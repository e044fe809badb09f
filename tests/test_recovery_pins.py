"""Pins of the phase-recovery oracle (Algorithms 3, 4, 5; Sec. 2.2, Scenario 1).

What fixes the answer independently of the oracle:
* Mathematics of Algorithm 3: on a vector whose third differences stay far
  below half a turn, nearest-integer choices rebuild v up to an integer
  polynomial of degree <= 2 (the first three choices), and v = u mod 1 holds.
* Discontinuities planted at known indices, and the kink of the paper's
  Figure (vec): a row of Phi = x xi + c(x)|xi| is found discontinuous at its
  start and in its middle.
* Consistency: rows and columns of one Psi agree where they cross.
* The paper's printed recovery errors eps^K of Table 1D-FIO (N = 1024, 4096).
Planted mistakes at the end break these pins.
"""
import os

import numpy as np
import pytest

from oracle import direct as d
from oracle import recovery as rc

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def frac(x):
    return x - np.floor(x)


def is_integer_quadratic(w, lo=0, hi=None):
    """w[lo:hi] takes integer values and has zero third differences."""
    w = w[lo:hi]
    k = np.rint(w)
    return np.abs(w - k).max() < 1e-6 and np.abs(np.diff(k, 3)).max() == 0


def eps_k(entry, P, Q, N, seed=1):
    """eps^K of Sec. 5 on 256 x 256 sampled entries: kernel rebuilt from the phase."""
    S = np.sort(np.random.default_rng(seed).choice(N, min(N, 256), replace=False))
    K = entry(S, S)
    psi = (P[:, S].T @ Q[:, S]).real
    Kr = np.abs(K) * np.exp(2j * np.pi * psi)
    return np.linalg.norm(K - Kr, 2) / np.linalg.norm(K, 2)


# ------------------------------------------------------------ Algorithm 3 ---
def test_unwrap_exact_up_to_integer_quadratic():
    # second differences of 0.7 turn (a linear extrapolation would pick wrong
    # integers), third differences ~1e-6: no discontinuity at tau = 1 turn
    a = np.arange(3000.0)
    v = 0.35 * a ** 2 + 0.37 * a + 3 * np.sin(a / 50)
    u = frac(v)
    w, S = rc.unwrap(u, rc.TAU_BLOCK)
    assert S == [0]
    assert np.array_equal(frac(w), frac(u + 0.0)) or np.abs(frac(w) - u).max() < 1e-9
    assert is_integer_quadratic(w - v)


def test_unwrap_detects_planted_jumps():
    a = np.arange(2000.0)
    v = 0.2 * a + 0.001 * a ** 2 + np.where(a >= 777, 0.4, 0.0) + np.where(a >= 1500, -0.35, 0.0)
    w, S = rc.unwrap(frac(v), rc.TAU_DETECT)
    assert S == [0, 777, 1500]
    d_ = w - v
    assert np.abs(d_ - np.rint(d_)).max() < 1e-9          # v = u mod 1 on every entry
    for lo, hi in ((0, 777), (777, 1500), (1500, 2000)):  # smooth pieces rebuilt exactly
        assert is_integer_quadratic(w - v, lo, hi)


def test_unwrap_paper_figure_row():
    # Figure (vec): one row of Phi = x xi + c(x)|xi|, c(x) = (2 + sin 2 pi x)/2, is
    # discontinuous (as a recovered vector) at its start and at the kink xi = 0.
    # At x = 85/1024, 2c(x) = 2.498 turns: the kink's second difference mod 1 is
    # about half a turn, above tau.  Index N/2 + 1 is the first whose second
    # difference spans xi = 0.
    N = 1024
    x = 85 / N
    xi = np.arange(N) - N / 2
    v = x * xi + (2 + np.sin(2 * np.pi * x)) / 2 * np.abs(xi)
    w, S = rc.unwrap(frac(v), rc.TAU_DETECT)
    assert S == [0, N // 2 + 1]
    assert np.abs((w - v) - np.rint(w - v)).max() < 1e-9


def test_unwrap_seeds_are_kept():
    a = np.arange(100.0)
    v = 0.45 * a + 0.003 * a ** 2
    w, _ = rc.unwrap(frac(v), rc.TAU_BLOCK, seed=list(v[:3] + 5.0))
    assert np.allclose(w, v + 5.0, atol=1e-9)             # the seeds fix the integer polynomial


# ------------------------------------------------------------ Algorithm 4 ---
def sampler_defects(ent, N, seed):
    """(entries where rows and columns of Psi disagree, max |Psi - Phi| mod 1) on 12 x 12 crossings."""
    rng = np.random.default_rng(seed)
    smp = rc.PsiSampler(ent, N, rng.choice(N, 10, replace=False), rng.choice(N, 10, replace=False))
    assert smp.rb[0] == 0 and smp.rb[-1] == N and smp.cb[0] == 0 and smp.cb[-1] == N
    I, J = rng.choice(N, 12, replace=False), rng.choice(N, 12, replace=False)
    rows = np.stack([smp.row(i) for i in I])
    cols = np.stack([smp.col(j) for j in J], axis=1)
    phi = frac(np.angle(ent(I, np.arange(N))) / (2 * np.pi))
    dd = frac(rows) - phi
    return int(np.sum(rows[:, J] != cols[I, :])), float(np.abs(dd - np.rint(dd)).max())


@pytest.mark.parametrize("s", [0.2, 1.0])
def test_sampler_rows_and_columns_agree(s):
    # the kink of c(x)|xi| at xi = 0 (second difference 2c(x) <= 0.375 turn) may or
    # may not cut the columns in two; either way rows and columns are one Psi
    N = 1024
    ent = lambda I, J: d.entries(d.FIO, N, np.asarray(I), np.asarray(J), s=s)
    disagree, dev = sampler_defects(ent, N, 3)
    assert disagree == 0                                       # same Psi entries, bitwise
    assert dev < 1e-9                                          # Psi = Phi mod 1


def test_sampler_blocks_at_planted_discontinuities():
    # Phi = x xi + c(x)|xi| + 0.4 [x >= 1/2] + 0.3 [xi >= 0]: jumps of 0.4 along every
    # column at row N/2 and of 0.3 along every row at column N/2 (both above 1/4 turn)
    N = 1024

    def ent(I, J):
        i = np.asarray(I, float)[:, None]
        j = np.asarray(J, float)[None, :]
        x, xi = i / N, j - N / 2
        ph = x * xi + (2 + 0.2 * np.sin(2 * np.pi * x)) / 16 * np.abs(xi) + 0.4 * (x >= 0.5) + 0.3 * (xi >= 0)
        return np.exp(2j * np.pi * ph)
    P, Q, smp = rc.phase_lowrank(ent, N, seed=4)
    assert smp.rb == [0, N // 2, N] and smp.cb == [0, N // 2, N]
    assert P.shape[0] <= 12
    assert eps_k(ent, P, Q, N) < 1e-10


# ------------------------------------------------------------ Algorithm 5 ---
def test_phase_lowrank_matches_paper_table_1dfio():
    tab = np.loadtxt(os.path.join(GOLDEN, "table_1dfio_recovery.txt"))
    for N in (1024, 4096):
        printed = tab[tab[:, 0] == N, 1]
        ent = lambda I, J: d.entries(d.FIO, N, np.asarray(I), np.asarray(J), s=0.2)
        P, Q, _ = rc.phase_lowrank(ent, N, r=20, q=5, seed=0)
        e = eps_k(ent, P, Q, N)
        # the rank of x xi + c(x)|xi| plus integer terms alpha i + a j + b is 3
        assert P.shape[0] == 3
        assert e < 10 * printed.max(), (N, e, printed)


def test_phase_lowrank_smooth_amplitude_dft():
    N = 2048
    for kind, amp in ((d.DFT, 0), (d.FIO, 1)):
        ent = lambda I, J: d.entries(kind, N, np.asarray(I), np.asarray(J), amp=amp)
        P, Q, _ = rc.phase_lowrank(ent, N, seed=5)
        assert eps_k(ent, P, Q, N) < 1e-10


# ----------------------------------------------- planted mistakes ---------
def test_planted_mistakes_are_caught(monkeypatch):
    a = np.arange(3000.0)
    v = 0.35 * a ** 2 + 0.37 * a + 3 * np.sin(a / 50)
    # (1) a dropped sign in the third-difference prediction
    monkeypatch.setattr(rc, "predict", lambda w, k: 3 * w[k - 1] - 3 * w[k - 2] - w[k - 3])
    w, _ = rc.unwrap(frac(v), rc.TAU_BLOCK)
    assert not is_integer_quadratic(w - v)
    monkeypatch.undo()
    # (2) a row seeded from the next row's values in the block's first three columns
    N = 1024
    ent = lambda I, J: d.entries(d.FIO, N, np.asarray(I), np.asarray(J), s=1.0)

    def off_by_one(self, i, bi, bj, u=None):
        r0, c0, c1 = self.rb[bi], self.cb[bj], self.cb[bj + 1]
        if u is None:
            u = self._u([i], np.arange(c0, c1))[0]
        k = min(i - r0 + 1, self.colseed[bi, bj].shape[1] - 1)
        return rc.unwrap(u, self.tau_block, seed=list(self.colseed[bi, bj][:, k]))[0]
    monkeypatch.setattr(rc.PsiSampler, "_row_block", off_by_one)
    disagree, dev = sampler_defects(ent, N, 3)
    assert disagree > 0 or dev > 1e-6
