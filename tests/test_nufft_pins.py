"""CPU pins of the NUFFT oracle (oracle/nufft.py, Eq. tg3 of Sec. 3 with the
column halves split as in Eq. FIOwq2).

The oracle's Gaussian gridding is held to things other than itself:
* the direct FP64 sum (oracle/direct.c) for the DFT, FIO and piecewise FIO
  phases with the smooth amplitude, with an error that follows the analytic
  rate exp(-2 pi msp / 3) of the truncation and aliasing terms (within a fixed
  band below it, for every msp from 3 to 12 and every N);
* numpy's FFT for the DFT phase (the unnormalised inverse DFT times (-1)^i);
* a single mode f = e_j, whose image is column j of K (oracle entries);
* planted mistakes (the halves' targets swapped, tau off by a factor 2, the
  deconvolution dropped, the centring phase's sign flipped): each fails.
"""
import numpy as np
import pytest

from oracle import direct as od
from oracle import lowrank
from oracle import nufft as nu
from paper_1803_04128_gb300 import inputs


def amp_split(N, amp=1):
    ent = lambda I, J: od.amplitude(amp, N, np.asarray(I)[:, None], np.asarray(J)[None, :]).astype(np.complex128)
    return lowrank.amplitude_split(ent, N, N)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("kind,okind", [(nu.FIO, od.FIO), (nu.FIOPW, od.FIOPW), (nu.DFT, od.DFT)])
@pytest.mark.parametrize("N", [256, 1024])
def test_nufft_meets_direct_at_the_analytic_rate(kind, okind, N):
    F = inputs.complex_gaussian(N, 3, seed=N + kind)
    a, b = amp_split(N)
    gd = od.direct(okind, N, F, None, amp=1)
    for msp in (3, 4, 6, 8, 10, 12):
        e = rel(nu.apply(kind, N, F, a, b, msp), gd)
        bound = nu.error_bound(msp)
        assert 0.03 * bound < e < bound, (msp, e, bound)


def test_nufft_dft_phase_equals_fft():
    N = 512
    F = inputs.complex_gaussian(N, 2, seed=3)
    one = np.ones((1, N), dtype=np.complex128)
    g = nu.apply(nu.DFT, N, F, one, one, 12)
    sign = (-1.0) ** np.arange(N)
    ref = sign[:, None] * N * np.fft.ifft(F, axis=0)      # sum_j e^{2 pi i i (j - N/2)/N} f_j
    assert rel(g, ref) < 2 * nu.error_bound(12)


def test_nufft_single_mode_is_a_column_of_k():
    N = 1024
    a, b = amp_split(N)
    for j in (0, N // 2 - 1, N // 2, 3 * N // 4 + 5, N - 1):   # both halves and both edges
        f = np.zeros((N, 1), dtype=np.complex128)
        f[j] = 1.0
        g = nu.apply(nu.FIO, N, f, a, b, 10)[:, 0]
        col = od.entries(od.FIO, N, np.arange(N), np.array([j]), amp=1)[:, 0]
        assert rel(g, col) < 20 * nu.error_bound(10), j


@pytest.mark.parametrize("mistake", ["swap_halves", "tau_x2", "no_deconvolution", "centring_sign"])
def test_nufft_planted_mistakes_fail(mistake, monkeypatch):
    N, msp = 512, 8
    F = inputs.complex_gaussian(N, 2, seed=9)
    a, b = amp_split(N)
    gd = od.direct(od.FIO, N, F, None, amp=1)
    if mistake == "swap_halves":
        orig = nu.targets
        monkeypatch.setattr(nu, "targets", lambda k, n, s=1.0: (lambda t: (t[1], t[0], t[2]))(orig(k, n, s)))
    elif mistake == "tau_x2":
        orig_tau = nu.tau_of
        monkeypatch.setattr(nu, "tau_of", lambda M, msp: 2 * orig_tau(M, msp))
    elif mistake == "no_deconvolution":
        orig2 = nu.type2

        def t2(u, t, msp):
            M = u.shape[0]
            tau = nu.tau_of(M, msp)
            jt = np.arange(-M // 2, M // 2)
            ph = np.sqrt(4 * np.pi * tau) * np.exp(-4 * np.pi ** 2 * jt.astype(float) ** 2 * tau)
            return orig2(u * ph[:, None], t, msp)       # cancels the division by phihat
        monkeypatch.setattr(nu, "type2", t2)
    else:
        monkeypatch.setattr(nu, "centring", lambda t1, shift, rho: np.exp(-2j * np.pi * (np.mod(t1 * shift, 1.0) + rho)))
    e = rel(nu.apply(nu.FIO, N, F, a, b, msp), gd)
    assert e > 100 * nu.error_bound(msp), (mistake, e)
