"""Pins of the oracle against facts the paper and the mathematics fix.

None of these re-derive the oracle's own formula: they compare it with a
library transform (FFT, Horner evaluation), an identity, a brute force in
higher precision, exactness cases of interpolation, or values printed in the
paper.  Planted-mistake tests at the end show that the pins catch plausible
errors in the oracle.
"""
import os

import numpy as np
import pytest

from conftest import relerr
from oracle import butterfly as bf
from oracle import direct as d
from oracle import lowrank as lr

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def cgauss(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


# ------------------------------------------------------------ direct ------
@pytest.mark.parametrize("N", [16, 256, 4096])
def test_direct_dft_equals_fft(N):
    # Phi = x xi, alpha = 1: K_ij = e^{2 pi i i (j - N/2)/N} = (-1)^i e^{2 pi i ij/N}
    rng = np.random.default_rng(1)
    f = cgauss(rng, N, 3)
    g = d.direct(d.DFT, N, f)
    ref = ((-1.0) ** np.arange(N))[:, None] * N * np.fft.ifft(f, axis=0)
    assert relerr(g, ref) < 1e-13


def test_direct_dft_naive_loop():
    N = 32
    rng = np.random.default_rng(2)
    f = cgauss(rng, N)
    ref = np.zeros(N, complex)
    for i in range(N):
        for j in range(N):
            ref[i] += np.exp(2j * np.pi * (i / N) * (j - N / 2)) * f[j]
    assert relerr(d.direct(d.DFT, N, f), ref) < 1e-13


def test_direct_parseval():
    N = 2048
    f = cgauss(np.random.default_rng(3), N)
    g = d.direct(d.DFT, N, f)
    assert abs(np.vdot(g, g).real / (N * np.vdot(f, f).real) - 1) < 1e-12


@pytest.mark.parametrize("kind,amp", [(d.FIO, 0), (d.FIO, 1), (d.FIOPW, 1), (d.DFT, 0)])
def test_direct_long_double_brute_force(kind, amp):
    N = 256
    f = cgauss(np.random.default_rng(4), N, 2)
    rows = np.arange(0, N, 3)
    assert relerr(d.direct(kind, N, f, rows, amp=amp), d.direct_ld(kind, N, f, rows, amp=amp)) < 1e-13


@pytest.mark.parametrize("kind,s", [(d.FIO, 1.0), (d.FIO, 0.2), (d.FIOPW, 1.0)])
def test_direct_half_spectrum_is_polynomial(kind, s):
    # For f supported on xi >= 0 (resp. xi < 0) the phase x xi + c(x)|xi| is
    # linear in xi, so g(x) is a polynomial in z = e^{2 pi i (x +- c(x))},
    # evaluated here by Horner's rule (np.polyval).  Second branch of FIOPW:
    # x xi - c(x)|xi|/2 for x >= 1/2.
    N = 1024
    rng = np.random.default_rng(5)
    x = np.arange(N) / N
    c = (2 + s * np.sin(2 * np.pi * x)) / 16
    cp = c if kind == d.FIO else np.where(x < 0.5, c, -0.5 * c)
    fpos = np.zeros(N, complex); fpos[N // 2:] = cgauss(rng, N // 2)
    gp = d.direct(kind, N, fpos, s=s)
    z = np.exp(2j * np.pi * (x + cp))
    refp = np.polyval(fpos[N // 2:][::-1], z)                 # sum_{xi=0}^{N/2-1} f(xi) z^xi
    assert relerr(gp, refp) < 1e-11
    fneg = np.zeros(N, complex); fneg[:N // 2] = cgauss(rng, N // 2)
    gn = d.direct(kind, N, fneg, s=s)
    w = np.exp(-2j * np.pi * (x - cp))                          # e^{2 pi i (x - c)(xi)}, xi = -k
    coeffs = np.concatenate([fneg[:N // 2], [0]])               # k = N/2 .. 1, highest first
    refn = np.polyval(coeffs, w)
    assert relerr(gn, refn) < 1e-11


def test_direct_amplitude_identity():
    # alpha = 1 + 0.25 sin(2 pi x) cos(2 pi xi/N)
    #   = 1 + 0.125 sin(2 pi x) (e^{2 pi i xi/N} + e^{-2 pi i xi/N})
    N = 512
    f = cgauss(np.random.default_rng(6), N)
    xi = np.arange(N) - N // 2
    x = np.arange(N) / N
    ga = d.direct(d.FIO, N, f, amp=1)
    g0 = d.direct(d.FIO, N, f)
    gp = d.direct(d.FIO, N, np.exp(2j * np.pi * xi / N) * f)
    gm = d.direct(d.FIO, N, np.exp(-2j * np.pi * xi / N) * f)
    assert relerr(ga, g0 + 0.125 * np.sin(2 * np.pi * x) * (gp + gm)) < 1e-12


def test_direct_linearity_and_impulse():
    N = 256
    rng = np.random.default_rng(7)
    f, h = cgauss(rng, N), cgauss(rng, N)
    a, b = 0.3 - 1.1j, 2.0 + 0.5j
    lhs = d.direct(d.FIOPW, N, a * f + b * h, amp=1)
    rhs = a * d.direct(d.FIOPW, N, f, amp=1) + b * d.direct(d.FIOPW, N, h, amp=1)
    assert relerr(lhs, rhs) < 1e-13
    for j in (0, 17, N // 2, N - 1):
        e = np.zeros(N, complex); e[j] = 1
        g = d.direct(d.FIO, N, e)
        assert np.allclose(np.abs(g), 1.0, atol=1e-14)          # |alpha e^{i...}| = 1
        assert np.allclose(g, d.entries(d.FIO, N, np.arange(N), [j])[:, 0], atol=1e-14)


def test_direct_rows_subset_and_columns():
    N = 512
    f = cgauss(np.random.default_rng(8), N, 5)
    full = d.direct(d.FIO, N, f, amp=1)
    rows = np.array([3, 100, 511])
    assert np.array_equal(d.direct(d.FIO, N, f, rows, amp=1), full[rows])
    assert np.allclose(d.direct(d.FIO, N, f[:, 2], amp=1), full[:, 2], atol=0)


# ------------------------------------------------------------ grids -------
@pytest.mark.parametrize("r", [2, 3, 6, 9, 10, 11, 12, 16])
@pytest.mark.parametrize("n", [4, 16, 17, 64, 1000, 4096, 65536])
def test_grid_properties(n, r):
    g = bf.grid(n, r)
    if n <= r:
        assert np.array_equal(g, np.arange(n))
        return
    assert g.size == r and g[0] == 0 and g[-1] == n - 1
    assert np.all(np.diff(g) >= 1)
    # mirror image about the middle, up to one index where a tie rounded down
    assert np.all(np.abs(g + g[::-1] - (n - 1)) <= 1)
    # the exact (real-arithmetic) grid, by rational evaluation where z_t is rational
    z = bf.chebyshev_z(r)
    assert np.allclose(np.sort(z), -z, atol=1e-15)                 # Chebyshev points are symmetric
    if r % 2 == 1 and (n - r) % 2 == 1:
        assert g[r // 2] == n // 2 - 1                            # exact tie -> lower index


def test_lagrange_basis():
    nodes = bf.grid(100, 10)
    pts = np.arange(100)
    M = bf.lagrange(nodes, pts)
    assert np.allclose(M.sum(axis=0), 1.0, atol=1e-11)           # partition of unity
    assert np.allclose(bf.lagrange(nodes, nodes), np.eye(10), atol=1e-14)
    # reproduces polynomials of degree < r (scipy's barycentric interpolator as library check)
    from scipy.interpolate import BarycentricInterpolator
    vals = np.sin(nodes / 17.0)
    ref = BarycentricInterpolator(nodes.astype(float), vals)(pts.astype(float))
    assert np.allclose(vals @ M, ref, atol=1e-9)


# -------------------------------------------------------- butterfly -------
@pytest.mark.parametrize("kind", [d.ONES, d.SEP])
@pytest.mark.parametrize("n0,r", [(1, 3), (1, 10), (2, 6), (4, 12)])
def test_butterfly_exact_when_R_vanishes(kind, n0, r):
    # Phi = p(x) + q(xi) makes R(A, B) of Eq. (RAB) identically zero, so every
    # interpolation in Algorithm 4.1 is exact and BF = K to rounding.
    N = 1024
    f = cgauss(np.random.default_rng(9), N, 2)
    assert relerr(bf.butterfly(bf.Kernel(kind, N), f, r, n0), d.direct(kind, N, f)) < 1e-12


@pytest.mark.parametrize("kind", [d.FIO, d.FIOPW, d.DFT])
def test_butterfly_exact_with_full_grids(kind):
    # r >= every node size: the grids hold every index, interpolation is exact.
    N = 64
    f = cgauss(np.random.default_rng(10), N)
    assert relerr(bf.butterfly(bf.Kernel(kind, N), f, 64), d.direct(kind, N, f)) < 1e-12


def test_butterfly_matches_paper_table_1dfio():
    # eps^b printed in Sec. 5, Table 1D-FIO (N = 1024, c(x) = (2 + 0.2 sin 2 pi x)/16)
    tab = np.loadtxt(os.path.join(GOLDEN, "table_1dfio_N1024.txt"))
    N = 1024
    rng = np.random.default_rng(11)
    f = cgauss(rng, N)
    rows = np.sort(rng.choice(N, 256, replace=False))          # 256 sampled rows, Sec. 5
    gd = d.direct(d.FIO, N, f, rows, s=0.2)
    kern = bf.Kernel(d.FIO, N, s=0.2)
    for r, eps_paper in tab:
        e = relerr(bf.butterfly(kern, f, int(r))[rows], gd)
        assert eps_paper / 4 < e < eps_paper * 4, (r, e, eps_paper)


def test_butterfly_error_decays_with_r():
    N = 2048
    f = cgauss(np.random.default_rng(12), N)
    gd = d.direct(d.FIO, N, f)
    kern = bf.Kernel(d.FIO, N)
    errs = [relerr(bf.butterfly(kern, f, r), gd) for r in (6, 8, 10, 12)]
    assert all(b < a / 10 for a, b in zip(errs, errs[1:])), errs
    assert errs[2] < 1e-6                                        # r = 10 meets eps = 1e-6


def test_butterfly_columns_independent():
    N = 512
    F = cgauss(np.random.default_rng(13), N, 4)
    kern = bf.Kernel(d.FIO, N)
    G = bf.butterfly(kern, F, 10)
    assert np.allclose(G[:, 1], bf.butterfly(kern, F[:, 1], 10), atol=1e-13)


# ---------------------------------------------------------- low rank ------
def test_lowrank_amplitude_rank_two():
    N = 2048
    ent = lambda I, J: d.amplitude(1, N, np.asarray(I)[:, None], np.asarray(J)[None, :])
    a, b = lr.amplitude_split(ent, N, N)
    assert a.shape == (2, N) and b.shape == (2, N)
    S = np.arange(0, N, 7)
    A = ent(S, S)
    eps_amp = np.linalg.norm(A - a[:, S].T @ b[:, S], 2) / np.linalg.norm(A, 2)
    assert eps_amp < 1e-12                                      # Table 1D-FIO: eps^amp ~ 1e-15


@pytest.mark.parametrize("amp,rank", [(0, 1), (1, 2)])
def test_lowrank_exact_low_rank_amplitudes(amp, rank):
    # alpha = 1 (rank 1) and the smooth amplitude (rank 2) are recovered exactly
    N = 1024
    ent = lambda I, J: d.amplitude(amp, N, np.asarray(I)[:, None], np.asarray(J)[None, :])
    a, b = lr.amplitude_split(ent, N, N)
    assert a.shape[0] == rank
    A = ent(np.arange(N), np.arange(N))
    assert np.abs(a.T @ b - A).max() < 1e-12


def test_lowrank_random_complex_matches_svd():
    rng = np.random.default_rng(14)
    m, n, k = 300, 200, 4
    K = cgauss(rng, m, k) @ cgauss(rng, k, n)
    U, S, V = lr.rsvd_sampled(lambda I, J: K[np.ix_(I, J)], m, n, r=8, q=3)
    assert np.allclose(S[:k], np.linalg.svd(K, compute_uv=False)[:k], rtol=1e-10)
    assert relerr((U[:, :k] * S[:k]) @ V[:, :k].conj().T, K) < 1e-12


def test_ibf_apply_with_amplitude():
    N = 1024
    rng = np.random.default_rng(15)
    F = cgauss(rng, N, 3)
    ent = lambda I, J: d.amplitude(1, N, np.asarray(I)[:, None], np.asarray(J)[None, :])
    a, b = lr.amplitude_split(ent, N, N)
    g = bf.ibf_apply(d.FIO, N, F, 10, a, b)
    assert relerr(g, d.direct(d.FIO, N, F, amp=1)) < 1e-6


# ------------------------------------------------------- Hankel entries ---
def test_hankel_entries_satisfy_bessel_identities():
    # oracle/special.py's entries H^(1)_nu(x) = J_nu + i Y_nu on the transform's grid:
    # the Wronskian J_{nu+1} Y_nu - J_nu Y_{nu+1} = 2 / (pi x) and the three-term
    # recurrence H_{nu-1} + H_{nu+1} = (2 nu / x) H_nu
    from oracle import special as sp
    N = 1024
    rows = np.array([0, 1, 100, 700, 1023])
    x = sp.hankel_x(N, rows)
    H = lambda n: sp.hankel_entries(N, rows, np.asarray(n))
    nu = np.array([0, 1, 333, 900, 1021])
    Jn, Yn = H(nu).real, H(nu).imag
    Jn1, Yn1 = H(nu + 1).real, H(nu + 1).imag
    wr = (Jn1 * Yn - Jn * Yn1) * (np.pi * x[:, None] / 2)
    assert np.abs(wr - 1).max() < 1e-10
    rec = H(nu[1:] - 1) + H(nu[1:] + 1) - (2 * nu[1:][None, :] / x[:, None]) * H(nu[1:])
    assert np.abs(rec).max() < 1e-10 * np.abs(H(nu[1:])).max()


# ----------------------------------------------- planted mistakes ---------
def test_planted_mistakes_are_caught(monkeypatch):
    """Each plausible oracle mistake below breaks at least one pin above."""
    N = 256
    f = cgauss(np.random.default_rng(16), N)
    ref = d.direct(d.SEP, N, f)
    kern = bf.Kernel(d.SEP, N)
    assert relerr(bf.butterfly(kern, f, 6), ref) < 1e-12
    # (1) wrong sign of one phase factor
    orig_e = bf.Kernel.e
    calls = {"n": 0}

    def e_flip(self, i, j, sign=1):
        calls["n"] += 1
        return orig_e(self, i, j, -sign if calls["n"] == 3 else sign)
    monkeypatch.setattr(bf.Kernel, "e", e_flip)
    assert relerr(bf.butterfly(kern, f, 6), ref) > 1e-3
    monkeypatch.setattr(bf.Kernel, "e", orig_e)
    # (2) Lagrange weights evaluated at the wrong points (reversed order): the
    # full-grid exactness pin catches it (R = 0 kernels cannot, since any
    # partition of unity reproduces a constant)
    orig_l = bf.lagrange
    f64 = f[:64]
    gfull = d.direct(d.FIO, 64, f64)
    monkeypatch.setattr(bf, "lagrange", lambda nodes, pts: orig_l(nodes, np.asarray(pts)[::-1]))
    assert relerr(bf.butterfly(bf.Kernel(d.FIO, 64), f64, 64), gfull) > 1e-3
    monkeypatch.setattr(bf, "lagrange", orig_l)
    # (3) centre off by one node (c_A outside the node) keeps R = 0 exactness for
    # SEP but breaks the accuracy pin for the FIO kernel
    Nf = 1024
    ff = cgauss(np.random.default_rng(17), Nf)
    gd = d.direct(d.FIO, Nf, ff, s=0.2)
    monkeypatch.setattr(bf, "centre", lambda start, n: start + n + (n - 1) // 2)
    e = relerr(bf.butterfly(bf.Kernel(d.FIO, Nf, 0.2), ff, 10), gd)
    assert e > 1.69e-8 * 4


# ------------------------------------------------------ Algorithm 6 -------
def _fio_factors(N):
    # Phi = x xi + c(x)|xi| is exactly rank 2: p = (x, c(x)), q = (xi, |xi|) (Sec. 3's lifting)
    x = np.arange(N) / N
    xi = np.arange(N) - N / 2.0
    c = (2 + np.sin(2 * np.pi * x)) / 16
    amp1 = (np.ones((1, N)), np.ones((1, N)))
    amp2 = (np.stack([np.ones(N), 0.25 * np.sin(2 * np.pi * x)]), np.stack([np.ones(N), np.cos(2 * np.pi * xi / N)]))
    return np.stack([x, c]), np.stack([xi, np.abs(xi)]), amp1, amp2


@pytest.mark.parametrize("N", [1024, 4096])
def test_decide_exact_lifting_of_fio_phase(N):
    # with r = 2 the lifting is the whole phase: the residual kernel is alpha itself, so n
    # and the number of NUFFTs equal the amplitude rank (1 or 2); with r = 1 the residual
    # phase c(x)|xi| - its projection winds hundreds of turns: every sampled column counts
    from oracle import decide as dc
    P1, Q1, amp1, amp2 = _fio_factors(N)
    assert dc.nufft_decide(P1, Q1, *amp1, r=2, r_eps=20) == (1, 1, 1)
    assert dc.nufft_decide(P1, Q1, *amp2, r=2, r_eps=20) == (1, 2, 2)
    assert dc.nufft_decide(P1, Q1, *amp1, r=1, r_eps=20) == (0, 100, 0)


@pytest.mark.parametrize("r,r_eps", [(1, 40), (1, 60), (2, 20)])
def test_decide_matches_brute_force_rank(r, r_eps):
    # N = 256: the numerical rank of the whole residual kernel by numpy's SVD.  Pivoted QR
    # reveals it up to the usual factor between |R_kk| and sigma_k, so n lies between the
    # SVD ranks at 10 eps and eps / 10 (for r = 1: 49 and 53), and y follows that band
    from oracle import decide as dc
    N, eps = 256, 1e-10
    P1, Q1, amp1, _ = _fio_factors(N)
    P, Q = dc.lifting(P1, Q1, r)
    K = dc.residual_kernel(P1, Q1, *amp1, P, Q, np.arange(N), np.arange(N))
    s = np.linalg.svd(K, compute_uv=False)
    lo, hi = (int(np.sum(s > t * s[0])) for t in (10 * eps, eps / 10))
    assert lo >= r_eps or hi < r_eps                     # the case is away from the threshold
    y, n, terms = dc.nufft_decide(P1, Q1, *amp1, r=r, r_eps=r_eps, q=5, eps=eps)
    assert lo <= n <= hi
    assert y == int(hi < r_eps)
    assert (terms > 0) == bool(y) and terms <= r_eps
    # the lifting is the best rank-r part of the phase (Eckart-Young against numpy's SVD)
    sv = np.linalg.svd(P1.T @ Q1, compute_uv=False)
    err = np.linalg.norm(P1.T @ Q1 - P.T @ Q, 2)
    assert abs(err - (sv[r] if r < sv.size else 0.0)) <= 1e-9 * sv[0]


def test_decide_planted_mistakes_are_caught(monkeypatch):
    # a lifting without its singular values, or a residual phase with the wrong sign,
    # turns the rank-2 case into a full-rank one
    from oracle import decide as dc
    P1, Q1, amp1, _ = _fio_factors(1024)
    real = dc.lifting
    monkeypatch.setattr(dc, "lifting", lambda A, B, r: (lambda P, Q: (P / np.linalg.norm(P, axis=1)[:, None], Q))(*real(A, B, r)))
    assert dc.nufft_decide(P1, Q1, *amp1, r=2, r_eps=20)[0] == 0
    monkeypatch.setattr(dc, "lifting", real)
    monkeypatch.setattr(dc, "residual_kernel", lambda P1, Q1, A2, B2, P, Q, I, J:
                        (A2[:, I].T @ B2[:, J]) * np.exp(2j * np.pi * (P1[:, I].T @ Q1[:, J] + P[:, I].T @ Q[:, J])))
    assert dc.nufft_decide(P1, Q1, *amp1, r=2, r_eps=20)[0] == 0
