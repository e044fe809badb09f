"""Oracle: the NUFFT evaluation of Eq. (tg3), Sec. 3, for phases that are rank 1
on each column half (the wave-equation split of Eq. FIOwq2, Sec. 5).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The transform is g_i = sum_j alpha(x_i, xi_j) e^{2 pi i Phi(x_i, xi_j)} f_j on the
grid x_i = i/N, xi_j = j - N/2.  For the phases here, on each half of the
columns (xi >= 0 and xi < 0) the phase is Phi = t_i xi + rho_i with one target
t_i per row:

    DFT     Phi = x xi                   t = x,               rho = 0
    FIO     Phi = x xi + c(x)|xi|        t = x +- c(x),       rho = 0
    FIO_PW  as FIO for x < 1/2, x xi - c(x)|xi|/2 above (t = x -+ c(x)/2)

with c(x) = (2 + s sin 2 pi x)/16 (Sec. 5).  So Algorithm 6's lifting with
r = 1 (p(x) = t, q(xi) = xi) removes the whole phase of each half, and with
the amplitude split alpha ~ sum_k a_k(x) b_k(xi) (Algorithm 1), Eq. (tg3)
becomes, per half and per k, one 1-D NUFFT "of type 2" (uniform modes xi,
non-uniform targets t_i):

    g_i = sum_k a_k(x_i) e^{2 pi i rho_i} sum_{halves} sum_{xi in half}
          e^{2 pi i t_i xi} (b_k(xi) f(xi)).

The paper names no NUFFT algorithm; the one here is Gaussian gridding.  Its
steps, for M = N/2 modes of one half, shifted to the centred set
jt in [-M/2, M/2) (xi = jt + s_h, s_h = +M/2 or -M/2), and an oversampled grid
of n = 2M points:

  1. e^{2 pi i t xi} = e^{2 pi i t s_h} e^{2 pi i t jt}  (the centring phase);
  2. deconvolve: u_jt = b_k(xi) f(xi) / phihat(jt), with the Gaussian
     phi(d) = sum_l exp(-(d - l)^2 / (4 tau)) (1-periodic) and its Fourier
     coefficients phihat(k) = sqrt(4 pi tau) exp(-4 pi^2 k^2 tau);
  3. h(s_p) = sum_jt u_jt e^{2 pi i p jt / n} on s_p = p/n (an inverse FFT of the
     zero-padded u; numpy's FFT is the library step);
  4. interpolate: sum_jt e^{2 pi i t jt} u_jt phihat(jt) = (phi * h)(t), by the
     trapezoid rule on the grid, (1/n) sum_p phi(t - p/n) h(s_p), over the 2 msp
     grid points nearest t.

tau = msp / (2 pi sigma (2 sigma - 1) M^2) with sigma = n / M = 2 balances the
truncation of phi at msp grid spacings against the aliasing of the trapezoid
rule; both then fall like exp(-2 pi msp (sigma - 1) / (2 sigma - 1)) =
exp(-2 pi msp / 3).  Pinned (tests/test_nufft_pins.py) against the direct sum,
the FFT (DFT phase) and single modes, at that rate.
"""
import numpy as np

DFT, FIO, FIOPW = 0, 1, 2
SIGMA = 2


def targets(kind, N, s=1.0):
    """(t_plus, t_minus, rho): the rank-1 lifting of each column half (targets per row)."""
    x = np.arange(N, dtype=np.float64) / N
    c = (2.0 + s * np.sin(2 * np.pi * x)) / 16.0
    if kind == DFT:
        kap = np.zeros(N)
    elif kind == FIO:
        kap = c
    elif kind == FIOPW:
        kap = np.where(np.arange(N) < N // 2, c, -0.5 * c)
    else:
        raise ValueError("phase kind %r is not rank 1 on the column halves" % kind)
    return x + kap, x - kap, np.zeros(N)


def tau_of(M, msp):
    return msp / (2 * np.pi * SIGMA * (2 * SIGMA - 1) * M * M)


def type2(u, t, msp):
    """sum_{jt} u[jt] e^{2 pi i t jt}, jt = -M/2 .. M/2-1 (u: (M, m)), at targets t (steps 2-4)."""
    M = u.shape[0]
    n = SIGMA * M
    tau = tau_of(M, msp)
    jt = np.arange(-M // 2, M // 2)
    phihat = np.sqrt(4 * np.pi * tau) * np.exp(-4 * np.pi ** 2 * jt.astype(np.float64) ** 2 * tau)
    U = np.zeros((n,) + u.shape[1:], dtype=np.complex128)
    U[jt % n] = u / phihat.reshape((-1,) + (1,) * (u.ndim - 1))          # step 2
    h = n * np.fft.ifft(U, axis=0)                                        # step 3: sum_j U_j e^{+2 pi i p j/n}
    t = np.mod(t, 1.0)
    out = np.zeros((t.size,) + u.shape[1:], dtype=np.complex128)
    base = np.floor(n * t).astype(np.int64)
    for q in range(-msp + 1, msp + 1):                                    # step 4
        p = base + q
        d = t - p / n                                                     # nearest image: |d| < msp/n
        w = np.exp(-d * d / (4 * tau)) / n
        out += w.reshape((-1,) + (1,) * (u.ndim - 1)) * h[np.mod(p, n)]
    return out


def centring(t1, shift, rho):
    """Step 1: e^{2 pi i (t s_h + rho)} per target (t1 = t mod 1, s_h = +-M/2)."""
    return np.exp(2j * np.pi * (np.mod(t1 * shift, 1.0) + rho))


def apply(kind, N, F, a, b, msp, s=1.0):
    """g = K F by Eq. (tg3) with the column halves split (F: (N, m); a, b: (r_alpha, N))."""
    F = np.asarray(F, dtype=np.complex128).reshape(N, -1)
    M = N // 2
    tp, tm, rho = targets(kind, N, s)
    jt = np.arange(-M // 2, M // 2)
    g = np.zeros_like(F)
    for t, shift in ((tp, M // 2), (tm, -(M // 2))):
        xi = jt + shift                       # the half's frequencies
        rows = xi + N // 2
        t1 = np.mod(t, 1.0)
        cent = centring(t1, shift, rho)       # step 1 (and e^{2 pi i rho})
        for k in range(a.shape[0]):
            v = type2(b[k, rows][:, None] * F[rows], t1, msp)
            g += (a[k] * cent)[:, None] * v
    return g


def error_bound(msp):
    """The rate both error terms fall at (sigma = 2): exp(-2 pi msp / 3)."""
    return float(np.exp(-2 * np.pi * msp / 3))
