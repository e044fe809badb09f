"""Oracle: the butterfly algorithm of Sec. 4 (Algorithm 4.1) in FP64, on the fly.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

This evaluates u = BF(y) ~ e^{2 pi i Phi} y exactly as Algorithm 4.1 states
it, step by step, recomputing every interpolation weight and phase from its
formula at each level (no stored factors, no fusion, no merging of levels).
It is the reference for what the product's stored IBF-MAT apply computes; the
difference between the two is then rounding only.

Notation follows the paper: T_X (rows, x) and T_Omega (columns, xi) are dyadic
trees of depth L; a pair (A, B) at level l has A at level l of T_X and B at
level L-l of T_Omega; lambda^{AB}_t are the expansion coefficients; xi^B_t and
x^A_t are the mock-Chebyshev index grids of Eq. (gdB)/(gdA); M^B_t, M^A_t are
their Lagrange polynomials; c_A, c_B are centre indices (Eq. RAB).

Readings of the paper taken here, where it is silent, garbled or ambiguous:
  * 0-based indices: x_i = i/N, xi_j = j - N/2 (Eq. 1D-xandxi, shifted).
  * Leaves of both trees hold n0 indices (the paper's Fig. "submatrices" uses
    n0 = 1, the default); L = log2(N/n0), h = floor(L/2) when L is odd.
  * Eq. (gdA)/(gdB): the printed grid t + (N_A - r)(z_t + 1/2) runs backwards
    and can repeat; the grid used is Round(t + (n - r)(1/2 - z_t)), t = 1..r,
    which is increasing, distinct and contains both end points.  Round takes
    the nearest integer and breaks ties toward the lower index, a value within
    1e-9 of a half integer counting as a tie, so that two implementations
    whose cos() differ in the last bit still pick the same indices
    (Round(v) = ceil(v - 1/2 - 1e-9)).  A node with n <= r indices uses all
    of them (the "only one kept if repeated" rule taken to its end).
  * c_A: of the two indices closest to the mean of an even-sized node, the
    lower one.
"""
import numpy as np

from . import direct as _d


# ---------------------------------------------------------------- grids ----
def chebyshev_z(r):
    """z_t = (1/2) cos((t-1) pi/(r-1)), t = 1..r: Chebyshev grid on [-1/2, 1/2] (Sec. 2.1)."""
    t = np.arange(1, r + 1)
    return 0.5 * np.cos((t - 1) * np.pi / (r - 1))


def grid(n, r):
    """0-based offsets of the r-point mock-Chebyshev grid of a node of n indices
    (Eq. gdA / gdB, with the reading stated in the module docstring)."""
    if n <= r:
        return np.arange(n, dtype=np.int64)
    t = np.arange(1, r + 1)
    v = t + (n - r) * (0.5 - chebyshev_z(r))
    return np.ceil(v - 0.5 - 1e-9).astype(np.int64) - 1


def lagrange(nodes, pts):
    """M[t, k] = prod_{j != t} (pts[k] - nodes[j]) / (nodes[t] - nodes[j])  (Sec. 2.1)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    pts = np.asarray(pts, dtype=np.float64)
    M = np.ones((nodes.size, pts.size))
    for t in range(nodes.size):
        for j in range(nodes.size):
            if j != t:
                M[t] *= (pts - nodes[j]) / (nodes[t] - nodes[j])
    return M


def centre(start, n):
    """Index of a node [start, start+n) closest to the mean index (lower on ties)."""
    return start + (n - 1) // 2


# ------------------------------------------------------------ butterfly ----
class Kernel:
    """e^{2 pi i Phi} of one of the built-in phase kinds of oracle/direct.c."""

    def __init__(self, kind, N, s=1.0):
        self.kind, self.N, self.s = kind, N, s

    def e(self, i, j, sign=1):
        return _d.expphase(self.kind, self.N, i, j, sign=sign, s=self.s)


def butterfly(kern, y, r, n0=1):
    """u ~ e^{2 pi i Phi} y by Algorithm 4.1 (steps 1-6), FP64.

    ``y`` is (N,) or (N, m) complex; returns the same shape.
    """
    N = kern.N
    y = np.asarray(y, dtype=np.complex128)
    vec = y.ndim == 1
    Y = y.reshape(N, -1)
    L = int(round(np.log2(N // n0)))
    assert n0 * 2 ** L == N and L >= 1
    h = L // 2
    E = kern.e

    # Step 1: trees.  Level-l node a of T_X covers rows [a N/2^l, (a+1) N/2^l);
    # level-l node b of T_Omega covers columns [b N/2^l, (b+1) N/2^l).

    # Step 2 (Eq. 1): A = root of T_X, B = each leaf of T_Omega.
    #   lambda^{AB}_t = e^{-2 pi i Phi(c_A, xi^B_t)} sum_{xi in B} M^B_t(xi) e^{2 pi i Phi(c_A, xi)} y(xi)
    nb = n0
    nB = N // nb
    gB = grid(nb, r)
    cA = centre(0, N)
    cols = np.arange(nB)[:, None] * nb + np.arange(nb)[None, :]            # [B, xi]
    MB = lagrange(gB, np.arange(nb))                                          # [t, xi]
    inner = np.einsum('tk,bkc->btc', MB, E(cA, cols)[:, :, None] * Y[cols])
    lam = (E(cA, np.arange(nB)[:, None] * nb + gB[None, :], -1)[:, :, None] * inner)[None]
    # lam[a, b, t, col]: pairs (A_a at level 0, B_b at level L)

    # Step 3 (Eq. 2), l = 1..h: P = parent of A, C = children of B.
    #   lambda^{AB}_t = e^{-2 pi i Phi(c_A, xi^B_t)} sum_{C > B} sum_s M^B_t(xi^C_s) e^{2 pi i Phi(c_A, xi^C_s)} lambda^{PC}_s
    for l in range(1, h + 1):
        nA, na = 2 ** l, N // 2 ** l
        nBl, nb = 2 ** (L - l), N // 2 ** (L - l)
        gB, gC = grid(nb, r), grid(nb // 2, r)
        assert lam.shape[2] == gC.size
        xiC = np.concatenate([gC, gC + nb // 2])                             # xi^C_s, both children
        MBC = lagrange(gB, xiC)                                               # M^B_t(xi^C_s)
        cA = centre(np.arange(nA) * na, na)
        lamPC = lam.reshape(nA // 2, nBl, 2 * gC.size, -1)[np.arange(nA) // 2]
        ph_in = E(cA[:, None, None], (np.arange(nBl)[:, None] * nb + xiC[None, :])[None])
        s = np.einsum('ts,absc->abtc', MBC, ph_in[..., None] * lamPC)
        ph_out = E(cA[:, None, None], (np.arange(nBl)[:, None] * nb + gB[None, :])[None], -1)
        lam = ph_out[..., None] * s

    # Step 4 (switch), l = h: lambda^{AB}_t := sum_s e^{2 pi i Phi(x^A_t, xi^B_s)} lambda^{AB}_s
    nA, na = 2 ** h, N // 2 ** h
    nBl, nb = 2 ** (L - h), N // 2 ** (L - h)
    gA, gB = grid(na, r), grid(nb, r)
    assert lam.shape[2] == gB.size
    xA = np.arange(nA)[:, None] * na + gA[None, :]
    xiB = np.arange(nBl)[:, None] * nb + gB[None, :]
    K = E(xA[:, None, :, None], xiB[None, :, None, :])                        # [a, b, t, s]
    lam = np.einsum('abts,absc->abtc', K, lam)

    # Step 5 (Eq. 3), l = h+1..L:
    #   lambda^{AB}_t = sum_{C > B} e^{2 pi i Phi(x^A_t, c_C)} sum_s M^P_s(x^A_t) e^{-2 pi i Phi(x^P_s, c_C)} lambda^{PC}_s
    for l in range(h + 1, L + 1):
        nA, na = 2 ** l, N // 2 ** l
        nP, npar = nA // 2, 2 * na
        nBl, nb = 2 ** (L - l), N // 2 ** (L - l)
        nc = nb // 2
        gA, gP = grid(na, r), grid(npar, r)
        assert lam.shape[2] == gP.size
        lamPC = lam.reshape(nP, nBl, 2, gP.size, -1)                          # [P, B, C, s, col]
        xP = np.arange(nP)[:, None] * npar + gP[None, :]
        cC = centre(np.arange(2 * nBl) * nc, nc).reshape(nBl, 2)
        v = E(xP[:, None, None, :], cC[None, :, :, None], -1)[..., None] * lamPC
        new = np.zeros((nA, nBl, gA.size, Y.shape[1]), dtype=np.complex128)
        for pos in (0, 1):                                                    # A = child pos of P
            MPA = lagrange(gP, gA + pos * na)                                  # M^P_s(x^A_t) [s, t]
            w = np.einsum('st,pbcsk->pbctk', MPA, v)
            xAt = (2 * np.arange(nP) + pos)[:, None] * na + gA[None, :]
            ph = E(xAt[:, None, None, :], cC[None, :, :, None])
            new[pos::2] = (ph[..., None] * w).sum(axis=2)
        lam = new

    # Step 6 (Eq. bf3): B = root of T_Omega, A = each leaf of T_X.
    #   u(x) = e^{2 pi i Phi(x, c_B)} sum_t M^A_t(x) e^{-2 pi i Phi(x^A_t, c_B)} lambda^{AB}_t
    nA, na = 2 ** L, n0
    gA = grid(na, r)
    cB = centre(0, N)
    MA = lagrange(gA, np.arange(na))                                          # [t, x]
    xAt = np.arange(nA)[:, None] * na + gA[None, :]
    v = E(xAt, cB, -1)[..., None] * lam[:, 0]
    u = np.einsum('tk,atc->akc', MA, v)
    rows = np.arange(nA)[:, None] * na + np.arange(na)[None, :]
    u = E(rows, cB)[..., None] * u
    u = u.reshape(N, -1)
    return u[:, 0] if vec else u


def ibf_apply(kind, N, F, r, a, b, n0=1, s=1.0):
    """g = sum_k diag(a_k) BF(diag(b_k) F)  (Eq. tg), BF = Algorithm 4.1.

    ``a``, ``b`` are (r_alpha, N) with alpha(x_i, xi_j) ~ sum_k a[k, i] b[k, j].
    ``F`` is (N,) or (N, m).
    """
    F = np.asarray(F, dtype=np.complex128)
    vec = F.ndim == 1
    F2 = F.reshape(N, -1)
    kern = Kernel(kind, N, s)
    g = np.zeros_like(F2)
    for k in range(a.shape[0]):
        g += a[k][:, None] * butterfly(kern, b[k][:, None] * F2, r, n0)
    return g[:, 0] if vec else g
