"""Oracle: Algorithm 1 (randomised sampling rank-r approximate SVD), Sec. 2.1.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Used by the oracle to split the amplitude alpha(x, xi) ~ sum_k a_k(x) b_k(xi)
for Eq. (tg).  Steps follow Algorithm 1 in order; scipy's pivoted QR and
numpy's pseudo-inverse and SVD serve as the library steps the algorithm names.
"""
import numpy as np
import scipy.linalg as sla


def rsvd_sampled(entry, m, n, r, q=5, sweeps=2, seed=0):
    """K ~ U0 diag(S0) V0^* from sampled rows/columns of K (Algorithm 1).

    ``entry(I, J)`` returns K[I][:, J] for index arrays I, J.
    Returns (U0 [m, r'], S0 [r'], V0 [n, r']) with r' <= r.
    """
    rng = np.random.default_rng(seed)
    pi_col = np.zeros(0, dtype=np.int64)
    pi_row = np.zeros(0, dtype=np.int64)
    allr, allc = np.arange(m), np.arange(n)
    for _ in range(sweeps):
        # rq random rows plus the important rows; pivoted QR of K(I, :) picks columns
        I = np.union1d(rng.choice(m, min(m, r * q), replace=False), pi_row)
        _, _, piv = sla.qr(entry(I, allc), mode='economic', pivoting=True)
        pi_col = np.sort(piv[:min(r, piv.size)])
        # rq random columns plus the important columns; pivoted LQ of K(:, J) picks rows
        J = np.union1d(rng.choice(n, min(n, r * q), replace=False), pi_col)
        _, _, piv = sla.qr(entry(allr, J).conj().T, mode='economic', pivoting=True)
        pi_row = np.sort(piv[:min(r, piv.size)])
    # column and row bases: the leading r columns of Q, with r capped at the
    # numerical rank the pivoted QR reveals (|R_kk| > 1e-14 |R_00|); columns past
    # it span nothing of K and would make the sampled core below singular.
    def basis(A):
        Q, R, _ = sla.qr(A, mode='economic', pivoting=True)
        d = np.abs(np.diag(R))
        k = int(np.sum(d > 1e-14 * d[0])) if d.size and d[0] > 0 else 0
        return Q[:, :min(r, max(k, 1))]
    Qc = basis(entry(allr, pi_col))
    Qr = basis(entry(pi_row, allc).conj().T)
    # core from a few extra sampled rows/columns
    J = np.union1d(pi_col, rng.choice(n, min(n, r * q), replace=False))
    I = np.union1d(pi_row, rng.choice(m, min(m, r * q), replace=False))
    M = np.linalg.pinv(Qc[I, :]) @ entry(I, J) @ np.linalg.pinv(Qr.conj().T[:, J])
    # thin SVD: the column and row bases may have different numerical ranks, and
    # U0 = Qc U_M, S0, V0 = Qr V_M then all have min of the two columns
    UM, SM, VMh = np.linalg.svd(M, full_matrices=False)
    return Qc @ UM, SM, (VMh @ Qr.conj().T).conj().T


def amplitude_split(entry, m, n, tol=1e-13, r=20, q=5, seed=0):
    """(a, b) of shape (r_alpha, m), (r_alpha, n) with alpha ~ sum_k a_k b_k^T.

    The rank r_alpha keeps the singular values above tol * sigma_1.
    """
    U, S, V = rsvd_sampled(entry, m, n, r=r, q=q, seed=seed)
    keep = S > tol * S[0]
    a = (U[:, keep] * S[keep]).T
    b = V[:, keep].conj().T
    return a, b
