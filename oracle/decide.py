"""Oracle: Algorithm 6 of Sec. 3 -- may the transform be evaluated by r-dimensional
NUFFTs after dimension lifting, or does it need the butterfly?

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper lifts the phase: if Phi ~ sum_{l<r} P_l(x) Q_l(xi) leaves a residual
kernel alpha e^{2 pi i (Phi - P Q^T)} of low rank r_eps, then g is r_eps
r-dimensional NUFFTs (Eq. tg3).  Algorithm 6 decides this in O(N) from low-rank
factorizations of the phase and amplitude matrices:

1. the r-leading SVD of the phase factorization U1 V1^T gives P Sigma Q^T; P Sigma -> P;
2. r_eps q random columns of the residual kernel are stacked into M, and M is
   factored by QR with column pivoting;
3. n = the number of diagonal entries of R above eps |R(1,1)|; y = 1 iff n < r_eps;
4. if y = 1, Algorithm 1 gives the residual kernel as U V^T with rank parameter r_eps.

Readings (where the printed algorithm is garbled or leaves a choice):
* Step 2 samples "r q" columns and step 3 tests "n < r"; with r <= 3 (the NUFFT
  dimensions) and r_eps up to O(100) (the paper's own remark), the sample and the
  test are read with r_eps: r_eps q columns, y = 1 iff n < r_eps.  Step 4's Algorithm 1
  runs with that same rank parameter r_eps.
* Step 1's r-leading SVD of a rank-r1 factorization is taken exactly: QR of both
  factors, then the SVD of the r1 x r1 core (a randomized truncated SVD converges to
  it).  numpy's QR and SVD serve as the library steps.  With r >= r1, P Q^T is the
  whole phase and the residual phase is zero.
* Factor conventions follow this package's other modules: phase Psi = P1^T Q1 and
  amplitude alpha = A2^T B2, factors stored as rows ([rank][N]); the paper's U1 V1^*
  is P1^T Q1.

Parity: pinned in tests/test_oracle_pins.py by the exact rank-2 lifting of the FIO
phase (n = the amplitude rank), by brute force (the numerical rank of the whole
residual kernel by SVD) at small N, and by the residual of a rank-1 lifting of that
phase being full rank.
"""
import numpy as np
import scipy.linalg as sla

from . import lowrank


def lifting(P1, Q1, r):
    """Step 1: (P, Q) of shape (r', N) with P^T Q the best rank-r' approximation of
    P1^T Q1, r' = min(r, rank); P carries the singular values."""
    Qa, Ra = np.linalg.qr(np.asarray(P1).T)
    Qb, Rb = np.linalg.qr(np.asarray(Q1).T)
    Uc, S, Vch = np.linalg.svd(Ra @ Rb.T)
    k = min(r, S.size)
    P = (Qa @ Uc[:, :k] * S[:k]).T
    Q = (Qb @ Vch[:k].T).T
    return P, Q


def residual_kernel(P1, Q1, A2, B2, P, Q, I, J):
    """alpha e^{2 pi i (Psi - P^T Q)} at rows I, columns J (complex128)."""
    I, J = np.asarray(I), np.asarray(J)
    amp = A2[:, I].T @ B2[:, J]
    ph = P1[:, I].T @ Q1[:, J] - P[:, I].T @ Q[:, J]
    ph = ph - np.rint(ph)
    return amp * np.exp(2j * np.pi * ph)


def nufft_decide(P1, Q1, A2, B2, r, r_eps, q=5, eps=1e-10, seed=0):
    """Algorithm 6.  Returns (y, n, terms): y = 1 if r-dimensional NUFFTs apply, n the
    numerical rank of the sampled residual columns, terms the rank of step 4's
    factorization (the number of NUFFTs; 0 when y = 0)."""
    P1, Q1 = np.real(np.asarray(P1)), np.real(np.asarray(Q1))
    A2, B2 = np.asarray(A2), np.asarray(B2)
    N = P1.shape[1]
    P, Q = lifting(P1, Q1, r)
    rng = np.random.default_rng(seed)
    J = np.sort(rng.choice(N, min(N, r_eps * q), replace=False))
    M = residual_kernel(P1, Q1, A2, B2, P, Q, np.arange(N), J)
    R = sla.qr(M, mode='r', pivoting=True)[0]
    d = np.abs(np.diag(R))
    n = int(np.sum(d > eps * d[0])) if d.size and d[0] > 0 else 0
    y = int(n < r_eps)
    terms = 0
    if y:
        a, _ = lowrank.amplitude_split(lambda I, J: residual_kernel(P1, Q1, A2, B2, P, Q, I, J), N, N,
                                       tol=eps, r=r_eps, q=q, seed=seed)
        terms = a.shape[0]
    return y, n, terms
