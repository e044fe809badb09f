"""Oracle: low-rank phase recovery from kernel entries (Sec. 2.2, Algorithms 3, 4, 5).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Scenario 1 of Table sc: K(x_i, xi_j) = alpha e^{2 pi i Phi} is known only through
its entries.  Only Phi mod 1 can be read off K / |K|.  The three algorithms
recover rows and columns of a Psi with Psi = Phi mod 1 that is smooth on each
block between discontinuities, hence low rank:

* ``unwrap``: Algorithm 3.  A vector v is rebuilt from u = v mod 1, entry by
  entry.  The first entry is u itself.  The second is the one nearest the
  first.  The third makes the second difference match the first's.  Every
  later one makes the third difference as small as it can be.  A second
  difference above tau marks a discontinuity, and the vector restarts there.
* ``PsiSampler``: Algorithm 4.  The discontinuities of one sampled column and
  one sampled row cut Psi into blocks.  In each block Algorithm 3 rebuilds
  the first row, then the first three columns, then the rows and columns.  Each one starts from values already fixed, so rows and
  columns agree where they cross.
* ``phase_lowrank``: Algorithm 5.  Algorithm 1 (oracle/lowrank.py) is run on
  Psi, whose rows and columns the sampler rebuilds on demand.

Readings (where the paper leaves a choice):
* tau is compared with second differences of Phi in turns.  The paper's
  tau = pi/2 is read as pi/2 of the phase 2 pi Phi, i.e. 1/4 turn.  After the
  nearest-integer choices a second difference of pi/2 turns could never occur.
* Inside a block, tau = 2 pi (of 2 pi Phi) = 1 turn, as in Algorithm 4.
* The second and third columns of a block are rebuilt through their
  differences with the column before.  Those differences are unwrapped along
  x from the first row's differences.  This is the reading of "no
  discontinuity along rows inside the first three columns".  It keeps the
  three columns' integer slopes equal even where one column's slope is a tie,
  e.g. the DFT's first column xi = -N/2, whose slope is exactly half a turn.
* The rows and columns of a block are seeded from its first three columns
  and its first three rows.  So any row or column can be rebuilt
  consistently, not only the sampled ones.
* Nearest integer: round half to even (numpy.rint); ties have measure zero.
"""
import numpy as np

from . import lowrank

TAU_DETECT = 0.25  # pi/2 of 2 pi Phi, in turns
TAU_BLOCK = 1.0    # 2 pi of 2 pi Phi, in turns


def predict(v, a):
    """The value at a that makes the third difference v[a] - 3 v[a-1] + 3 v[a-2] - v[a-3] zero."""
    return 3 * v[a - 1] - 3 * v[a - 2] + v[a - 3]


def unwrap(u, tau, seed=()):
    """Algorithm 3: v with v = u mod 1 from u (values in [0, 1)).

    ``seed``: up to 3 leading values already fixed (Algorithm 4 passes them).
    Returns (v, S) with S the start indices of the smooth pieces (S[0] = 0).
    """
    u = np.asarray(u, dtype=np.float64)
    n = u.size
    v = np.empty(n)
    S = [0]
    if n == 0:
        return v, S

    def near(p, a):  # the value of u[a] + integer nearest the prediction p
        return u[a] + np.rint(p - u[a])

    seed = list(seed)
    k = len(seed)
    # first piece: v[0], v[1], v[2]
    v[0] = seed[0] if k >= 1 else u[0]
    if n > 1:
        v[1] = seed[1] if k >= 2 else near(v[0], 1)           # |v1 - v0| smallest
    if n > 2:
        v[2] = seed[2] if k >= 3 else near(2 * v[1] - v[0], 2)  # v2 - v1 nearest v1 - v0
    a = 3
    while a < n:
        # third difference smallest: v[a] + v[a-2] - 2 v[a-1] nearest v[a-1] + v[a-3] - 2 v[a-2]
        v[a] = near(predict(v, a), a)
        if abs(v[a] + v[a - 2] - 2 * v[a - 1]) > tau:
            # a discontinuity at a: a new piece starts there
            S.append(a)
            st = a
            v[st] = near(v[st - 1], st)                        # nearest the entry before it
            if st + 1 < n:
                v[st + 1] = near(2 * v[st] - v[st - 1], st + 1)  # slope continued
            a = st + 2
            continue
        a += 1
    return v, S


def phase_turns(K):
    """Phi mod 1 in [0, 1) from entries K = alpha e^{2 pi i Phi} (alpha > 0)."""
    t = np.angle(K) / (2 * np.pi)
    return t - np.floor(t)


class PsiSampler:
    """Algorithm 4 on the N x N phase matrix seen through ``entry(I, J)`` (complex K).

    ``C``, ``R``: sampled column and row indices; the first of each finds the
    discontinuities.  ``row(i)`` and ``col(j)`` return full rows/columns of Psi.
    """

    def __init__(self, entry, N, C, R, tau=TAU_DETECT, tau_block=TAU_BLOCK):
        self.entry, self.N, self.tau_block = entry, N, tau_block
        allidx = np.arange(N)
        _, Sr = unwrap(self._u(allidx, [C[0]])[:, 0], tau)
        _, Sc = unwrap(self._u([R[0]], allidx)[0], tau)
        self.rb = list(Sr) + [N]   # row blocks [rb[k], rb[k+1])
        self.cb = list(Sc) + [N]   # column blocks
        self.colseed, self.rowseed = {}, {}
        for bi in range(len(self.rb) - 1):
            r0, r1 = self.rb[bi], self.rb[bi + 1]
            for bj in range(len(self.cb) - 1):
                c0, c1 = self.cb[bj], self.cb[bj + 1]
                # the block's first row
                first, _ = unwrap(self._u([r0], np.arange(c0, c1))[0], tau_block)
                # its first three columns: the first from the first row's value, the
                # second and third through their differences with the column before,
                # unwrapped from the first row's differences, so that along every row
                # the three values are continuous
                nc = min(3, c1 - c0)
                ucols = self._u(np.arange(r0, r1), np.arange(c0, c0 + nc))
                cols = [unwrap(ucols[:, 0], tau_block, seed=[first[0]])[0]]
                for t in range(1, nc):
                    dt = ucols[:, t] - ucols[:, t - 1]
                    dt = dt - np.floor(dt)
                    cols.append(cols[-1] + unwrap(dt, tau_block, seed=[first[t] - first[t - 1]])[0])
                self.colseed[bi, bj] = np.stack(cols)
                # its first three rows, from the first three columns
                nr = min(3, r1 - r0)
                self.rowseed[bi, bj] = np.stack([self._row_block(r0 + t, bi, bj) for t in range(nr)])

    def _u(self, I, J):
        return phase_turns(self.entry(np.asarray(I), np.asarray(J)))

    def _block(self, edges, i):
        return int(np.searchsorted(edges, i, side='right') - 1)

    def _row_block(self, i, bi, bj, u=None):
        r0 = self.rb[bi]
        c0, c1 = self.cb[bj], self.cb[bj + 1]
        if u is None:
            u = self._u([i], np.arange(c0, c1))[0]
        return unwrap(u, self.tau_block, seed=list(self.colseed[bi, bj][:, i - r0]))[0]

    def row(self, i):
        bi = self._block(self.rb, i)
        u = self._u([i], np.arange(self.N))[0]
        return np.concatenate([self._row_block(i, bi, bj, u[self.cb[bj]:self.cb[bj + 1]])
                               for bj in range(len(self.cb) - 1)])

    def col(self, j):
        bj = self._block(self.cb, j)
        c0 = self.cb[bj]
        u = self._u(np.arange(self.N), [j])[:, 0]
        parts = []
        for bi in range(len(self.rb) - 1):
            r0, r1 = self.rb[bi], self.rb[bi + 1]
            parts.append(unwrap(u[r0:r1], self.tau_block, seed=list(self.rowseed[bi, bj][:, j - c0]))[0])
        return np.concatenate(parts)

    def entries(self, I, J):
        """Psi[I][:, J], built from whole rows (or whole columns when fewer)."""
        I, J = np.asarray(I), np.asarray(J)
        if I.size <= J.size:
            return np.stack([self.row(i)[J] for i in I])
        return np.stack([self.col(j)[I] for j in J], axis=1)


def phase_lowrank(entry, N, r=20, q=5, seed=0, tol=1e-13, tau=TAU_DETECT):
    """Algorithm 5 (Scenario 1): (P, Q) with Psi ~ P^T Q and e^{2 pi i Psi} ~ e^{2 pi i Phi}.

    P: (r_phi, N), Q: (r_phi, N), real up to rounding.  The C and R samples of
    Algorithm 4 are rq random columns and rows (seeded); Algorithm 1 then draws
    the rows and columns it needs from the sampler.
    """
    rng = np.random.default_rng(seed)
    C = rng.choice(N, min(N, r * q), replace=False)
    R = rng.choice(N, min(N, r * q), replace=False)
    sampler = PsiSampler(entry, N, C, R, tau=tau)
    a, b = lowrank.amplitude_split(lambda I, J: sampler.entries(I, J).astype(np.complex128), N, N,
                                   tol=tol, r=r, q=q, seed=seed)
    return a, b, sampler
