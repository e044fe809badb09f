"""Oracle: the Hankel-function transform of Sec. 5 (Eq. HK), in FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

g_i = sum_j H^(1)_j(x_i) f_j with x_i = N + 2 pi i / 3, i, j = 0 .. N-1 (the 0-based
form of the paper's x_i = N + 2 pi (i-1)/3 and orders j-1).  Every argument exceeds
every order, so each entry lies in the oscillatory regime, where H = |H| e^{i arg H}
has a smooth amplitude and phase.  scipy.special.hankel1 evaluates the entries (a
library routine standing for a step); tests/test_oracle_pins.py pins it with the
Wronskian and the three-term recurrence of the Bessel functions.
"""
import numpy as np
from scipy.special import hankel1


def hankel_x(N, i):
    return N + 2.0 * np.pi * np.asarray(i, dtype=np.float64) / 3.0


def hankel_entries(N, rows, cols):
    """K[rows][:, cols] = H^(1)_j(x_i) as a complex128 matrix."""
    rows = np.asarray(rows)
    cols = np.asarray(cols)
    return hankel1(cols.astype(np.float64)[None, :], hankel_x(N, rows)[:, None])


def hankel_direct(N, F, rows=None):
    """g = K F on the given rows (all rows if None), plain dense products."""
    rows = np.arange(N) if rows is None else np.asarray(rows)
    F = np.asarray(F, dtype=np.complex128).reshape(N, -1)
    out = np.empty((rows.size, F.shape[1]), dtype=np.complex128)
    for s in range(0, rows.size, 256):
        out[s:s + 256] = hankel_entries(N, rows[s:s + 256], np.arange(N)) @ F
    return out
