"""Test helper: evaluate a plan's exported FP64 factors stage by stage in numpy.

This reads the factor arrays through bf_plan_view and applies them with the
stage formulas of the factored form (V, H levels, switch, G levels, U), so
that the host construction can be compared with the oracle's Algorithm 4.1
on the CPU, before and independently of the CUDA kernels.
"""
import numpy as np


def apply_block(plan, F, block=0):
    info = plan.info()
    r, L, h, l1 = info["r"], info["L"], info["h"], info["l1"]
    n0 = info["n0"]
    a = plan.view(0, block=block)
    b = plan.view(1, block=block)
    N = F.shape[0]
    ra = a.size // N
    a = a.reshape(ra, N); b = b.reshape(ra, N)
    nv = n0 << l1
    P = N // n0
    Mv = plan.view(2, block=block).reshape(r, nv)
    EV = plan.view(3, block=block).reshape(1 << l1, N)
    out = np.zeros_like(F, dtype=np.complex128)
    for k in range(ra):
        Y = b[k][:, None] * F                                              # [N, m]
        # V: mu[a, b, t] = sum_x Mv[t, x] EV[a, b nv + x] Y[b nv + x]
        Yb = Y.reshape(P >> l1, nv, -1)                                     # [b, x, m]
        Eb = EV.reshape(1 << l1, P >> l1, nv)                               # [a, b, x]
        mu = np.einsum('tx,abx,bxm->abtm', Mv, Eb, Yb).reshape(P, r, -1)
        for l in range(l1 + 1, h + 1):
            MH = plan.view(4, l, block).reshape(r, 2 * r)
            EH = plan.view(5, l, block).reshape(P, 2 * r)
            nB = 1 << (L - l)
            q = np.arange(P); A = q // nB; B = q % nB
            qin0 = (A >> 1) * 2 * nB + 2 * B
            lam = np.concatenate([mu[qin0], mu[qin0 + 1]], axis=1)          # [P, 2r, m]
            mu = np.einsum('ts,qsm->qtm', MH, EH[:, :, None] * lam)
        S = plan.view(6, block=block).reshape(P, r, r)
        nu = np.einsum('qts,qsm->qtm', S, mu)
        for l in range(h + 1, L - l1 + 1):
            MG = plan.view(7, l, block).reshape(2, r, r)
            FG = plan.view(8, l, block).reshape(P, 2, r)
            nB = 1 << (L - l)
            q = np.arange(P); A = q // nB; B = q % nB
            qin0 = (A >> 1) * 2 * nB + 2 * B
            Mp = MG[A & 1]                                                   # [P, r, r]
            w0 = np.einsum('qts,qsm->qtm', Mp, nu[qin0])
            w1 = np.einsum('qts,qsm->qtm', Mp, nu[qin0 + 1])
            nu = FG[:, 0, :, None] * w0 + FG[:, 1, :, None] * w1
        MU = plan.view(9, block=block).reshape(nv, r)
        EU = plan.view(10, block=block).reshape(1 << l1, N)
        nuA = nu.reshape(P >> l1, 1 << l1, r, -1)                           # [A, C, s, m]
        w = np.einsum('is,acsm->acim', MU, nuA)                              # [A, C, i, m]
        EUr = EU.reshape(1 << l1, P >> l1, nv).transpose(1, 0, 2)            # [A, C, i]
        u = np.einsum('aci,acim->aim', EUr, w).reshape(N, -1)
        out += a[k][:, None] * u
    return out


def apply(plan, F):
    info = plan.info()
    if info["split"] == 1:
        return apply_block(plan, F)
    N = F.shape[0]; Nb = N // 2
    out = np.zeros_like(F, dtype=np.complex128)
    for rh in range(2):
        for ch in range(2):
            out[rh * Nb:(rh + 1) * Nb] += apply_block(plan, F[ch * Nb:(ch + 1) * Nb], 2 * rh + ch)
    return out
