"""GPU parity of the NUFFT evaluation (bf_nufft_apply, Sec. 3 Eq. tg3 with the
column halves split at xi = 0 as in Eq. FIOwq2) through the C ABI.

Two oracles:
  (i) oracle/nufft.py, the same Gaussian gridding with the same msp in FP64:
      the difference is FP32 rounding only.  Tolerance 2e-6: the deconvolution
      (one complex product), 2 log2 N radix-2 butterfly levels with unit-modulus
      twiddles, and an interpolation sum of 2 msp positive weights of total
      ~1: about 2 log2 N + 2 msp + 4 rounding steps of relative size
      u = 2^-24, i.e. 6e-8 * sqrt(50) ~ 4e-7 as a random walk and ~3e-6 in the
      worst case; 2e-6 sits between.
  (ii) the direct FP64 sum (oracle/direct.c): 1e-5, the stated FP32 target
      (the NUFFT's own error at eps = 1e-6 is below 2e-7).
Both amplitude splits (the library's Algorithm 1 and the oracle's) reproduce
the amplitude to ~1e-13, far below either tolerance.
"""
import numpy as np
import pytest

from conftest import relerr
from oracle import direct as od
from oracle import lowrank as olr
from oracle import nufft as onu
from paper_1803_04128_gb300 import _lib as L
from paper_1803_04128_gb300 import api, inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ORACLE_KIND = {L.PHASE_FIO: (onu.FIO, od.FIO), L.PHASE_FIO_PW: (onu.FIOPW, od.FIOPW),
               L.PHASE_DFT: (onu.DFT, od.DFT)}


@pytest.fixture(scope="module", autouse=True)
def gpu_ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1803_04128_gb300 import build
    build.build()
    torch.cuda.init()


def gpu_nufft(plan, F):
    Ft = torch.from_numpy(np.ascontiguousarray(F)).to(torch.complex64).cuda()
    G = plan.nufft_apply(Ft)
    torch.cuda.synchronize()
    return G.cpu().numpy().astype(np.complex128)


def oracle_nufft(kind, N, F, msp, amp=1):
    ent = lambda I, J: od.amplitude(amp, N, np.asarray(I)[:, None], np.asarray(J)[None, :]).astype(np.complex128)
    a, b = olr.amplitude_split(ent, N, N)
    return onu.apply(ORACLE_KIND[kind][0], N, F, a, b, msp)


@pytest.mark.parametrize("N,m", [(256, 1), (1024, 3), (2048, 64), (4096, 5), (8192, 130), (32768, 2)])
@pytest.mark.parametrize("kind", [L.PHASE_FIO, L.PHASE_FIO_PW, L.PHASE_DFT])
def test_nufft_matches_oracle_gridding(N, m, kind):
    plan = api.Plan(N, eps=1e-6, phase_kind=kind, amp_kind=L.AMP_SMOOTH, factor=False)
    msp = plan.nufft_prepare(1e-6)
    assert msp == 7
    F = inputs.complex_gaussian(N, m, seed=N + m + kind)
    g = gpu_nufft(plan, F)
    assert relerr(g, oracle_nufft(kind, N, F, msp)) < 2e-6
    gd = od.direct(ORACLE_KIND[kind][1], N, F, None if N <= 8192 else inputs.sample_rows(N, 256, seed=1), amp=1)
    rows = slice(None) if N <= 8192 else inputs.sample_rows(N, 256, seed=1)
    assert relerr(g[rows], gd) < 1e-5
    plan.close()


@pytest.mark.parametrize("eps", [1e-3, 1e-5, 1e-8])
def test_nufft_error_follows_eps(eps):
    # msp from eps: the error against the direct sum stays below eps (down to FP32 rounding)
    N, m = 4096, 4
    plan = api.Plan(N, eps=1e-6, phase_kind=L.PHASE_FIO, amp_kind=L.AMP_SMOOTH, factor=False)
    msp = plan.nufft_prepare(eps)
    F = inputs.complex_gaussian(N, m, seed=3)
    e = relerr(gpu_nufft(plan, F), od.direct(od.FIO, N, F, None, amp=1))
    assert e < max(eps, 2e-6), (msp, e)
    plan.close()


@pytest.mark.parametrize("N,m,kind", [(65536, 64, L.PHASE_FIO), (262144, 256, L.PHASE_FIO_PW),
                                      (1 << 20, 4, L.PHASE_FIO)])
def test_nufft_full_size_sampled_rows(N, m, kind):
    # the configurations' shapes (and the largest N the NUFFT takes): sampled rows vs direct
    plan = api.Plan(N, eps=1e-6, phase_kind=kind, amp_kind=L.AMP_SMOOTH, factor=False)
    plan.nufft_prepare(1e-6)
    F = inputs.complex_gaussian(N, m, seed=7)
    g = gpu_nufft(plan, F)
    rows = inputs.sample_rows(N, 96 if N < (1 << 20) else 48, seed=2)
    gd = od.direct(ORACLE_KIND[kind][1], N, F, rows, amp=1)
    assert relerr(g[rows], gd) < 1e-5
    plan.close()


def test_nufft_matches_butterfly_apply():
    # the two evaluations of Sec. 3 and Sec. 4 of the same operator agree to their tolerances
    N, m = 16384, 16
    plan = api.Plan(N, eps=1e-6, phase_kind=L.PHASE_FIO, amp_kind=L.AMP_SMOOTH)
    plan.nufft_prepare(1e-6)
    F = torch.from_numpy(inputs.complex_gaussian(N, m, seed=11)).to(torch.complex64).cuda()
    gb = plan.apply(F, prec=api.F32)
    gn = plan.nufft_apply(F)
    torch.cuda.synchronize()
    assert float((gb - gn).norm() / gb.norm()) < 2e-6 + 2e-6
    plan.close()


def test_nufft_refusals():
    p = api.Plan(4096, eps=1e-6, phase_kind=L.PHASE_SEP, factor=False)
    with pytest.raises(L.BFError) as e:
        p.nufft_prepare(1e-6)
    assert e.value.status == L.BF_ERR_UNSUPPORTED
    q = api.Plan(4096, eps=1e-6, phase_kind=L.PHASE_FIO, factor=False)
    F = torch.zeros((4096, 2), dtype=torch.complex64, device="cuda")
    with pytest.raises(L.BFError) as e:
        q.nufft_apply(F)
    assert e.value.status == L.BF_ERR_STATE
    p.close()
    q.close()
