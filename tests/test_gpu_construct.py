"""GPU tests of bf_factor_device: the phase tables built on the device.

The device tables are the host construction's formulas evaluated in FP64 on
the GPU, so a plan built either way applies to the same result up to rounding.
The host evaluates c(x) = (2 + s sin 2 pi x)/16 with a rounded argument 2 pi x
(a few ulp of error in sin), and that error is multiplied by |xi| <= N/2 in the
phase c(x)|xi|: at N = 4096 about 2048/16 x 4.4e-16 x 2 pi ~ 3.5e-13 rad per
entry.  The device uses sinpi(2 i / N), exact in its argument.  Hence FP64
applies agree to 1e-12, FP32 applies to 1e-6, and against the direct oracle
the usual FP32 bound holds.
"""
import numpy as np
import pytest

from conftest import relerr
from oracle import direct as od
from paper_1803_04128_gb300 import _lib as L
from paper_1803_04128_gb300 import api, inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def gpu_ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1803_04128_gb300 import build
    build.build()


def apply(plan, F, prec):
    dt = torch.complex128 if prec == api.F64 else torch.complex64
    G = plan.apply(torch.from_numpy(F).to(dt).cuda(), prec=prec)
    torch.cuda.synchronize()
    return G.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("kind,amp,split", [(L.PHASE_FIO, L.AMP_SMOOTH, 1), (L.PHASE_FIO_PW, L.AMP_SMOOTH, 2),
                                            (L.PHASE_DFT, L.AMP_ONE, 1), (L.PHASE_SEP, L.AMP_ONE, 1),
                                            (L.PHASE_ONES, L.AMP_SMOOTH, 1)])
def test_device_tables_match_host_construction(kind, amp, split):
    N, m = 4096, 3
    ph = api.Plan(N, r=10, phase_kind=kind, amp_kind=amp, split=split)
    pd = api.Plan(N, r=10, phase_kind=kind, amp_kind=amp, split=split, factor_on_device=True)
    F = inputs.complex_gaussian(N, m, seed=5)
    assert relerr(apply(pd, F, api.F64), apply(ph, F, api.F64)) < 1e-12
    assert relerr(apply(pd, F, api.F32), apply(ph, F, api.F32)) < 1e-6


def test_device_factored_fio2_shape_vs_direct():
    N, m = 65536, 4
    pd = api.Plan(N, eps=1e-6, phase_kind=L.PHASE_FIO, amp_kind=L.AMP_SMOOTH, factor_on_device=True)
    F = inputs.complex_gaussian(N, m, seed=6)
    rows = inputs.sample_rows(N, 64, seed=7)
    gd = od.direct(od.FIO, N, F, rows, amp=1)
    assert relerr(apply(pd, F, api.F32)[rows], gd) < 1e-5


def test_device_factor_refusals(tmp_path):
    with pytest.raises(L.BFError) as e:
        api.Plan(1024, r=10, phase_kind=L.PHASE_USER, phi=lambda x, xi: x * xi, factor_on_device=True)
    assert e.value.status == L.BF_ERR_UNSUPPORTED
    pd = api.Plan(1024, r=10, factor_on_device=True)
    with pytest.raises(L.BFError) as e:
        pd.save(str(tmp_path / "plan.bin"))
    assert e.value.status == L.BF_ERR_STATE
