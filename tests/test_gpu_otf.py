"""GPU tests of the on-the-fly apply (bf_factor_otf): no phase tables; the FP32
kernels evaluate every phase factor of Eqs. 1, 2, 3, bf3 and the switch step
of Algorithm 4.1 from the closed form of Phi.

Error budget.  A stored FP32 table entry is the FP64 value rounded to FP32
(relative error <= 2^-24 = 6e-8 per component).  An on-the-fly entry forms
Phi mod 1 exactly as a 32-bit count of turns (argument error < 2^-32 turn =
1.5e-9 rad), takes sincospif of the top 24 bits (about 1 ulp, 1.2e-7) and
rotates by the low 8 bits to first order (dropped term < 1e-13).  Both are at
FP32 rounding level, like the FP32 arithmetic of the apply itself, whose own
error against the FP64 apply is a few 1e-7 at these sizes.  So the on-the-fly
and table FP32 applies agree to 2e-6, both agree with the FP64 apply to 2e-6,
and against the direct oracle the FP32 bound (1e-5 at eps = 1e-6) holds.
The sharded apply runs the same tiles, so it is bitwise the unsharded one.
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


def apply(plan, F, prec=api.F32):
    dt = torch.complex128 if prec == api.F64 else torch.complex64
    G = plan.apply(torch.from_numpy(F).to(dt).cuda(), prec=prec)
    torch.cuda.synchronize()
    assert plan.sync_status() == 0
    return G.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("kind,amp,split", [(L.PHASE_FIO, L.AMP_SMOOTH, 1), (L.PHASE_FIO_PW, L.AMP_SMOOTH, 2),
                                            (L.PHASE_DFT, L.AMP_ONE, 1), (L.PHASE_SEP, L.AMP_ONE, 1),
                                            (L.PHASE_ONES, L.AMP_SMOOTH, 1)])
def test_otf_matches_table_apply(kind, amp, split):
    N, m = 4096, 3
    pt = api.Plan(N, r=10, phase_kind=kind, amp_kind=amp, split=split)
    po = api.Plan(N, r=10, phase_kind=kind, amp_kind=amp, split=split, on_the_fly=True)
    F = inputs.complex_gaussian(N, m, seed=31)
    g64 = apply(pt, F, api.F64)
    go = apply(po, F)
    assert relerr(go, apply(pt, F)) < 2e-6
    assert relerr(go, g64) < 2e-6


@pytest.mark.parametrize("r", [6, 8, 12, 14, 16])
def test_otf_ranks(r):
    N, m = 8192, 2
    pt = api.Plan(N, r=r, phase_kind=L.PHASE_FIO, amp_kind=L.AMP_SMOOTH)
    po = api.Plan(N, r=r, phase_kind=L.PHASE_FIO, amp_kind=L.AMP_SMOOTH, on_the_fly=True)
    F = inputs.complex_gaussian(N, m, seed=r)
    assert relerr(apply(po, F), apply(pt, F, api.F64)) < 2e-6


@pytest.mark.parametrize("m", [1, 5, 64, 200])
def test_otf_column_counts(m):
    # m = 200: several column slices, the last one ragged
    N = 16384
    pt = api.Plan(N, r=10, phase_kind=L.PHASE_FIO, amp_kind=L.AMP_SMOOTH)
    po = api.Plan(N, r=10, phase_kind=L.PHASE_FIO, amp_kind=L.AMP_SMOOTH, on_the_fly=True)
    F = inputs.complex_gaussian(N, m, seed=100 + m)
    assert relerr(apply(po, F), apply(pt, F, api.F64)) < 2e-6


def test_otf_fio2_shape_vs_direct_and_memory():
    N, m = 65536, 4
    po = api.Plan(N, eps=1e-6, phase_kind=L.PHASE_FIO, amp_kind=L.AMP_SMOOTH, on_the_fly=True)
    pt = api.Plan(N, eps=1e-6, phase_kind=L.PHASE_FIO, amp_kind=L.AMP_SMOOTH).upload()
    F = inputs.complex_gaussian(N, m, seed=41)
    rows = inputs.sample_rows(N, 64, seed=42)
    gd = od.direct(od.FIO, N, F, rows, amp=1)
    assert relerr(apply(po, F)[rows], gd) < 1e-5
    io, it = po.info(), pt.info()
    # O(N): 16 B of phase coefficients per row, a_k and b_k, small matrices and grids
    assert io["dev_bytes_f64"] == 0
    assert io["dev_bytes_f32"] <= (16 + 2 * 8 * io["r_alpha"]) * N + (1 << 20)
    assert it["dev_bytes_f32"] > 10 * io["dev_bytes_f32"]


def test_otf_large_n_vs_direct():
    # N = 2^20: 20 levels, phases with |xi| up to 2^19
    N, m = 1 << 20, 2
    po = api.Plan(N, eps=1e-6, phase_kind=L.PHASE_FIO, amp_kind=L.AMP_SMOOTH, on_the_fly=True)
    F = inputs.complex_gaussian(N, m, seed=43)
    rows = inputs.sample_rows(N, 12, seed=44)
    gd = od.direct(od.FIO, N, F, rows, amp=1)
    assert relerr(apply(po, F)[rows], gd) < 1e-5


@pytest.mark.parametrize("G", [2, 4])
def test_otf_sharded_equals_unsharded(G):
    N, m = 16384, 6
    po = api.Plan(N, r=10, phase_kind=L.PHASE_FIO, amp_kind=L.AMP_SMOOTH, on_the_fly=True)
    F = torch.from_numpy(inputs.complex_gaussian(N, m, seed=45)).to(torch.complex64).cuda()
    ref = po.apply(F, prec=api.F32)
    sh = api.ShardedApply(po, G, m)
    out = torch.full_like(F, float("nan"))
    sh.apply_local(F, out)
    torch.cuda.synchronize()
    assert po.sync_status() == 0
    assert torch.equal(out, ref)


def test_otf_refusals(tmp_path):
    po = api.Plan(4096, r=10, phase_kind=L.PHASE_FIO, amp_kind=L.AMP_SMOOTH, on_the_fly=True)
    F = torch.zeros((4096, 2), dtype=torch.complex64, device="cuda")
    for prec, dt in ((api.F64, torch.complex128), (api.BF16X3, torch.complex64)):
        with pytest.raises(L.BFError) as e:
            po.apply(F.to(dt), prec=prec)
        assert e.value.status == L.BF_ERR_UNSUPPORTED
    G = torch.empty_like(F)
    with pytest.raises(L.BFError) as e:
        api.Batch([(po, F, G)])
    assert e.value.status == L.BF_ERR_UNSUPPORTED
    srv = api.Server(n_slots=2)
    with pytest.raises(L.BFError) as e:
        srv.add(po)
    assert e.value.status == L.BF_ERR_UNSUPPORTED
    srv.close()
    with pytest.raises(L.BFError) as e:
        po.save(str(tmp_path / "otf.bin"))
    assert e.value.status == L.BF_ERR_STATE
    # the FP32 apply still works after the refusals
    assert torch.equal(po.apply(F, prec=api.F32), torch.zeros_like(F))
