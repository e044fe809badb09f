"""GPU tests of the level passes of the plain FP32 apply.

When kH or kG exceeds 5 levels (N >= 2^20 at r = 10; with on-the-fly phases from
5 levels, N >= 2^17), bf_apply runs the H and G levels in several passes of at most
4 levels each.  The passes share an HBM
workspace.  Every (group, column) item performs the same operations in the same
order in either form, and values round-trip through HBM exactly.  So the split
apply must equal, bit for bit, the single-pass kernels that the batched apply
(table phases) and the one-shard sharded apply (on-the-fly phases) still run.
Accuracy against the FP64 apply and the direct oracle is checked as well.
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


def gauss(N, m, seed):
    return torch.from_numpy(inputs.complex_gaussian(N, m, seed=seed)).to(torch.complex64).cuda()


@pytest.mark.parametrize("r,m", [(10, 5), (10, 64), (6, 3), (12, 1)])
def test_split_apply_equals_single_pass_batch(r, m):
    N = 1 << 20    # r = 10: kH = kG = 6 -> passes 3 + 3; r = 6: 7 -> 4 + 3; r = 12: 6 -> 3 + 3
    plan = api.Plan(N, r=r, phase_kind=L.PHASE_FIO, amp_kind=L.AMP_SMOOTH, factor_on_device=True)
    F = gauss(N, m, 50 + r + m)
    G1 = plan.apply(F, prec=api.F32)
    G2 = torch.full_like(F, float("nan"))
    api.apply_batched([(plan, F, G2)])
    torch.cuda.synchronize()
    api.apply_batched_release()
    assert plan.sync_status() == 0
    assert torch.equal(G1, G2)
    g64 = plan.apply(F.to(torch.complex128), prec=api.F64)
    torch.cuda.synchronize()
    assert relerr(G1.cpu().numpy().astype(np.complex128), g64.cpu().numpy()) < 2e-6


@pytest.mark.parametrize("lg,m", [(20, 2), (20, 40), (18, 16), (17, 3)])
def test_split_otf_apply_equals_single_pass_shard(lg, m):
    # on-the-fly plans split from 5 levels up: 2^18 -> 3 + 2 on each side, 2^17 -> G only
    N = 1 << lg
    po = api.Plan(N, r=10, phase_kind=L.PHASE_FIO, amp_kind=L.AMP_SMOOTH, on_the_fly=True)
    F = gauss(N, m, 60 + m)
    G1 = po.apply(F, prec=api.F32)
    G2 = torch.full_like(F, float("nan"))
    api.ShardedApply(po, 1, m).apply_local(F, G2)
    torch.cuda.synchronize()
    assert po.sync_status() == 0
    assert torch.equal(G1, G2)


def test_split_otf_n22_vs_direct():
    # N = 2^22: kH = kG = 7, passes 4 + 3 on each side; on-the-fly (tables would take ~42 GB)
    N, m = 1 << 22, 2
    po = api.Plan(N, eps=1e-6, phase_kind=L.PHASE_FIO, amp_kind=L.AMP_SMOOTH, on_the_fly=True)
    Fh = inputs.complex_gaussian(N, m, seed=70)
    G = po.apply(torch.from_numpy(Fh).to(torch.complex64).cuda(), prec=api.F32)
    torch.cuda.synchronize()
    assert po.sync_status() == 0
    rows = inputs.sample_rows(N, 6, seed=71)
    gd = od.direct(od.FIO, N, Fh, rows, amp=1)
    assert relerr(G.cpu().numpy().astype(np.complex128)[rows], gd) < 1e-5
