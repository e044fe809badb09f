"""GPU tests of the sharded apply (include/bf_shard.h) on one device.

All G shards run in this process: the fronts write per-peer blocks, the
exchange is a block transpose, the backs read them.  Every output element must
be bitwise what the unsharded FP32 apply gives: each tile's arithmetic is the
same, only which CTA runs it and where W lives change.
"""
import pytest

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


@pytest.mark.parametrize("N,m", [(16384, 5), (8192, 1), (16384, 40), (65536, 64)])
@pytest.mark.parametrize("G", [1, 2, 4, 8])
def test_sharded_equals_unsharded(N, m, G):
    plan = api.Plan(N, r=10, phase_kind=L.PHASE_FIO, amp_kind=L.AMP_SMOOTH)
    F = torch.from_numpy(inputs.complex_gaussian(N, m, seed=N + m)).to(torch.complex64).cuda()
    ref = plan.apply(F, prec=api.F32)
    sh = api.ShardedApply(plan, G, m)
    out = torch.full_like(F, float("nan"))
    sh.apply_local(F, out)
    torch.cuda.synchronize()
    assert plan.sync_status() == 0
    assert torch.equal(out, ref)


def test_shard_rejections():
    plan = api.Plan(4096, r=10)
    import ctypes
    c = ctypes.c_int64()
    lib = L.lib()
    assert lib.bf_shard_info(plan._h, 3, 4, ctypes.byref(c)) == L.BF_ERR_ARG        # not a power of two
    assert lib.bf_shard_info(plan._h, 1 << 12, 4, ctypes.byref(c)) == L.BF_ERR_ARG  # above min(2^l1, 2^h)
    assert lib.bf_shard_info(plan._h, 2, 0, ctypes.byref(c)) == L.BF_ERR_ARG
    split = api.Plan(4096, r=10, phase_kind=L.PHASE_FIO_PW, split=2)
    assert lib.bf_shard_info(split._h, 2, 4, ctypes.byref(c)) == L.BF_ERR_UNSUPPORTED
