"""GPU tests of the continuous-batching server (bf_server_*).

The central property: a request's result is the same alone and in the mix.
Each served result is compared bitwise with bf_apply of its operator on that
request alone, while many requests of several operators are batched and run
concurrently on several slots; a sample is also checked against the direct
FP64 oracle within the FP32 tolerance (1e-5).
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


def test_results_same_alone_and_in_the_mix():
    Ns = [1024, 4096, 16384]
    plans = [api.Plan(N, eps=1e-6, amp_kind=L.AMP_SMOOTH) for N in Ns]
    srv = api.Server(n_slots=3, max_batch_rhs=64)
    ops = [srv.add(p) for p in plans]
    srv.start()
    rng = np.random.default_rng(0)
    reqs = []
    for k in range(48):
        o = int(rng.integers(0, 3))
        m = int(rng.choice([1, 4, 16]))
        F = inputs.complex_gaussian(Ns[o], m, seed=100 + k).astype(np.complex64)
        G = np.full_like(F, np.nan)
        reqs.append((o, F, G, srv.submit(ops[o], F, G)))
    lat = [srv.wait(rid, 60000.0) for _, _, _, rid in reqs]
    st = srv.stats()
    assert st["completed"] == 48 and st["pending"] == 0
    assert st["mean_batch_rhs"] >= 1.0 and st["launches"] <= 48
    assert st["p99_ms"] >= st["p50_ms"] > 0 and min(lat) > 0
    for o, F, G, _ in reqs:
        alone = plans[o].apply(torch.from_numpy(F).cuda(), prec=api.F32).cpu().numpy()
        assert np.array_equal(G, alone)
    o, F, G, _ = next(r for r in reqs if r[0] == 2)
    rows = inputs.sample_rows(16384, 24, seed=1)
    gd = od.direct(od.FIO, 16384, F.astype(np.complex128), rows, amp=1)
    assert relerr(G[rows], gd) < 1e-5
    srv.close()


def test_per_request_plain_fp64_server():
    plan = api.Plan(2048, eps=1e-6, amp_kind=L.AMP_SMOOTH)
    srv = api.Server(n_slots=1, precision=api.F64, per_request=True)
    op = srv.add(plan)
    srv.start()
    items = []
    for k in range(6):
        F = inputs.complex_gaussian(2048, 1 + k % 3, seed=200 + k)
        G = np.zeros_like(F)
        items.append((F, G, srv.submit(op, F, G)))
    srv.drain(60000.0)
    st = srv.stats()
    assert st["launches"] == 6 and st["completed"] == 6
    for F, G, rid in items:
        srv.wait(rid, 1000.0)
        alone = plan.apply(torch.from_numpy(F).cuda(), prec=api.F64).cpu().numpy()
        assert np.array_equal(G, alone)
    srv.close()


def test_admission_by_hbm_budget():
    plan = api.Plan(65536, eps=1e-6, amp_kind=L.AMP_SMOOTH)
    srv = api.Server(hbm_budget=64 << 20)            # 64 MB: the factors do not fit
    with pytest.raises(L.BFError) as e:
        srv.add(plan)
    assert e.value.status == L.BF_ERR_NOMEM
    small = api.Plan(1024, eps=1e-6)
    srv2 = api.Server(hbm_budget=64 << 20, n_slots=2)
    op = srv2.add(small)
    srv2.start()
    F = inputs.complex_gaussian(1024, 300, seed=3).astype(np.complex64)
    with pytest.raises(L.BFError):                   # wider than a slot's batch width
        srv2.submit(op, F, np.empty_like(F))
    srv.close()
    srv2.close()
