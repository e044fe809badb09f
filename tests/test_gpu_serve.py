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
    assert st["device_busy_ms"] > 0
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


def _burst(srv, ops, Ns, n, ms, seed, pinned=True):
    """n requests (operator, m drawn from ms) with page-locked buffers, all built first and
    then submitted back to back, so that they queue while the slots are busy."""
    rng = np.random.default_rng(seed)
    reqs = []
    for k in range(n):
        o = int(rng.integers(0, len(Ns)))
        m = int(rng.choice(ms))
        F = torch.from_numpy(inputs.complex_gaussian(Ns[o], m, seed=seed + k).astype(np.complex64))
        G = torch.full_like(F, float("nan"))
        if pinned:
            F, G = F.pin_memory(), G.pin_memory()
        reqs.append([o, F, G, None])
    for r in reqs:
        r[3] = srv.submit(ops[r[0]], r[1], r[2])
    for r in reqs:
        srv.wait(r[3], 120000.0)
    return reqs


def test_batches_form_and_slots_overlap_on_the_device():
    # continuous batching: requests that arrive while slots are busy are packed into fewer
    # applies, and the slots' batches (copies and kernels, CUDA-event intervals) overlap in time
    Ns = [16384, 65536]
    plans = [api.Plan(N, eps=1e-6, amp_kind=L.AMP_SMOOTH) for N in Ns]
    srv = api.Server(n_slots=4, max_batch_rhs=64)
    ops = [srv.add(p) for p in plans]
    srv.start()
    reqs = _burst(srv, ops, Ns, 40, (1, 4, 16), seed=300)
    st = srv.stats()
    assert st["completed"] == 40
    assert st["launches"] < 40, st             # requests were batched
    assert st["overlap_ms"] > 0.0, st          # two slots' device work overlapped
    assert st["overlap_ms"] <= st["device_busy_ms"]
    for o, F, G, _ in reqs:
        alone = plans[o].apply(F.cuda(), prec=api.F32).cpu()
        assert torch.equal(G, alone)
    srv.close()


def test_auto_method_serves_nufft_where_the_phase_allows():
    # Sec. 3's choice per operator: the FIO operator (rank 1 on the column halves) by the NUFFT,
    # the separable phase with a xi^2 term by the butterfly; each result equals its method's
    # apply of that request alone, and meets the direct sum
    plans = [api.Plan(16384, eps=1e-6, phase_kind=L.PHASE_FIO, amp_kind=L.AMP_SMOOTH),
             api.Plan(4096, eps=1e-6, phase_kind=L.PHASE_SEP, amp_kind=L.AMP_SMOOTH)]
    Ns = [16384, 4096]
    srv = api.Server(n_slots=3, max_batch_rhs=64, method=1)
    ops = [srv.add(p) for p in plans]
    srv.start()
    assert srv.stats()["nufft_operators"] == 1
    reqs = _burst(srv, ops, Ns, 24, (1, 4, 16), seed=500)
    assert srv.stats()["completed"] == 24
    for o, F, G, _ in reqs:
        if o == 0:
            alone = plans[0].nufft_apply(F.cuda()).cpu()
        else:
            alone = plans[1].apply(F.cuda(), prec=api.F32).cpu()
        assert torch.equal(G, alone)
    o, F, G, _ = next(r for r in reqs if r[0] == 0)
    rows = inputs.sample_rows(16384, 24, seed=4)
    gd = od.direct(od.FIO, 16384, F.numpy().astype(np.complex128), rows, amp=1)
    assert relerr(G.numpy()[rows], gd) < 1e-5
    o, F, G, _ = next(r for r in reqs if r[0] == 1)
    rows = inputs.sample_rows(4096, 24, seed=5)
    gd = od.direct(od.SEP, 4096, F.numpy().astype(np.complex128), rows, amp=1)
    assert relerr(G.numpy()[rows], gd) < 1e-5
    srv.close()


@pytest.mark.parametrize("prec,max_rhs,ms,n", [
    (api.F64, 64, (1, 4, 16), 24),      # batches of several requests, 16-byte elements
    (api.F32, 256, (1,), 120),          # more requests in a batch than the staged copy takes
    (api.F32, 2048, (200, 300), 12),    # batches wider than the staged copy takes
])
def test_batch_copies_keep_results_bitwise(prec, max_rhs, ms, n):
    # a batch moves its requests' rows either as one contiguous copy per request plus a device
    # interleave, or (many or wide requests) as one strided copy per request; both give each
    # request exactly its apply alone
    Ns = [1024, 2048]
    plans = [api.Plan(N, eps=1e-6, amp_kind=L.AMP_SMOOTH) for N in Ns]
    srv = api.Server(n_slots=2, max_batch_rhs=max_rhs, precision=prec, n_priority_slots=0)
    ops = [srv.add(p) for p in plans]
    srv.start()
    rng = np.random.default_rng(7)
    dt = np.complex128 if prec == api.F64 else np.complex64
    reqs = []
    for k in range(n):
        o = int(rng.integers(0, 2))
        m = int(rng.choice(ms))
        F = torch.from_numpy(inputs.complex_gaussian(Ns[o], m, seed=900 + k).astype(dt)).pin_memory()
        G = torch.full_like(F, float("nan")).pin_memory()
        reqs.append((o, F, G))
    rids = [srv.submit(ops[o], F, G) for o, F, G in reqs]
    for rid in rids:
        srv.wait(rid, 120000.0)
    st = srv.stats()
    assert st["completed"] == n and st["launches"] < n, st
    for o, F, G in reqs:
        alone = plans[o].apply(F.cuda(), prec=prec).cpu()
        assert torch.equal(G, alone)
    srv.close()


def test_large_nufft_requests_in_column_chunks_are_bitwise_alone():
    # a single NUFFT request of m >= 32 columns (N m >= 2^20), with no other request waiting,
    # runs in two column chunks whose copies overlap the other chunk's kernels; every column is
    # computed on its own, so the result is that of the request's nufft_apply alone.  The first
    # two requests go one at a time (chunked), the rest back to back (a queue: not chunked).
    N = 16384
    plan = api.Plan(N, eps=1e-6, phase_kind=L.PHASE_FIO, amp_kind=L.AMP_SMOOTH)
    srv = api.Server(n_slots=2, max_batch_rhs=64, method=1, n_priority_slots=0)
    op = srv.add(plan)
    srv.start()
    reqs = []
    for k, m in enumerate((64, 32, 64, 4, 64)):
        F = torch.from_numpy(inputs.complex_gaussian(N, m, seed=700 + k).astype(np.complex64)).pin_memory()
        G = torch.full_like(F, float("nan")).pin_memory()
        reqs.append((F, G, srv.submit(op, F, G)))
        if k < 2:
            srv.wait(reqs[-1][2], 120000.0)
    for F, G, rid in reqs[2:]:
        srv.wait(rid, 120000.0)
    for F, G, _ in reqs:
        assert torch.equal(G, plan.nufft_apply(F.cuda()).cpu())
    F, G, _ = reqs[0]
    rows = inputs.sample_rows(N, 24, seed=6)
    gd = od.direct(od.FIO, N, F.numpy().astype(np.complex128), rows, amp=1)
    assert relerr(G.numpy()[rows], gd) < 1e-5
    srv.close()
