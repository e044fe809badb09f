"""GPU tests of the batched uneven apply, CUDA-graph replay and the autotuner.

Each operator in a batch must produce exactly (bitwise) what bf_apply gives
for it alone: columns never mix and the per-column arithmetic is the same
code, so batching, slicing and graph replay cannot change a result.
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


def make_ops(shapes, seed=0):
    ops = []
    for k, (N, m) in enumerate(shapes):
        plan = api.Plan(N, r=10, phase_kind=L.PHASE_FIO, amp_kind=L.AMP_SMOOTH)
        F = torch.from_numpy(inputs.complex_gaussian(N, m, seed=seed + k)).to(torch.complex64).cuda()
        G = torch.full_like(F, float("nan"))
        ops.append((plan, F, G))
    return ops


SHAPES = [(4096, 1), (1024, 7), (16384, 33), (8192, 64), (2048, 128), (4096, 3)]


def test_batch_equals_individual_applies():
    ops = make_ops(SHAPES)
    b = api.Batch(ops)
    b.run()
    assert b.status() == 0
    for plan, F, G in ops:
        ref = plan.apply(F, prec=api.F32)
        torch.cuda.synchronize()
        assert torch.equal(G, ref)
    # and against the direct oracle on a few rows of one operator
    plan, F, G = ops[2]
    rows = inputs.sample_rows(16384, 32, seed=3)
    gd = od.direct(od.FIO, 16384, F.cpu().numpy().astype(np.complex128), rows, amp=1)
    assert relerr(G.cpu().numpy()[rows], gd) < 1e-5


def test_graph_replay_repeats_exactly():
    ops = make_ops(SHAPES[:4], seed=10)
    b = api.Batch(ops)
    s = torch.cuda.Stream()
    b.capture(s)
    b.replay(s)
    s.synchronize()
    first = [G.clone() for _, _, G in ops]
    for _, _, G in ops:
        G.fill_(0)
    b.replay(s)
    b.replay(s)
    assert b.status(s) == 0
    for (plan, F, G), g0 in zip(ops, first):
        assert torch.equal(G, g0)
        assert torch.equal(G, plan.apply(F, prec=api.F32))


def test_autotune_choice_does_not_change_results(tmp_path):
    N, m = 8192, 40
    plan = api.Plan(N, r=10, amp_kind=L.AMP_SMOOTH)
    F = torch.from_numpy(inputs.complex_gaussian(N, m, seed=5)).to(torch.complex64).cuda()
    before = plan.apply(F, prec=api.F32).clone()
    cache = tmp_path / "tune.txt"
    mr = api.autotune(plan, m, cache)
    assert mr >= 1 and (mr & (mr - 1)) == 0
    assert "m=40 mr=%d" % mr in cache.read_text()
    after = plan.apply(F, prec=api.F32)
    torch.cuda.synchronize()
    assert torch.equal(before, after)
    plan2 = api.Plan(N, r=10, amp_kind=L.AMP_SMOOTH)
    assert api.autotune(plan2, m, cache) == mr           # served from the cache
    assert api.tile_shapes(plan2, m) == api.tile_shapes(plan, m)


@pytest.mark.parametrize("N,m", [(65536, 1), (65536, 64), (1 << 20, 3)])
def test_level_tile_autotuner_keeps_results_bitwise(N, m, tmp_path):
    # the autotuner searches mr, the levels per pass (N = 2^20 splits its level ranges) and
    # the tiles per CTA; whatever it picks, every column sees the same arithmetic
    plan = api.Plan(N, eps=1e-6, amp_kind=L.AMP_SMOOTH, factor_on_device=True)
    F = torch.from_numpy(inputs.complex_gaussian(N, m, seed=N + m)).to(torch.complex64).cuda()
    before = plan.apply(F, prec=api.F32).clone()
    rule = api.tile_shapes(plan, m)
    api.autotune(plan, m, tmp_path / "tune.txt")
    tuned = api.tile_shapes(plan, m)
    assert tuned["mr"] >= 1 and tuned["tpc_front"] >= 1 and tuned["tpc_back"] >= 1
    assert tuned["levels_per_pass"] >= 1 and rule["levels_per_pass"] >= 1
    after = plan.apply(F, prec=api.F32)
    torch.cuda.synchronize()
    assert plan.sync_status() == 0
    assert torch.equal(before, after), (rule, tuned)
    rows = inputs.sample_rows(N, 16, seed=3)
    gd = od.direct(od.FIO, N, F.cpu().numpy().astype(np.complex128), rows, amp=1)
    assert relerr(after.cpu().numpy()[rows], gd) < 1e-5
    plan.close()


def test_wait_timeout_is_reported_not_hung():
    # every back tile waits for a front completion that never arrives; each
    # wait gives up after a few thousand polls and the status says so
    ops = make_ops([(1024, 2), (2048, 1)], seed=20)
    b = api.Batch(ops)
    b.set_spin_limit(2000)
    b.debug_hold(True)
    b.run()
    assert b.status() == L.BF_ERR_TIMEOUT
    b.debug_hold(False)
    b.run()
    assert b.status() == 0
    for plan, F, G in ops:
        assert torch.equal(G, plan.apply(F, prec=api.F32))


def test_batch_rejects_mixed_rank_and_split():
    p10 = api.Plan(1024, r=10)
    p12 = api.Plan(1024, r=12)
    F = torch.zeros((1024, 1), dtype=torch.complex64, device="cuda")
    G1, G2 = torch.empty_like(F), torch.empty_like(F)
    with pytest.raises(L.BFError):
        api.Batch([(p10, F, G1), (p12, F, G2)])
    ps = api.Plan(2048, r=10, split=2)
    F2 = torch.zeros((2048, 1), dtype=torch.complex64, device="cuda")
    with pytest.raises(L.BFError):
        api.Batch([(ps, F2, torch.empty_like(F2))])


def test_apply_batched_one_call_reuses_kept_batch():
    ops = make_ops(SHAPES[:4], seed=30)
    s = torch.cuda.current_stream()
    api.apply_batched(ops, s)                    # builds and keeps the batch
    torch.cuda.synchronize()
    for plan, F, G in ops:
        assert torch.equal(G, plan.apply(F, prec=api.F32))
    # same plans and m, new buffers: only the F/G pointers change
    ops2 = [(plan, torch.from_numpy(inputs.complex_gaussian(F.shape[0], F.shape[1], seed=40 + k))
             .to(torch.complex64).cuda(), torch.full_like(G, float("nan"))) for k, (plan, F, G) in enumerate(ops)]
    api.apply_batched(ops2, s)
    torch.cuda.synchronize()
    for plan, F, G in ops2:
        assert torch.equal(G, plan.apply(F, prec=api.F32))
    # a different m list rebuilds
    plan0, F0, _ = ops[0]
    F3 = torch.cat([F0, F0], dim=1).contiguous()
    G3 = torch.empty_like(F3)
    api.apply_batched([(plan0, F3, G3)], s)
    torch.cuda.synchronize()
    assert torch.equal(G3, plan0.apply(F3, prec=api.F32))
    api.apply_batched_release()


def test_apply_batched_rejects_bad_items():
    plan, F, G = make_ops([(1024, 2)])[0]
    lib = L.lib()
    import ctypes
    plans = (ctypes.c_void_p * 1)(plan._h.value)
    arr = (L.ApplyItem * 1)()
    arr[0].F, arr[0].G, arr[0].m = F.data_ptr(), G.data_ptr(), 0
    assert lib.bf_apply_batched(ctypes.cast(plans, ctypes.c_void_p), ctypes.cast(arr, ctypes.c_void_p), 1,
                                None) == L.BF_ERR_ARG
    assert lib.bf_apply_batched(None, ctypes.cast(arr, ctypes.c_void_p), 1, None) == L.BF_ERR_ARG


def test_two_phase_mode_is_bitwise_the_same_and_tunable():
    # mode 1 (a front launch and a back launch over every operator) against mode 0 and the
    # single applies, eager and replayed from a graph; the tuner keeps one of the three modes
    ops = make_ops([(4096, 3), (16384, 40), (2048, 1), (65536, 17), (8192, 128)], seed=40)
    b = api.Batch(ops)
    assert b.mode() == 0
    b.set_mode(1)
    b.run()
    assert b.status() == 0
    ref = [plan.apply(F, prec=api.F32) for plan, F, G in ops]
    for (plan, F, G), r in zip(ops, ref):
        assert torch.equal(G, r)
    for _, _, G in ops:
        G.fill_(float("nan"))
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    b.capture(s)
    b.replay(s)
    assert b.status(s) == 0
    for (plan, F, G), r in zip(ops, ref):
        assert torch.equal(G, r)
    mode, ms = b.tune()
    assert mode in (0, 1, 2) and min(ms) > 0 and b.mode() == mode
    for (plan, F, G), r in zip(ops, ref):
        assert torch.equal(G, r)
    b.close()


def test_stream_mode_is_bitwise_the_same_and_replays():
    # mode 2 (each operator's own apply on four forked streams) against the single applies,
    # run directly and replayed from a CUDA graph (the fork and join are captured)
    ops = make_ops(SHAPES + [(65536, 5)], seed=40)
    b = api.Batch(ops)
    b.set_mode(2)
    assert b.mode() == 2
    b.run()
    assert b.status() == 0
    for plan, F, G in ops:
        assert torch.equal(G, plan.apply(F, prec=api.F32))
    s = torch.cuda.Stream()
    b.capture(s)
    for _, _, G in ops:
        G.fill_(float("nan"))
    b.replay(s)
    b.replay(s)
    assert b.status(s) == 0
    for plan, F, G in ops:
        assert torch.equal(G, plan.apply(F, prec=api.F32))
