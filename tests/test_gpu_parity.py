"""GPU parity: the CUDA apply (through the C ABI) against the oracle.

Two oracles: (i) Algorithm 4.1 evaluated on the fly in FP64
(oracle/butterfly.py) -- the same approximation the library stores, so the
difference is rounding only; (ii) the direct FP64 matvec (oracle/direct.c) --
the plain definition, so the difference is the BF error plus rounding.

Tolerances (relative l2 over the compared entries, eps^b of Sec. 5):
  * FP64 plain form vs (i): 1e-12 (rounding of ~2L+3 stages of short sums).
  * FP32 vs (i): 2e-6.  Each stage multiplies by unit-modulus phases and
    applies Lagrange weights with sum of |weights| <= ~3 (Lebesgue constant of
    the mock-Chebyshev grids, r <= 16); over <= 2L+3 <= 40 stages with
    u = 2^-24 the worst-case relative growth is ~40 * 3 * 6e-8 = 7e-6 and the
    random-walk estimate sqrt(40) * 3 * 6e-8 = 1.1e-6; 2e-6 sits between.
  * FP32 vs (ii): 1e-5, the stated FP32 target; FP64 vs (ii): eps = 1e-6.
"""
import numpy as np
import pytest

from conftest import relerr
from oracle import butterfly as obf
from oracle import direct as od
from oracle import lowrank as olr
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
    torch.cuda.init()


def oracle_ibf(kind, N, F, r, amp, n_global=None):
    ent = lambda I, J: od.amplitude(amp, N, np.asarray(I)[:, None], np.asarray(J)[None, :])
    a, b = olr.amplitude_split(ent, N, N)
    return obf.ibf_apply(kind, N, F, r, a, b)


def run(plan, F, prec):
    dt = torch.complex128 if prec == api.F64 else torch.complex64
    Ft = torch.from_numpy(np.ascontiguousarray(F)).to(dt).cuda()
    G = plan.apply(Ft, prec=prec)
    torch.cuda.synchronize()
    assert plan.sync_status() == 0
    return G.cpu().numpy().astype(np.complex128)


# ------------------------------------------------ precision-only parity ----
@pytest.mark.parametrize("N,r,m", [(256, 8, 1), (1024, 10, 3), (1024, 10, 37), (4096, 12, 5),
                                   (2048, 16, 2), (4096, 6, 130), (8192, 10, 17)])
@pytest.mark.parametrize("kind", [L.PHASE_FIO, L.PHASE_FIO_PW])
def test_f32_and_f64_match_algorithm_4_1(N, r, m, kind):
    plan = api.Plan(N, r=r, phase_kind=kind, amp_kind=L.AMP_SMOOTH)
    F = inputs.complex_gaussian(N, m, seed=N + m)
    ref = oracle_ibf(kind, N, F, r, 1)
    g32 = run(plan, F, api.F32)
    assert relerr(g32, ref) < 2e-6
    g64 = run(plan, F, api.F64)
    assert relerr(g64, ref) < 1e-12


@pytest.mark.parametrize("kind", [L.PHASE_DFT, L.PHASE_ONES, L.PHASE_SEP])
def test_special_kernels(kind):
    N, m = 2048, 4
    plan = api.Plan(N, r=10, phase_kind=kind)
    F = inputs.complex_gaussian(N, m, seed=3)
    gd = od.direct(kind, N, F)
    assert relerr(run(plan, F, api.F32), gd) < 1e-5
    if kind != L.PHASE_DFT:                      # R(A,B) = 0: the BF is exact
        assert relerr(run(plan, F, api.F64), gd) < 1e-12


def test_split_plan():
    N, m = 4096, 6
    plan = api.Plan(N, r=10, phase_kind=L.PHASE_FIO_PW, amp_kind=L.AMP_SMOOTH, split=2)
    F = inputs.complex_gaussian(N, m, seed=5)
    gd = od.direct(od.FIOPW, N, F, amp=1)
    assert relerr(run(plan, F, api.F32), gd) < 1e-5
    assert relerr(run(plan, F, api.F64), gd) < 1e-6


# ------------------------------------------------------- direct oracle -----
def test_config1_fp64_n1024():
    # 1D FIO, N = 1024, alpha = 1, eps = 1e-6, one RHS, FP64 apply
    N = 1024
    plan = api.Plan(N, eps=1e-6, phase_kind=L.PHASE_FIO, amp_kind=L.AMP_ONE)
    F = inputs.complex_gaussian(N, 1, seed=0)
    g = run(plan, F, api.F64)
    gd = od.direct(od.FIO, N, F)
    assert relerr(g, gd) < 1e-6


def test_config2_fp32_full_size_sampled_rows():
    # N = 65536, m = 64, smooth amplitude, complex FP32: 128 sampled rows
    N, m = 65536, 64
    plan = api.Plan(N, eps=1e-6, phase_kind=L.PHASE_FIO, amp_kind=L.AMP_SMOOTH)
    F = inputs.complex_gaussian(N, m, seed=0)
    g = run(plan, F, api.F32)
    rows = inputs.sample_rows(N, 128, seed=0)
    gd = od.direct(od.FIO, N, F, rows, amp=1)
    assert relerr(g[rows], gd) < 1e-5


def test_config3_shape_fp32_sampled():
    # N = 262144 piecewise phase, four N/2 sub-BFs; 48 rows x 8 columns sampled
    N, m = 262144, 8
    plan = api.Plan(N, eps=1e-6, phase_kind=L.PHASE_FIO_PW, amp_kind=L.AMP_SMOOTH, split=2)
    F = inputs.complex_gaussian(N, m, seed=0)
    g = run(plan, F, api.F32)
    rows = np.concatenate([inputs.sample_rows(N // 2, 24, seed=1), N // 2 + inputs.sample_rows(N // 2, 24, seed=2)])
    gd = od.direct(od.FIOPW, N, F, rows, amp=1)
    assert relerr(g[rows], gd) < 1e-5


# ----------------------------------------------------------- edge cases ----
def test_columns_are_independent_and_bitwise_batch_invariant():
    N, m = 4096, 24
    plan = api.Plan(N, r=10, amp_kind=L.AMP_SMOOTH)
    F = inputs.complex_gaussian(N, m, seed=7)
    Gall = run(plan, F, api.F32)
    for c in (0, 5, 23):
        g1 = run(plan, F[:, c:c + 1], api.F32)
        assert np.array_equal(g1[:, 0], Gall[:, c])
    # repeated applies are deterministic
    assert np.array_equal(run(plan, F, api.F32), Gall)


def test_zero_impulse_linearity():
    N = 1024
    plan = api.Plan(N, r=10)
    assert np.all(run(plan, np.zeros((N, 3), complex), api.F32) == 0)
    e = np.zeros((N, 1), complex); e[17] = 1
    col = od.entries(od.FIO, N, np.arange(N), [17])
    assert relerr(run(plan, e, api.F32), col) < 1e-5
    F = inputs.complex_gaussian(N, 2, seed=9)
    a, b = 0.5 - 2j, 1.5 + 0.25j
    lhs = run(plan, a * F[:, :1] + b * F[:, 1:], api.F64)
    rhs = a * run(plan, F[:, :1], api.F64) + b * run(plan, F[:, 1:], api.F64)
    assert relerr(lhs, rhs) < 1e-13


def test_apply_host_matches_device_apply():
    N, m = 2048, 9
    plan = api.Plan(N, r=10, amp_kind=L.AMP_SMOOTH)
    F = inputs.complex_gaussian(N, m, seed=11).astype(np.complex64)
    Gh = plan.apply_host(F)
    Gd = run(plan, F, api.F32)
    assert np.array_equal(Gh.astype(np.complex128), Gd)


@pytest.mark.parametrize("otf", [False, True])
def test_apply_host_row_ranges_bitwise(otf):
    """The host apply copies F and G in row ranges that overlap the front and back
    launches of the other ranges (one sub-BF, one pass per side): the same tiles as
    bf_apply, so bitwise the same result, at the benchmark's shape (N = 65536, m = 64)
    and on a ragged column count; two calls in a row reuse the copy stream and events."""
    N = 65536
    plan = api.Plan(N, eps=1e-6, amp_kind=L.AMP_SMOOTH, on_the_fly=otf)
    for m, seed in ((64, 21), (7, 22)):
        F = inputs.complex_gaussian(N, m, seed=seed).astype(np.complex64)
        Gd = run(plan, F, api.F32)
        for _ in range(2):
            Gh = plan.apply_host(F)
            assert np.array_equal(Gh.astype(np.complex128), Gd)


def test_apply_host_whole_buffer_paths():
    """Host applies that copy F and G in one piece (FP64; a plan of four sub-BFs) are
    bitwise the device applies."""
    N, m = 4096, 3
    plan = api.Plan(N, r=10, amp_kind=L.AMP_SMOOTH)
    F = inputs.complex_gaussian(N, m, seed=23)
    assert np.array_equal(plan.apply_host(np.ascontiguousarray(F), prec=api.F64), run(plan, F, api.F64))
    pw = api.Plan(N, r=10, phase_kind=L.PHASE_FIO_PW, amp_kind=L.AMP_SMOOTH, split=2)
    F32 = F.astype(np.complex64)
    assert np.array_equal(pw.apply_host(F32).astype(np.complex128), run(pw, F32, api.F32))


def test_bad_calls_return_errors():
    plan = api.Plan(1024, r=10)
    F = torch.zeros((1024, 2), dtype=torch.complex64, device="cuda")
    lib = L.lib()
    import ctypes
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.bf_apply(plan._h, api.F32, ctypes.c_void_p(F.data_ptr()), 0, ctypes.c_void_p(F.data_ptr()), s) == L.BF_ERR_ARG
    assert lib.bf_apply(plan._h, api.F32, ctypes.c_void_p(F.data_ptr()), 2, ctypes.c_void_p(F.data_ptr()), s) == L.BF_ERR_ARG
    assert lib.bf_apply(plan._h, 7, ctypes.c_void_p(F.data_ptr()), 2, ctypes.c_void_p(F.data_ptr() + 64), s) == L.BF_ERR_ARG
    assert lib.bf_apply(None, api.F32, ctypes.c_void_p(F.data_ptr()), 2, ctypes.c_void_p(F.data_ptr() + 64), s) == L.BF_ERR_ARG


# ------------------------------------------------------ split-BF16 path ----
# Tolerance: operands are split x = hi + lo in BF16 (8-bit significands), so
# hi + lo carries x to about 2^-16 relative; the dropped lo*lo term is
# ~2^-18; with unit-modulus phases and Lagrange weights of Lebesgue constant
# ~3 over <= 2L+3 stages this gives ~1e-5 .. 1e-4; 3e-4 against Algorithm 4.1
# and the stated 1e-3 against the direct oracle.
@pytest.mark.parametrize("N,r,m", [(1024, 8, 3), (4096, 10, 5), (16384, 8, 64), (8192, 12, 2), (2048, 10, 130)])
def test_bf16x3_matches_algorithm_4_1(N, r, m):
    plan = api.Plan(N, r=r, phase_kind=L.PHASE_FIO, amp_kind=L.AMP_SMOOTH)
    F = inputs.complex_gaussian(N, m, seed=N + r)
    cols = slice(0, min(m, 4))
    ref = oracle_ibf(L.PHASE_FIO, N, F[:, cols], r, 1)
    g = run(plan, F, api.BF16X3)
    assert relerr(g[:, cols], ref) < 3e-4
    assert relerr(g, run(plan, F, api.F32)) < 3e-4


def test_bf16x3_full_size_config2_sampled():
    N, m = 65536, 64
    plan = api.Plan(N, eps=1e-6, phase_kind=L.PHASE_FIO, amp_kind=L.AMP_SMOOTH)
    F = inputs.complex_gaussian(N, m, seed=0)
    g = run(plan, F, api.BF16X3)
    rows = inputs.sample_rows(N, 64, seed=0)
    gd = od.direct(od.FIO, N, F[:, :16], rows, amp=1)
    assert relerr(g[rows, :16], gd) < 1e-3


def test_bf16x3_config3_shape_r8_split():
    # piecewise phase, N = 262144 as four N/2 sub-BFs, r = 8: back tiles of 32 pairs
    N, m = 262144, 4
    plan = api.Plan(N, r=8, phase_kind=L.PHASE_FIO_PW, amp_kind=L.AMP_SMOOTH, split=2)
    F = inputs.complex_gaussian(N, m, seed=0)
    g = run(plan, F, api.BF16X3)
    rows = np.concatenate([inputs.sample_rows(N // 2, 16, seed=1), N // 2 + inputs.sample_rows(N // 2, 16, seed=2)])
    gd = od.direct(od.FIOPW, N, F, rows, amp=1)
    assert relerr(g[rows], gd) < 1e-3


@pytest.mark.parametrize("N,m,kind,okind,split", [(262144, 4, L.PHASE_FIO_PW, od.FIOPW, 2),
                                                  (65536, 130, L.PHASE_FIO, od.FIO, 1)])
def test_bf16x3_at_eps_1e6_with_v_and_u_one_level_higher(N, m, kind, okind, split):
    # config 3 at the contract's eps = 1e-6 (r = 10): with V and U at level 5 (32-index leaf
    # groups) the N/2 sub-BFs have kH = 3 and kG = 4, tiles that fit tensor memory.  Against
    # the same plan's FP64 apply (precision only, 3e-4) and the direct sum (1e-3); the FP64
    # apply of this plan meets the direct sum to eps; the FP32 kernels have no 32-index
    # leaf groups at r = 10 and refuse
    plan = api.Plan(N, eps=1e-6, phase_kind=kind, amp_kind=L.AMP_SMOOTH, split=split, l1=5)
    assert plan.info()["r"] == 10 and plan.info()["l1"] == 5
    F = inputs.complex_gaussian(N, m, seed=N + m)
    g = run(plan, F, api.BF16X3)
    g64 = run(plan, F, api.F64)
    assert relerr(g, g64) < 3e-4
    if split == 2:
        rows = np.concatenate([inputs.sample_rows(N // 2, 24, seed=1), N // 2 + inputs.sample_rows(N // 2, 24, seed=2)])
    else:
        rows = inputs.sample_rows(N, 48, seed=3)
    gd = od.direct(okind, N, F, rows, amp=1)
    assert relerr(g[rows], gd) < 1e-3
    assert relerr(g64[rows], gd) < 1e-6
    Ft = torch.from_numpy(F).to(torch.complex64).cuda()
    with pytest.raises(L.BFError) as e:
        plan.apply(Ft, prec=api.F32)
    assert e.value.status == L.BF_ERR_UNSUPPORTED


def test_bf16x3_refuses_tiles_that_do_not_fit():
    plan = api.Plan(262144, r=10, phase_kind=L.PHASE_FIO, amp_kind=L.AMP_SMOOTH, split=2)
    F = torch.zeros((262144, 1), dtype=torch.complex64, device="cuda")
    with pytest.raises(L.BFError) as e:
        plan.apply(F, prec=api.BF16X3)
    assert e.value.status == L.BF_ERR_UNSUPPORTED


def test_largest_serving_operator_n_2_20_sampled():
    # the largest operator of the serving workload (N = 2^20): FP32 and FP64 on 48 sampled rows
    N, m = 1 << 20, 3
    plan = api.Plan(N, eps=1e-6, phase_kind=L.PHASE_FIO, amp_kind=L.AMP_SMOOTH)
    F = inputs.complex_gaussian(N, m, seed=21)
    rows = inputs.sample_rows(N, 48, seed=22)
    gd = od.direct(od.FIO, N, F, rows, amp=1)
    assert relerr(run(plan, F, api.F32)[rows], gd) < 1e-5
    assert relerr(run(plan, F, api.F64)[rows], gd) < 1e-6


# ------------------------------------------------------- more edge cases ----
@pytest.mark.parametrize("n0", [4, 8])
def test_leaves_of_n0_indices_match_algorithm_4_1(n0):
    # leaves of n0 > 1 indices (Sec. 4 uses n0 = 1; the levels of <= r indices fold into V and U)
    N, r, m = 4096, 10, 3
    plan = api.Plan(N, r=r, n0=n0, phase_kind=L.PHASE_FIO, amp_kind=L.AMP_SMOOTH)
    F = inputs.complex_gaussian(N, m, seed=n0)
    ent = lambda I, J: od.amplitude(1, N, np.asarray(I)[:, None], np.asarray(J)[None, :])
    a, b = olr.amplitude_split(ent, N, N)
    ref = obf.ibf_apply(L.PHASE_FIO, N, F, r, a, b, n0=n0)
    assert relerr(run(plan, F, api.F32), ref) < 2e-6
    assert relerr(run(plan, F, api.F64), ref) < 1e-12


def test_many_ragged_columns_sampled():
    # m = 1000 (62 full slices of 16 and a ragged one of 8), sampled rows vs the direct oracle
    N, m = 4096, 1000
    plan = api.Plan(N, eps=1e-6, phase_kind=L.PHASE_FIO, amp_kind=L.AMP_SMOOTH)
    F = inputs.complex_gaussian(N, m, seed=31)
    rows = inputs.sample_rows(N, 24, seed=32)
    gd = od.direct(od.FIO, N, F, rows, amp=1)
    g = run(plan, F, api.F32)
    assert relerr(g[rows], gd) < 1e-5
    # every column equals its own single-column apply (slices never mix columns)
    for c in (0, 15, 16, 991, 999):
        assert np.array_equal(run(plan, F[:, c:c + 1], api.F32)[:, 0], g[:, c])


def test_zero_amplitude_gives_zero():
    # alpha = 0 has numerical rank 0: the apply writes G = 0 in every precision
    N, m = 1024, 4
    plan = api.Plan(N, r=10, phase_kind=L.PHASE_FIO, amp_kind=L.AMP_USER, alpha=lambda x, xi: 0.0)
    assert plan.info()["r_alpha"] == 0
    F = inputs.complex_gaussian(N, m, seed=33)
    for prec in (api.F32, api.F64):
        assert np.all(run(plan, F, prec) == 0)
