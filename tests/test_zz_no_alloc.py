"""The allocation-free apply entry point (bf_apply_f32_noalloc).

It exists for callers that may not allocate device memory while applying
(an application that owns all device memory through its own pool, or a
latency-critical path that must stay out of the CUDA allocator).  The test
calls it through the C ABI twice in a row and checks both results against
bf_apply, the ordinary FP32 entry point: the two run the same tiles in the
same order, so the results must be bitwise equal (and so within the FP32
parity tolerance of the other GPU tests).  Sampled rows are also held to the
FP64 direct oracle at the FP32 tolerance.  Free device memory must not change
across those calls, and an oversized request is refused.
This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from paper_1803_04128_gb300 import _lib as L
from paper_1803_04128_gb300 import api, inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


from oracle import direct as od  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_matches_bf_apply_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1803_04128_gb300 import build
    build.build()
    lib = L.lib()
    N, m = 4096, 12
    plan = api.Plan(N, r=10, phase_kind=L.PHASE_FIO, amp_kind=L.AMP_SMOOTH).upload()
    F = torch.from_numpy(inputs.complex_gaussian(N, m, seed=21)).to(torch.complex64).cuda()
    ref = plan.apply(F, prec=api.F32)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # outputs allocated up front, so that only the library calls fall between the
    # two free-memory readings (torch's caching allocator stays out of it)
    Gs = [torch.empty_like(F) for _ in range(3)]
    torch.cuda.synchronize()
    outs = []
    free_before = None
    for call, G in enumerate(Gs):
        if call == 1:
            torch.cuda.synchronize()
            free_before = torch.cuda.mem_get_info()[0]
        st = lib.bf_apply_f32_noalloc(plan._h, ctypes.c_void_p(F.data_ptr()), m, ctypes.c_void_p(G.data_ptr()), s)
        assert st == L.BF_OK, lib.bf_last_error().decode()
        torch.cuda.synchronize()
        if call == 2:
            assert torch.cuda.mem_get_info()[0] == free_before
    for G in Gs:
        outs.append(G.cpu().numpy())
    for g in outs[1:]:                       # two calls in a row after the set-up call
        assert np.array_equal(g, ref), rel(g, ref)
        assert rel(g, ref) < 2e-6
    rows = inputs.sample_rows(N, 64, seed=5)
    gd = od.direct(od.FIO, N, inputs.complex_gaussian(N, m, seed=21), rows, amp=1)
    assert rel(outs[2][rows], gd) < 1e-5
    # a request whose workspace exceeds the fixed scratch is refused, not allocated
    big = api.Plan(65536, r=10, phase_kind=L.PHASE_FIO, amp_kind=L.AMP_SMOOTH).upload()
    Fb = torch.zeros((65536, 64), dtype=torch.complex64, device="cuda")
    Gb = torch.empty_like(Fb)
    st = lib.bf_apply_f32_noalloc(big._h, ctypes.c_void_p(Fb.data_ptr()), 64, ctypes.c_void_p(Gb.data_ptr()), s)
    assert st == L.BF_ERR_ARG and b"scratch" in lib.bf_last_error()
