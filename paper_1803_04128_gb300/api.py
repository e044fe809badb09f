"""Python binding of the butterfly-factorisation apply (same names as the C ABI).

Only argument marshalling lives here: every step of the apply runs in the
library's CUDA kernels.  PyTorch supplies device memory and streams.
"""
import ctypes

import numpy as np

from . import _lib as L

F64, F32, BF16X3 = L.PREC_F64, L.PREC_F32, L.PREC_BF16X3
PREC_NAMES = {"f64": F64, "f32": F32, "bf16x3": BF16X3}


def grid_indices(n, r):
    """Mock-Chebyshev index grid of Eq. (gdA)/(gdB) (0-based offsets)."""
    out = (ctypes.c_int64 * max(1, min(n, r)))()
    cnt = ctypes.c_int()
    L.check(L.lib().bf_grid_indices(n, r, out, ctypes.byref(cnt)), "bf_grid_indices")
    return np.array(out[:cnt.value], dtype=np.int64)


def default_options():
    o = L.Options()
    L.check(L.lib().bf_default_options(ctypes.byref(o)), "bf_default_options")
    return o


def unwrap(u, tau=0.25, seed=()):
    """Algorithm 3 (bf_unwrap): (v, starts) with v = u + integers, from u = v mod 1."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    sd = np.ascontiguousarray(seed, dtype=np.float64)
    v = np.empty_like(u)
    starts = np.zeros(max(16, u.size // 2 + 1), dtype=np.int64)
    cnt = ctypes.c_int64()
    L.check(L.lib().bf_unwrap(u.ctypes.data, u.size, tau, sd.ctypes.data if sd.size else None, sd.size,
                              v.ctypes.data, starts.ctypes.data, starts.size, ctypes.byref(cnt)), "bf_unwrap")
    return v, [int(t) for t in starts[:cnt.value]]


def _stream_ptr(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Plan:
    """A factored operator g = K f (bf_plan_create + bf_factor)."""

    def __init__(self, N, eps=1e-6, phase_kind=L.PHASE_FIO, phase_param=1.0, amp_kind=L.AMP_ONE,
                 r=0, n0=1, split=1, seed=0, keep_host=True, device=0, factor=True, phi=None, alpha=None,
                 factor_on_device=False, on_the_fly=False, indirect=False, entry=None, entries=None,
                 matvec=None, amp_rank=0, amp_oversample=0, phase_rank=0, phase_oversample=0, l1=0, _handle=None):
        """``indirect``: factor from the kernel's entries alone (amplitude and phase
        recovered, Algorithms 1 and 3-5).  A kernel without a built-in kind is given by
        ``entry(x, xi) -> complex`` or, in bulk, ``entries(i, j) -> complex array`` over
        grid index arrays (x_i = i/N, xi_j = j - N/2); either implies indirect.  A kernel
        known only through products (Scenario 2) is given by ``matvec(X, transpose) -> Y``,
        Y = K X or K^T X for a complex array X of shape (N, m); it implies indirect too.
        ``amp_rank``, ``amp_oversample`` (``phase_rank``, ``phase_oversample``): Algorithm 1's
        rank parameter and oversampling for the amplitude (the recovered phase); 0: the
        library's defaults.  ``l1``: level of the V and U stages (0: the first level whose
        nodes hold more than r indices; see bf_options.l1)."""
        self._lib = L.lib()
        self._h = ctypes.c_void_p()
        self._keep = []
        if _handle is not None:
            self._h = _handle
        else:
            d = L.KernelDesc()
            d.N = N
            d.phase_kind = phase_kind
            d.phase_param = phase_param
            d.amp_kind = amp_kind
            if phi is not None:
                cb = L.PHASE_FN(lambda x, xi, u: phi(x, xi))
                self._keep.append(cb)
                d.phi = cb
            if alpha is not None:
                def _amp(x, xi, u, re, im):
                    v = complex(alpha(x, xi))
                    re[0], im[0] = v.real, v.imag
                cb2 = L.AMP_FN(_amp)
                self._keep.append(cb2)
                d.alpha = cb2
            if entry is not None:
                def _ent(x, xi, u, re, im):
                    v = complex(entry(x, xi))
                    re[0], im[0] = v.real, v.imag
                cb3 = L.AMP_FN(_ent)
                self._keep.append(cb3)
                d.entry = cb3
                d.phase_kind = L.PHASE_ENTRIES
            if entries is not None:
                def _ents(ip, jp, n, u, out):
                    I = np.ctypeslib.as_array(ip, shape=(n,))
                    J = np.ctypeslib.as_array(jp, shape=(n,))
                    o = np.ctypeslib.as_array(out, shape=(2 * n,)).view(np.complex128)
                    o[:] = np.asarray(entries(I, J), dtype=np.complex128).reshape(n)
                cb4 = L.ENTRIES_FN(_ents)
                self._keep.append(cb4)
                d.entries = cb4
                d.phase_kind = L.PHASE_ENTRIES
            if matvec is not None:
                def _mv(xp, m, tr, u, yp):
                    X = np.ctypeslib.as_array(xp, shape=(2 * N * m,)).view(np.complex128).reshape(N, m)
                    Y = np.ctypeslib.as_array(yp, shape=(2 * N * m,)).view(np.complex128).reshape(N, m)
                    Y[:] = np.asarray(matvec(X, bool(tr)), dtype=np.complex128).reshape(N, m)
                cb5 = L.MATVEC_FN(_mv)
                self._keep.append(cb5)
                d.matvec = cb5
                d.phase_kind = L.PHASE_ENTRIES
            o = default_options()
            o.r, o.n0, o.split, o.seed, o.keep_host, o.device = r, n0, split, seed, int(keep_host), device
            o.indirect = int(indirect or entry is not None or entries is not None or matvec is not None)
            if amp_rank:
                o.amp_rank = amp_rank
            if amp_oversample:
                o.amp_oversample = amp_oversample
            if phase_rank:
                o.phase_rank = phase_rank
            if phase_oversample:
                o.phase_oversample = phase_oversample
            o.l1 = l1
            L.check(self._lib.bf_plan_create(ctypes.byref(d), eps, ctypes.byref(o), ctypes.byref(self._h)),
                    "bf_plan_create")
            if on_the_fly:
                self.factor_otf()
            elif factor_on_device:
                self.factor_device()
            elif factor:
                self.factor()

    # -- life cycle
    def factor(self):
        L.check(self._lib.bf_factor(self._h), "bf_factor")
        return self

    def factor_device(self):
        """Factor with the phase tables built on the GPU (bf_factor_device)."""
        L.check(self._lib.bf_factor_device(self._h), "bf_factor_device")
        return self

    def factor_otf(self):
        """Factor for the on-the-fly FP32 apply (bf_factor_otf): no phase tables,
        the apply kernels evaluate the phases; O(r_alpha N) device memory."""
        L.check(self._lib.bf_factor_otf(self._h), "bf_factor_otf")
        return self

    def upload(self):
        L.check(self._lib.bf_upload(self._h), "bf_upload")
        return self

    def reserve(self, prec, m_max):
        L.check(self._lib.bf_reserve(self._h, prec, int(m_max)), "bf_reserve")
        return self

    def close(self):
        if self._h:
            self._lib.bf_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- inspection
    def info(self):
        i = L.PlanInfo()
        L.check(self._lib.bf_plan_get_info(self._h, ctypes.byref(i)), "bf_plan_get_info")
        return {k: getattr(i, k) for k, _ in L.PlanInfo._fields_}

    def view(self, what, level=0, block=0):
        """Copy of a host FP64 factor array (see bf_plan_view); complex ones as complex128."""
        ptr = ctypes.POINTER(ctypes.c_double)()
        cnt = ctypes.c_int64()
        L.check(self._lib.bf_plan_view(self._h, block, what, level, ctypes.byref(ptr), ctypes.byref(cnt)),
                "bf_plan_view")
        a = np.ctypeslib.as_array(ptr, shape=(cnt.value,)).copy() if cnt.value else np.zeros(0)
        if what in (0, 1, 3, 5, 6, 8, 10, 11, 12):
            a = a.view(np.complex128)
        return a

    def nufft_decide(self, r, r_eps=20, q=5, eps=1e-10, seed=0, block=0):
        """Algorithm 6 (bf_nufft_decide) on a plan factored from its entries: (y, n, terms),
        y = 1 if r-dimensional NUFFTs after lifting the phase evaluate the transform, n the
        numerical rank of the sampled residual columns, terms the number of NUFFTs."""
        y, n, t = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        L.check(self._lib.bf_nufft_decide(self._h, block, r, r_eps, q, eps, seed, ctypes.byref(y), ctypes.byref(n),
                                          ctypes.byref(t)), "bf_nufft_decide")
        return y.value, n.value, t.value

    def save(self, path):
        L.check(self._lib.bf_plan_save(self._h, str(path).encode()), "bf_plan_save")

    @classmethod
    def load(cls, path, device=0):
        o = default_options()
        o.device = device
        h = ctypes.c_void_p()
        L.check(L.lib().bf_plan_load(str(path).encode(), ctypes.byref(o), ctypes.byref(h)), "bf_plan_load")
        return cls(0, _handle=h)

    # -- apply
    def apply(self, F, G=None, prec=F32, stream=None):
        """G = K F on the GPU.  F: torch CUDA tensor (N,) or (N, m), complex64
        (F32, BF16X3) or complex128 (F64), contiguous.  Returns G."""
        import torch
        dt = torch.complex128 if prec == F64 else torch.complex64
        if F.dtype != dt or not F.is_cuda or not F.is_contiguous():
            raise ValueError("F must be a contiguous CUDA %s tensor" % dt)
        m = 1 if F.dim() == 1 else F.shape[1]
        if G is None:
            G = torch.empty_like(F)
        elif G.dtype != dt or not G.is_contiguous() or G.shape != F.shape:
            raise ValueError("G must match F")
        L.check(self._lib.bf_apply(self._h, prec, ctypes.c_void_p(F.data_ptr()), m,
                                   ctypes.c_void_p(G.data_ptr()), _stream_ptr(stream)), "bf_apply")
        return G

    def apply_host(self, F, G=None, prec=F32, stream=None):
        """G = K F with HOST buffers (numpy arrays or CPU tensors, pinned preferred):
        copies in, applies, copies out, synchronises."""
        if isinstance(F, np.ndarray):
            dt = np.complex128 if prec == F64 else np.complex64
            if F.dtype != dt or not F.flags.c_contiguous:
                raise ValueError("F must be C-contiguous %s" % dt)
            m = 1 if F.ndim == 1 else F.shape[1]
            if G is None:
                G = np.empty_like(F)
            fp, gp = F.ctypes.data, G.ctypes.data
        else:
            m = 1 if F.dim() == 1 else F.shape[1]
            if G is None:
                G = F.new_empty(F.shape)
            fp, gp = F.data_ptr(), G.data_ptr()
        L.check(self._lib.bf_apply_host(self._h, prec, ctypes.c_void_p(fp), m, ctypes.c_void_p(gp),
                                        _stream_ptr(stream)), "bf_apply_host")
        return G

    # -- NUFFT evaluation (Sec. 3, Eq. tg3) of phases rank 1 on each column half
    def nufft_prepare(self, eps=1e-6):
        """Plan the NUFFT evaluation (bf_nufft_prepare); returns msp."""
        msp = ctypes.c_int()
        L.check(self._lib.bf_nufft_prepare(self._h, float(eps), ctypes.byref(msp)), "bf_nufft_prepare")
        return msp.value

    def nufft_apply(self, F, G=None, stream=None):
        """G = K F by 2 r_alpha 1-D NUFFTs (bf_nufft_apply); F, G contiguous CUDA complex64."""
        import torch
        if F.dtype != torch.complex64 or not F.is_cuda or not F.is_contiguous():
            raise ValueError("F must be a contiguous CUDA complex64 tensor")
        m = 1 if F.dim() == 1 else F.shape[1]
        if G is None:
            G = torch.empty_like(F)
        L.check(self._lib.bf_nufft_apply(self._h, ctypes.c_void_p(F.data_ptr()), m, ctypes.c_void_p(G.data_ptr()),
                                         _stream_ptr(stream)), "bf_nufft_apply")
        return G

    def nufft_info(self):
        msp, ra, wb = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
        L.check(self._lib.bf_nufft_info(self._h, ctypes.byref(msp), ctypes.byref(ra), ctypes.byref(wb)),
                "bf_nufft_info")
        return {"msp": msp.value, "r_alpha": ra.value, "ws_bytes_per_rhs": wb.value}

    def sync_status(self, stream=None):
        return self._lib.bf_sync_status(self._h, _stream_ptr(stream))


def tile_shapes(plan, m):
    """The FP32 apply's level-tile shapes for (plan, m) (bf_autotune_get): dict of mr,
    levels_per_pass, tpc_front, tpc_back."""
    v = [ctypes.c_int() for _ in range(4)]
    L.check(L.lib().bf_autotune_get(plan._h, int(m), *[ctypes.byref(x) for x in v]), "bf_autotune_get")
    return dict(zip(("mr", "levels_per_pass", "tpc_front", "tpc_back"), (x.value for x in v)))


def autotune(plan, m, cache_path=None):
    """Time the level-tile shape candidates of the FP32 apply for (plan, m); returns mr
    (the other chosen shapes: tile_shapes)."""
    mr = ctypes.c_int()
    L.check(L.lib().bf_autotune(plan._h, int(m), None if cache_path is None else str(cache_path).encode(),
                                ctypes.byref(mr)), "bf_autotune")
    return mr.value


def apply_batched(items, stream=None):
    """One-call batched FP32 apply (bf_apply_batched): ``items`` is a list of
    (plan, F, G), F and G contiguous CUDA complex64 tensors of shape (N, m).
    Asynchronous on ``stream``; repeated calls with the same plans and m reuse
    the thread's kept batch (no allocation)."""
    lib = L.lib()
    n = len(items)
    plans = (ctypes.c_void_p * n)()
    arr = (L.ApplyItem * n)()
    for i, (plan, F, G) in enumerate(items):
        plans[i] = plan._h.value
        arr[i].F, arr[i].G, arr[i].m = F.data_ptr(), G.data_ptr(), 1 if F.dim() == 1 else F.shape[1]
    L.check(lib.bf_apply_batched(ctypes.cast(plans, ctypes.c_void_p), ctypes.cast(arr, ctypes.c_void_p), n,
                                 _stream_ptr(stream)), "bf_apply_batched")


def apply_batched_release():
    """Free the calling thread's kept batch (bf_apply_batched_release)."""
    L.lib().bf_apply_batched_release()


class ShardedApply:
    """One operator applied by ``nshard`` shards (bf_shard.h): shard s holds the
    rows [s N/G, (s+1) N/G) of F and of G, applies the xi-side half (front) to
    its rows, the switch-level coefficients are exchanged all-to-all, and it
    applies the x-side half (back).  ``apply_distributed`` runs one shard per
    rank of a torch.distributed group; ``apply_local`` runs every shard in this
    process on one device (the exchange becomes a block transpose)."""

    def __init__(self, plan, nshard, m):
        self.plan, self.G, self.m = plan, int(nshard), int(m)
        c = ctypes.c_int64()
        L.check(L.lib().bf_shard_info(plan._h, self.G, self.m, ctypes.byref(c)), "bf_shard_info")
        self.chunk = c.value                      # c64 elements per peer block
        self.rows = plan.info()["N"] // self.G

    def front(self, shard, F_rows, W_send, stream=None):
        L.check(L.lib().bf_apply_shard_front(self.plan._h, self.G, int(shard), ctypes.c_void_p(F_rows.data_ptr()),
                                             self.m, ctypes.c_void_p(W_send.data_ptr()), _stream_ptr(stream)),
                "bf_apply_shard_front")

    def back(self, shard, W_recv, G_rows, stream=None):
        L.check(L.lib().bf_apply_shard_back(self.plan._h, self.G, int(shard), ctypes.c_void_p(W_recv.data_ptr()),
                                            self.m, ctypes.c_void_p(G_rows.data_ptr()), _stream_ptr(stream)),
                "bf_apply_shard_back")

    def apply_distributed(self, F_rows, G_rows, group=None, stream=None):
        """This rank's shard: front, one all-to-all of equal blocks, back."""
        import torch
        import torch.distributed as dist
        rank = dist.get_rank(group)
        send = torch.empty(self.G * self.chunk, dtype=torch.complex64, device=F_rows.device)
        recv = torch.empty_like(send)
        self.front(rank, F_rows, send, stream)
        dist.all_to_all_single(torch.view_as_real(recv), torch.view_as_real(send), group=group)
        self.back(rank, recv, G_rows, stream)

    def apply_local(self, F, G):
        """All shards in this process: F, G (N, m) complex64 on one device."""
        import torch
        send = torch.empty((self.G, self.G * self.chunk), dtype=torch.complex64, device=F.device)
        for s in range(self.G):
            self.front(s, F[s * self.rows:(s + 1) * self.rows], send[s])
        recv = send.view(self.G, self.G, self.chunk).transpose(0, 1).contiguous().view(self.G, -1)
        for d in range(self.G):
            self.back(d, recv[d], G[d * self.rows:(d + 1) * self.rows])


class Batch:
    """Many operators of different N and m applied in one persistent launch
    (bf_batch_*).  ``items``: list of (plan, F, G) with F, G contiguous CUDA
    complex64 tensors of shape (N, m); they must outlive the batch."""

    def __init__(self, items):
        self._lib = L.lib()
        self._keep = list(items)
        arr = (L.BatchItem * len(items))()
        for i, (plan, F, G) in enumerate(items):
            m = 1 if F.dim() == 1 else F.shape[1]
            arr[i].plan, arr[i].F, arr[i].G, arr[i].m = plan._h.value, F.data_ptr(), G.data_ptr(), m
        self._h = ctypes.c_void_p()
        L.check(self._lib.bf_batch_create(ctypes.cast(arr, ctypes.c_void_p), len(items), ctypes.byref(self._h)),
                "bf_batch_create")

    def run(self, stream=None):
        L.check(self._lib.bf_batch_run(self._h, _stream_ptr(stream)), "bf_batch_run")

    def capture(self, stream):
        L.check(self._lib.bf_batch_capture_graph(self._h, _stream_ptr(stream)), "bf_batch_capture_graph")

    def replay(self, stream=None):
        L.check(self._lib.bf_batch_replay(self._h, _stream_ptr(stream)), "bf_batch_replay")

    def status(self, stream=None):
        return self._lib.bf_batch_status(self._h, _stream_ptr(stream))

    def info(self):
        w, g, ws, sm = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64()
        L.check(self._lib.bf_batch_get_info(self._h, ctypes.byref(w), ctypes.byref(g), ctypes.byref(ws),
                                            ctypes.byref(sm)), "bf_batch_get_info")
        return {"work_items": w.value, "grid": g.value, "ws_bytes": ws.value, "smem": sm.value}

    def set_spin_limit(self, polls):
        L.check(self._lib.bf_batch_set_spin_limit(self._h, int(polls)), "bf_batch_set_spin_limit")

    def set_mode(self, mode):
        """0: one persistent launch (default); 1: a front and a back launch over all operators."""
        L.check(self._lib.bf_batch_set_mode(self._h, int(mode)), "bf_batch_set_mode")

    def mode(self):
        v = ctypes.c_int()
        L.check(self._lib.bf_batch_get_mode(self._h, ctypes.byref(v)), "bf_batch_get_mode")
        return v.value

    def tune(self, stream=None):
        """Time the three modes and keep the fastest; returns (mode, [ms of modes 0, 1, 2])."""
        mo = ctypes.c_int()
        ms = (ctypes.c_double * 2)()
        L.check(self._lib.bf_batch_tune(self._h, _stream_ptr(stream), ctypes.byref(mo), ms), "bf_batch_tune")
        al = (ctypes.c_double * 3)()
        L.check(self._lib.bf_batch_tune_times(self._h, al, 3), "bf_batch_tune_times")
        return mo.value, [al[0], al[1], al[2]]

    def debug_hold(self, on=True):
        L.check(self._lib.bf_batch_debug_hold(self._h, int(on)), "bf_batch_debug_hold")

    def close(self):
        if self._h:
            self._lib.bf_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request loop over resident operators (bf_server_*)."""

    def __init__(self, n_slots=4, hbm_budget=0, max_batch_rhs=256, precision=F32, per_request=False, device=0,
                 n_priority_slots=-1, small_units=0, method=0, nufft_eps=1e-6):
        """``method``: 0 = the butterfly apply for every operator; 1 = Sec. 3's choice per operator
        (the NUFFT where the phase is rank 1 on the column halves, the butterfly otherwise)."""
        self._lib = L.lib()
        o = L.ServerOptions()
        L.check(self._lib.bf_server_default_options(ctypes.byref(o)), "bf_server_default_options")
        o.n_slots, o.hbm_budget, o.max_batch_rhs = n_slots, hbm_budget, max_batch_rhs
        o.precision, o.per_request, o.device = precision, int(per_request), device
        o.n_priority_slots, o.small_units = n_priority_slots, small_units
        o.method, o.nufft_eps = method, nufft_eps
        self._h = ctypes.c_void_p()
        L.check(self._lib.bf_server_create(ctypes.byref(o), ctypes.byref(self._h)), "bf_server_create")
        self._plans = []

    def add(self, plan):
        i = ctypes.c_int()
        L.check(self._lib.bf_server_add_operator(self._h, plan._h, ctypes.byref(i)), "bf_server_add_operator")
        self._plans.append(plan)
        return i.value

    def start(self):
        L.check(self._lib.bf_server_start(self._h), "bf_server_start")

    def submit(self, op, F, G):
        """F, G: C-contiguous host arrays (numpy or pinned CPU tensors) of shape (N, m)."""
        if isinstance(F, np.ndarray):
            m = 1 if F.ndim == 1 else F.shape[1]
            fp, gp = F.ctypes.data, G.ctypes.data
        else:
            m = 1 if F.dim() == 1 else F.shape[1]
            fp, gp = F.data_ptr(), G.data_ptr()
        rid = ctypes.c_uint64()
        L.check(self._lib.bf_server_submit(self._h, op, ctypes.c_void_p(fp), m, ctypes.c_void_p(gp),
                                           ctypes.byref(rid)), "bf_server_submit")
        return rid.value

    def wait(self, rid, timeout_ms=-1.0):
        lat = ctypes.c_double()
        L.check(self._lib.bf_server_wait(self._h, rid, timeout_ms, ctypes.byref(lat)), "bf_server_wait")
        return lat.value

    def drain(self, timeout_ms=-1.0):
        L.check(self._lib.bf_server_drain(self._h, timeout_ms), "bf_server_drain")

    def stats(self):
        st = L.ServerStats()
        L.check(self._lib.bf_server_get_stats(self._h, ctypes.byref(st)), "bf_server_get_stats")
        return {k: getattr(st, k) for k, _ in L.ServerStats._fields_}

    def reset_stats(self):
        L.check(self._lib.bf_server_reset_stats(self._h), "bf_server_reset_stats")

    def close(self):
        if self._h:
            self._lib.bf_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class KernelTimer:
    """Context manager: CUDA-event times of every library kernel launched inside
    (bf_profile_begin/end).  ``.result`` maps kernel name -> (launches, total_ms)."""

    def __enter__(self):
        L.check(L.lib().bf_profile_begin(), "bf_profile_begin")
        return self

    def __exit__(self, *exc):
        lib = L.lib()
        L.check(lib.bf_profile_end(), "bf_profile_end")
        self.result = {}
        for i in range(lib.bf_profile_count()):
            name = ctypes.c_char_p()
            n = ctypes.c_int64()
            ms = ctypes.c_double()
            L.check(lib.bf_profile_get(i, ctypes.byref(name), ctypes.byref(n), ctypes.byref(ms)), "bf_profile_get")
            self.result[name.value.decode()] = (n.value, ms.value)
        return False


def version():
    return L.lib().bf_version().decode()


def fp32_peak(device=0):
    """(SM count, measured FP32 FMA TFLOP/s) of ``device`` (bf_fp32_peak)."""
    sms, tf = ctypes.c_int(), ctypes.c_double()
    L.check(L.lib().bf_fp32_peak(int(device), ctypes.byref(sms), ctypes.byref(tf)), "bf_fp32_peak")
    return sms.value, tf.value


def fp64_peak(device=0):
    """Measured FP64 FMA TFLOP/s of ``device`` (bf_fp64_peak)."""
    tf = ctypes.c_double()
    L.check(L.lib().bf_fp64_peak(int(device), ctypes.byref(tf)), "bf_fp64_peak")
    return tf.value
