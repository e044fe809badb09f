#!/usr/bin/env python
"""Benchmark of the butterfly-factorisation apply (one JSON line on rank 0).

Default workload: the 1D FIO of Sec. 5 with the smooth rank-2 amplitude,
N = 65536, m = 64 complex right-hand sides, complex FP32 apply, BF built to
eps = 1e-6.  One step = one full apply G = K F (amplitude split-in, V, all H
levels, switch, all G levels, U, amplitude split-out).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload fio2|fio1|fio3|fio4|serve5] [--prec f32|f64|bf16x3]

The fio2 line also carries two side measurements of the same operator: the
plan without phase tables ("on_the_fly") and the plan factored from kernel
entries alone ("indirect").

Under torchrun each rank applies its own operator replica to its own m
right-hand sides (weak scaling, no data-path collective).
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BF-apply complex GN·RHS/s at stated rel err vs FP64; % HBM peak; serve p99 ms"
UNIT = "GN·RHS/s"

WORKLOADS = {
    # name: N, m, phase, amp, eps, prec, split, description
    "fio2": dict(N=65536, m=64, phase=1, amp=1, eps=1e-6, prec="f32", split=1,
                 desc="1D FIO Phi=x xi+c(x)|xi|, c=(2+sin 2pi x)/16, alpha=1+0.25 sin(2pi x)cos(2pi xi/N), "
                      "N=65536, m=64 complex Gaussian RHS, complex FP32 apply, eps=1e-6"),
    "fio1": dict(N=1024, m=1, phase=1, amp=0, eps=1e-6, prec="f64", split=1,
                 desc="1D FIO, alpha=1, N=1024, one RHS, FP64 apply, eps=1e-6"),
    "fio4": dict(N=0, m=0, phase=1, amp=1, eps=1e-6, prec="f32", split=1, n_ops=32,
                 desc="32 operators of the fio2 kernel, N = 2^floor(U(12,19)), m ~ U{1..128} (seed 0), one "
                      "persistent batched launch replayed from a CUDA graph, autotuned column slices, complex FP32"),
    "serve5": dict(N=0, m=0, phase=1, amp=1, eps=1e-6, prec="f32", split=1, rate=2000.0, seconds=6.0,
                   rate_light=100.0, seconds_light=4.0,
                   desc="serving: Poisson arrivals (mean 2000 req/s) against 4 resident operators N=2^14,2^16,2^18,2^20 "
                        "of the fio2 kernel, m uniform in {1,4,16,64}, host buffers, continuous batching on 4 slots, "
                        "complex FP32; compared with the plain per-request FP64 form; latency also at 100 req/s"),
    "fio_big": dict(N=1 << 22, m=16, phase=1, amp=1, eps=1e-6, prec="f32", split=1, otf=True,
                    desc="1D FIO as fio2 at N=2^22, m=16, on-the-fly plan (no phase tables; FP32+FP64 tables "
                         "would take ~42 GB), complex FP32 apply, eps=1e-6"),
    "nufft2": dict(N=65536, m=64, phase=1, amp=1, eps=1e-6, prec="f32", split=1,
                   desc="fio2's operator (1D FIO, smooth rank-2 amplitude, N=65536, m=64, complex FP32) evaluated "
                        "by 1-D NUFFTs on the column halves xi >= 0 and xi < 0 (Sec. 3, Eq. tg3), eps=1e-6"),
    "fio3": dict(N=262144, m=256, phase=2, amp=1, eps=1e-6, prec="bf16x3", split=2, l1=5,
                 desc="piecewise FIO (jump at x=1/2), N=262144 as four N/2 sub-BFs, m=256, alpha as fio2, "
                      "split-BF16 tensor-core apply (hi/lo operands, FP32 accumulation), BF eps=1e-6 (r=10) with V "
                      "and U at level 5 (32-index leaf groups: tiles of 2^3 and 2^4 pairs fit tensor memory)"),
}

FP32_LANES_PER_SM = 128
NUM_SMS = 152


def max_over_ranks(x, world, device):
    """The timing rule across ranks: each rank's value reduced with MAX (over the
    process group of the run: NCCL with GPUs, gloo for CPU ranks)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, units_per_rank_step, steps, ms_max):
    """Whole-job throughput in G units/s: the units every rank processed over the
    slowest rank's time (weak scaling: each rank applies its own replica)."""
    return world * units_per_rank_step * steps / (ms_max * 1e-3) / 1e9


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, "fallback"


def tensor_flops(info, m, N, split):
    """Tensor-core FLOPs one launch of front_tc / back_tc issues (all sub-BFs)."""
    r, l1, ra, L, h = info["r"], info["l1"], info["r_alpha"], info["L"], info["h"]
    Nb = N // split
    kH, kG = h - l1, L - l1 - h
    D2 = 2 * r
    SLOT = 16 if D2 <= 16 else 32
    KS = (D2 + 7) // 8 * 8
    KG = 2 * KS
    mr = 128 // ra
    nslice = -(-m // mr)
    mma = 2 * 128 * SLOT * 16
    group = 2 * 3 * (KG // 16) * mma
    TF, TB = 2 ** kH, 2 ** kG
    ntile = (2 ** l1) * (2 ** (L - h)) * nslice
    # the switch runs per region of two pairs: a group-shaped chain with a block-diagonal weight
    front = ntile * (kH * (TF // 2) * group + TF * 3 * (KG // 16) * mma)
    back = (2 ** h) * nslice * (2 ** l1) * kG * (TB // 2) * group
    nblk = split * split
    return {"front_tc": front * nblk, "back_tc": back * nblk}


def algorithmic(info, m, N, split):
    """Algorithmic flops per launch of the front and back kernels and the
    algorithmic bytes of one apply (c64), from the factored form's stages.
    Per column (1 complex mul = 6 flops, real x complex MAC = 4, complex
    MAC = 8): front = 6N + 2^l1 N (6 + 4r) + kH P (12r + 8r^2) + 8 P r^2;
    back = kG P (8r^2 + 16r) + 2^l1 N (4r + 8) + 8N.  Bytes: the phase
    tables EV, EU (2^l1 N each), EH/FG (2r P per level), S (r^2 P), a and b
    (r_alpha N each), all c64, plus F and G (N m each)."""
    r, l1, ra = info["r"], info["l1"], info["r_alpha"]
    L, h = info["L"], info["h"]
    Nb = N // split
    P = Nb // info["n0"]
    kH, kG = h - l1, L - l1 - h
    M = ra * m
    front = M * (6 * Nb + (2 ** l1) * Nb * (6 + 4 * r) + kH * P * (12 * r + 8 * r * r) + 8 * P * r * r)
    back = M * (kG * P * (8 * r * r + 16 * r) + (2 ** l1) * Nb * (4 * r + 8) + 8 * Nb)
    nblk = split * split
    fac = 8 * ((2 ** l1) * Nb * 2 + (kH + kG) * P * 2 * r + P * r * r + 2 * ra * Nb)  # EV, EU, EH/FG, S, a/b
    bytes_apply = nblk * fac + 2 * 8 * N * m
    return front, back, bytes_apply


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while running."""

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        return False

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


KERNEL_SOURCES = {"f32": ("bf_f32_tile.h", "bf_kernels_f32.cu"), "otf": ("bf_f32_tile.h", "bf_kernels_otf.cu"),
                  "tc": ("bf_kernels_tc.cu", "bf_tc.h"), "f64": ("bf_kernels_f64.cu",), "nufft": ("bf_nufft.cu",)}


def kernel_hash(kernel):
    """Hash of the source file(s) of a kernel family ('front_f32' -> f32, 'back_tc' -> tc,
    'front_f32_otf' -> otf, ...)."""
    fam = "nufft" if kernel.startswith("nufft") else next((f for f in ("tc", "f64", "otf") if kernel.endswith("_" + f)),
                                                          "f32")
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[fam]:
        with open(os.path.join(ROOT, "paper_1803_04128_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, workload, m):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or None
    if it was captured from a different kernel source or right-hand-side count."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(workload, {}).get(kernel)
    if not e or e.get("kernel_hash") != kernel_hash(kernel) or e.get("m") != m:
        return None
    return e.get("dram_bytes_per_launch")


def host_cores():
    """Host cores this process may run on (a multi-process launcher's one-thread default
    for OpenMP does not limit the timed CPU baseline, which rank 0 runs alone)."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def cpu_oracle_rate(w, F, G_gpu, budget_s, max_rows=None):
    """Time the FP64 direct oracle on sampled rows (all m RHS); also the rel.
    error of the GPU result on those rows.  Returns a dict."""
    import numpy as np
    from oracle import direct as od
    from paper_1803_04128_gb300 import inputs
    N, m = w["N"], w["m"]
    kind = w["phase"]
    od.set_threads(host_cores())
    # enough rows to keep every host thread busy, fewer for very long rows
    probe = inputs.sample_rows(N, int(min(N, 64, max(8, (1 << 28) // (N * m)))), seed=11)
    t0 = time.perf_counter()
    od.direct(kind, N, F, probe, amp=w["amp"])
    per_row = (time.perf_counter() - t0) / probe.size
    k = int(max(8, min(N, budget_s / max(per_row, 1e-9))))
    if max_rows:
        k = min(k, max_rows)
    rows = inputs.sample_rows(N, k, seed=12)
    t0 = time.perf_counter()
    gd = od.direct(kind, N, F, rows, amp=w["amp"])
    dt = time.perf_counter() - t0
    out = {"value": rows.size * m / dt / 1e9, "unit": UNIT, "cores": od.num_threads(), "kind": "oracle",
           "sample": "%d of N=%d rows x all %d RHS, FP64 direct O(N^2) oracle (compensated sums), %.1f s"
                     % (rows.size, N, m, dt), "seconds": dt}
    if G_gpu is not None:
        g = G_gpu[rows].astype(np.complex128)
        out["rel_err_gpu"] = float(np.linalg.norm(g - gd) / np.linalg.norm(gd))
        out["rows_compared"] = int(rows.size)
    return out


def run_reference(args, w, rank, world):
    if rank != 0:
        return 0
    import numpy as np
    from oracle import direct as od
    from paper_1803_04128_gb300 import inputs
    F = inputs.complex_gaussian(w["N"], w["m"], seed=0)
    od.set_threads(host_cores())
    rows_all = inputs.sample_rows(w["N"], 4096, seed=13)
    probe = rows_all[:4]
    t0 = time.perf_counter()
    od.direct(w["phase"], w["N"], F, probe, amp=w["amp"])
    per_row = (time.perf_counter() - t0) / probe.size
    k = int(max(1, min(rows_all.size // max(1, args.steps + args.warmup), 8.0 / max(per_row, 1e-9))))
    t_total, done = 0.0, 0
    for s in range(args.warmup + args.steps):
        rows = rows_all[(s * k) % rows_all.size:][:k]
        t0 = time.perf_counter()
        od.direct(w["phase"], w["N"], F, rows, amp=w["amp"])
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            t_total += dt
            done += rows.size
    v = done * w["m"] / t_total / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded complex Gaussian F; analytic kernel)",
            "config": {"workload": w["desc"], "N": w["N"], "m": w["m"]},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": od.num_threads(), "kind": "oracle",
                             "sample": "%d rows x all %d RHS per step, FP64 direct oracle" % (k, w["m"])},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def serve_trace(srv, ops, pools, times, opi, ms, warm_s):
    """Submit a request trace at its arrival times; stats of the window after warm_s."""
    start = time.perf_counter()
    reset = False
    for t, o, m in zip(times, opi, ms):
        if not reset and t >= warm_s:
            srv.reset_stats()
            reset = True
        while True:
            dt = start + t - time.perf_counter()
            if dt <= 0:
                break
            if dt > 3e-4:
                time.sleep(dt - 2e-4)
        F, G = pools[(o, int(m))]
        srv.submit(ops[o], F, G)
    st = srv.stats()                       # at the end of the arrival window
    return st


def oracle_rows_err(w, Fh, Gh, nrows, seed=17, G_rows=None, F_dev=None):
    """Relative l2 error (the paper's eps^b over the sampled set) of a GPU result
    against the FP64 direct oracle on ``nrows`` sampled rows, all RHS."""
    import numpy as np
    from oracle import direct as od
    from paper_1803_04128_gb300 import inputs
    if Fh is None:
        Fh = F_dev.cpu().numpy()
    rows = inputs.sample_rows(w["N"], nrows, seed=seed)
    gd = od.direct(w["phase"], w["N"], Fh, rows, amp=w["amp"])
    g = (Gh[rows] if G_rows is None else G_rows).astype(np.complex128)
    return float(np.linalg.norm(g - gd) / np.linalg.norm(gd)), int(rows.size)


def alu_peak_info(local):
    """FP32 FMA peak: derived from the device's SM count and the measured maximum SM
    clock (128 FP32 lanes x 2 flop per SM per clock), with the register-only FMA
    loop's measured figure beside it."""
    import torch
    from paper_1803_04128_gb300 import api
    peaks, src = load_peaks()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    mhz = peaks.get("sm_max_mhz", 2070.0)
    derived = sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
    try:
        sms2, loop = api.fp32_peak(local)
    except Exception:
        loop = None
    return {"peak": derived, "sms": sms, "sm_max_mhz": mhz, "ffma_loop_tflops": loop,
            "peak_source": "%d SMs (from the device) x 128 FP32 lanes x 2 flop x %.0f MHz (%s sm_max_mhz)"
                           % (sms, mhz, src)}


def alu_roof(kernel, flops, avg_ms, alu, traffic=None, **extra):
    achieved = flops / (avg_ms * 1e-3) / 1e12
    d = {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": alu["peak"], "unit": "TFLOP/s",
         "frac": achieved / alu["peak"], "traffic": traffic, "peak_source": alu["peak_source"],
         "ffma_loop_tflops": alu["ffma_loop_tflops"],
         "frac_of_ffma_loop": (achieved / alu["ffma_loop_tflops"]) if alu["ffma_loop_tflops"] else None}
    d.update(extra)
    return d


def run_serving(args, w, rank, world, local, side=False):
    """Continuous-batching server vs the plain per-request FP64 form (config 5).
    Returns the JSON line (side=True: shorter windows, for the default run)."""
    import numpy as np
    import torch

    from paper_1803_04128_gb300 import api, inputs

    Ns = [2 ** 14, 2 ** 16, 2 ** 18, 2 ** 20]
    mset = (1, 4, 16, 64)
    t0 = time.perf_counter()
    # phase tables built on the device (same factors as the host build, seconds faster at N = 2^20)
    plans = [api.Plan(N, eps=w["eps"], phase_kind=w["phase"], amp_kind=w["amp"], device=local,
                      factor_on_device=True) for N in Ns]
    t_factor = time.perf_counter() - t0
    warm = 1.0
    secs, secs_light = (4.0, 6.0) if side else (w["seconds"], w["seconds_light"])

    def pools_for(cdt):
        out = {}
        for o, N in enumerate(Ns):
            for m in mset:
                f = torch.from_numpy(inputs.complex_gaussian(N, m, seed=o * 100 + m)).to(cdt).pin_memory()
                out[(o, m)] = (f, torch.empty_like(f).pin_memory())
        return out

    results = {}
    errs = {}
    # the offered rate of the workload (above the GPU's capacity: throughput under
    # overload), a light rate the server sustains (latency), and the plain form
    # method 0: the butterfly apply for every operator; method 1: Sec. 3's choice per operator
    # (the NUFFT of Eq. tg3 where the phase is rank 1 on the column halves -- all four here)
    # the light (latency) runs first, so that no run follows an overloaded one
    runs = (("batched_f32_light", api.F32, 4, False, torch.complex64, w["rate_light"], secs_light, 0),
            ("auto_method_f32_light", api.F32, 4, False, torch.complex64, w["rate_light"], secs_light, 1),
            ("batched_f32", api.F32, 4, False, torch.complex64, w["rate"], secs, 0),
            ("auto_method_f32", api.F32, 4, False, torch.complex64, w["rate"], secs, 1))
    pools = pools_for(torch.complex64)     # one fixed F per (operator, m), shared by the runs
    for name, prec, slots, per_req, cdt, rate, secs_run, method in runs:
        window = warm + secs_run
        times, opi, ms = inputs.poisson_requests(rate, window, len(Ns), mset, seed=rank)
        # batch width: 256 right-hand sides under overload (throughput); 64 at the light rate,
        # so that a large request never waits for a batch four times its own size (latency)
        srv = api.Server(n_slots=slots, max_batch_rhs=64 if "light" in name else 256, precision=prec,
                         per_request=per_req, device=local, method=method)
        ops = [srv.add(p) for p in plans]
        srv.start()
        # start-up: every (operator, m) served once before the trace, so that first-use costs
        # (kernel loading, first touches) stay out of the statistics
        for (o, mm), (F, G) in pools.items():
            srv.wait(srv.submit(ops[o], F, G), 120000.0)
        srv.reset_stats()
        with ClockSampler(local) as clk:
            st = serve_trace(srv, ops, pools, times, opi, ms, warm)
        st["clocks"] = clk.summary()
        st["offered_req_per_s"] = rate
        st["window_s"] = window - warm
        st["served_req_per_s"] = st["completed"] / st["wall_s"] if st["wall_s"] > 0 else 0.0
        results[name] = st
        if name in ("batched_f32_light", "auto_method_f32_light"):
            # the light run's queue empties: once drained, every pool buffer that served a
            # request holds that request's result (one fixed F per (operator, m)); sampled
            # rows of the N = 2^16 operator's m = 16 result against the oracle
            srv.drain()
            o, mm = 1, 16
            if any(int(a) == o and int(b) == mm for a, b in zip(opi, ms)):
                Fh = inputs.complex_gaussian(Ns[o], mm, seed=o * 100 + mm)
                errs[name.replace("_light", "")] = oracle_rows_err(dict(w, N=Ns[o]), Fh, pools[(o, mm)][1].numpy(),
                                                                     48)[0]
        srv.close()                        # drops requests still queued (the overloaded runs)
    # the plain per-request form: one request at a time, FP64 stage launches, host buffers
    # (bf_apply_host: copies in, apply, copies out).  Its capacity for the trace's mix (operator
    # and m independent and uniform) is sum_N N E[m] / sum_N t_N(E[m]); with the time linear in m
    # (measured at m = 16 per operator) that is sum_N N / sum_N (t_N(16) / 16).  At small m the
    # plain form is latency-bound, so this overstates it, which only lowers the ratio below.
    t_col = []
    for pl, N in zip(plans, Ns):
        Fh = inputs.complex_gaussian(N, 16, seed=116 + N)
        Fp = torch.from_numpy(Fh).pin_memory()
        Gp = torch.empty_like(Fp).pin_memory()
        pl.apply_host(Fp, Gp, api.F64)            # warm-up (graph capture of the stage launches)
        t0 = time.perf_counter()
        pl.apply_host(Fp, Gp, api.F64)
        t_col.append((time.perf_counter() - t0) / 16)
        if N == Ns[1]:
            errs["plain_f64_per_request"] = oracle_rows_err(dict(w, N=N), Fh, Gp.numpy(), 48)[0]
    p = {"units_per_s": sum(Ns) / sum(t_col), "seconds_per_column": dict(zip(map(str, Ns), t_col)),
         "method": "bf_apply_host FP64 (plain per-stage form) of one m = 16 request per operator, timed on the "
                   "host; capacity of the trace's mix = sum_N N / sum_N t_N(16)/16"}
    b = results["batched_f32"]
    bl = results["batched_f32_light"]
    units_all = b["units_per_s"]
    if world > 1:  # each rank serves its own trace on its own GPU: the job's rate is the sum
        import torch.distributed as dist
        t = torch.tensor([b["units_per_s"]], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        units_all = float(t.item())
    # algorithmic flops per served N.RHS unit, averaged over the trace's operator mix
    flops_per_unit = 0.0
    for pl, N in zip(plans, Ns):
        fr, bk, _ = algorithmic(pl.info(), 1, N, 1)
        flops_per_unit += (fr + bk) / N / len(Ns)
    r_used = plans[0].info()["r"]
    for pl in plans:
        pl.close()
    cfg = {"workload": w["desc"], "operators_N": Ns, "m_choices": list(mset), "r": r_used,
           "eps": w["eps"], "t_factor_s": round(t_factor, 2), "warmup_s": warm,
           "batched_f32": {k: v for k, v in b.items() if k != "clocks"},
           "batched_f32_light": {k: v for k, v in bl.items() if k != "clocks"},
           "auto_method_f32": {k: v for k, v in results["auto_method_f32"].items() if k != "clocks"},
           "auto_method_f32_light": {k: v for k, v in results["auto_method_f32_light"].items() if k != "clocks"},
           "auto_method_note": "the same trace served with Sec. 3's choice per operator: every operator here has a "
                               "phase that is rank 1 on the column halves, so all four are evaluated by the NUFFT "
                               "of Eq. tg3 (bf_nufft_apply) instead of the butterfly",
           "plain_f64_per_request": p,
           "throughput_ratio_vs_plain": (b["units_per_s"] / p["units_per_s"]) if p["units_per_s"] else None,
           "rel_err_vs_fp64_oracle": errs,
           "rel_err_note": "48 sampled rows, all 16 RHS, of an N = 2^16, m = 16 request's result (served by the "
                           "light run; the plain form's apply of an m = 16 request)",
           "note": "stats over the arrival window after warm-up; requests still queued at its end are "
                   "counted in 'pending' and not in the latency percentiles.  At the offered 2000 req/s the "
                   "work arriving exceeds the GPU's capacity, so its p50/p99 measure queue growth over the "
                   "window; p50_ms/p99_ms of this line are those of the light rate, which the server sustains"}
    alu = alu_peak_info(local)
    ach = b["units_per_s"] * flops_per_unit / 1e12
    roof = {"bound": "alu", "kernel": "all kernels of the served applies (front_f32, back_f32, level passes)",
            "achieved": ach, "peak": alu["peak"], "unit": "TFLOP/s", "frac": ach / alu["peak"], "traffic": None,
            "note": "algorithmic flops of the served N.RHS units (mean over the 4 operators) per second of the "
                    "offered-rate window: a whole-server figure, copies and scheduling included",
            "peak_source": alu["peak_source"]}
    line = {"metric": METRIC, "value": units_all / 1e9, "unit": UNIT, "n_gpus": world,
            "steps": int(b["completed"]), "warmup": warm, "ms_per_step": b["mean_ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded complex Gaussian F; analytic kernel; Poisson arrivals)", "config": cfg,
            "p50_ms": bl["p50_ms"], "p99_ms": bl["p99_ms"], "p99_ms_at_offered_rate": b["p99_ms"],
            "auto_method": {"units_per_s": results["auto_method_f32"]["units_per_s"],
                            "p50_ms": results["auto_method_f32_light"]["p50_ms"],
                            "p99_ms": results["auto_method_f32_light"]["p99_ms"],
                            "throughput_ratio_vs_plain": results["auto_method_f32"]["units_per_s"] / p["units_per_s"]},
            "roofline": roof, "cpu_baseline": None,
            "e2e": {"value": units_all / 1e9, "unit": UNIT, "h2d_bytes_per_step": None,
                    "d2h_bytes_per_step": None, "note": "requests are served from host buffers"},
            "gpu_launches": int(b["launches"]), "clocks": b["clocks"]}
    return line


def run_batched(args, w, rank, world, local, steps=None, warmup=None):
    """32 uneven operators applied in one persistent launch replayed from a CUDA graph.
    Returns the JSON line."""
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1803_04128_gb300 import api, inputs

    steps = steps or args.steps
    warmup = warmup if warmup is not None else args.warmup
    shapes = inputs.uneven_batch(w["n_ops"], 12, 18, 1, 128, seed=0)
    t0 = time.perf_counter()
    plans = {}
    for N, _ in shapes:
        if N not in plans:
            plans[N] = api.Plan(N, eps=w["eps"], phase_kind=w["phase"], amp_kind=w["amp"], device=local)
    t_factor = time.perf_counter() - t0
    tune_path = os.path.join(tempfile.gettempdir(), "bf_autotune_%d.txt" % os.getpid())
    t0 = time.perf_counter()
    for N, m in shapes:
        api.autotune(plans[N], m, tune_path)
    t_tune = time.perf_counter() - t0
    ops, Fh = [], []
    for k, (N, m) in enumerate(shapes):
        f = inputs.complex_gaussian(N, m, seed=1000 * rank + k)
        Fh.append(f)
        F = torch.from_numpy(f).to(torch.complex64).cuda()
        ops.append((plans[N], F, torch.empty_like(F)))
    batch = api.Batch(ops)
    stream = torch.cuda.Stream()
    # one persistent launch (mode 0) or a front and a back launch over all operators (mode 1):
    # timed on the device, the faster kept (bitwise the same results)
    mode, mode_ms = batch.tune(stream)
    batch.capture(stream)
    units = sum(N * m for N, m in shapes)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            flush.zero_()
            batch.replay(stream)
    stream.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with ClockSampler(local) as clk:
        with torch.cuda.stream(stream):
            for i in range(steps):
                flush.zero_()
                ev[i][0].record(stream)
                batch.replay(stream)
                ev[i][1].record(stream)
        stream.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    assert batch.status(stream) == 0
    ms = sum(a.elapsed_time(b) for a, b in ev)
    ms_max = max_over_ranks(ms, world, "cuda")
    value = job_rate(world, units, steps, ms_max)
    # sampled rows of every operator's result against the FP64 oracle
    num = den = 0.0
    for k, ((N, m), (plan, F, G)) in enumerate(zip(shapes, ops)):
        rows = inputs.sample_rows(N, 8, seed=100 + k)
        from oracle import direct as od
        gd = od.direct(w["phase"], N, Fh[k], rows, amp=w["amp"])
        g = G.cpu().numpy()[rows].astype(np.complex128)
        num += float(np.linalg.norm(g - gd) ** 2)
        den += float(np.linalg.norm(gd) ** 2)
    rel_err = (num / den) ** 0.5
    # kernel time of the persistent launch, issued eagerly (graph replays bypass the launch hooks)
    with api.KernelTimer() as kt_eager:
        with torch.cuda.stream(stream):
            for _ in range(3):
                flush.zero_()
                batch.run(stream)
        stream.synchronize()
    # the same 32 applies issued one operator at a time (2 launches each), for comparison,
    # with the same L2 flush before each step
    torch.cuda.synchronize()
    seq = []
    for _ in range(steps):
        flush.zero_()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record()
        for plan, F, G in ops:
            plan.apply(F, G, api.F32)
        s1.record()
        seq.append((s0, s1))
    torch.cuda.synchronize()
    seq_ms = sum(a.elapsed_time(b) for a, b in seq) / steps
    peaks, peak_src = load_peaks()
    alu = alu_peak_info(local)
    flops = 0
    bytes_apply = 0
    for N, m in shapes:
        info = plans[N].info()
        fr, bk, by = algorithmic(info, m, N, 1)
        flops += fr + bk
        bytes_apply += by
    roof = None
    nb, tb = kt_eager.result.get("batch_f32", (0, 0.0))
    if nb:
        roof = alu_roof("batch_f32", flops, tb / nb, alu, ncu_traffic("batch_f32", "fio4", None),
                        kernel_ms={k: v[1] / v[0] for k, v in kt_eager.result.items()})
    elif "batch_front_f32" in kt_eager.result:
        # mode 1: the apply's algorithmic flops over the two phase launches' summed time
        tot = sum(v[1] for v in kt_eager.result.values())
        n3 = kt_eager.result["batch_front_f32"][0]
        roof = alu_roof("batch_front_f32 + batch_back_f32", flops, tot / n3, alu, None,
                        kernel_ms={k: v[1] / v[0] for k, v in kt_eager.result.items()})
    elif kt_eager.result:
        # mode 2: the operators' own front / back launches run concurrently on four streams, so
        # the batch's algorithmic flops are taken over its whole step time (graph replay)
        roof = alu_roof("front_f32 + back_f32 (each operator's own apply, 4 streams)", flops, ms_max / steps, alu,
                        None, kernel_ms={k: v[1] / v[0] for k, v in kt_eager.result.items()},
                        launches_per_step={k: v[0] / 3 for k, v in kt_eager.result.items()})
    launches_per_step = sum(v[0] for v in kt_eager.result.values()) / 3 if kt_eager.result else 1
    # end to end: pinned host F in, graph replay, G out
    Fp = [torch.from_numpy(f).to(torch.complex64).pin_memory() for f in Fh]
    Gp = [torch.empty_like(x).pin_memory() for x in Fp]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for _ in range(steps):
            for (plan, F, G), fp in zip(ops, Fp):
                F.copy_(fp, non_blocking=True)
            batch.replay(stream)
            for (plan, F, G), gp in zip(ops, Gp):
                gp.copy_(G, non_blocking=True)
            stream.synchronize()
    t_e2e = time.perf_counter() - t0
    nbytes = sum(x.numel() * x.element_size() for x in Fp)
    cfg = {"workload": w["desc"], "n_ops": len(shapes), "shapes": shapes, "units_per_step": units,
           "r": plans[shapes[0][0]].info()["r"], "eps": w["eps"], "l2": "flushed (512 MB write) between timed steps",
           "t_factor_s": round(t_factor, 2), "t_autotune_s": round(t_tune, 2),
           "tile_shapes": [dict(api.tile_shapes(plans[N], m), N=N, m=m) for N, m in shapes],
           "batch_mode": {"chosen": mode, "ms_mode0_one_persistent_launch": mode_ms[0],
                          "ms_mode1_front_and_back_launches": mode_ms[1],
                          "ms_mode2_own_applies_on_4_streams": mode_ms[2]},
           "sequential_single_op_ms_per_step": seq_ms, "batched_ms_per_step": ms_max / steps,
           "speedup_batched_vs_sequential": seq_ms / (ms_max / steps),
           "hbm_frac_of_measured": bytes_apply / (ms_max / steps * 1e-3) / (peaks["hbm_gbs"] * 1e9),
           "algorithmic_flops_per_step": flops, "algorithmic_bytes_per_step": bytes_apply,
           "rel_err_vs_fp64_oracle": rel_err, "rel_err_rows": "8 sampled rows of each of the 32 results, all RHS",
           "parallelism": "replicas" if world > 1 else "single GPU"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
            "warmup": warmup, "ms_per_step": ms_max / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded complex Gaussian F; analytic kernel)", "config": cfg, "roofline": roof,
            "cpu_baseline": None,
            "e2e": {"value": world * units * steps / t_e2e / 1e9, "unit": UNIT,
                    "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes},
            "gpu_launches": int(round(steps * launches_per_step)), "clocks": clk.summary()}
    batch.close()
    for pl in plans.values():
        pl.close()
    return line


def otf_side(args, w, plan, F, G, flush, stream, world, local, alu_peak, front, back):
    """Time the on-the-fly plan of the same operator (bf_factor_otf) with the main
    line's protocol; its result is compared with the table apply's G."""
    import torch
    from paper_1803_04128_gb300 import api
    N, m = w["N"], w["m"]
    t0 = time.perf_counter()
    po = api.Plan(N, eps=w["eps"], phase_kind=w["phase"], amp_kind=w["amp"], split=w["split"], device=local,
                  on_the_fly=True)
    t_factor = time.perf_counter() - t0
    tune_path = os.path.join(tempfile.gettempdir(), "bf_autotune_bench_otf_%d.txt" % os.getpid())
    mr = api.autotune(po, m, tune_path)
    po.reserve(api.F32, m)
    Go = torch.empty_like(F)
    for _ in range(args.warmup):
        flush.zero_()
        po.apply(F, Go, api.F32)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with api.KernelTimer() as kt:
        torch.cuda.nvtx.range_push("timed_otf")
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            po.apply(F, Go, api.F32)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    assert po.sync_status() == 0
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), world, "cuda")
    rel = float((Go - G).norm() / G.norm())
    io, it = po.info(), plan.info()
    km = {k: v[1] / v[0] for k, v in kt.result.items()}
    out = {"value": job_rate(world, N * m, args.steps, ms), "unit": UNIT, "ms_per_step": ms / args.steps,
           "dev_bytes_f32": io["dev_bytes_f32"], "dev_bytes_f32_with_tables": it["dev_bytes_f32"],
           "dev_bytes_f64_with_tables": it["dev_bytes_f64"], "t_factor_s": round(t_factor, 3),
           "mr_autotuned": mr, "rel_diff_vs_table_apply": rel, "kernel_ms": km,
           "traffic": {k: ncu_traffic(k, args.workload, m) for k in ("front_f32_otf", "back_f32_otf")}}
    if "front_f32_otf" in km:
        out["alu_frac_algorithmic"] = {
            "front_f32_otf": front / (km["front_f32_otf"] * 1e-3) / 1e12 / alu_peak,
            "back_f32_otf": back / (km["back_f32_otf"] * 1e-3) / 1e12 / alu_peak}
        out["note"] = ("algorithmic flops of the apply (the phase evaluation is extra work) over each kernel's "
                       "CUDA-event time, against the FP32 FMA peak")
    po.close()
    return out


def nufft_bytes(N, m, ra, msp):
    """Algorithmic DRAM bytes of the three NUFFT kernels (c64 = 8 B): pass 1 reads F and the
    deconvolution factors and writes the four-step intermediate T (both column halves, n = N
    grid points, r_alpha m columns); pass 2 reads T and writes the grid H; the interpolation
    reads H, its weights, windows and prefactors, and writes G.  T and H are each written and
    read once: a grid of n r_alpha m points per half does not fit on chip, so this is the
    traffic of a two-pass FFT."""
    M, n, Mc = N // 2, N, ra * m
    grid = 2 * n * Mc * 8
    return {"nufft_pass1": N * m * 8 + 2 * ra * M * 8 + grid,
            "nufft_pass2": 2 * grid,
            "nufft_interp": grid + 2 * N * (2 * msp * 4 + 4 + ra * 8) + N * m * 8}


def nufft_side(w, F, G, flush, stream, local, steps, warmup):
    """The same operator evaluated by 1-D NUFFTs on the two column halves (Sec. 3, Eq. tg3;
    bf_nufft_apply), timed with the main line's protocol; error against the oracle on sampled
    rows and difference from the butterfly apply's G."""
    import torch
    from paper_1803_04128_gb300 import api
    N, m = w["N"], w["m"]
    t0 = time.perf_counter()
    pn = api.Plan(N, eps=w["eps"], phase_kind=w["phase"], amp_kind=w["amp"], device=local, factor=False)
    msp = pn.nufft_prepare(w["eps"])
    t_prep = time.perf_counter() - t0
    Gn = torch.empty_like(F)
    for _ in range(warmup):
        flush.zero_()
        pn.nufft_apply(F, Gn)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with api.KernelTimer() as kt:
        for i in range(steps):
            flush.zero_()
            ev[i][0].record(stream)
            pn.nufft_apply(F, Gn)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    info = pn.nufft_info()
    peaks, src = load_peaks()
    byt = nufft_bytes(N, m, info["r_alpha"], msp)
    km = {k: v[1] / v[0] for k, v in kt.result.items()}
    tot = sum(v[1] for v in kt.result.values())
    dom = max(km, key=lambda k: kt.result[k][1])
    ach = byt[dom] / (km[dom] * 1e-3) / 1e9
    roof = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": ach / peaks["hbm_gbs"], "traffic": ncu_traffic(dom, "fio2", m),
            "algorithmic_bytes_per_launch": byt, "kernel_ms": km,
            "share": {k: v[1] / tot for k, v in kt.result.items()},
            "apply_frac": sum(byt.values()) / (ms / steps * 1e-3) / 1e9 / peaks["hbm_gbs"],
            "peak_source": "measured copy bandwidth (%s)" % src}
    Gh = Gn.cpu().numpy()
    err, nrows = oracle_rows_err(w, None, Gh, w.get("err_rows", 256), G_rows=None, F_dev=F)
    out = {"value": N * m * steps / (ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ms / steps, "msp": msp,
           "t_prepare_s": round(t_prep, 3), "rel_err_vs_fp64_oracle": err, "rel_err_rows": nrows,
           "rel_diff_vs_butterfly_apply": None if G is None else float((Gn - G).norm() / G.norm()),
           "roofline": roof,
           "gpu_launches": sum(v[0] for v in kt.result.values()),
           "method": "2 r_alpha 1-D type-2 NUFFTs (Gaussian gridding, grid 2x the modes, msp points each side) "
                     "on the column halves xi >= 0 and xi < 0, where the phase is (x +- c(x)) xi"}
    pn.close()
    return out


def run_nufft(args, w, rank, world, local):
    """The NUFFT evaluation as the main line (bf_nufft_apply; same protocol as the butterfly
    line, L2 flushed between timed applies); its own roofline and oracle error."""
    import torch
    import torch.distributed as dist
    from paper_1803_04128_gb300 import inputs
    Fh = inputs.complex_gaussian(w["N"], w["m"], seed=rank)
    F = torch.from_numpy(Fh).to(torch.complex64).cuda()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    if world > 1:
        dist.barrier()
    with ClockSampler(local) as clk:
        d = nufft_side(w, F, None, flush, stream, local, args.steps, args.warmup)
    ms = max_over_ranks(d["ms_per_step"] * args.steps, world, "cuda")
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_rate(w, Fh, None, args.cpu_budget)
    line = {"metric": METRIC, "value": job_rate(world, w["N"] * w["m"], args.steps, ms), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded complex Gaussian F; analytic kernel)",
            "config": {"workload": w["desc"], "N": w["N"], "m": w["m"], "eps": w["eps"], "msp": d["msp"],
                       "l2": "flushed (512 MB write) between timed steps",
                       "rel_err_vs_fp64_oracle": d["rel_err_vs_fp64_oracle"], "rel_err_rows": d["rel_err_rows"]},
            "roofline": d["roofline"], "cpu_baseline": cpu, "e2e": None, "gpu_launches": d["gpu_launches"],
            "clocks": clk.summary()}
    return line


def indirect_side(w, F, G, local):
    """The same operator factored from its entries alone (indirect access, Scenario 1
    of Sec. 2.2): amplitude by Algorithm 1 on |K|, phase by Algorithms 3-5, on the
    host.  One FP32 apply of it is compared with the table apply's G."""
    import torch
    from paper_1803_04128_gb300 import api
    N = w["N"]
    t0 = time.perf_counter()
    pi = api.Plan(N, eps=w["eps"], phase_kind=w["phase"], amp_kind=w["amp"], split=w["split"], device=local,
                  indirect=True)
    t_factor = time.perf_counter() - t0
    Gi = torch.empty_like(F)
    pi.apply(F, Gi, api.F32)
    torch.cuda.synchronize()
    assert pi.sync_status() == 0
    info = pi.info()
    pi.close()
    return {"t_recover_s": round(info["t_recover_s"], 3), "t_factor_s": round(t_factor, 3),
            "phase_rank": info["phase_rank"], "recover_err_k": info["recover_err_k"],
            "recover_err_amp": info["recover_err_amp"],
            "rel_diff_vs_table_apply": float((Gi - G).norm() / G.norm()),
            "note": "t_recover_s: host recovery of amplitude and phase from kernel entries (part of t_factor_s, "
                    "which adds the butterfly construction); recover_err_k/amp: eps^K, eps^amp of Sec. 5 on "
                    "256 x 256 sampled entries"}


def run_single(args, w, rank, world, local, steps, warmup, plan=None, sides=True, cpu_budget=None):
    """One operator (or one split operator) applied to m right-hand sides: W warm-up
    applies, then ``steps`` timed applies (CUDA events on the launching stream, L2
    flushed between them).  Returns the JSON line.  ``plan``: an already factored plan
    of the same operator (shared by two precisions of one workload)."""
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1803_04128_gb300 import api, inputs

    def barrier():
        if world > 1:
            dist.barrier()

    N, m = w["N"], w["m"]
    prec = {"f64": api.F64, "f32": api.F32, "bf16x3": api.BF16X3}[w["prec"]]
    cdt = torch.complex128 if prec == api.F64 else torch.complex64
    otf = bool(w.get("otf"))
    own_plan = plan is None
    t_factor = t_factor_dev = None
    if own_plan:
        t0 = time.perf_counter()
        plan = api.Plan(N, eps=w["eps"], phase_kind=w["phase"], amp_kind=w["amp"], split=w["split"], device=local,
                        on_the_fly=otf, factor_on_device=bool(w.get("factor_on_device")), l1=w.get("l1", 0))
        t_factor = time.perf_counter() - t0
        # the same operator with its phase tables built on the GPU (bf_factor_device), for the record
        if sides and not otf and not w.get("factor_on_device"):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            api.Plan(N, eps=w["eps"], phase_kind=w["phase"], amp_kind=w["amp"], split=w["split"], device=local,
                     factor_on_device=True, l1=w.get("l1", 0)).close()
            torch.cuda.synchronize()
            t_factor_dev = time.perf_counter() - t0
    info = plan.info()
    mr_tuned = None
    if prec == api.F32:
        # column-slice width of the fused FP32 apply chosen by timing (off the timed region)
        tune_path = os.path.join(tempfile.gettempdir(), "bf_autotune_bench_%d.txt" % os.getpid())
        mr_tuned = api.autotune(plan, m, tune_path)
    plan.reserve(prec, m)
    Fh = inputs.complex_gaussian(N, m, seed=rank)
    F = torch.from_numpy(Fh).to(cdt).cuda()
    G = torch.empty_like(F)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")   # > L2 (129 MB)
    stream = torch.cuda.current_stream()

    for _ in range(warmup):
        flush.zero_()
        plan.apply(F, G, prec)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()

    fk, bk = ("front_f32_otf", "back_f32_otf") if otf else ("front_f32", "back_f32")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with ClockSampler(local) as clk:
        with api.KernelTimer() as kt:
            torch.cuda.nvtx.range_push("timed")    # lets an ncu capture select the timed launches
            for i in range(steps):
                flush.zero_()                      # L2 flush between timed steps (not timed)
                ev[i][0].record(stream)
                plan.apply(F, G, prec)
                ev[i][1].record(stream)
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_pop()
    barrier()
    torch.cuda.synchronize()
    assert plan.sync_status() == 0
    ms = sum(a.elapsed_time(b) for a, b in ev)
    ms_max = max_over_ranks(ms, world, "cuda")
    value = job_rate(world, N * m, steps, ms_max)

    peaks, peak_src = load_peaks()
    alu = alu_peak_info(local)
    front, back, bytes_apply = algorithmic(info, m, N, w["split"])
    roof = None
    launches = sum(n for n, _ in kt.result.values())
    tot = sum(v[1] for v in kt.result.values())
    kms = {k: v[1] / v[0] for k, v in kt.result.items()}
    share = {k: v[1] / tot for k, v in kt.result.items()} if tot else {}
    if prec == api.F32 and any(k.startswith("mid_") for k in kt.result):
        # level ranges split into passes (front, middle H and G passes, back): the
        # apply's algorithmic flops over the summed time of all its passes
        roof = alu_roof("all passes of one apply (front, mid_h, mid_g, back)", (front + back) * w["split"] ** 2,
                        tot / steps, alu, None, kernel_ms=kms, share=share)
    elif prec == api.F32 and fk in kt.result:
        nf, tf = kt.result[fk]
        nb, tb = kt.result[bk]
        dom, n_l, t_l, flops = (fk, nf, tf, front) if tf >= tb else (bk, nb, tb, back)
        roof = alu_roof(dom, flops, t_l / n_l, alu, ncu_traffic(dom, w["name"], m), kernel_ms=kms, share=share)
    elif prec == api.BF16X3 and "front_tc" in kt.result:
        tflops = tensor_flops(info, m, N, w["split"])
        dom = max(("front_tc", "back_tc"), key=lambda k: kt.result[k][1])
        n_l, t_l = kt.result[dom]
        achieved = tflops[dom] / (t_l / n_l * 1e-3) / 1e12
        roof = {"bound": "tensor", "kernel": dom, "achieved": achieved, "peak": peaks["bf16_tflops_sustained"],
                "unit": "TFLOP/s", "frac": achieved / peaks["bf16_tflops_sustained"],
                "traffic": ncu_traffic(dom, w["name"], m),
                "note": "tensor FLOPs issued (3 BF16 products per split product, zero padding to the MMA shape); "
                        "peak: sustained cuBLAS BF16 (%s)" % peak_src,
                "useful_alu_frac": (front + back) * w["split"] ** 2 / (tot / steps * 1e-3) / 1e12 / alu["peak"],
                "kernel_ms": kms, "share": share}
    elif kt.result:
        # plain FP64 form: one launch per stage, state through HBM.  Its stage kernels do the
        # apply's algorithmic flops in FP64 (flop/B ~ M_eff / 2 in c128), bound by the FP64
        # pipes: the apply's flops over the summed stage-kernel time against the measured
        # DFMA-loop rate; the HBM fraction of its algorithmic bytes beside it
        import torch  # noqa: F401
        from paper_1803_04128_gb300 import api as _api
        f64_peak = _api.fp64_peak(local)
        achieved = (front + back) * w["split"] ** 2 / (tot / steps * 1e-3) / 1e12
        roof = {"bound": "alu", "kernel": "plain FP64 stages (v/h/s/g/u_f64) per apply", "achieved": achieved,
                "peak": f64_peak, "unit": "TFLOP/s", "frac": achieved / f64_peak, "traffic": None,
                "peak_source": "register-only DFMA loop on this device (bf_fp64_peak)",
                "hbm_frac_algorithmic_bytes": 2 * bytes_apply / (tot / steps * 1e-3) / 1e9 / peaks["hbm_gbs"],
                "note": "algorithmic flops of one apply over the summed stage-kernel time",
                "kernel_ms": kms, "share": share}
    if prec == api.F64:
        bytes_apply *= 2  # complex128 factors and vectors
    hbm_frac = bytes_apply / (ms_max / steps * 1e-3) / (peaks["hbm_gbs"] * 1e9)

    # end to end through bf_apply_host with pinned host buffers
    e2e = None
    if sides and not args.no_e2e:
        Fp = torch.from_numpy(Fh).to(cdt).pin_memory()
        Gp = torch.empty_like(Fp).pin_memory()
        for _ in range(2):
            plan.apply_host(Fp, Gp, prec)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(steps):
            plan.apply_host(Fp, Gp, prec)
        t_e2e = max_over_ranks(time.perf_counter() - t0, world, "cuda")
        nbytes = Fp.numel() * Fp.element_size()
        e2e = {"value": job_rate(world, N * m, steps, 1e3 * t_e2e), "unit": UNIT,
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes}

    # the same operator factored for the on-the-fly apply (no phase tables), timed alike
    otf_d = None
    if sides and prec == api.F32 and not otf and not args.no_otf_side:
        otf_d = otf_side(args, w, plan, F, G, flush, stream, world, local, alu["peak"], front, back)
    ind = None
    if sides and prec == api.F32 and not otf and not args.no_indirect_side and w["N"] > 0:
        ind = indirect_side(w, F, G, local)
    nu = None
    if sides and prec == api.F32 and not otf and w["split"] == 1 and w["phase"] in (0, 1, 2, 3):
        nu = nufft_side(w, F, G, flush, stream, local, steps, warmup)

    Gh = G.cpu().numpy() if rank == 0 else None
    cpu = None
    rel_err = None
    if rank == 0 and world == 1 and sides and not args.no_cpu_baseline:
        cpu = cpu_oracle_rate(w, Fh, Gh, cpu_budget or args.cpu_budget)
        rel_err = (cpu.pop("rel_err_gpu"), cpu.pop("rows_compared"))
    elif rank == 0:
        rel_err = oracle_rows_err(w, Fh, Gh, w.get("err_rows", 32))

    cfg = {"workload": w["desc"], "N": N, "m": m, "r": info["r"], "r_alpha": info["r_alpha"],
           "eps": w["eps"], "L": info["L"], "split": w["split"], "l2": "flushed (512 MB write) between timed steps",
           "t_factor_s": None if t_factor is None else round(t_factor, 3),
           "t_factor_device_s": None if t_factor_dev is None else round(t_factor_dev, 3),
           "plan": "on-the-fly (bf_factor_otf)" if otf else "phase tables",
           "dev_bytes_f32": info["dev_bytes_f32"], "dev_bytes_f64": info["dev_bytes_f64"],
           "mr_autotuned": mr_tuned,
           "tile_shapes": api.tile_shapes(plan, m) if prec == api.F32 else None,
           "parallelism": "replicas" if world > 1 else "single GPU",
           "hbm_frac_of_measured": hbm_frac, "algorithmic_bytes_per_step": bytes_apply,
           "algorithmic_flops_per_step": (front + back) * w["split"] ** 2}
    if rel_err is not None:
        cfg["rel_err_vs_fp64_oracle"], cfg["rel_err_rows"] = rel_err
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
            "warmup": warmup, "ms_per_step": ms_max / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": {api.F64: "f64", api.F32: "f32", api.BF16X3: "bf16x3"}[prec],
            "data": "synthetic (seeded complex Gaussian F; analytic kernel)", "config": cfg,
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk.summary()}
    if otf_d is not None:
        line["on_the_fly"] = otf_d
    if ind is not None:
        line["indirect"] = ind
    if nu is not None:
        line["nufft"] = nu
    if own_plan:
        plan.close()
    del F, G, flush
    torch.cuda.empty_cache()
    return line


def side_lines(args, rank, world, local):
    """The other configurations, measured in the default run beside the headline:
    the plain FP64 per-stage form at the headline's shape, config 1, config 3 (split-BF16 and
    FP32 on the same plan), config 4 (one batched launch against one by one) and
    config 5 (serving).  Each is a full JSON object with its own roofline and error
    against the FP64 oracle on sampled rows."""
    import torch
    from paper_1803_04128_gb300 import api
    out = {}
    st, wu = min(args.steps, 5), 3
    # the plain form: FP64, one launch per stage, state through HBM, on the fio2 operator
    w = dict(WORKLOADS["fio2"], name="fio2", prec="f64", factor_on_device=True, err_rows=32)
    w["desc"] = ("plain FP64 per-stage form (one launch per stage, CUDA-graph replay) at the fio2 shape: "
                 "N=65536, m=64, eps=1e-6")
    out["fp64_plain_fio2"] = run_single(args, w, rank, world, local, st, wu, sides=False)
    # config 1: the plain FP64 form at N = 1024, one right-hand side (every row against the oracle)
    out["fio1"] = run_single(args, dict(WORKLOADS["fio1"], name="fio1", err_rows=1024), rank, world, local, 50, wu,
                             sides=False)
    # config 3: split-BF16 tensor cores (V and U at level 5) and FP32 (the built-in level) on
    # the same operator at the same eps
    w3 = dict(WORKLOADS["fio3"], name="fio3", factor_on_device=True, err_rows=24)
    out["fio3_bf16x3"] = run_single(args, w3, rank, world, local, st, wu, sides=False)
    w3f = dict(w3, prec="f32", l1=0,
               desc="piecewise FIO (jump at x=1/2), N=262144 as four N/2 sub-BFs, m=256, alpha as fio2, complex "
                    "FP32 apply, BF eps=1e-6 (r=10), V and U at the built-in level 4")
    out["fio3_f32"] = run_single(args, w3f, rank, world, local, st, wu, sides=False)
    # the same operator by the NUFFT of Eq. tg3 (its phase is rank 1 on each column half)
    from paper_1803_04128_gb300 import inputs
    F3 = torch.from_numpy(inputs.complex_gaussian(w3["N"], w3["m"], seed=rank)).to(torch.complex64).cuda()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    out["fio3_nufft"] = nufft_side(dict(w3f, err_rows=24), F3, None, flush, torch.cuda.current_stream(), local, st, wu)
    del F3, flush
    torch.cuda.empty_cache()
    torch.cuda.empty_cache()
    out["fio4"] = run_batched(args, dict(WORKLOADS["fio4"], name="fio4"), rank, world, local, steps=st, warmup=wu)
    torch.cuda.empty_cache()
    out["serve5"] = run_serving(args, dict(WORKLOADS["serve5"], name="serve5"), rank, world, local, side=True)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="fio2", choices=sorted(WORKLOADS))
    ap.add_argument("--prec", default=None, choices=["f32", "f64", "bf16x3"])
    ap.add_argument("--eps", type=float, default=None, help="override the BF tolerance of the workload")
    ap.add_argument("--m", type=int, default=None, help="override the right-hand-side count (single-operator workloads)")
    ap.add_argument("--cpu-budget", type=float, default=12.0, help="seconds of oracle work for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-indirect-side", action="store_true",
                    help="skip the plan factored from kernel entries alone (indirect access)")
    ap.add_argument("--otf", action="store_true",
                    help="time the on-the-fly plan (bf_factor_otf, FP32 only) as the main line")
    ap.add_argument("--no-otf-side", action="store_true",
                    help="skip the on-the-fly side measurement of FP32 workloads")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other configurations' side objects of the default fio2 run")
    args = ap.parse_args()
    w = dict(WORKLOADS[args.workload], name=args.workload)
    if args.prec and args.prec != w["prec"]:
        w["prec"] = args.prec
        w["desc"] += " [apply precision overridden to %s]" % args.prec
        if args.prec != "bf16x3" and w.get("l1"):
            w["l1"] = 0                     # the FP32 / FP64 kernels take the built-in V level
            w["desc"] += " [V and U at the built-in level]"
    if args.eps:
        w["eps"] = args.eps
        w["desc"] += " [BF eps overridden to %g]" % args.eps
    if args.m:
        w["m"] = args.m
        w["desc"] += " [m overridden to %d]" % args.m
    if args.otf and not w.get("otf"):
        w["prec"] = "f32"
        w["otf"] = True
        w["desc"] += " [on-the-fly plan: phases evaluated in the kernels]"

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, w, rank, world)

    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if args.workload == "fio4":
        line = run_batched(args, w, rank, world, local)
    elif args.workload == "serve5":
        line = run_serving(args, w, rank, world, local)
    elif args.workload == "nufft2":
        line = run_nufft(args, w, rank, world, local)
    else:
        line = run_single(args, w, rank, world, local, args.steps, args.warmup)
        # the default run also measures the other configurations (one GPU, rank 0 only)
        default_run = (args.workload == "fio2" and not (args.prec or args.eps or args.m or args.otf))
        if default_run and world == 1 and not args.no_configs:
            line["configs"] = side_lines(args, rank, world, local)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
