"""Single-process host logic of bench.py on CPU.

* The algorithmic bytes of one apply (the roofline's numerator for the HBM
  figure) must equal what the plan actually stores in complex form -- the
  phase tables, switch blocks and amplitude factors, counted here from the
  library's own FP64 arrays through bf_plan_view -- plus one read of F and
  one write of G.  This ties the formula to the construction, not to itself.
* The clock summary turns nvidia-smi samples into the median SM clock and
  the set of active throttle reasons that decide whether a run is kept.
* ncu traffic is only reported while the committed capture matches the
  kernel's current source and the right-hand-side count.
"""
import json
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1803_04128_gb300 import _lib as L  # noqa: E402
from paper_1803_04128_gb300 import api  # noqa: E402

# bf_plan_view kinds holding complex entries (c128 on the host, c64 on the device):
# a, b, EV, S, EU once per sub-BF; EH and FG once per H / G level
_ONCE = (0, 1, 3, 6, 10)
_EH, _FG = 5, 8


def _complex_entries(plan):
    info = plan.info()
    L_, h, l1, split = info["L"], info["h"], info["l1"], info["split"]
    total = 0
    for blk in range(split * split):
        total += sum(plan.view(w, block=blk).size for w in _ONCE)
        total += sum(plan.view(_EH, lev, block=blk).size for lev in range(l1 + 1, h + 1))
        total += sum(plan.view(_FG, lev, block=blk).size for lev in range(h + 1, L_ - l1 + 1))
    return total


@pytest.mark.parametrize("N,r,kind,amp,split,m", [
    (4096, 8, L.PHASE_FIO, L.AMP_SMOOTH, 1, 3),
    (8192, 10, L.PHASE_FIO, L.AMP_ONE, 1, 64),
    (8192, 10, L.PHASE_FIO_PW, L.AMP_SMOOTH, 2, 5),
    (16384, 12, L.PHASE_DFT, L.AMP_ONE, 1, 1),
])
def test_algorithmic_bytes_equal_stored_complex_factors(N, r, kind, amp, split, m):
    plan = api.Plan(N, r=r, phase_kind=kind, amp_kind=amp, split=split)
    info = plan.info()
    _, _, bytes_apply = bench.algorithmic(info, m, N, split)
    stored = 8 * _complex_entries(plan)           # c64 bytes the FP32 apply reads
    assert bytes_apply == stored + 2 * 8 * N * m   # + F read once, G written once


def test_algorithmic_flops_scale_with_columns():
    # every stage's work is per column: r_alpha * m columns go through the butterfly
    plan = api.Plan(4096, r=8, amp_kind=L.AMP_SMOOTH)
    info = plan.info()
    f1, b1, _ = bench.algorithmic(info, 1, 4096, 1)
    f7, b7, _ = bench.algorithmic(info, 7, 4096, 1)
    assert (f7, b7) == (7 * f1, 7 * b1)
    assert info["r_alpha"] == 2 and f1 > 0 and b1 > 0


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _summary(tmp_path, lines):
    p = tmp_path / "clocks.csv"
    p.write_text("".join(l + "\n" for l in lines))
    cs = bench.ClockSampler(0)
    cs.proc, cs.path = _Done(), str(p)
    return cs.summary()


def test_clock_summary_median_and_reasons(tmp_path):
    ok = "0, {}, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, {}"
    s = _summary(tmp_path, [ok.format(2070, "Not Active"), ok.format(1980, "Active"),
                            ok.format(2055, "Not Active"), "garbage line", "0, [N/A], 2070, 1, 0, a, b, c, d"])
    assert s["samples"] == 3 and s["sm_mhz"] == 2055 and s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["sw_power_cap"]
    hot = "0, 1500, 2070, 1300, 0x0000000000000048, Active, Active, Not Active, Not Active"
    s = _summary(tmp_path, [hot])
    assert s["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"] and s["sm_mhz"] == 1500


def test_clock_summary_without_nvidia_smi():
    cs = bench.ClockSampler(0)
    assert cs.summary()["reasons"] == ["nvidia-smi unavailable"]


def test_ncu_traffic_is_keyed_by_kernel_source_and_m(tmp_path, monkeypatch):
    src = tmp_path / "paper_1803_04128_gb300" / "csrc"
    src.mkdir(parents=True)
    for f in ("bf_f32_tile.h", "bf_kernels_f32.cu"):
        shutil.copy(os.path.join(ROOT, "paper_1803_04128_gb300", "csrc", f), src / f)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.kernel_hash("front_f32")
    assert h == bench.kernel_hash("back_f32")      # one hash per kernel family
    entry = {"dram_bytes_per_launch": 123456, "kernel_hash": h, "m": 64}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"fio2": {"front_f32": entry}}))
    assert bench.ncu_traffic("front_f32", "fio2", 64) == 123456
    assert bench.ncu_traffic("front_f32", "fio2", 32) is None        # other RHS count
    assert bench.ncu_traffic("back_f32", "fio2", 64) is None         # not captured
    assert bench.ncu_traffic("front_f32", "fio3", 64) is None        # other workload
    with open(src / "bf_f32_tile.h", "a") as f:                     # kernel source changed
        f.write("\n// edited\n")
    assert bench.ncu_traffic("front_f32", "fio2", 64) is None
