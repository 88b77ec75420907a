"""The reference arm of bench.py (the oracle on the host cores) prints the contract's JSON line."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.strip().splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["unit"] == "steps/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and abs(d["ms_per_step"] - 1000.0 / d["value"]) < 1e-6 * d["ms_per_step"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "D=4 chi=64" in d["config"]["workload"]


class _Event:
    def __init__(self, enable_timing=False):
        self.t = None

    def record(self, stream=None):
        import time
        self.t = time.perf_counter()

    def elapsed_time(self, other):
        return 1000.0 * (other.t - self.t)


class _Cuda:
    Event = _Event

    @staticmethod
    def synchronize():
        pass


class _Torch:
    cuda = _Cuda


class _Flush:
    def zero_(self):
        pass


class _Ctx:
    """Stand-in for the library context: records the call sequence, no device."""

    def __init__(self, log, D):
        self.log, self.D = log, D

    def __getattr__(self, name):
        def call(*a, **k):
            self.log.append(name)
            if name == "tn_ctmrg":
                return dict(svd_calls=8, svd_iterations=32, iterations=4, converged=True)
            if name == "tn_get_state":
                import numpy as np
                return [np.zeros((2,) + (self.D,) * 4) for _ in range(2)]
            if name == "tn_recycle":
                return 0.9999
            return None
        return call


class _Lib:
    def __init__(self):
        self.log, self.n = [], 0

    def Context(self, D, chi, device=None, precision=0):
        return _Ctx(self.log, D)

    def tn_launch_count(self):
        self.n += 10
        return self.n


def test_time_form_schedule_and_keys():
    """The GPU arm's per-form timing loop, run against a stand-in library: warm-up steps,
    timed converged steps, end-to-end steps through the public API (H2D, tn_fu_step, D2H),
    fixed-budget steps and recycled windows, and the keys the JSON line is built from."""
    sys.path.insert(0, ROOT)
    import bench
    L = _Lib()
    ctx, out = bench.time_form(L, _Torch, None, None, "f64s7", None, 2, _Flush(), 3, recycled=True, fixed=True,
                               e2e=True)
    log = L.log
    assert log.count("tn_fu_step") == 2 + 3                  # warm-up + end-to-end steps
    assert log.count("tn_set_state") == 1 + 3 and log.count("tn_recycle") == 3
    assert log.count("tn_ctmrg") == 3 + 3 + 3                # timed, fixed-budget, recycled
    first_e2e = log.index("tn_set_state", 1)
    assert "tn_recycle" not in log[:first_e2e]               # e2e continues the timed trajectory
    for key in ("total", "t_ctm", "launches", "svd_calls", "ctm_iters", "steps_total", "state", "t_e2e",
                "e2e_bytes", "t_fixed", "t_rec", "fidelity"):
        assert key in out, key
    assert out["steps_total"] == 5 and out["e2e_bytes"] == 2 * 2 * 4 ** 4 * 8 and out["ctm_iters"] == 12
    summ = bench.form_summary(out, 1)
    assert summ["k_ctm"] == 4 and summ["recycled"]["n_re"] == bench.N_RE
