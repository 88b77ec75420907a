"""Host logic of the field sweep: stage schedules and recycling modes, against a recording
stand-in for the library context (no GPU)."""
import pytest

from paper_1411_0391_gb300 import sweep


class FakeContext:
    calls = []

    def __init__(self, D, chi, device=None, precision=None):
        self.D, self.chi = D, chi

    def __getattr__(self, name):
        def rec(*a, **k):
            FakeContext.calls.append((name, a, k))
            if name == "tn_evolve":
                return {"env_computations": 2}
            if name == "tn_ctmrg":
                return {"converged": True}
            if name == "tn_measure":
                return {"e_site": -3.0, "mx": [0.5, 0.5], "mz": [0.1, -0.1]}
            return None
        return rec


@pytest.fixture(autouse=True)
def fake(monkeypatch):
    FakeContext.calls = []
    monkeypatch.setattr(sweep.L, "Context", FakeContext)
    monkeypatch.setattr(sweep, "random_peps", lambda *a, **k: [0.0])


def test_two_stage_threshold_schedule():
    """tau 0.01 then 0.001 (the second workload's schedule), threshold recycling, plain warm-up
    steps only in the first stage; the measurement follows the last stage."""
    r = sweep.run_field(3.04, 3, 32, [0.01, 0.001], [1000, 1000], method="fu", n_re=50, recycle_eps=1e-8,
                        warmup_plain=20)
    names = [c[0] for c in FakeContext.calls]
    assert names == ["tn_set_hamiltonian", "tn_set_state", "tn_set_time_step", "tn_evolve", "tn_set_time_step",
                     "tn_evolve", "tn_build_double_layer", "tn_reset_env", "tn_ctmrg", "tn_measure",
                     "tn_get_state", "close"]
    ev = [c for c in FakeContext.calls if c[0] == "tn_evolve"]
    taus = [c[1][0] for c in FakeContext.calls if c[0] == "tn_set_time_step"]
    assert taus == [0.01, 0.001]
    assert [e[1][0] for e in ev] == [1000, 1000]
    assert all(e[2]["recycle"] == "threshold" and e[2]["recycle_eps"] == 1e-8 and e[2]["n_re"] == 50 for e in ev)
    assert [e[2]["warmup_plain"] for e in ev] == [20, 0]
    assert r["env_computations"] == 4 and r["mz"] == pytest.approx(0.1) and r["tau"] == [0.01, 0.001]


def test_single_stage_modes():
    sweep.run_field(2.5, 2, 8, 0.01, 5, method="fu")
    ev = [c for c in FakeContext.calls if c[0] == "tn_evolve"][0]
    assert ev[2]["recycle"] is False and ev[2]["recycle_eps"] is None
    FakeContext.calls = []
    sweep.run_field(2.5, 2, 8, 0.01, 5, method="fu", n_re=5)
    ev = [c for c in FakeContext.calls if c[0] == "tn_evolve"][0]
    assert ev[2]["recycle"] is True and ev[2]["n_re"] == 5
    FakeContext.calls = []
    sweep.run_field(2.5, 2, 8, 0.01, 3, method="su")
    assert [c[0] for c in FakeContext.calls].count("tn_su_step") == 3


def test_mismatched_stages_rejected():
    with pytest.raises(ValueError):
        sweep.run_field(2.5, 2, 8, [0.01, 0.001], [10], method="fu")
