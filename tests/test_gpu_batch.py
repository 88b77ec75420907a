"""Batched form: independent instances of mixed (D, chi, h) evolved concurrently
(tn_evolve_batch, each instance on its own stream and host thread), with the
FP64 product tile autotuner on.

Every instance is deterministic and the autotuner's tiles sum in one order, so
the batched run must reproduce, bit for bit, the same instances evolved one
after the other on the default stream with the autotuner off.
"""
import numpy as np
import pytest

from paper_1411_0391_gb300 import _lib as L
from paper_1411_0391_gb300 import build as B
from paper_1411_0391_gb300.inputs import random_peps

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# (D, chi, h, seed instance): mixed bond dimensions and fields, as the batched workload mixes them
INSTANCES = [(2, 8, 2.5, 8), (2, 12, 3.5, 11), (3, 12, 3.0, 12), (2, 8, 4.0, 3)]
OPTS = dict(recycle=True, n_re=2, ctm_tol=1e-10, ctm_max=300)
N_STEPS = 4


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    L.lib()


def _make(D, chi, h, inst, stream=None):
    ctx = L.Context(D, chi, stream=stream)
    ctx.tn_set_hamiltonian(1.0, h)
    ctx.tn_set_time_step(0.01)
    ctx.tn_set_state(random_peps(2, D, instance=inst))
    return ctx


def test_batched_instances_match_sequential_runs():
    ref = []
    L.tn_set_autotune(False)
    for D, chi, h, inst in INSTANCES:
        ctx = _make(D, chi, h, inst)
        rep = ctx.tn_evolve(N_STEPS, **OPTS)
        ref.append((ctx.tn_get_state(), rep))
        ctx.close()
    streams = [torch.cuda.Stream() for _ in INSTANCES]
    ctxs = [_make(D, chi, h, inst, stream=s) for (D, chi, h, inst), s in zip(INSTANCES, streams)]
    L.tn_set_autotune(True)
    try:
        reps = L.tn_evolve_batch(ctxs, N_STEPS, n_threads=len(ctxs), **OPTS)
        assert L.tn_set_autotune(True) > 0           # shapes were tuned
    finally:
        L.tn_set_autotune(False)
    for ctx, rep, (state, rref) in zip(ctxs, reps, ref):
        assert rep["status"] == L.TN_OK and rep["steps"] == N_STEPS
        assert rep["env_computations"] == rref["env_computations"] == N_STEPS // 2
        for a, b in zip(ctx.tn_get_state(), state):
            np.testing.assert_array_equal(a, b)
        ctx.close()


def test_batch_rejects_shared_stream():
    s = torch.cuda.Stream()
    a, b = _make(2, 8, 3.0, 8, stream=s), _make(2, 8, 3.0, 9, stream=s)
    with pytest.raises(L.TnError) as err:
        L.tn_evolve_batch([a, b], 1, **OPTS)
    assert err.value.status == L.TN_EINVAL
    a.close()
    b.close()
