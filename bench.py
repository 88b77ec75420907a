#!/usr/bin/env python3
"""Benchmark of the imaginary-time-evolution hot path at D = 4, chi = 64.

Workload (one "step"): one full-update imaginary-time step of the 2D
transverse-field Ising model (h = 3.04, tau = 0.005) on the 2-site
checkerboard iPEPS, D = 4, chi = 64, FP64:
  canonical form + iPEPO + simple-update pre-truncation + double layers,
  a warm-started CTMRG budget of CTM_ITERS iterations (4 directional moves each),
  bond environments + ALS + assembly of every link type.
The CTMRG budget is fixed so that every implementation does the same work per
step; the energy error against the FP64 oracle is measured on the converged
D = 2, chi = 8 workload and reported beside the throughput.

Prints one JSON line.  --impl reference times the CPU oracle on the same
workload (a bounded sample, scaled to steps/s).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CTMRG moves/s and ITE steps/s at D=4,χ=64; energy err vs FP64 oracle"
WL = dict(D=4, chi=64, h=3.04, tau=0.005, cell="checkerboard")
CTM_ITERS = 4
MOVES_PER_STEP = 4 * CTM_ITERS
N_RE = 5                            # recycled steps per environment computation (Sec. VI.C)
FP64_NOMINAL_TFLOPS = 1.25          # GB300 FP64 (SIMT) at the 2070 MHz boost clock


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    p.add_argument("--profile-moves", type=int, default=0,
                   help="run only this many CTMRG moves and one update at the workload shape (for ncu)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    return p.parse_args()


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.lines, self.proc = index, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
def oracle_sample():
    """Time the oracle on a bounded sample of one step: prepare, one CTMRG move, update."""
    import numpy as np
    from oracle import ctmrg as OC
    from oracle import recycle as OR
    from oracle import fullupdate as OF
    from oracle import canonical as OK
    from oracle import model as OM
    from paper_1411_0391_gb300.inputs import random_peps
    cell = OC.checkerboard()
    D, chi = WL["D"], WL["chi"]
    A = random_peps(2, D)
    g = OM.ipepo(WL["h"], WL["tau"])
    t0 = time.perf_counter()
    can = OK.canonicalize(A, cell)
    Theta = [OM.apply_pepo(g, a) for a in can["A"]]
    pre = OF.pretruncation(Theta, cell, can["lam"], D)
    a_list = [OC.double_layer(x) for x in OF.pretruncated_sites(Theta, cell, pre)]
    t1 = time.perf_counter()
    # a dense environment (seeded values): the cost of a move does not depend on them,
    # but the near-empty start environment would let LAPACK take zero shortcuts
    from paper_1411_0391_gb300.inputs import random_matrix
    env = OC.init_env(cell, chi, D * D)
    for i, site in enumerate(sorted(env)):
        for j, name in enumerate(sorted(env[site])):
            env[site][name] = random_matrix(env[site][name].shape, instance=100 + 8 * i + j)
    st = OC.State(cell, a_list, env)
    t2 = time.perf_counter()
    OC.left_move(st, chi)
    t3 = time.perf_counter()
    for _ in range(3):
        st = st.rotated()
    fu, _ = OF.full_update(Theta, cell, st, pre)
    OF.assemble(Theta, cell, fu)
    t4 = time.perf_counter()
    t_prep, t_move, t_upd = t1 - t0, t3 - t2, t4 - t3
    t_step = t_prep + MOVES_PER_STEP * t_move + t_upd
    return dict(t_prepare=t_prep, t_move=t_move, t_update=t_upd, t_step=t_step,
                sample="oracle at D=4 chi=64: one prepare, one CTMRG move (dense env), one bond-env+ALS update, "
                       "scaled to %d moves per step" % MOVES_PER_STEP)


def threads_used():
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        n = max((i.get("num_threads", 1) for i in info), default=1)
        return int(n)
    except Exception:
        return os.cpu_count() or 1


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    vals = []
    for _ in range(args.warmup):
        oracle_sample()
    samples = [oracle_sample() for _ in range(max(args.steps, 1))]
    t_step = statistics.median(s["t_step"] for s in samples)
    t_move = statistics.median(s["t_move"] for s in samples)
    value = 1.0 / t_step
    line = {
        "metric": METRIC, "value": value, "unit": "steps/s", "impl": "reference", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * t_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "moves_per_s": 1.0 / t_move,
        "config": dict(workload="ITE full-update step, 2D TFIM h=3.04 tau=0.005, checkerboard iPEPS D=4 chi=64, "
                                "CTMRG budget %d iterations per step" % CTM_ITERS, **WL,
                       ctm_iterations_per_step=CTM_ITERS),
        "cpu_baseline": {"value": value, "unit": "steps/s", "cores": threads_used(), "kind": "oracle",
                         "sample": samples[0]["sample"]},
        "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ---------------------------------------------------------------------------
def energy_error_small():
    """|E_gpu - E_oracle| / |E| after 3 plain steps of the D=2, chi=8 workload (h=3, tau=0.01)."""
    from oracle import ctmrg as OC
    from oracle import recycle as OR
    from paper_1411_0391_gb300 import _lib as L
    from paper_1411_0391_gb300.inputs import random_peps
    D, chi, h, tau = 2, 8, 3.0, 0.01
    A = random_peps(2, D)
    ctx = L.Context(D, chi)
    ctx.tn_set_hamiltonian(1.0, h)
    ctx.tn_set_time_step(tau)
    ctx.tn_set_state(A)
    cfg = OR.Config(h=h, tau=tau, D=D, chi=chi, ctm_tol=1e-10, ctm_max=500)
    env, Ao = None, A
    for _ in range(3):
        ctx.tn_fu_step(1e-10, 500)
        Ao, env, _ = OR.fu_step(Ao, OC.checkerboard(), cfg, env)
    ctx.tn_build_double_layer()
    ctx.tn_reset_env()
    ctx.tn_ctmrg(1e-12, 500)
    g = ctx.tn_measure()
    o = OR.energy(Ao, OC.checkerboard(), cfg, tol=1e-12)
    ctx.close()
    return abs(g["e_site"] - o["e_site"]) / abs(o["e_site"]), g["e_site"], o["e_site"]


def run_gpu(args):
    import torch
    import __graft_entry__ as G
    G.build()
    from paper_1411_0391_gb300 import _lib as L
    from paper_1411_0391_gb300.inputs import random_peps

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    D, chi = WL["D"], WL["chi"]
    ctx = L.Context(D, chi, device=dev)
    ctx.tn_set_hamiltonian(1.0, WL["h"])
    ctx.tn_set_time_step(WL["tau"])
    state = random_peps(2, D, instance=rank)          # replicas: independent instances per rank
    ctx.tn_set_state(state)

    if args.profile_moves:
        ctx.tn_step_prepare()
        ctx.tn_ctmrg_moves(args.profile_moves)
        ctx.tn_step_update()
        torch.cuda.synchronize()
        print(json.dumps({"profile_moves": args.profile_moves, "launches": L.tn_launch_count()}))
        return

    for _ in range(args.warmup):
        ctx.tn_step_prepare()
        ctx.tn_ctmrg(0.0, CTM_ITERS)
        ctx.tn_step_update()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)       # larger than the 129 MB L2
    t_prep = t_ctm = t_upd = 0.0
    launches = 0
    svd_calls = svd_iters = 0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            l0 = L.tn_launch_count()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            ev[0].record(stream)
            ctx.tn_step_prepare()
            ev[1].record(stream)
            rep = ctx.tn_ctmrg(0.0, CTM_ITERS)
            ev[2].record(stream)
            svd_calls += rep["svd_calls"]
            svd_iters += rep["svd_iterations"]
            ctx.tn_step_update()
            ev[3].record(stream)
            torch.cuda.synchronize()
            launches += L.tn_launch_count() - l0
            t_prep += ev[0].elapsed_time(ev[1]) / 1e3
            t_ctm += ev[1].elapsed_time(ev[2]) / 1e3
            t_upd += ev[2].elapsed_time(ev[3]) / 1e3
    total = t_prep + t_ctm + t_upd
    if dist:
        t = torch.tensor([total, t_ctm], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total, t_ctm = float(t[0]), float(t[1])
    value = world * args.steps / total
    moves_per_s = world * args.steps * MOVES_PER_STEP / t_ctm

    # recycled form (Sec. VI.C): one environment computation, then N_RE steps with the renormalised gate
    t_rec = 0.0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.tn_step_prepare()
        ctx.tn_ctmrg(0.0, CTM_ITERS)
        ctx.tn_step_update()
        F = ctx.tn_recycle(N_RE)
        e1.record(stream)
        torch.cuda.synchronize()
        t_rec += e0.elapsed_time(e1) / 1e3
    recycled = {"n_re": N_RE, "steps_per_s": world * args.steps * N_RE / t_rec,
                "speedup_vs_plain": (args.steps * N_RE / t_rec) / (args.steps / total), "last_fidelity": F}

    # end to end through the public API with host buffers: H2D of the state, the step, D2H of the result
    import numpy as np
    host = [np.ascontiguousarray(a) for a in ctx.tn_get_state()]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.tn_set_state(host)
        ctx.tn_step_prepare()
        ctx.tn_ctmrg(0.0, CTM_ITERS)
        ctx.tn_step_update()
        host = ctx.tn_get_state()
    torch.cuda.synchronize()
    e2e_t = time.perf_counter() - t0
    state_bytes = sum(a.nbytes for a in host)

    # roofline of the dominant kernel: the FP64 GEMM of the N x N half-system and loop products
    N = chi * D * D
    A = torch.randn(N, N, dtype=torch.float64, device=dev)
    B = torch.randn(N, N, dtype=torch.float64, device=dev)
    C = torch.empty(N, N, dtype=torch.float64, device=dev)
    for _ in range(3):
        L.tn_gemm_f64(0, 0, N, N, N, 1.0, A, N, 0, B, N, 0, 0.0, C, N, 0, 1, stream)
    reps = 10
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        L.tn_gemm_f64(0, 0, N, N, N, 1.0, A, N, 0, B, N, 0, 0.0, C, N, 0, 1, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    t_gemm = e0.elapsed_time(e1) / 1e3 / reps
    achieved = 2.0 * N ** 3 / t_gemm / 1e12
    csum = clk.summary()
    sm_mhz = csum.get("sm_mhz") or 2070.0
    peak = FP64_NOMINAL_TFLOPS * sm_mhz / 2070.0

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "moves_per_s": moves_per_s,
        "time_split_s": {"prepare": t_prep, "ctmrg": t_ctm, "update": t_upd},
        "projector_svd": {"calls": svd_calls, "iterations_per_call": svd_iters / max(svd_calls, 1)},
        "recycled": recycled,
        "config": dict(workload="ITE full-update step, 2D TFIM h=3.04 tau=0.005, checkerboard iPEPS D=4 chi=64, "
                                "CTMRG budget %d iterations per step" % CTM_ITERS, **WL,
                       ctm_iterations_per_step=CTM_ITERS, parallelism="replicas" if world > 1 else "single",
                       l2="flushed between timed steps (256 MB write)"),
        "e2e": {"value": world * args.steps / e2e_t, "unit": "steps/s", "h2d_bytes_per_step": state_bytes,
                "d2h_bytes_per_step": state_bytes},
        "gpu_launches": int(launches),
        "clocks": csum,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": None, "kernel": "dgemm_kernel %dx%dx%d (FP64 SIMT; GB300 has no FP64 tensor path)"
                     % (N, N, N), "peak_source": "derived: 1.25 TFLOP/s FP64 at 2070 MHz scaled to the median "
                     "sampled SM clock"},
    }
    try:
        err, eg, eo = energy_error_small()
        line["energy_err"] = {"rel": err, "workload": "D=2 chi=8 h=3 tau=0.01, 3 plain steps, CTMRG tol 1e-10",
                              "e_gpu": eg, "e_oracle": eo}
    except Exception as ex:                                 # reported, never hidden
        line["energy_err"] = {"error": repr(ex)}
    if world == 1 and not args.no_cpu_baseline:
        s = oracle_sample()
        line["cpu_baseline"] = {"value": 1.0 / s["t_step"], "unit": "steps/s", "cores": threads_used(),
                                "kind": "oracle", "sample": s["sample"], "moves_per_s": 1.0 / s["t_move"]}
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
