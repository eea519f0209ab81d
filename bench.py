"""Benchmark of the IREBM time step on GB300 (one JSON line on stdout).

Headline: D2Q9 MLUPS of the step in the FP32 form (FP32 populations, FP64
Newton; five launches per step: rows 1 .. ny-2 of the left and the right
half of the strips, and on a second stream the wall nodes and the Newton
solves of the left half beside the right half, then the right half's) on the 4096 x 4096 melting workload, timed with CUDA events on
the launching stream over --steps steps after --warmup untimed steps.  The
timed window sits at the middle of the 10,000-step job (the state is first
advanced, untimed, to step 5,000 - (warmup + steps)/2) so the Newton front band
has its average width.  The state (1.2 GB) is larger than L2 (129 MB), so
every step reads and writes HBM; no flush is needed.

Also reported: the FP64 form on the same workload, the 2048^2 FP64 corner
workload for Ste in {0.01, 0.1, 1}, EEBM (Algorithm 2) on the same window, 256
batched problems in one persistent graph-captured launch per step, the
adjoint/forward time ratio on 1024^2 with sqrt(T) checkpointing, the 512-node
D1Q3 workload (all steps of a call in one launch), the paper's 2D cavity on D2Q5 (4096^2, Eq. 17
closure; IREBM FP32 and FP64, EEBM), the paper's 1D bar (N = 801) and its 2D
cavity on D2Q9 (N = 801, FP64) with the three schemes (IREBM, EEBM, ILFBM).

--impl reference times the FP64 CPU oracle (the reference of this build) on
a bounded sample of the same workload.
Multi-GPU (torchrun): each rank runs an independent replica (the problems
do not exchange data); value = all nodes updated / max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "D2Q9 MLUPS incl. local Newton (FP32 vs FP64 form) and adjoint/forward time ratio"
BYTES_FP32 = 9 * 4 * 2   # algorithmic bytes per node update: each population read once, written once
BYTES_FP64 = 9 * 8 * 2
BYTES_D2Q5_FP32 = 5 * 4 * 2   # D2Q5: five populations
BYTES_D2Q5_FP64 = 5 * 8 * 2
# DRAM bytes (read + write) per node of one launch of the flat FP32 D2Q9 kernel,
# from an ncu capture of a smaller case scaled by the node count (None: not
# captured since the kernel changed)
FLAT_TRAFFIC_PER_NODE = (77219072 + 29094656) / 2086920
FLAT_TRAFFIC_NOTE = ("ncu capture of one launch (left half of the strips) on the 2048^2 melting workload at "
                     "step 301: 77.2 MB read + 29.1 MB written for 2,086,920 nodes, 50.9 B per node; writes "
                     "still in L2 when the launch ends are written back during the next; scaled by nodes")


def flat_nodes(nx, ny):
    """Nodes of one step in the flat kernel: rows 1 .. ny-2 outside the W and E four-column groups."""
    xe = max(4, ((nx - 1) >> 2) << 2)
    cold = min(4, nx) + max(0, nx - xe)
    return max(0, ny - 2) * (nx - cold)


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, n in enumerate(names):
                if f[5 + k].lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ replicas
def max_over_ranks(torch, dist, value, device):
    """The largest `value` over the ranks of the process group (the job ends with
    its slowest replica); `value` itself without a process group."""
    if dist is None:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(world, nodes, steps, ms_max):
    """Whole-job throughput: every replica's node updates over the slowest replica's time."""
    return world * nodes * steps / ms_max / 1e3


# ------------------------------------------------------------------ GPU measurements
def time_steps(torch, S, steps, stream):
    """Device time of `steps` steps (ms), CUDA events on the launching stream."""
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    S.step(steps)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def melt_window(case, steps, warmup, centre=None):
    centre = case.steps // 2 if centre is None else centre
    return max(0, centre - (steps + warmup) // 2)


def bench_single(torch, solver, case, steps, warmup, stream, barrier=None, centre=None):
    S = solver.Stefan.from_case(case, stream=stream)
    S.set_ic(case.theta0())
    pre = melt_window(case, steps, warmup, centre)
    if pre:
        S.step(pre)
    S.step(warmup)
    S.sync()
    if barrier:
        barrier()
    ms = time_steps(torch, S, steps, stream)
    st = S.stats()
    # per-kernel device times (CUDA events between the two launches of a step)
    if case.lattice == 2 and case.precision == 1:
        k0, k1, kf = S.step_timed(min(steps, 50), flat=True)
        st["kernel_ms"], st["flat_ms"] = (k0, k1), kf
    else:
        st["kernel_ms"] = S.step_timed(min(steps, 50)) if case.lattice in (2, 3) else None
    S.close()
    return ms, st


def bench_eebm(torch, solver, case, steps, warmup, stream, nodes, irebm_ms):
    """EEBM (Algorithm 2) on the melting workload, FP32 populations, same window."""
    S = solver.Stefan.from_case(case, stream=stream)
    S.set_method("EEBM")
    S.set_ic(case.theta0())
    S.step(melt_window(case, steps, warmup) + warmup)
    S.sync()
    ms = time_steps(torch, S, steps, stream)
    k = S.step_timed(min(steps, 50))
    S.close()
    return {"mlups": nodes * steps / ms / 1e3, "ms_per_step": ms / steps, "kernel_ms": k[0],
            "kernel_gbs": BYTES_FP32 * nodes / (k[0] * 1e-3) / 1e9, "irebm_over_eebm": irebm_ms / ms}


def bench_d2q5(torch, solver, workloads, steps, warmup, stream, peak, n=4096, fp64=True, centre=None):
    """The paper's 2D cavity (Sec. 6.2) on its D2Q5 lattice with the Eq. (17)
    closure, n^2, FP32 and FP64 populations, window centred on step 2,500."""
    out = {}
    legs = [(workloads.FP32, "fp32", BYTES_D2Q5_FP32)] + ([(workloads.FP64, "fp64", BYTES_D2Q5_FP64)] if fp64 else [])
    for prec, tag, bpn in legs:
        c = workloads.cavity_2d(n=n, precision=prec)
        nodes = c.nx * c.ny
        ms, st = bench_single(torch, solver, c, steps, warmup, stream, centre=centre)
        k_step, k_job = st["kernel_ms"]
        gbs = bpn * nodes / (k_step * 1e-3) / 1e9
        out[tag] = {"workload": c.name, "mlups": nodes * steps / ms / 1e3, "ms_per_step": ms / steps,
                    "kernel": "d2q5_step_kernel<%s,false>" % ("float" if prec == workloads.FP32 else "double"),
                    "kernel_ms": k_step, "job_kernel_ms": k_job, "bytes_per_node": bpn,
                    "kernel_gbs": gbs, "kernel_frac": gbs / peak,
                    "whole_step_gbs": bpn * nodes / (ms / steps * 1e-3) / 1e9,
                    "newton_nodes_last_step": st["newton_nodes"]}
        if prec == workloads.FP32 and fp64:
            # the paper's comparison scheme on the same lattice, workload and window
            # (its 2D timing table compares EEBM and IREBM on D2Q5)
            S = solver.Stefan.from_case(c, stream=stream)
            S.set_method("EEBM")
            S.set_ic(c.theta0())
            S.step(melt_window(c, steps, warmup, centre) + warmup)
            S.sync()
            mse = time_steps(torch, S, steps, stream)
            ke = S.step_timed(min(steps, 50))
            S.close()
            out["eebm_fp32"] = {"mlups": nodes * steps / mse / 1e3, "ms_per_step": mse / steps, "kernel_ms": ke[0],
                                "kernel_gbs": bpn * nodes / (ke[0] * 1e-3) / 1e9, "irebm_over_eebm": ms / mse}
    return out


def bench_e2e(torch, solver, case, steps, stream, centre=None):
    """Through the public C ABI with host buffers, on the headline's window:
    the state at the window's start is saved to pinned host memory (untimed);
    the timed region then loads it (lbm_stefan_set_state, host -> device),
    runs `steps` steps and reads theta back (lbm_stefan_get_fields, device ->
    pinned host)."""
    import ctypes
    from paper_2505_13097_gb300 import _abi
    n = case.nx * case.ny
    out = torch.empty((case.ny, case.nx), dtype=torch.float64, pin_memory=True)
    S = solver.Stefan.from_case(case, stream=stream)
    S.set_ic(case.theta0())
    S.step(melt_window(case, steps, 0, centre))
    host_state = torch.empty(S.state_bytes, dtype=torch.uint8, pin_memory=True)
    S.get_state(host_state.numpy())
    S.set_state(host_state.numpy())
    S.step(3)
    S.sync()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    S.set_state(host_state.numpy())
    S.step(steps)
    _abi.check(S.lib.lbm_stefan_get_fields(S.h, ctypes.c_void_p(out.data_ptr()), None, None, 0))
    t1 = time.perf_counter()
    nbytes = S.state_bytes
    S.close()
    return (t1 - t0) * 1e3, nbytes, 8 * n


def bench_batch(torch, solver, workloads, steps, warmup, stream, count=256, hi=1024, centre=None):
    cases = workloads.batch_2d(count=count, hi=hi)
    B = solver.StefanBatch(cases, stream=stream)
    for k, c in enumerate(cases):
        B.set_ic(k, c.theta0())
    tile_h = B.autotune(trial_steps=5)
    centre = cases[0].steps // 2 if centre is None else centre
    pre = max(0, centre - steps // 2 - warmup)
    B.step(pre + warmup)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    B.step(steps)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    nodes = sum(c.nx * c.ny for c in cases)
    err = max(B.stats(k)["error"] for k in range(len(cases)))
    B.close()
    return {"problems": len(cases), "nodes": nodes, "steps": steps, "mlups": nodes * steps / ms / 1e3,
            "tile_h": tile_h, "error": err, "window_start_step": pre + warmup}


def bench_adjoint(torch, solver, workloads, stream, n=1024, repeats=3):
    """n^2, 2,000 steps, FP32 forward with FP64 Newton, sqrt(T) checkpoints.
    One untimed forward + backward first creates the run's handle, checkpoint
    buffers and CUDA graphs; then `repeats` forward and backward passes are
    timed (wall clock between device synchronizations) and their medians
    reported, with the spread (max - min) / median of each.  The forward pass
    is also compared with T times the steady per-step time of the same step
    (CUDA events, 200 steps mid-run), and one adjoint step with one forward
    step (the kernels alone)."""
    from paper_2505_13097_gb300.autograd import clear_pool, misfit
    base = workloads.adjoint_2d(n=n)
    tcase = workloads.adjoint_target_case(base)
    T = base.steps
    with torch.cuda.stream(stream):
        St = solver.Stefan.from_case(tcase, stream=stream)
        St.set_ic(workloads.adjoint_target_theta0(base))
        St.step(T)
        _, ph, _ = St.fields(device=True)
        St.close()
    torch.cuda.synchronize()
    th0 = torch.tensor(base.theta0(), device="cuda", requires_grad=True)
    tw = torch.tensor([base.walls["W"][1], 0.0, 0.0, 0.0], dtype=torch.float64, device="cuda", requires_grad=True)
    ste = torch.tensor(base.ste, dtype=torch.float64, device="cuda", requires_grad=True)

    def once():
        th0.grad = tw.grad = ste.grad = None
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        L = misfit(th0, tw, ste, base, T, ph)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        L.backward()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        return (t1 - t0) * 1e3, (t2 - t1) * 1e3, float(L.detach())

    once()
    runs = [once() for _ in range(repeats)]
    fwd = statistics.median(r[0] for r in runs)
    bwd = statistics.median(r[1] for r in runs)
    spread_f = (max(r[0] for r in runs) - min(r[0] for r in runs)) / fwd
    spread_b = (max(r[1] for r in runs) - min(r[1] for r in runs)) / bwd
    clear_pool()
    # steady forward step, and one adjoint step against one forward step (kernels alone)
    S = solver.Stefan.from_case(base, stream=stream)
    S.set_ic(base.theta0())
    S.step(T // 2)
    S.sync()
    steady_ms = time_steps(torch, S, 200, stream) / 200
    traj = S.new_theta_planes(2)
    S.theta_plane(traj[0])
    a = S.new_state_buffer()
    b = S.new_state_buffer()
    S.step_record(1, traj[1:])
    S.adjoint_seed(traj[1], ph, a, want_loss=False)
    reps = 50
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    e[0].record(stream)
    S.step(reps)
    e[1].record(stream)
    for _ in range(reps):
        S.adjoint_step(traj[0], traj[1], a, b)
        a, b = b, a
    e[2].record(stream)
    e[2].synchronize()
    f_ms, a_ms = e[0].elapsed_time(e[1]) / reps, e[1].elapsed_time(e[2]) / reps
    S.close()
    return {"grid": "%dx%d" % (base.nx, base.ny), "steps": T, "state_mb": 9 * 4 * base.nx * base.ny / 1e6,
            "repeats": repeats, "forward_ms": fwd, "backward_ms": bwd, "backward_over_forward": bwd / fwd,
            "forward_spread": spread_f, "backward_spread": spread_b,
            "steady_forward_ms_per_step": steady_ms, "backward_over_T_steady_forward": bwd / (T * steady_ms),
            "kernel_forward_ms": f_ms, "kernel_adjoint_ms": a_ms, "kernel_adjoint_over_forward": a_ms / f_ms,
            "loss": runs[-1][2], "checkpoints": int(math.ceil(T / math.ceil(math.sqrt(T)))),
            "timing": "wall clock between torch.cuda.synchronize() calls, median of %d after one untimed "
                      "forward+backward (handle, checkpoints and graphs created there)" % repeats}


def bench_d1q3(torch, solver, workloads, stream):
    c = workloads.melt_1d()
    S = solver.Stefan.from_case(c, stream=stream)
    S.set_ic(c.theta0())
    S.step(100)
    S.set_ic(c.theta0())
    S.sync()
    ms = time_steps(torch, S, c.steps, stream)
    S.close()
    return {"nodes": c.nx, "steps": c.steps, "ms": ms, "steps_per_s": c.steps / ms * 1e3,
            "mlups": c.nx * c.steps / ms / 1e3}


def bench_bar_1d(torch, solver, workloads, stream, steps=20000):
    """The paper's 1D bar (N = 801, tau 0.62, delta 0.01) with IREBM, EEBM
    (Algorithm 2) and ILFBM (Algorithm 1), `steps` steps each, and the time of
    the full 160 s run (204,800 steps) at that rate: the GPU counterpart of the
    paper's 1D timing table (one M1 core at N = 801: EEBM 1.538 s, IREBM
    5.586 s, ILFBM 22.01 s)."""
    c = workloads.bar_1d()
    out = {"workload": c.name, "steps_timed": steps}
    from paper_2505_13097_gb300 import _abi
    for method in ("IREBM", "EEBM", "ILFBM"):
        # ILFBM: the inner loop's tolerance on l and its iteration limit
        kw = dict(newton_tol=1e-12, newton_max_iter=200) if method == "ILFBM" else {}
        S = solver.Stefan.from_case(c, stream=stream, **kw)
        try:
            S.set_method(method)
            S.set_ic(c.theta0())
            S.step(200)
            S.sync()
            ms = time_steps(torch, S, steps, stream)
            st = S.stats()
            S.sync()
            out[method.lower()] = {"steps_per_s": steps / ms * 1e3, "full_run_s": c.steps * ms / steps / 1e3,
                                   "iterations_last_step": st["newton_max_iter"]}
        except _abi.LBMError as e:   # reported, not fatal
            out[method.lower()] = {"error": str(e)}
        finally:
            S.close()
    if all("full_run_s" in out[m] for m in ("irebm", "eebm", "ilfbm")):
        out["ilfbm_over_irebm"] = out["ilfbm"]["full_run_s"] / out["irebm"]["full_run_s"]
        out["irebm_over_eebm"] = out["irebm"]["full_run_s"] / out["eebm"]["full_run_s"]
    return out


def bench_cavity_d2q9_801(torch, solver, workloads, stream, steps=20, warmup_steps=200):
    """The paper's 2D cavity on D2Q9 at its largest size (N = 801), FP64 as the
    paper computes, with the three schemes: ms per step after `warmup_steps`
    steps (the paper's 2D timing table covers EEBM and IREBM; its ILFBM did not
    converge there, ours does on D2Q9)."""
    c = workloads.cavity_2d(n=801, precision=workloads.FP64).scaled(lattice=2, bb_mode=0)
    out = {"workload": "cavity_2d_d2q9_801 (FP64, mirror bounce-back on the symmetry lines)", "steps_timed": steps}
    from paper_2505_13097_gb300 import _abi
    for method in ("IREBM", "EEBM", "ILFBM"):
        kw = dict(newton_tol=1e-12, newton_max_iter=400) if method == "ILFBM" else {}
        S = solver.Stefan.from_case(c, stream=stream, **kw)
        try:
            S.set_method(method)
            S.set_ic(c.theta0())
            S.step(warmup_steps)
            S.sync()
            ms = time_steps(torch, S, steps, stream)
            st = S.stats()
            S.sync()
            out[method.lower()] = {"ms_per_step": ms / steps, "mlups": c.nx * c.ny * steps / ms / 1e3,
                                   "iterations_last_step": st["newton_max_iter"]}
        except _abi.LBMError as e:   # e.g. ILFBM's inner loop at its limit: reported, not fatal
            out[method.lower()] = {"error": str(e)}
        finally:
            S.close()
    if "ms_per_step" in out["irebm"] and "ms_per_step" in out["eebm"]:
        out["irebm_over_eebm"] = out["irebm"]["ms_per_step"] / out["eebm"]["ms_per_step"]
    if "ms_per_step" in out["irebm"] and "ms_per_step" in out["ilfbm"]:
        out["ilfbm_over_irebm"] = out["ilfbm"]["ms_per_step"] / out["irebm"]["ms_per_step"]
    return out


# ------------------------------------------------------------------ error against the oracle
def _err(th, ph, refs, key):
    tr = refs[key + "/theta"]
    out = {"max_rel_dtheta": float(abs(th - tr).max() / max(abs(tr).max(), 1e-300))}
    if ph is not None:
        out["max_abs_dphi"] = float(abs(ph - refs[key + "/phi"]).max())
    return out


def oracle_errors(torch, solver, workloads, stream):
    """Every leg's small version (workloads.bench_parity_cases, same kernels and
    launch path) against the FP64 oracle's stored results
    (tests/golden/bench_refs.npz, written by tests/golden/make_bench_refs.py):
    max |d theta| / max |theta_ref| and max |d phi|; for the adjoint the
    relative errors of the gradient and of the loss."""
    import numpy as np
    refs = np.load(os.path.join(ROOT, "tests", "golden", "bench_refs.npz"))
    out = {}
    for name, (c, method, kw) in workloads.bench_parity_cases().items():
        S = solver.Stefan.from_case(c, stream=stream, **kw)
        try:
            if method != "IREBM":
                S.set_method(method)
            S.set_ic(c.theta0())
            S.step(c.steps)
            th, ph, _ = S.fields()
            out[name] = _err(th, ph, refs, name)
            out[name]["case"] = "%s %dx%d, %d steps, %s" % (c.name, c.nx, c.ny, c.steps, method)
        finally:
            S.close()
    cases = workloads.bench_parity_batch()
    B = solver.StefanBatch(cases, stream=stream)
    try:
        for k, c in enumerate(cases):
            B.set_ic(k, c.theta0())
        B.step(cases[0].steps)
        errs = [_err(B.theta(k), None, refs, "batch%d" % k)["max_rel_dtheta"] for k in range(len(cases))]
    finally:
        B.close()
    out["batched"] = {"max_rel_dtheta": max(errs), "case": "%d problems, sides %d-%d, %d steps" % (
        len(cases), min(c.nx for c in cases), max(c.nx for c in cases), cases[0].steps)}
    from paper_2505_13097_gb300.autograd import misfit
    a = workloads.bench_parity_adjoint()
    th0 = torch.tensor(a.theta0(), device="cuda", requires_grad=True)
    tw = torch.tensor([a.walls.get(k, (0, 0.0))[1] for k in "WESN"], dtype=torch.float64, device="cuda",
                      requires_grad=True)
    ste = torch.tensor(a.ste, dtype=torch.float64, device="cuda", requires_grad=True)
    with torch.cuda.stream(stream):
        L = misfit(th0, tw, ste, a, a.steps, torch.tensor(refs["adjoint/target"], device="cuda"))
        L.backward()
    torch.cuda.synchronize()
    g0 = th0.grad.cpu().numpy()
    r0 = refs["adjoint/g_theta0"]
    out["adjoint"] = {
        "case": "%s %dx%d, %d steps, FP32 forward; oracle FP64 adjoint" % (a.name, a.nx, a.ny, a.steps),
        "g_theta0_max_rel": float(abs(g0 - r0).max() / abs(r0).max()),
        "g_wall_rel": float(abs(float(tw.grad[0]) - refs["adjoint/g_wall"][0]) / abs(refs["adjoint/g_wall"][0])),
        "g_ste_rel": float(abs(float(ste.grad) - float(refs["adjoint/g_ste"])) / abs(float(refs["adjoint/g_ste"]))),
        "loss_rel": float(abs(float(L.detach()) - float(refs["adjoint/loss"])) / abs(float(refs["adjoint/loss"])))}
    return out


def _oracle_sample(rows, nsteps):
    """nsteps oracle steps of a 4096 x rows problem with the melting workload's
    parameters and the first rows of its initial field: (node updates, seconds).
    Module-level so that spawned worker processes can run it."""
    import oracle
    from paper_2505_13097_gb300 import workloads
    c = workloads.melt_2d()
    P = oracle.Problem(2, c.nx, rows, tau=c.tau, delta=c.delta, ste=c.ste, walls=c.walls)
    f = P.init(c.theta0()[:rows])
    f = P.step(f)
    t = time.perf_counter()
    for _ in range(nsteps):
        f = P.step(f)
    return c.nx * rows * nsteps, time.perf_counter() - t


def cpu_baseline_sample(workloads, budget_s=8.0):
    """The FP64 oracle as it stands on the host cores, on a bounded sample of the
    melting workload: one thread, then one independent copy of the same
    sample per core (worker processes started with spawn) timed together;
    `value` is the all-core aggregate."""
    import multiprocessing as mp
    rows = 64
    n1, t1 = _oracle_sample(rows, 1)
    nsteps = max(2, min(400, int(budget_s / max(t1, 1e-6))))
    u, el = _oracle_sample(rows, nsteps)
    single = u / el / 1e6
    cores = os.cpu_count() or 1
    sample = "%d steps of a 4096x%d problem with the 4096^2 melting workload's parameters (first %d rows of its " \
             "initial field)" % (nsteps, rows, rows)
    try:
        with mp.get_context("spawn").Pool(cores) as pool:
            res = pool.starmap(_oracle_sample, [(rows, nsteps)] * cores)
        agg = sum(r[0] for r in res) / max(r[1] for r in res) / 1e6
        return {"value": agg, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                "sample": "FP64 C oracle, %d independent single-thread copies (one per host core) of %s, "
                          "aggregate node updates / slowest copy's time" % (cores, sample),
                "single_thread": {"value": single, "unit": "MLUPS", "cores": 1, "seconds": el,
                                  "sample": "FP64 C oracle, 1 thread, " + sample}}
    except Exception as e:   # reported, not fatal
        return {"value": single, "unit": "MLUPS", "cores": 1, "kind": "oracle",
                "sample": "FP64 C oracle, 1 thread, " + sample, "all_cores_error": str(e)}


# ------------------------------------------------------------------ arms
def run_reference(args):
    from paper_2505_13097_gb300 import workloads
    import oracle
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    c = workloads.melt_2d()
    rows = 64
    P = oracle.Problem(2, c.nx, rows, tau=c.tau, delta=c.delta, ste=c.ste, walls=c.walls)
    f = P.init(c.theta0()[:rows])
    for _ in range(args.warmup):
        f = P.step(f)
    t = time.perf_counter()
    for _ in range(args.steps):
        f = P.step(f)
    el = time.perf_counter() - t
    v = c.nx * rows * args.steps / el / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "melt_2d_d2q9_4096 sample: 4096x64 rows, Ste 0.1, delta 0.01, tau 1.0, FP64 CPU oracle"},
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": 1, "kind": "oracle",
                             "sample": "%d oracle steps of a 4096x64 problem with the melting workload's parameters" % args.steps},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import torch
    from paper_2505_13097_gb300 import solver, workloads

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    barrier = (lambda: dist.barrier(device_ids=[local])) if dist else None
    stream = torch.cuda.Stream()
    peak, peak_kind = load_peaks()
    if args.only_bar:
        # profiling aid: the 1D bar with the three schemes, --steps steps each
        if rank == 0:
            print(json.dumps({"bar_1d": bench_bar_1d(torch, solver, workloads, stream, steps=args.steps)}), flush=True)
        return 0
    if args.only_corner:
        # profiling aid: the FP64 corner leg alone, Ste 0.1, side --n (default 2048)
        if rank == 0:
            cc = workloads.corner_2d(n=args.n or 2048, ste=0.1)
            msc, stc = bench_single(torch, solver, cc, args.steps, args.warmup, stream, centre=args.window_step)
            print(json.dumps({"corner": {"workload": cc.name, "mlups": cc.nx * cc.ny * args.steps / msc / 1e3,
                                         "kernel_ms": stc["kernel_ms"], "newton_nodes": stc["newton_nodes"]}}),
                  flush=True)
        return 0
    if args.only_batch:
        # profiling aid: the batch leg alone (--batch-count problems, sides up to --batch-hi)
        if rank == 0:
            print(json.dumps({"batch": bench_batch(torch, solver, workloads, args.steps, args.warmup, stream,
                                                   count=args.batch_count, hi=args.batch_hi,
                                                   centre=args.window_step)}), flush=True)
        return 0
    if args.only_d2q5:
        # profiling aid: the D2Q5 cavity leg alone, FP32
        if rank == 0:
            print(json.dumps({"d2q5_cavity": bench_d2q5(torch, solver, workloads, args.steps, args.warmup, stream, peak,
                                                       n=args.n or 4096, fp64=False, centre=args.window_step)}),
                  flush=True)
        return 0

    case = workloads.melt_2d() if args.n is None else workloads.melt_2d(n=args.n)
    nodes = case.nx * case.ny
    with ClockSampler(local) as clk:
        ms, st = bench_single(torch, solver, case, args.steps, args.warmup, stream, barrier, args.window_step)
    ms_max = max_over_ranks(torch, dist, ms, "cuda")
    value = job_mlups(world, nodes, args.steps, ms_max)
    per_step_ms = ms / args.steps
    k_step_ms, k_job_ms = st["kernel_ms"]
    # the dominant kernel: the flat kernel, two launches per step (the left and the
    # right half of the strips), timed with events on the handle's stream around each
    # launch (the wall kernel and the left half's Newton solves run beside the right
    # half on a second stream); 72 algorithmic bytes per node it updates
    fnodes = flat_nodes(case.nx, case.ny)
    flat_launch_ms = st["flat_ms"] / 2
    achieved = BYTES_FP32 * (fnodes / 2) / (flat_launch_ms * 1e-3) / 1e9

    extra = {}
    if rank == 0 and not args.quick:
        # FP64 form, same workload and window
        c64 = case.scaled(precision=workloads.FP64)
        ms64, _ = bench_single(torch, solver, c64, args.steps, args.warmup, stream)
        extra["fp64_form"] = {"workload": c64.name, "mlups": nodes * args.steps / ms64 / 1e3,
                              "gbs": BYTES_FP64 * nodes / (ms64 / args.steps * 1e-3) / 1e9,
                              "fp32_over_fp64": ms64 / ms}
        corner = {}
        for ste in workloads.CORNER_STE:
            cc = workloads.corner_2d(ste=ste)
            k = max(20, args.steps // 2)
            msc, stc = bench_single(torch, solver, cc, k, args.warmup, stream)
            corner["ste%g" % ste] = {"mlups": cc.nx * cc.ny * k / msc / 1e3,
                                     "newton_nodes": stc["newton_nodes"], "newton_max_iter": stc["newton_max_iter"]}
        extra["corner_2d_fp64_2048"] = corner
        # the paper's comparison scheme on the same workload and window (Sec. 6 compares run times)
        extra["eebm_form"] = bench_eebm(torch, solver, case, args.steps, args.warmup, stream, nodes, ms)
        extra["batched_256"] = bench_batch(torch, solver, workloads, max(20, args.steps // 2), args.warmup, stream)
        extra["adjoint_1024"] = bench_adjoint(torch, solver, workloads, stream)
        extra["adjoint_2048"] = bench_adjoint(torch, solver, workloads, stream, n=2048)
        extra["d1q3_512"] = bench_d1q3(torch, solver, workloads, stream)
        extra["bar_1d_801_three_schemes"] = bench_bar_1d(torch, solver, workloads, stream)
        extra["cavity_d2q9_801_three_schemes"] = bench_cavity_d2q9_801(torch, solver, workloads, stream)
        extra["d2q5_cavity_4096"] = bench_d2q5(torch, solver, workloads, args.steps, args.warmup, stream, peak)
    e2e_ms, h2d, d2h = bench_e2e(torch, solver, case, args.steps, stream, args.window_step) if rank == 0 else (0, 0, 0)
    errs = oracle_errors(torch, solver, workloads, stream) if rank == 0 else {}
    # every result carries its error against the FP64 oracle (the leg's small version)
    legs = {"fp64_form": ["melt_2d_fp64"], "eebm_form": ["eebm_fp32"], "batched_256": ["batched"],
            "adjoint_1024": ["adjoint"], "adjoint_2048": ["adjoint"], "d1q3_512": ["d1q3_melt_512"],
            "bar_1d_801_three_schemes": ["bar_1d_irebm", "bar_1d_eebm", "bar_1d_ilfbm"],
            "cavity_d2q9_801_three_schemes": ["cavity_d2q9_irebm", "cavity_d2q9_eebm", "cavity_d2q9_ilfbm"],
            "d2q5_cavity_4096": ["d2q5_cavity_fp32", "d2q5_cavity_fp64", "d2q5_eebm_fp32"],
            "corner_2d_fp64_2048": ["corner_ste%g" % s_ for s_ in workloads.CORNER_STE]}
    for leg, keys in legs.items():
        if leg in extra:
            extra[leg]["error_vs_oracle"] = {k: errs[k] for k in keys}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "dtype_detail": "FP32 populations and relaxation, FP32 m0 at saturated nodes, float-float moments at Newton and Dirichlet nodes, FP64 Newton refinement, fixed-point energy sums",
            "data": "synthetic",
            "config": {"workload": "%s: D2Q9 %dx%d, FP32 populations with FP64 Newton, west wall +1, other "
                                   "walls adiabatic, Ste 0.1, delta 0.01, tau 1.0, theta0 -0.2 + U(+-1e-3) seed 0; "
                                   "timed window centred on step %d of the 10,000-step job"
                                   % (case.name, case.nx, case.ny,
                                      args.window_step if args.window_step is not None else case.steps // 2),
                       "l2": "state 1.2 GB > 129 MB L2 (no flush needed)", "parallelism": "replicas" if world > 1 else "1 GPU"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak,
                         # dram__bytes_read.sum + dram__bytes_write.sum of one launch of this kernel in an ncu
                         # capture, per launch at this node count (None: not captured since the kernel changed)
                         "traffic": FLAT_TRAFFIC_PER_NODE * fnodes / 2 if FLAT_TRAFFIC_PER_NODE else None,
                         "traffic_note": FLAT_TRAFFIC_NOTE,
                         "bytes_per_node": BYTES_FP32, "units_per_launch": fnodes / 2,
                         "kernel": "d2q9_flat_kernel<false,false> (two launches per step: the left and the right "
                                   "half of the strips; d2q9_wall_kernel<false>, d2q9_wall_cols_kernel<false> and "
                                   "the left half's newton_jobs_kernel<float,false,9> on a second stream)",
                         "kernel_ms": flat_launch_ms,
                         "launches_per_step": 6,
                         "step_kernels_ms": k_step_ms,
                         "second_kernel": "newton_jobs_kernel<float,false,9> (the last job launch: the rest of "
                                          "the left half's list, the right half's, the publication)",
                         "second_kernel_ms": k_job_ms,
                         "whole_step_gbs": BYTES_FP32 * nodes / (per_step_ms * 1e-3) / 1e9,
                         "whole_step_frac": BYTES_FP32 * nodes / (per_step_ms * 1e-3) / 1e9 / peak,
                         "timing": "kernel_ms: mean of the flat launches' CUDA-event times (on the handle's "
                                   "stream) over 50 steps launched one by one right after the timed window; "
                                   "step_kernels_ms: every launch but the last job launch, same steps; "
                                   "whole_step: the timed window (graph replays)",
                         "peak_source": peak_kind},
            "error_vs_oracle": errs.get("melt_2d_fp32"),
            "cpu_baseline": cpu_baseline_sample(workloads) if (world == 1 and not args.no_cpu) else None,
            "e2e": {"value": nodes * args.steps / e2e_ms / 1e3, "unit": "MLUPS",
                    "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
                    "what": "lbm_stefan_set_state from a pinned host copy of the state at the start of the "
                            "headline's window (all populations), %d steps, lbm_stefan_get_fields to pinned host "
                            "theta; wall clock" % args.steps},
            "gpu_launches": 6 * args.steps,   # two flat halves, two wall kernels, two Newton launches
            "clocks": clk.summary(),
            "energy_imbalance_last_step": st["imbalance"],
            "newton_nodes_last_step": st["newton_nodes"],
            "newton_mean_iterations_last_step": st["newton_iters"] / max(1, st["newton_nodes"]),
            "newton_max_iterations_last_step": st["newton_max_iter"],
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier(device_ids=[local])
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--quick", action="store_true", help="headline only")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle baseline")
    ap.add_argument("--n", type=int, default=None,
                    help="side of the melting workload (default 4096, the benchmark); a profiling aid")
    ap.add_argument("--window-step", type=int, default=None,
                    help="centre the timed window on this step (default: mid-run, step 5,000); a profiling aid")
    ap.add_argument("--only-bar", action="store_true",
                    help="time the 1D bar (IREBM, EEBM, ILFBM) alone, --steps steps each; a profiling aid")
    ap.add_argument("--only-d2q5", action="store_true",
                    help="time the D2Q5 cavity leg alone, FP32, side --n (default 4096); a profiling aid")
    ap.add_argument("--only-corner", action="store_true",
                    help="time the FP64 corner leg alone (Ste 0.1, side --n, default 2048); a profiling aid")
    ap.add_argument("--only-batch", action="store_true",
                    help="time the batch leg alone (--batch-count problems, sides log-uniform in [64, --batch-hi]); "
                         "a profiling aid")
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--batch-hi", type=int, default=1024)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
