"""Write bench_refs.npz: the FP64 oracle's results on the small versions of
the benchmark legs (paper_2505_13097_gb300.workloads.bench_parity_cases,
bench_parity_batch, bench_parity_adjoint).

bench.py runs the same cases through the CUDA library and reports, beside
each leg's speed, the error against these stored results: max |d theta| /
max |theta_ref| and max |d phi|.  Every value here comes from the oracle
(oracle/) on the seeded inputs of workloads.py; nothing comes from the CUDA
path.  Run from the repository root:

    python tests/golden/make_bench_refs.py

Stored per case: theta (ny x nx) and phi, the liquid fraction of the method
(IREBM: phi(theta) = (1 + tanh(theta/delta))/2; EEBM: the lever rule of the
enthalpy, min(max(Ste H, 0), 1); ILFBM: the liquid-fraction field l).  For
the adjoint: the target liquid fraction (from the oracle's perturbed run),
the loss, dL/dtheta0, dL/dtheta_wall and dL/dSte of the oracle's FP64 adjoint.
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2505_13097_gb300 import workloads  # noqa: E402

OUT = os.path.join(HERE, "bench_refs.npz")


def problem(c, **kw):
    return oracle.Problem(c.lattice, c.nx, c.ny, tau=c.tau, delta=c.delta, ste=c.ste, walls=c.walls,
                          bb_mode=c.bb_mode, **kw)


def phi_field(theta, delta):
    return np.vectorize(lambda x: oracle.phi(x, delta))(theta)


def lever_field(H, ste):
    return np.vectorize(lambda h: oracle.ilfbm_lever(h, ste))(H)


def run_case(c, method, kw):
    if method == "IREBM":
        P = problem(c, **kw)
        _, th = P.run(c.theta0(), c.steps)
        return th, phi_field(th, c.delta)
    if method == "EEBM":
        P = problem(c)
        f, th = P.eebm_run(c.theta0(), c.steps)
        _, H = P.eebm_fields(f)
        return th, lever_field(H, c.ste)
    if method == "ILFBM":
        P = problem(c)
        _, ell, th, bad, _ = P.ilfbm_run(c.theta0(), c.steps, tol=kw["newton_tol"], maxit=kw["newton_max_iter"])
        if bad:
            raise RuntimeError("oracle ILFBM inner loop did not converge in %d steps" % bad)
        return th, ell
    raise ValueError(method)


def adjoint_refs():
    base = workloads.bench_parity_adjoint()
    tcase = workloads.adjoint_target_case(base)
    Pt = problem(tcase)
    _, thT = Pt.run(workloads.adjoint_target_theta0(base), base.steps)
    target = phi_field(thT, base.delta)
    P = problem(base)
    L, g0, gw, gs = P.adjoint(base.theta0(), base.steps, target)
    return {"adjoint/target": target, "adjoint/loss": np.array(L), "adjoint/g_theta0": g0,
            "adjoint/g_wall": np.asarray(gw), "adjoint/g_ste": np.array(gs)}


def main():
    out = {}
    for name, (c, method, kw) in workloads.bench_parity_cases().items():
        th, ph = run_case(c, method, kw)
        out[name + "/theta"] = th
        out[name + "/phi"] = ph
        print(name, c.nx, c.ny, c.steps, method, flush=True)
    for k, c in enumerate(workloads.bench_parity_batch()):
        th, ph = run_case(c, "IREBM", {})
        out["batch%d/theta" % k] = th
        out["batch%d/phi" % k] = ph
    out.update(adjoint_refs())
    np.savez_compressed(OUT, **out)
    print("wrote", OUT, os.path.getsize(OUT), "bytes")


if __name__ == "__main__":
    main()
