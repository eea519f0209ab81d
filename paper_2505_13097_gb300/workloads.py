"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This module holds random numbers, shapes and boundary settings only: none of
the method's arithmetic.  Every workload below is a synthetic stand-in shaped
like the paper's benchmarks (Sec. 6.1: a 1D bar melting from a hot wall;
Sec. 6.2: a square cavity cooled from two walls), at the sizes of the
benchmark configurations:

* ``melt_1d``        D1Q3, 512 nodes on [0,1], FP64, solid at -0.5, hot wall +1 on
                     the west, adiabatic east, Ste 0.1, delta 0.01, 20,000 steps;
* ``melt_2d``        D2Q9 4096 x 4096, FP32 populations / FP64 Newton, -0.2 plus
                     uniform noise of amplitude 1e-3 (seed 0), west wall +1, other
                     walls adiabatic, Ste 0.1, delta 0.01, 10,000 steps;
* ``corner_2d``      D2Q9 2048 x 2048, FP64, liquid at +0.3, south and west walls
                     at -1, north/east adiabatic, delta 0.005, tau 0.84,
                     Ste in {0.01, 0.1, 1}, 20,000 steps;
* ``batch_2d``       256 D2Q9 problems, sides log-uniform in [64, 1024] (seed 0),
                     Ste log-uniform in [0.01, 1], west wall uniform in [0.5, 2],
                     other walls adiabatic, -0.2 plus noise 1e-3, delta 0.01,
                     5,000 steps, FP32 populations;
* ``adjoint_2d``     D2Q9 1024 x 1024, 2,000 steps, FP32 forward; the target
                     liquid fraction comes from a run with Ste and the wall
                     temperature raised 5 % and theta0 + 1e-3 N(0,1) (seed 1);
* ``bar_1d``         the paper's 1D bar (Sec. 6.1) for timing: D1Q3, 801 nodes,
                     Ste = 100/350, solid at theta = -0.5 with the hot end at +1
                     and the cold end held at -0.5, tau 0.62, delta 0.01 (the
                     timing table's values), 204,800 steps (160 s), FP64;
* ``cavity_2d``      the paper's 2D case (Sec. 6.2) on D2Q5: the lower-left
                     quarter of a square cavity of liquid at theta = 1
                     (T_i = 10 C over T_f = 0 C) frozen from the west and south
                     walls at theta = -2 (T = -20 C), the north and east walls
                     symmetry lines closed by Eq. (17); Ste = c (T_i - T_f)/h_sl
                     = 1.762 * 10 / 338, tau 0.84 and delta 0.01 (the timing
                     table's values), FP32 populations; 4096 x 4096 by default.

tau = 1.0 wherever the configuration does not fix it (a reading: the paper
gives tau only for its own cases).  Walls are given as {"W": (kind, theta), ...} with kind 0 =
adiabatic, 1 = Dirichlet.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Tuple

import numpy as np

ADIABATIC, DIRICHLET = 0, 1
FP64, FP32 = 0, 1


@dataclasses.dataclass
class Case:
    name: str
    lattice: int                  # 1 = D1Q3, 2 = D2Q9, 3 = D2Q5
    nx: int
    ny: int
    tau: float
    delta: float
    ste: float
    walls: Dict[str, Tuple[int, float]]
    steps: int
    precision: int = FP64
    theta_init: float = 0.0
    noise: float = 0.0
    seed: int = 0
    bb_mode: int = 0              # adiabatic walls: 0 mirror, 1 link-wise bounce-back, 2 Eq. (17)

    def theta0(self) -> np.ndarray:
        """Initial temperature field, shape (ny, nx), float64."""
        th = np.full((self.ny, self.nx), self.theta_init, dtype=np.float64)
        if self.noise:
            rng = np.random.Generator(np.random.PCG64(self.seed))
            th += rng.uniform(-self.noise, self.noise, size=th.shape)
        return th

    def scaled(self, nx=None, ny=None, steps=None, **kw) -> "Case":
        """Same physics at another size or step count (parity cases)."""
        d = dataclasses.asdict(self)
        if nx is not None:
            d["nx"] = nx
        if ny is not None:
            d["ny"] = ny
        if steps is not None:
            d["steps"] = steps
        d.update(kw)
        return Case(**d)


def melt_1d(n=512, steps=20000) -> Case:
    return Case("melt_1d_d1q3_%d" % n, 1, n, 1, 1.0, 0.01, 0.1,
                {"W": (DIRICHLET, 1.0), "E": (ADIABATIC, 0.0)}, steps, FP64, theta_init=-0.5)


def melt_2d(n=4096, steps=10000, precision=FP32, seed=0) -> Case:
    return Case("melt_2d_d2q9_%d" % n, 2, n, n, 1.0, 0.01, 0.1,
                {"W": (DIRICHLET, 1.0), "E": (ADIABATIC, 0.0), "S": (ADIABATIC, 0.0), "N": (ADIABATIC, 0.0)},
                steps, precision, theta_init=-0.2, noise=1e-3, seed=seed)


def corner_2d(n=2048, ste=0.1, steps=20000, precision=FP64) -> Case:
    return Case("corner_2d_d2q9_%d_ste%g" % (n, ste), 2, n, n, 0.84, 0.005, ste,
                {"W": (DIRICHLET, -1.0), "S": (DIRICHLET, -1.0), "E": (ADIABATIC, 0.0), "N": (ADIABATIC, 0.0)},
                steps, precision, theta_init=0.3)


CORNER_STE = (0.01, 0.1, 1.0)


def batch_2d(count=256, lo=64, hi=1024, steps=5000, seed=0, precision=FP32) -> List[Case]:
    """Independent problems of uneven size, Ste and wall temperature."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sides = np.exp(rng.uniform(math.log(lo), math.log(hi), size=count))
    stes = np.exp(rng.uniform(math.log(0.01), math.log(1.0), size=count))
    walls = rng.uniform(0.5, 2.0, size=count)
    cases = []
    for k in range(count):
        n = int(round(sides[k]))
        cases.append(Case("batch%03d_%d" % (k, n), 2, n, n, 1.0, 0.01, float(stes[k]),
                          {"W": (DIRICHLET, float(walls[k])), "E": (ADIABATIC, 0.0),
                           "S": (ADIABATIC, 0.0), "N": (ADIABATIC, 0.0)},
                          steps, precision, theta_init=-0.2, noise=1e-3, seed=seed * 100003 + k + 1))
    return cases


def adjoint_2d(n=1024, steps=2000, precision=FP32) -> Case:
    return Case("adjoint_2d_d2q9_%d" % n, 2, n, n, 1.0, 0.01, 0.1,
                {"W": (DIRICHLET, 1.0), "E": (ADIABATIC, 0.0), "S": (ADIABATIC, 0.0), "N": (ADIABATIC, 0.0)},
                steps, precision, theta_init=-0.2, noise=1e-3, seed=0)


def adjoint_target_case(base: Case, rel=0.05) -> Case:
    """The perturbed-parameter run that produces the target liquid fraction."""
    walls = {k: (kind, th * (1.0 + rel) if kind == DIRICHLET else th) for k, (kind, th) in base.walls.items()}
    return base.scaled(ste=base.ste * (1.0 + rel), walls=walls)


def adjoint_target_theta0(base: Case, amp=1e-3, seed=1) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return base.theta0() + amp * rng.standard_normal(size=(base.ny, base.nx))


def bar_1d(n=801, steps=204800) -> Case:
    return Case("bar_1d_d1q3_%d" % n, 1, n, 1, 0.62, 0.01, 100.0 / 350.0,
                {"W": (DIRICHLET, 1.0), "E": (DIRICHLET, -0.5)}, steps, FP64, theta_init=-0.5)


CAVITY_STE = 1.762 * 10.0 / 338.0


def cavity_2d(n=4096, steps=5000, precision=FP32) -> Case:
    return Case("cavity_2d_d2q5_%d" % n, 3, n, n, 0.84, 0.01, CAVITY_STE,
                {"W": (DIRICHLET, -2.0), "S": (DIRICHLET, -2.0), "E": (ADIABATIC, 0.0), "N": (ADIABATIC, 0.0)},
                steps, precision, theta_init=1.0, bb_mode=2)


def random_field(shape, lo, hi, seed) -> np.ndarray:
    """Uniform random field (test inputs)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, size=shape)


def random_direction(shape, seed) -> np.ndarray:
    """Unit-variance normal direction (finite-difference checks)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(size=shape)


# ------------------------------------------------------------------ bench parity cases
# Small versions of the benchmark legs: the same lattices, precisions, methods,
# walls and parameters, at sizes the FP64 oracle finishes in seconds.  The
# oracle's results on them are stored in tests/golden/bench_refs.npz (written
# by tests/golden/make_bench_refs.py); bench.py runs each case through the
# same kernels as its leg and reports the error against those results beside
# the leg's speed.  Entries: name -> (case, method, extra solver arguments).
ILFBM_BAR_KW = {"newton_tol": 1e-12, "newton_max_iter": 200}
ILFBM_CAVITY_KW = {"newton_tol": 1e-12, "newton_max_iter": 400}


def bench_parity_cases():
    melt = melt_2d(n=130, steps=300).scaled(ny=64)
    cav5 = cavity_2d(n=64, steps=200)
    cav9 = cavity_2d(n=64, steps=100, precision=FP64).scaled(lattice=2, bb_mode=0)
    bar = bar_1d(steps=2000)
    cases = {
        "melt_2d_fp32": (melt, "IREBM", {}),
        "melt_2d_fp64": (melt.scaled(precision=FP64), "IREBM", {}),
        "eebm_fp32": (melt, "EEBM", {}),
        "d2q5_cavity_fp32": (cav5, "IREBM", {}),
        "d2q5_cavity_fp64": (cav5.scaled(precision=FP64), "IREBM", {}),
        "d2q5_eebm_fp32": (cav5, "EEBM", {}),
        "d1q3_melt_512": (melt_1d(), "IREBM", {}),
        "bar_1d_irebm": (bar, "IREBM", {}),
        "bar_1d_eebm": (bar, "EEBM", {}),
        "bar_1d_ilfbm": (bar, "ILFBM", dict(ILFBM_BAR_KW)),
        "cavity_d2q9_irebm": (cav9, "IREBM", {}),
        "cavity_d2q9_eebm": (cav9, "EEBM", {}),
        "cavity_d2q9_ilfbm": (cav9, "ILFBM", dict(ILFBM_CAVITY_KW)),
    }
    for ste in CORNER_STE:
        cases["corner_ste%g" % ste] = (corner_2d(n=64, ste=ste, steps=300), "IREBM", {})
    return cases


def bench_parity_batch() -> List[Case]:
    """Six problems drawn like the batched workload, sides 40 to 80, 100 steps."""
    return batch_2d(count=6, lo=40, hi=80, steps=100)


def bench_parity_adjoint() -> Case:
    """The adjoint workload at 48 x 48 over 40 steps (FP32 forward)."""
    return adjoint_2d(n=48, steps=40)
