"""FP64 CPU oracle of the IREBM step (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  It shares
no code with the CUDA library in ``paper_2505_13097_gb300``; both only take
their inputs from the seeded generators in ``paper_2505_13097_gb300.workloads``.

``irebm_oracle.c`` holds the method (Algorithm 3 of the paper, the boundary
closures of Sec. 4.2, the discrete adjoint, and the explicit enthalpy based
method of Algorithm 2 for comparison); this module only marshals
numpy arrays into it.  ``neumann`` holds the closed-form solution of Sec. 2.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "irebm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

WALLS = {"W": 0, "E": 1, "S": 2, "N": 3}
ADIABATIC, DIRICHLET = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("tau", ctypes.c_double), ("delta", ctypes.c_double), ("ste", ctypes.c_double),
        ("newton_tol", ctypes.c_double), ("newton_max_iter", ctypes.c_int),
        ("bb_mode", ctypes.c_int),
        ("wall_kind", ctypes.c_int * 4), ("wall_theta", ctypes.c_double * 4),
    ]


class Diag(ctypes.Structure):
    _fields_ = [
        ("energy_before", ctypes.c_double), ("energy_after", ctypes.c_double),
        ("flux", ctypes.c_double), ("max_iter", ctypes.c_int), ("failed", ctypes.c_int),
    ]


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_P = ctypes.POINTER(Params)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            l = ctypes.CDLL(build())
            l.orc_phi.restype = ctypes.c_double
            l.orc_phi.argtypes = [ctypes.c_double, ctypes.c_double]
            l.orc_dphi.restype = ctypes.c_double
            l.orc_dphi.argtypes = [ctypes.c_double, ctypes.c_double]
            l.orc_newton.restype = ctypes.c_double
            l.orc_newton.argtypes = [ctypes.c_double] * 5 + [ctypes.c_int, _I, _I]
            l.orc_init.restype = None
            l.orc_init.argtypes = [_P, _D, _D]
            l.orc_theta.restype = None
            l.orc_theta.argtypes = [_P, _D, _D]
            l.orc_energy.restype = ctypes.c_double
            l.orc_energy.argtypes = [_P, _D]
            l.orc_step.restype = ctypes.c_int
            l.orc_step.argtypes = [_P, _D, _D, _D, _D, _D, _I, ctypes.POINTER(Diag)]
            l.orc_run.restype = ctypes.c_int
            l.orc_run.argtypes = [_P, _D, ctypes.c_int, _D, _D]
            l.orc_loss.restype = ctypes.c_double
            l.orc_loss.argtypes = [_P, _D, ctypes.c_int, _D]
            l.orc_adjoint.restype = ctypes.c_double
            l.orc_adjoint.argtypes = [_P, _D, ctypes.c_int, _D, _D, _D, _D]
            l.orc_eebm_theta.restype = ctypes.c_double
            l.orc_eebm_theta.argtypes = [ctypes.c_double, ctypes.c_double]
            l.orc_eebm_enthalpy.restype = ctypes.c_double
            l.orc_eebm_enthalpy.argtypes = [ctypes.c_double, ctypes.c_double]
            l.orc_eebm_init.restype = None
            l.orc_eebm_init.argtypes = [_P, _D, _D]
            l.orc_eebm_fields.restype = None
            l.orc_eebm_fields.argtypes = [_P, _D, _D, _D]
            l.orc_eebm_step.restype = ctypes.c_int
            l.orc_eebm_step.argtypes = [_P, _D, _D, ctypes.POINTER(Diag)]
            l.orc_eebm_run.restype = ctypes.c_int
            l.orc_eebm_run.argtypes = [_P, _D, ctypes.c_int, _D, _D]
            l.orc_ilfbm_lever.restype = ctypes.c_double
            l.orc_ilfbm_lever.argtypes = [ctypes.c_double, ctypes.c_double]
            l.orc_ilfbm_init.restype = None
            l.orc_ilfbm_init.argtypes = [_P, _D, _D, _D]
            l.orc_ilfbm_energy.restype = ctypes.c_double
            l.orc_ilfbm_energy.argtypes = [_P, _D, _D]
            l.orc_ilfbm_step.restype = ctypes.c_int
            l.orc_ilfbm_step.argtypes = [_P, _D, _D, _D, _D, ctypes.c_double, ctypes.c_int, _I,
                                         ctypes.POINTER(Diag)]
            l.orc_ilfbm_run.restype = ctypes.c_int
            l.orc_ilfbm_run.argtypes = [_P, _D, ctypes.c_int, ctypes.c_double, ctypes.c_int, _D, _D, _D, _I]
            _lib = l
    return _lib


def _dp(a):
    return a.ctypes.data_as(_D) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Problem:
    """One Stefan problem: lattice, sizes, tau, delta, Ste, Newton settings, walls.

    ``lattice`` is 1 (D1Q3, ``ny`` = 1), 2 (D2Q9) or 3 (D2Q5).  ``walls`` maps "W", "E",
    "S", "N" to ``(kind, theta)`` with kind 0 = adiabatic, 1 = Dirichlet.
    ``bb_mode`` closes the adiabatic walls: 0 mirror bounce-back, 1 link-wise
    bounce-back (Sec. 4.2.2), 2 the D2Q5 Neumann closure of Eq. (17).
    """

    def __init__(self, lattice, nx, ny=1, tau=1.0, delta=0.01, ste=0.1, walls=None,
                 newton_tol=1e-14, newton_max_iter=60, bb_mode=0):
        self.lattice, self.nx, self.ny = int(lattice), int(nx), int(ny)
        self.q = {1: 3, 2: 9, 3: 5}[self.lattice]
        if int(bb_mode) == 2 and (self.lattice != 3 or self.nx < 3 or self.ny < 3):
            raise ValueError("the Neumann closure of Eq. (17) is the D2Q5 one, nx and ny >= 3")
        p = Params()
        p.lattice, p.nx, p.ny = self.lattice, self.nx, self.ny
        p.tau, p.delta, p.ste = float(tau), float(delta), float(ste)
        p.newton_tol, p.newton_max_iter, p.bb_mode = float(newton_tol), int(newton_max_iter), int(bb_mode)
        for name, k in WALLS.items():
            kind, th = (walls or {}).get(name, (ADIABATIC, 0.0))
            p.wall_kind[k] = int(kind)
            p.wall_theta[k] = float(th)
        self.p = p

    def _no_eq17(self, what):
        if self.p.bb_mode == 2:
            raise NotImplementedError(what + " is written for the bounce-back closures")

    @property
    def shape(self):
        return (self.ny, self.nx)

    def init(self, theta0):
        f = np.empty((self.q, self.ny, self.nx))
        lib().orc_init(ctypes.byref(self.p), _dp(_f64(theta0).reshape(self.shape)), _dp(f))
        return f

    def theta(self, f):
        th = np.empty(self.shape)
        lib().orc_theta(ctypes.byref(self.p), _dp(_f64(f)), _dp(th))
        return th

    def energy(self, f):
        return lib().orc_energy(ctypes.byref(self.p), _dp(_f64(f)))

    def step(self, f, detail=False):
        """One step of Algorithm 3.  With ``detail`` also returns per-node
        m0, theta(t), root and Newton iterations, and the step diagnostics."""
        f = _f64(f)
        fn = np.empty_like(f)
        if not detail:
            r = lib().orc_step(ctypes.byref(self.p), _dp(f), _dp(fn), None, None, None, None, None)
            if r < 0:
                raise MemoryError("oracle step")
            return fn
        m0, th, rt = (np.empty(self.shape) for _ in range(3))
        it = np.empty(self.shape, dtype=np.int32)
        d = Diag()
        r = lib().orc_step(ctypes.byref(self.p), _dp(f), _dp(fn), _dp(m0), _dp(th), _dp(rt),
                           it.ctypes.data_as(_I), ctypes.byref(d))
        if r < 0:
            raise MemoryError("oracle step")
        return fn, dict(m0=m0, theta=th, root=rt, iters=it, energy_before=d.energy_before,
                        energy_after=d.energy_after, flux=d.flux, max_iter=d.max_iter, failed=d.failed)

    def run(self, theta0, nsteps):
        """``nsteps`` steps from the equilibrium state of ``theta0``: (f, theta)."""
        f = np.empty((self.q, self.ny, self.nx))
        th = np.empty(self.shape)
        r = lib().orc_run(ctypes.byref(self.p), _dp(_f64(theta0).reshape(self.shape)), int(nsteps), _dp(f), _dp(th))
        if r < 0:
            raise MemoryError("oracle run")
        if r > 0:
            raise RuntimeError("oracle Newton did not converge at %d node updates" % r)
        return f, th

    def loss(self, theta0, nsteps, phi_target):
        self._no_eq17("the adjoint")
        return lib().orc_loss(ctypes.byref(self.p), _dp(_f64(theta0).reshape(self.shape)), int(nsteps),
                              _dp(_f64(phi_target).reshape(self.shape)))

    def adjoint(self, theta0, nsteps, phi_target):
        """Loss and its gradient: (L, dL/dtheta0, dL/dtheta_wall[4], dL/dSte)."""
        self._no_eq17("the adjoint")
        g0 = np.empty(self.shape)
        gw = np.zeros(4)
        gs = np.zeros(1)
        L = lib().orc_adjoint(ctypes.byref(self.p), _dp(_f64(theta0).reshape(self.shape)), int(nsteps),
                              _dp(_f64(phi_target).reshape(self.shape)), _dp(g0), _dp(gw), _dp(gs))
        if not np.isfinite(L):
            raise MemoryError("oracle adjoint")
        return L, g0, gw, float(gs[0])


    # ---- explicit enthalpy based method (EEBM, Algorithm 2): f carries H = M0(f)
    def eebm_init(self, theta0):
        f = np.empty((self.q, self.ny, self.nx))
        lib().orc_eebm_init(ctypes.byref(self.p), _dp(_f64(theta0).reshape(self.shape)), _dp(f))
        return f

    def eebm_fields(self, f):
        """(theta, H) of an EEBM state: H = M0(f), theta = Theta(H)."""
        th, H = np.empty(self.shape), np.empty(self.shape)
        lib().orc_eebm_fields(ctypes.byref(self.p), _dp(_f64(f)), _dp(th), _dp(H))
        return th, H

    def eebm_step(self, f, detail=False):
        f = _f64(f)
        fn = np.empty_like(f)
        d = Diag()
        if lib().orc_eebm_step(ctypes.byref(self.p), _dp(f), _dp(fn), ctypes.byref(d)) < 0:
            raise MemoryError("oracle step")
        if not detail:
            return fn
        return fn, dict(energy_before=d.energy_before, energy_after=d.energy_after, flux=d.flux)

    def eebm_run(self, theta0, nsteps):
        """``nsteps`` EEBM steps from the equilibrium state of ``theta0``: (f, theta)."""
        f = np.empty((self.q, self.ny, self.nx))
        th = np.empty(self.shape)
        if lib().orc_eebm_run(ctypes.byref(self.p), _dp(_f64(theta0).reshape(self.shape)), int(nsteps),
                              _dp(f), _dp(th)) < 0:
            raise MemoryError("oracle run")
        return f, th

    # ---- implicit liquid fraction based method (ILFBM, Algorithm 1): state (f, l)
    def ilfbm_init(self, theta0):
        self._no_eq17("ILFBM")
        f = np.empty((self.q, self.ny, self.nx))
        ell = np.empty(self.shape)
        lib().orc_ilfbm_init(ctypes.byref(self.p), _dp(_f64(theta0).reshape(self.shape)), _dp(f), _dp(ell))
        return f, ell

    def ilfbm_energy(self, f, ell):
        """sum theta + l/Ste, theta = M0(f)."""
        return lib().orc_ilfbm_energy(ctypes.byref(self.p), _dp(_f64(f)), _dp(_f64(ell)))

    def ilfbm_step(self, f, ell, tol=1e-12, maxit=200):
        """One step of Algorithm 1: (f~, l~, inner iterations, converged, diagnostics)."""
        self._no_eq17("ILFBM")
        f, ell = _f64(f), _f64(ell)
        fn, ln = np.empty_like(f), np.empty_like(ell)
        it = ctypes.c_int()
        d = Diag()
        r = lib().orc_ilfbm_step(ctypes.byref(self.p), _dp(f), _dp(ell), _dp(fn), _dp(ln), float(tol), int(maxit),
                                 ctypes.byref(it), ctypes.byref(d))
        if r < 0:
            raise MemoryError("oracle step")
        return fn, ln, it.value, r == 0, dict(energy_before=d.energy_before, energy_after=d.energy_after,
                                              flux=d.flux)

    def ilfbm_run(self, theta0, nsteps, tol=1e-12, maxit=200):
        """``nsteps`` ILFBM steps from (w_i theta0, [theta0 > 0]): (f, l, theta,
        steps whose inner loop did not converge, largest inner iteration count)."""
        self._no_eq17("ILFBM")
        f = np.empty((self.q, self.ny, self.nx))
        ell, th = np.empty(self.shape), np.empty(self.shape)
        mx = ctypes.c_int()
        r = lib().orc_ilfbm_run(ctypes.byref(self.p), _dp(_f64(theta0).reshape(self.shape)), int(nsteps), float(tol),
                                int(maxit), _dp(f), _dp(ell), _dp(th), ctypes.byref(mx))
        if r < 0:
            raise MemoryError("oracle run")
        return f, ell, th, r, mx.value


def ilfbm_lever(H, ste):
    """Lever rule of Algorithm 1: l(H) = 0 below 0, Ste H on [0, 1/Ste], 1 above."""
    return lib().orc_ilfbm_lever(float(H), float(ste))


def eebm_theta(H, ste):
    return lib().orc_eebm_theta(float(H), float(ste))


def eebm_enthalpy(theta, ste):
    return lib().orc_eebm_enthalpy(float(theta), float(ste))


def phi(x, delta):
    return lib().orc_phi(float(x), float(delta))


def newton(m0, theta, ste, delta, tol=1e-14, maxit=60):
    """Local Newton root of Eq. (14) for one node: (root, iterations, converged)."""
    it, ok = ctypes.c_int(), ctypes.c_int()
    r = lib().orc_newton(float(m0), float(theta), float(ste), float(delta), float(tol), int(maxit),
                         ctypes.byref(it), ctypes.byref(ok))
    return r, it.value, bool(ok.value)
