"""The benchmark configurations run to their end on the GPU and checked against
what the mathematics fixes at that size.

* 1D melting (D1Q3, 512 nodes, 20,000 steps, FP64): the oracle's result, and
  the first-zero front against the Neumann solution x_f = 2 lambda sqrt(t)
  (Sec. 2, Eqs. 2-3), within the bound of the oracle's own pin (5e-4).
* 2D melting (D2Q9 4096^2, 10,000 steps, FP32 populations / FP64 Newton):
  the front stays planar (the initial noise of 1e-3 moves it by far less
  than a node); its mean first zero follows 2 lambda sqrt(t) to within half a
  lattice spacing (the oracle's planar D1Q3 run of the same size is 0.07
  nodes from it) and the oracle's planar run to within 0.02 nodes; the
  Dirichlet column holds and the energy balance closes.  The same run in the
  FP64 form gives the FP32 form's error at full size, within the FP32-form
  tolerance (2e-5 on theta, 1e-4 on phi).
* 2D corner solidification (D2Q9 2048^2, FP64, 20,000 steps, Ste in
  {0.01, 0.1, 1}): theta at the diagonal probes i = 16, 64, 256 (Sec. 6.2
  plots such histories), sampled every 20 steps, has no plateau: once a
  probe starts cooling, no two samples are equal.  The explicit enthalpy
  method (Algorithm 2) on the same case does hold theta at exactly 0 while a
  probe's latent heat is released, which shows the check can fail.
"""
import numpy as np
import pytest

from paper_2505_13097_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_13097_gb300 import solver
    return solver


def rel_err(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def first_zero(row):
    """First sign change of theta from the hot wall, linearly interpolated (node units)."""
    j = int(np.argmax(row < 0.0))
    return j - 1 + row[j - 1] / (row[j - 1] - row[j])


def test_config1_melt_1d_to_the_end(gpu, orc):
    from oracle import neumann
    c = workloads.melt_1d()
    S = gpu.Stefan.from_case(c)
    S.set_ic(c.theta0())
    S.step(c.steps)
    th = S.theta()
    fz = S.front_position("W")[0]
    st = S.stats()
    S.close()
    assert st["error"] == 0 and st["steps"] == c.steps
    P = orc.Problem(1, c.nx, 1, tau=c.tau, delta=c.delta, ste=c.ste, walls=c.walls)
    _, ref = P.run(c.theta0(), c.steps)
    # FP64 tolerance: 1e-12, or ten times the oracle's own rounding floor over 20,000 steps
    rng = np.random.Generator(np.random.PCG64(12345))
    th0 = c.theta0()
    pert = th0 + np.spacing(th0) * rng.choice([-1, 0, 1], size=th0.shape)
    _, alt = P.run(pert, c.steps)
    tol = max(1e-12, 10 * rel_err(alt, ref))
    err = rel_err(th, ref)
    print("config 1: GPU vs oracle %.2e (tolerance %.2e)" % (err, tol))
    assert err < tol
    lam = neumann.stefan_lambda(c.ste, c.theta_init)
    dx = 1.0 / (c.nx - 1)
    t = neumann.lattice_time(c.steps, c.nx, c.tau)
    e_front = abs(fz * dx - neumann.front(t, lam))
    print("config 1: front %.6f, Neumann %.6f, |diff| %.2e" % (fz * dx, neumann.front(t, lam), e_front))
    assert e_front < 5e-4


@pytest.fixture(scope="module")
def melt_full(gpu):
    """The 4096^2 melting workload run to its end in both forms."""
    out = {}
    for prec in (workloads.FP32, workloads.FP64):
        c = workloads.melt_2d(precision=prec)
        S = gpu.Stefan.from_case(c)
        S.set_ic(c.theta0())
        S.step(c.steps)
        th, ph, _ = S.fields()
        fz, _, lines, _ = S.front_position("W")
        st = S.stats()
        S.close()
        out[prec] = dict(theta=th, phi=ph, front=fz, lines=lines, stats=st, case=c)
    return out


def test_config2_melt_2d_front_to_the_end(melt_full, orc):
    from oracle import neumann
    r = melt_full[workloads.FP32]
    c, st = r["case"], r["stats"]
    assert st["error"] == 0 and st["steps"] == c.steps
    lam = neumann.stefan_lambda(c.ste, c.theta_init)
    xn = 2.0 * lam * np.sqrt(c.steps * (c.tau - 0.5) / 3.0)   # node units (dx = 1, lattice time)
    # the oracle's planar run (the y-uniform D2Q9 problem is D1Q3 row by row) without the noise
    P = orc.Problem(1, c.nx, 1, tau=c.tau, delta=c.delta, ste=c.ste, walls={"W": c.walls["W"], "E": c.walls["E"]})
    _, th1 = P.run(np.full((1, c.nx), c.theta_init), c.steps)
    xo = first_zero(th1[0])
    spread = r["lines"].max() - r["lines"].min()
    print("config 2: mean front %.4f nodes, Neumann %.4f, oracle planar %.4f, spread over rows %.2e; "
          "energy %.6e, last step's imbalance %.2e (max %.2e)"
          % (r["front"], xn, xo, spread, st["energy"], st["imbalance"], st["imbalance_max"]))
    assert abs(r["front"] - xn) < 0.5
    assert abs(r["front"] - xo) < 0.02
    assert spread < 0.05
    assert np.max(np.abs(r["theta"][:, 0] - 1.0)) < 1e-6
    # energy balance: FP64 form to 1e-9 of E; FP32 form to the rounding of its
    # stored populations in one step (each of the 9 per node rounded once by the
    # relaxation and once by its product w_i c: 18 half-ulps of the largest)
    st64 = melt_full[workloads.FP64]["stats"]
    assert abs(st64["imbalance"]) < 1e-9 * abs(st64["energy"])
    bound32 = c.nx * c.ny * 18 * 0.5 * 2.0 ** -24 * np.max(np.abs(r["theta"]))
    print("config 2 energy balance: FP32 form %.2e (bound %.2e), FP64 form %.2e of E = %.4e"
          % (st["imbalance"], bound32, st64["imbalance"], st64["energy"]))
    assert abs(st["imbalance"]) < bound32


def test_config2_fp32_form_against_fp64_form_full_size(melt_full):
    a, b = melt_full[workloads.FP32], melt_full[workloads.FP64]
    et = rel_err(a["theta"], b["theta"])
    ep = np.max(np.abs(a["phi"] - b["phi"]))
    print("config 2 at full size: FP32 form vs FP64 form, max|d theta|/max|theta| %.2e, max|d phi| %.2e" % (et, ep))
    assert et < 2e-5 and ep < 1e-4
    assert abs(a["front"] - b["front"]) < 1e-3


def probe_history(gpu, c, method, probes, every=20):
    import torch
    S = gpu.Stefan.from_case(c)
    if method != "IREBM":
        S.set_method(method)
    S.set_ic(c.theta0())
    plane = S.new_theta_planes(1)
    idx = torch.tensor([p * S.row_stride + p for p in probes], device="cuda")
    hist = []
    for _ in range(c.steps // every):
        S.step(every)
        S.theta_plane(plane[0])
        hist.append(plane[0].reshape(-1)[idx])
    S.sync()
    S.close()
    return torch.stack(hist).cpu().numpy()


def plateau_samples(h, theta0):
    """Pairs of consecutive equal samples after the probe has started to cool."""
    active = np.abs(h[:-1] - theta0) > 1e-12
    return int(np.sum(active & (np.abs(np.diff(h)) < 1e-14)))


@pytest.mark.parametrize("ste", workloads.CORNER_STE)
def test_config3_corner_probe_histories(gpu, ste):
    c = workloads.corner_2d(ste=ste)
    probes = [16, 64, 256]
    hi = probe_history(gpu, c, "IREBM", probes)
    he = probe_history(gpu, c, "EEBM", probes)
    for j, p in enumerate(probes):
        pi, pe = plateau_samples(hi[:, j], c.theta_init), plateau_samples(he[:, j], c.theta_init)
        print("config 3, Ste %g, probe (%d, %d): theta %.4f -> %.4f, plateau samples IREBM %d, EEBM %d"
              % (ste, p, p, hi[0, j], hi[-1, j], pi, pe))
        assert np.all(np.isfinite(hi[:, j]))
        assert pi == 0
    if ste >= 0.1:
        # the probe at i = 16 is reached by the front within 20,000 steps: the
        # explicit enthalpy method holds it at theta = 0 while it solidifies
        assert plateau_samples(he[:, 0], c.theta_init) > 0
