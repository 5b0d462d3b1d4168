"""GPU discrete adjoint (xflat_adjoint): against the oracle's discrete adjoint on small problems,
invariance under the checkpoint interval, and at the full adjoint workload size (200 E x 400 u,
5000 RK4 steps, checkpoints every 64 steps) against central differences of the CUDA forward run.

The full-size window is 100 -> 300 km: with 5000 steps from r = R the configured step is ~1e4
times too long for explicit RK4 near the neutrino sphere and the forward run itself diverges.
"""
import numpy as np
import pytest

from bulb_inputs import Workload, workload_adjoint
from oracle.physics import Bulb, Grid
from oracle.adjoint import rk4_adjoint

pytestmark = pytest.mark.gpu


def solver(xf, wl, N=None, theta=None, **over):
    cfg = xf.config_from_workload(wl, **over)
    if theta is not None:
        cfg.theta[0] = theta
    s = xf.Solver(cfg)
    s.set_spectra(Grid.from_workload(wl).N if N is None else N)
    return s


# (inputs, window, steps, checkpoint interval, tolerance relative to the largest gradient).  The
# r^-3 matter case: matter (~2e3 /km at 100 km) suppresses flavour change, P_ee stays within 1e-8
# of 1 and the largest luminosity gradient (1.5e-10) is dominated by the objective's own weights,
# du_j (P_ee - J) / sum W, a difference of two numbers near 1 that either side knows only to the
# ~1e-16 rounding of its state: 1e-5 of the largest gradient.
SMALL = [
    (dict(n_energy=13, n_angle=9), (100.0, 104.0), 80, 7, 1e-9),
    (dict(n_energy=5, n_angle=17, dm2=(2.4e-3, 0.0), theta=(0.2, 0.0, 0.0), matter="constant",
          lambda_const=3.0, L={"nue": 4e51, "nuebar": 3e51, "nux": 1e51, "nuxbar": 1e51}),
     (100.0, 104.0), 120, 64, 1e-9),
    (dict(n_energy=4, n_angle=6, matter="power_law"), (100.0, 100.5), 500, 100, 1e-5),
]


@pytest.mark.parametrize("kw,win,n,K,tol", SMALL)
def test_adjoint_matches_oracle_adjoint(xf, kw, win, n, K, tol):
    wl = Workload(name="adj", integrator="rk4", n_steps=n, **kw)
    r0, r1 = win
    s = solver(xf, wl)
    J, dN, dth = s.adjoint(r0, r1, n, K)
    b = Bulb(wl)
    Jo, GNo, Gtho = rk4_adjoint(b, b.initial_state(), r0, r1, n)
    assert J == pytest.approx(Jo, rel=1e-12)
    scale = np.abs(GNo * b.grid.N).max()
    assert scale > 0
    assert np.abs((dN - GNo) * b.grid.N).max() < tol * scale
    assert dth == pytest.approx(Gtho, rel=tol, abs=1e-15)


def test_adjoint_objective_matches_forward_and_checkpoint_interval_is_exact(xf):
    wl = Workload(name="adj", n_energy=11, n_angle=7, integrator="rk4", n_steps=50)
    r0, r1, n = 100.0, 103.0, 50
    outs = [solver(xf, wl).adjoint(r0, r1, n, K) for K in (1, 8, 50, 1000)]
    for J, dN, dth in outs[1:]:
        assert J == outs[0][0] and dth == outs[0][2]
        assert np.array_equal(dN, outs[0][1])
    s = solver(xf, wl, fixed_dr_km=(r1 - r0) / n)
    s.reset(r0)
    s.evolve(r0, r1)
    _, mean = s.pee(per_beam=False)
    assert outs[0][0] == pytest.approx(mean, rel=1e-13)


def test_adjoint_full_size_against_central_differences(xf):
    wl = workload_adjoint()
    r0, r1, n = 100.0, 300.0, wl.n_steps
    g = Grid.from_workload(wl)
    N0 = g.N
    th0 = wl.theta[0]
    J, dN, dth = solver(xf, wl).adjoint(r0, r1, n, 64)

    def J_of(N, theta=th0):
        s = solver(xf, wl, N=N, theta=theta, fixed_dr_km=(r1 - r0) / n)
        s.reset(r0)
        s.evolve(r0, r1)
        _, mean = s.pee(per_beam=False)
        s.close()
        return mean

    assert J == pytest.approx(J_of(N0), rel=1e-12)
    eps = 1e-5
    # the three luminosities (nu_e, nubar_e, and nu_x = nubar_x) and four nu_e bin weights, as
    # multiplicative factors around 1
    masks = []
    for sel in ([(0, 0)], [(1, 0)], [(0, 1), (1, 1)]):
        m = np.zeros_like(N0)
        for sp, fl in sel:
            m[sp, fl, :] = 1.0
        masks.append(m)
    for k in (0, 57, 123, 199):
        m = np.zeros_like(N0)
        m[0, 0, k] = 1.0
        masks.append(m)
    for m in masks:
        fd = (J_of(N0 * (1 + eps * m)) - J_of(N0 * (1 - eps * m))) / (2 * eps)
        adj = float((dN * N0 * m).sum())
        assert adj == pytest.approx(fd, rel=1e-5, abs=1e-8), (adj, fd)
    d = 1e-6
    fdth = (J_of(N0, th0 + d) - J_of(N0, th0 - d)) / (2 * d)
    assert abs(fdth) > 1e-4
    assert dth == pytest.approx(fdth, rel=1e-5, abs=1e-8)


def test_autograd_function(xf):
    torch = pytest.importorskip("torch")
    from paper_1912_10596_gb300.autograd import mean_survival
    wl = Workload(name="adj", n_energy=6, n_angle=5, integrator="rk4", n_steps=30)
    cfg = xf.config_from_workload(wl)
    N = torch.tensor(Grid.from_workload(wl).N, dtype=torch.float64, requires_grad=True)
    th = torch.tensor(0.1, dtype=torch.float64, requires_grad=True)
    J = mean_survival(N, th, cfg, 100.0, 102.0, 30, 8)
    (2.0 * J).backward()
    b = Bulb(wl)
    Jo, GNo, Gtho = rk4_adjoint(b, b.initial_state(), 100.0, 102.0, 30)
    assert float(J.detach()) == pytest.approx(Jo, rel=1e-12)
    assert np.allclose(N.grad.numpy(), 2.0 * GNo, rtol=1e-8, atol=1e-9 * np.abs(GNo).max())
    assert float(th.grad) == pytest.approx(2.0 * Gtho, rel=1e-8)


def test_autograd_parameters_match_central_differences(xf):
    """Gradients of J with respect to the three luminosities, the per-energy nu_e weights and
    theta_v through autograd (the adjoint's dJ/dN carried through the spectra by torch) against
    central differences of J itself."""
    torch = pytest.importorskip("torch")
    from paper_1912_10596_gb300.autograd import mean_survival_from_parameters
    wl = Workload(name="adjp", n_energy=6, n_angle=5, integrator="rk4", n_steps=30)
    cfg = xf.config_from_workload(wl)
    unit = Workload(name="unit", n_energy=6, n_angle=5,
                    L={k: 1e51 for k in ("nue", "nuebar", "nux", "nuxbar")})
    base = torch.tensor(Grid.from_workload(unit).N, dtype=torch.float64)
    L = torch.tensor([1.0, 1.3, 0.8], dtype=torch.float64, requires_grad=True)
    w = torch.linspace(0.8, 1.2, 6, dtype=torch.float64).requires_grad_(True)
    th = torch.tensor(0.1, dtype=torch.float64, requires_grad=True)
    J = mean_survival_from_parameters(L, w, th, base, cfg, 100.0, 102.0, 30, 8)
    J.backward()

    def J_at(Lv, wv, tv):
        with torch.no_grad():
            return float(mean_survival_from_parameters(Lv, wv, tv, base, cfg, 100.0, 102.0, 30, 8))

    h = 1e-6
    for i in range(3):
        e = torch.zeros(3, dtype=torch.float64)
        e[i] = h
        fd = (J_at(L.detach() + e, w.detach(), th.detach()) - J_at(L.detach() - e, w.detach(), th.detach())) / (2 * h)
        assert float(L.grad[i]) == pytest.approx(fd, rel=1e-5, abs=1e-9)
    for k in (0, 3, 5):
        e = torch.zeros(6, dtype=torch.float64)
        e[k] = h
        fd = (J_at(L.detach(), w.detach() + e, th.detach()) - J_at(L.detach(), w.detach() - e, th.detach())) / (2 * h)
        assert float(w.grad[k]) == pytest.approx(fd, rel=1e-5, abs=1e-9)
    fd = (J_at(L.detach(), w.detach(), th.detach() + h) - J_at(L.detach(), w.detach(), th.detach() - h)) / (2 * h)
    assert abs(fd) > 1e-4
    assert float(th.grad) == pytest.approx(fd, rel=1e-5)


def test_adjoint_argument_checks(xf):
    wl = Workload(name="adj", n_energy=4, n_angle=3, integrator="rk4", n_steps=10)
    s = solver(xf, wl)
    for args in ((100.0, 99.0, 10, 4), (100.0, 101.0, 0, 4), (100.0, 101.0, 10, 0), (5.0, 101.0, 10, 4)):
        with pytest.raises(xf.XflatError) as e:
            s.adjoint(*args)
        assert e.value.code == xf.ERR_INVAL
    w3 = Workload(name="adj3", n_flavor=3, n_energy=4, n_angle=3, dm2=(7.5e-5, 2.4e-3),
                  theta=(0.59, 0.15, 0.785), integrator="rk4", n_steps=10)
    s3 = solver(xf, w3)
    with pytest.raises(xf.XflatError) as e:
        s3.adjoint(100.0, 101.0, 10, 4)
    assert e.value.code == xf.ERR_UNSUPPORTED
