"""Pins of the oracle's whole time step against closed-form solutions,
invariants and convergence orders that the paper and the mathematics fix.

* porous Brinkman Poiseuille flow (steady x-momentum of Eq. GoverneEq with F of
  Eq. ForceEq and F_eps = 0) -- exact profile, second-order convergence
  (Sec. 4.1 reports second order for the flow field);
* the same channel with the Forchheimer term, against a 1-D boundary-value
  solve of the same ODE to 1e-12;
* conservation in a periodic box: sum f = N rho0 and sum g constant
  (sum f^eq = rho0, sum F_i = 0, sum g^eq = sigma T, sum P_i = 0);
* a uniform heat source: sigma dT/dt = Q exactly;
* an advected, diffusing sine wave with eps != sigma and B != 0, against
  sigma dT/dt + u . grad T = alpha_e lap T with alpha_e = sigma cs2 (tau_T - B - 1/2)
  (Eq. Therdiff): decay rate and phase speed converge at second order;
* pure conduction in the cavity: T is exactly linear, Nu = 1;
* stable stratification: hydrostatic pressure gradient rho0 g beta (T - T0);
* the cavity's centro-symmetry.
"""
import numpy as np
import pytest
from scipy.integrate import solve_bvp

import oracle
from paper_1505_02976_gb300 import workloads as W

CS2 = 1.0 / 3.0


def _relerr(a, n):
    """Relative global error E of Sec. 4: sum |a - n| / sum |a|."""
    return np.abs(a - n).sum() / np.abs(a).sum()


def _steady_channel(p, chunk=200, max_chunks=400):
    o = oracle.Oracle(p)
    prev = None
    for _ in range(max_chunks):
        o.run(chunk)
        u = o.moments()["ux"][:, 0]
        if prev is not None and np.abs(u - prev).max() <= 1e-14 * np.abs(u).max():
            break
        prev = u
    return o, u


def _brinkman(H, G, K, nu, nu_e, eps):
    y = np.arange(H + 1.0)
    r = np.sqrt(eps * nu / (K * nu_e))
    return G * K / nu * (1.0 - np.cosh(r * (y - H / 2.0)) / np.cosh(r * H / 2.0))


def _channel(H, A, Da=1e-2, eps=0.5, umax=1e-4, forchheimer=0, G=None):
    nu_e = CS2 * (1.0 - A - 0.5)
    K = Da * H * H
    if G is None:
        G = umax * nu_e / K
    p = W.poiseuille(nx=2, ny=H + 1, G=G, eps=eps, Da=Da, nu=nu_e, A=A, forchheimer=forchheimer)
    return p, G, K, nu_e


@pytest.mark.parametrize("A", [0.2, -0.2])
def test_brinkman_poiseuille_second_order(A):
    errs = []
    for H in (16, 32, 64):
        p, G, K, nu = _channel(H, A)
        _, u = _steady_channel(p)
        errs.append(_relerr(_brinkman(H, G, K, nu, nu, p["eps"]), u))
    order = np.log2(errs[1] / errs[2])
    assert errs[2] < 1e-3
    assert order > 1.7, errs


def test_brinkman_poiseuille_standard_lbgk_limit():
    """A = 0 is the standard LBGK model (Sec. 3.1)."""
    p, G, K, nu = _channel(32, 0.0)
    _, u = _steady_channel(p)
    assert _relerr(_brinkman(32, G, K, nu, nu, p["eps"]), u) < 1e-5


def test_forchheimer_channel_against_bvp():
    H, eps, Da, A = 48, 0.5, 1e-2, 0.0
    nu = CS2 * (1.0 - A - 0.5)
    K = Da * H * H
    G = 9e-2 * nu / K
    p = W.poiseuille(nx=2, ny=H + 1, G=G, eps=eps, Da=Da, nu=nu, A=A, forchheimer=1)
    _, u = _steady_channel(p)
    Feps = 1.75 / np.sqrt(150.0 * eps ** 3)  # Ergun (Sec. 2)

    def rhs(y, Y):
        return np.vstack([Y[1], (eps * nu / K * Y[0] + eps * Feps / np.sqrt(K) * np.abs(Y[0]) * Y[0]
                                 - eps * G) / nu])

    ys = np.linspace(0.0, H, 2001)
    sol = solve_bvp(rhs, lambda a, b: np.array([a[0], b[0]]), ys, np.zeros((2, ys.size)),
                    tol=1e-12, max_nodes=200000)
    assert sol.status == 0
    ub = sol.sol(np.arange(H + 1.0))[0]
    assert u.max() > 0.04  # the quadratic drag matters at this speed
    assert _relerr(_brinkman(H, G, K, nu, nu, eps), u) > 0.1
    assert _relerr(ub, u) < 1e-5


def test_periodic_box_conservation():
    p = W.problem(nx=12, ny=10, bc=("periodic",) * 4, Ra=1e4, Da=1e-3, eps=0.5, sigma=1.3,
                  tau_f=0.8, tau_T=1.2)
    T, ux, uy = W.random_fields(p, seed=3, amp_u=2e-3)
    o = oracle.Oracle(p, T=T, ux=ux, uy=uy)
    m0, e0 = o.totals()
    N = p["nx"] * p["ny"]
    assert m0 == pytest.approx(N * p["rho0"], rel=1e-14)
    o.run(300)
    m1, e1 = o.totals()
    assert m1 == pytest.approx(N * p["rho0"], rel=1e-13)
    assert e1 == pytest.approx(e0, rel=1e-13)
    assert np.abs(o.moments()["ux"]).max() > 1e-5  # the box did move


def test_uniform_heat_source():
    """sigma T = sum g + Q/2 and sum_i g*_i = sum_i g_i + Q per node, so after
    n steps T = T_init + (n + 1/2) Q / sigma on every node."""
    Q, sigma, n = 1e-4, 1.5, 40
    p = W.problem(nx=6, ny=5, bc=("periodic",) * 4, Q=Q, sigma=sigma, gbeta=0.0, nu=0.1,
                  alpha_e=0.1, T_init=0.3)
    o = oracle.Oracle(p)
    o.run(n)
    T = o.moments()["T"]
    assert np.allclose(T, 0.3 + (n + 0.5) * Q / sigma, rtol=0, atol=1e-14)


def _sine(N, u0=0.1, eps=0.6, sigma=1.5, B=0.2):
    p = W.problem(nx=N, ny=1, bc=("periodic",) * 4, da_infinite=1, gbeta=0.0, nu=0.1, eps=eps,
                  sigma=sigma, B=B)
    x = np.arange(N)
    k = 2.0 * np.pi / N
    T = 0.5 + 0.1 * np.sin(k * x)[None, :]
    o = oracle.Oracle(p, T=T, ux=np.full((1, N), u0), uy=np.zeros((1, N)))
    alpha = sigma * CS2 * (1.0 - B - 0.5)
    lam, om = alpha * k * k / sigma, k * u0 / sigma

    def coef():
        return np.sum((o.moments()["T"][0] - 0.5) * np.exp(-1j * k * x))

    o.run(int(0.2 / lam))
    c1 = c = coef()
    dt, done, phase = int(1.0 / lam), 0, 0.0
    while done < dt:
        s = min(N, dt - done)
        o.run(s)
        done += s
        cn = coef()
        phase += np.angle(cn / c)
        c = cn
    return np.log(abs(c1) / abs(c)) / dt / lam - 1.0, -phase / dt / om - 1.0


def test_advected_sine_wave_recovers_energy_equation():
    e = [_sine(N) for N in (32, 64, 128)]
    lam_err = np.abs([v[0] for v in e])
    om_err = np.abs([v[1] for v in e])
    assert lam_err[-1] < 1e-4 and om_err[-1] < 2e-4
    assert np.log2(lam_err[1] / lam_err[2]) > 1.8
    assert np.log2(om_err[1] / om_err[2]) > 1.8


def test_pure_conduction_is_exactly_linear():
    p = W.cavity(12, 1e3, 1e-2, 0.6, gbeta=0.0, nu=0.1, alpha_e=0.1)
    o = oracle.Oracle(p)
    o.run(6000)
    m = o.moments()
    Tl = 1.0 - np.arange(12) / 11.0
    assert np.abs(m["T"] - Tl[None, :]).max() < 1e-12
    assert np.abs(m["ux"]).max() == 0.0 and np.abs(m["uy"]).max() == 0.0
    for side in ("W", "E"):
        nu_mean, nu_loc = o.nusselt(side)
        assert nu_mean == pytest.approx(1.0, abs=1e-12)
        assert np.allclose(nu_loc, 1.0, atol=1e-12)


def test_hydrostatic_pressure_under_stable_stratification():
    """Cold bottom, hot top, periodic in x: the rest state has T linear in y
    and dp/dy = rho0 g beta (T - T0) (Eqs. GoverneEq, ForceEq at u = 0).  The
    model is weakly compressible, so the interior matches to O(Ma^2)."""
    H, gb = 15, 1e-4
    p = W.problem(nx=2, ny=H + 1, bc=("periodic", "periodic", "dirichlet", "dirichlet"),
                  T_bc=(0.0, 0.0, 0.0, 1.0), gbeta=gb, nu=0.1, alpha_e=0.1, da_infinite=1, eps=0.5)
    o = oracle.Oracle(p)
    o.run(20000)
    m = o.moments()
    y = np.arange(H + 1.0)
    pe = gb * (y ** 2 / (2 * H) - y / 2)
    pn = m["p"][:, 0]
    d = (pn - pn[H // 2]) - (pe - pe[H // 2])
    assert np.abs(d[1:-1]).max() < 3e-3 * np.abs(pe - pe[H // 2]).max()
    assert np.abs(m["T"][:, 0] - y / H).max() < 1e-3
    assert np.abs(m["uy"]).max() < 1e-4 * gb * H * H / 0.1


def test_cavity_centro_symmetry():
    """Rotation by pi maps the cavity onto itself with T - T0 -> -(T - T0),
    u -> -u, p -> p.  The products T u and T p in g^eq (Eq. TeEDFEQ) keep this
    symmetry of the discrete model exactly only when T0 = 0, so the walls are
    set to +-1/2."""
    n = 20
    p = W.cavity(n, 1e4, 1e-2, 0.6, Th=0.5, Tc=-0.5, T_init=0.0)
    o = oracle.Oracle(p)
    o.run(1500)
    m = o.moments()
    rot = lambda a: a[::-1, ::-1]
    assert np.abs(m["T"] + rot(m["T"]) - (p["Th"] + p["Tc"])).max() < 1e-12
    assert np.abs(m["ux"] + rot(m["ux"])).max() < 1e-14
    assert np.abs(m["uy"] + rot(m["uy"])).max() < 1e-14
    assert np.abs(m["ux"]).max() > 1e-3
    # Nu on the hot and cold walls agree by symmetry
    assert o.nusselt("W")[0] == pytest.approx(o.nusselt("E")[0], rel=1e-12)
