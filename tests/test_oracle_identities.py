"""Pins of the oracle's one-cell building blocks against facts the paper and
the mathematics fix independently of the oracle's code:

* lattice isotropy of D2Q9 (Sec. 3.1);
* velocity moments of f^{e(0)}, f^{e(1)}, F_i (Appendix A, Eqs. EqZEqu,
  EqFEqu, FmomEq);
* the closed forms of s_0 and F_0 (Appendix A, end);
* velocity moments of g^{e(0)}, g^{e(1)}, P_i, Q_i (Sec. 3.2, Eq. MeOtEq);
* the implicit velocity relation behind the quadratic solve (Sec. 3.1).

Each identity is a sum over the nine directions computed here by brute force;
a dropped term, a wrong sign or a transposed index in any of the oracle's
per-direction formulas breaks at least one of them.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_1505_02976_gb300 import workloads as W

CS2 = 1.0 / 3.0
RNG = np.random.Generator(np.random.PCG64(7))


def _lat():
    cx, cy, w, varpi = oracle.lattice()
    c = np.stack([cx, cy], axis=1).astype(float)
    return c, w, varpi


def _cases(n=6):
    for _ in range(n):
        eps = RNG.uniform(0.2, 1.0)
        sigma = RNG.uniform(0.5, 2.0)
        tau_f = RNG.uniform(0.6, 2.0)
        tau_T = RNG.uniform(0.6, 2.0)
        A = RNG.uniform(-0.3, min(0.4, tau_f - 0.51))
        B = RNG.uniform(-0.3, min(0.4, tau_T - 0.51))
        Q = RNG.uniform(-1e-3, 1e-3)
        rho0 = RNG.uniform(0.8, 1.2)
        p = W.problem(eps=eps, sigma=sigma, A=A, B=B, tau_f=tau_f, tau_T=tau_T, Q=Q, rho0=rho0,
                      nu=0.05, alpha_e=0.05, gbeta=1e-3)
        u = RNG.uniform(-0.1, 0.1, 2)
        S = RNG.uniform(-1e-2, 1e-2, (2, 2))
        S = 0.5 * (S + S.T)
        F = RNG.uniform(-1e-3, 1e-3, 2)
        gradT = RNG.uniform(-1e-2, 1e-2, 2)
        T = RNG.uniform(0.0, 1.0)
        pr = RNG.uniform(-1e-2, 1e-2)
        yield dict(p=p, eps=eps, sigma=sigma, A=A, B=B, tau_f=tau_f, tau_T=tau_T, Q=Q, rho0=rho0,
                   u=u, S=S, F=F, gradT=gradT, T=T, pr=pr)


def _m0(v):
    return v.sum()


def _m1(v, c):
    return c.T @ v


def _m2(v, c):
    return np.einsum("i,ia,ib->ab", v, c, c)


def _m3(v, c):
    return np.einsum("i,ia,ib,ig->abg", v, c, c, c)


def _delta_u(u):
    d = np.eye(2)
    return (np.einsum("a,bg->abg", u, d) + np.einsum("b,ag->abg", u, d)
            + np.einsum("g,ab->abg", u, d))


def test_lattice_isotropy():
    c, w, varpi = _lat()
    # velocity set of Sec. 3.1: rest, four axis, four diagonal directions
    assert np.all(np.abs(c).sum(axis=1) == [0, 1, 1, 1, 1, 2, 2, 2, 2])
    assert sorted(map(tuple, c.astype(int))) == sorted(itertools.product((-1, 0, 1), repeat=2))
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    assert np.allclose(_m1(w, c), 0.0, atol=1e-16)
    assert np.allclose(_m2(w, c), CS2 * np.eye(2), atol=1e-16)
    assert np.allclose(_m3(w, c), 0.0, atol=1e-16)
    m4 = np.einsum("i,ia,ib,ig,id->abgd", w, c, c, c, c)
    d = np.eye(2)
    iso = (np.einsum("ab,gd->abgd", d, d) + np.einsum("ag,bd->abgd", d, d)
           + np.einsum("ad,bg->abgd", d, d))
    assert np.allclose(m4, CS2 ** 2 * iso, atol=1e-16)
    # varpi_0 = -sum_{i != 0} varpi_i, varpi_i = w_i otherwise (Eq. TeEDFEQ)
    assert varpi[0] == pytest.approx(-5.0 / 9.0, abs=1e-15)
    assert np.allclose(varpi[1:], w[1:])


@pytest.mark.parametrize("case", list(_cases()))
def test_flow_equilibrium_moments(case):
    c, w, _ = _lat()
    k = case
    fe0 = oracle.cell_eval(k["p"], "feq0", k["eps"], u=k["u"], pr=k["pr"], S=k["S"])
    fe = oracle.cell_eval(k["p"], "feq", k["eps"], u=k["u"], pr=k["pr"], S=k["S"])
    rho0, eps, u, pr = k["rho0"], k["eps"], k["u"], k["pr"]
    # Eq. (EqZEqu)
    assert _m0(fe0) == pytest.approx(rho0, abs=1e-14)
    assert np.allclose(_m1(fe0, c), rho0 * u, atol=1e-15)
    assert np.allclose(_m2(fe0, c), eps * pr * np.eye(2) + rho0 * np.outer(u, u) / eps, atol=1e-15)
    assert np.allclose(_m3(fe0, c), CS2 * rho0 * _delta_u(u), atol=1e-15)
    # Eq. (EqFEqu): f^{e(1)} = f^{eq} - f^{e(0)}
    fe1 = fe - fe0
    assert _m0(fe1) == pytest.approx(0.0, abs=1e-15)
    assert np.allclose(_m1(fe1, c), 0.0, atol=1e-16)
    assert np.allclose(_m2(fe1, c), CS2 * rho0 * k["A"] * k["S"], atol=1e-15)


@pytest.mark.parametrize("case", list(_cases()))
def test_forcing_moments_and_closed_forms(case):
    c, w, _ = _lat()
    k = case
    Fi = oracle.cell_eval(k["p"], "F", k["eps"], u=k["u"], F=k["F"])
    kf = 1.0 - 1.0 / (2.0 * k["tau_f"])
    u, F, eps, rho0 = k["u"], k["F"], k["eps"], k["rho0"]
    # Eq. (FmomEq)
    assert _m0(Fi) == pytest.approx(0.0, abs=1e-17)
    assert np.allclose(_m1(Fi, c), kf * rho0 * F, atol=1e-17)
    uF = np.outer(u, F)
    assert np.allclose(_m2(Fi, c), kf * rho0 * (uF + uF.T) / eps, atol=1e-17)
    # closed forms of F_0 and s_0 (Appendix A): F_0 = -w0 (1 - 1/2tau) u.F / (eps cs2),
    # s_0 = -w0 |u|^2 / (2 eps cs2)
    w0 = w[0]
    assert Fi[0] == pytest.approx(-w0 * kf * rho0 * (u @ F) / (eps * CS2), rel=1e-13, abs=1e-19)
    fe0 = oracle.cell_eval(k["p"], "feq0", eps, u=u, pr=0.0)
    s0 = (fe0[0] - rho0) / rho0
    assert s0 == pytest.approx(-w0 * (u @ u) / (2.0 * eps * CS2), rel=1e-12)


@pytest.mark.parametrize("case", list(_cases()))
def test_thermal_equilibrium_and_source_moments(case):
    c, w, _ = _lat()
    k = case
    T, u, pr, eps, sigma, rho0 = k["T"], k["u"], k["pr"], k["eps"], k["sigma"], k["rho0"]
    ge0 = oracle.cell_eval(k["p"], "geq0", eps, T=T, u=u, pr=pr, gradT=k["gradT"])
    ge = oracle.cell_eval(k["p"], "geq", eps, T=T, u=u, pr=pr, gradT=k["gradT"])
    # Eq. (MeOtEq), first line
    assert _m0(ge0) == pytest.approx(sigma * T, abs=1e-14)
    assert np.allclose(_m1(ge0, c), T * u, atol=1e-15)
    m2 = T * np.outer(u, u) / eps + CS2 * sigma * T * np.eye(2) + eps * pr * T / rho0 * np.eye(2)
    assert np.allclose(_m2(ge0, c), m2, atol=1e-15)
    assert np.allclose(_m3(ge0, c), CS2 * T * _delta_u(u), atol=1e-15)
    # second line: g^{e(1)}
    ge1 = ge - ge0
    assert _m0(ge1) == pytest.approx(0.0, abs=1e-16)
    assert np.allclose(_m1(ge1, c), sigma * CS2 * k["B"] * k["gradT"], atol=1e-16)
    assert np.allclose(_m2(ge1, c), 0.0, atol=1e-16)
    # third line: P_i
    kT = 1.0 - 1.0 / (2.0 * k["tau_T"])
    Pi = oracle.cell_eval(k["p"], "P", eps, T=T, u=u, pr=pr, F=k["F"], gradT=k["gradT"])
    gT = k["gradT"]
    m1 = kT * (T * k["F"] + eps * pr * gT / rho0 + (1.0 / eps - 1.0 / sigma) * u * (u @ gT))
    assert _m0(Pi) == pytest.approx(0.0, abs=1e-17)
    assert np.allclose(_m1(Pi, c), m1, atol=1e-17)
    assert np.allclose(_m2(Pi, c), 0.0, atol=1e-17)
    # fourth line: Q_i
    Qi = oracle.cell_eval(k["p"], "Q", eps, u=u)
    assert _m0(Qi) == pytest.approx(kT * k["Q"], abs=1e-18)
    assert np.allclose(_m1(Qi, c), kT * u * k["Q"] / sigma, atol=1e-18)


@pytest.mark.parametrize("seed", range(5))
def test_quadratic_velocity_solve(seed):
    """u = v / (c0 + sqrt(c0^2 + c1 |v|)) is the root of u (2 c0 + c1 |u|) = v
    (Sec. 3.1), equivalently u = m/rho0 + F(u)/2 with F of Eq. (ForceEq)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    eps = rng.uniform(0.3, 0.9)
    p = W.problem(eps=eps, Da=10 ** rng.uniform(-6, -2), nx=64, ny=64, Ra=1e5)
    d = oracle.derived(p)
    v = rng.uniform(-0.05, 0.05, 2)
    u, c0, c1 = oracle.cell_velocity(p, eps, v)
    assert c0 == pytest.approx(0.5 * (1.0 + 0.5 * eps * d["nu"] / d["K"]), rel=1e-14)
    assert c1 == pytest.approx(0.5 * eps * d["Feps"] / np.sqrt(d["K"]), rel=1e-14)
    lhs = u * (2.0 * c0 + c1 * np.linalg.norm(u))
    assert np.allclose(lhs, v, rtol=1e-13, atol=1e-18)
    # no Forchheimer term: u = v / (2 c0)
    p0 = dict(p, forchheimer=0)
    u0, c00, c10 = oracle.cell_velocity(p0, eps, v)
    assert c10 == 0.0
    assert np.allclose(u0, v / (2.0 * c00), rtol=1e-15)


def test_parameter_derivation_matches_eq_A_B():
    """A and B from Eq. (EQA&B) with Ma = 0.1, and the admissibility checks
    A < tau_f - 1/2, B < tau_T - 1/2."""
    for n, Ra, Pr in ((32, 1e3, 1.0), (256, 1e6, 1.0), (100, 1e4, 0.71)):
        p = W.cavity(n, Ra, 1e-2, 0.6, Pr=Pr)
        d = oracle.derived(p)
        L = n - 1
        A = 1.0 - 0.5 - 0.1 * L * np.sqrt(3.0 * Pr / Ra)
        B = 1.0 - 0.5 - 0.1 * L * np.sqrt(3.0 / (Pr * Ra))
        assert d["A"] == pytest.approx(A, rel=1e-13)
        assert d["B"] == pytest.approx(B, rel=1e-13)
        # Ra and Pr recomputed from the derived lattice constants (Sec. 2)
        assert d["gbeta"] * d["dT"] * L ** 3 / (d["nu"] * d["alpha_e"]) == pytest.approx(Ra, rel=1e-12)
        assert d["nu"] / d["alpha_e"] == pytest.approx(Pr, rel=1e-13)
        assert d["K"] == pytest.approx(1e-2 * L * L, rel=1e-15)
        assert d["Feps"] == pytest.approx(1.75 / np.sqrt(150 * 0.6 ** 3), rel=1e-15)
    with pytest.raises(ValueError):
        oracle.derived(W.problem(A=0.5))
    with pytest.raises(ValueError):
        oracle.derived(W.problem(eps=1.5))
