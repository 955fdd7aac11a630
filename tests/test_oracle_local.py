"""Pins of the oracle's local gradient schemes (Sec. 3.3).

Populations are built with prescribed macroscopic moments: the equilibrium
moments of Appendix A / Sec. 3.2 plus a non-equilibrium part whose second
(flow) or first (thermal) moment encodes a chosen shear rate S or temperature
gradient through the relations the schemes invert (Eqs. Shear, TfFintemEq).
The oracle must return exactly the prescribed p, u, T, S and grad T.  The
eps = sigma shortcut of Sec. 3.3 is checked against the general 2x2 solve.
"""
import numpy as np
import pytest

import oracle
from paper_1505_02976_gb300 import workloads as W

CS2 = 1.0 / 3.0


def _lat():
    cx, cy, w, _ = oracle.lattice()
    return np.stack([cx, cy], axis=1).astype(float), w


def _solve_with_null(rows, rhs, rng, free0=True):
    """Minimum-norm solution of rows @ x = rhs plus a random null-space part."""
    x, *_ = np.linalg.lstsq(rows, rhs, rcond=None)
    _, s, vt = np.linalg.svd(rows)
    null = vt[np.sum(s > 1e-12):]
    x = x + null.T @ rng.uniform(-1e-3, 1e-3, null.shape[0])
    assert np.allclose(rows @ x, rhs, atol=1e-15)
    return x


def _problem(rng, eps, sigma):
    tau_f = rng.uniform(0.7, 1.5)
    tau_T = rng.uniform(0.7, 1.5)
    return W.problem(eps=eps, sigma=sigma, tau_f=tau_f, tau_T=tau_T,
                     A=rng.uniform(-0.2, tau_f - 0.55), B=rng.uniform(-0.2, tau_T - 0.55),
                     da_infinite=1, gbeta=0.0, nu=0.05, alpha_e=0.05,
                     ax=rng.uniform(-1e-4, 1e-4), ay=rng.uniform(-1e-4, 1e-4),
                     Q=rng.uniform(-1e-4, 1e-4), rho0=1.0)


def _build(pb, rng, eps, sigma):
    c, w = _lat()
    rho0, tau_f, tau_T = pb["rho0"], pb["tau_f"], pb["tau_T"]
    A, B, Q = pb["A"], pb["B"], pb["Q"]
    u = rng.uniform(-0.08, 0.08, 2)
    pr = rng.uniform(-1e-2, 1e-2)
    T = rng.uniform(0.2, 0.8)
    S = rng.uniform(-1e-2, 1e-2, (2, 2)); S = 0.5 * (S + S.T)
    gT = rng.uniform(-1e-2, 1e-2, 2)
    a = np.array([pb["ax"], pb["ay"]])
    F = eps * a  # K infinite and g beta = 0: F = eps G = eps a (Eq. ForceEq)
    kf = 1.0 - 1.0 / (2.0 * tau_f)
    w0 = w[0]
    F0 = -w0 * kf * rho0 * (u @ F) / (eps * CS2)      # closed form, Appendix A
    s0 = -w0 * (u @ u) / (2.0 * eps * CS2)           # closed form, Appendix A
    # --- flow populations: constraints on sum_{i!=0} f, sum c f, sum c c f
    rows = [np.r_[0.0, np.ones(8)], c[:, 0], c[:, 1], c[:, 0] ** 2, c[:, 0] * c[:, 1], c[:, 1] ** 2]
    Pi = (CS2 * rho0 * (A - tau_f) * S - 0.5 * rho0 * (np.outer(u, F) + np.outer(F, u)) / eps
          + eps * pr * np.eye(2) + rho0 * np.outer(u, u) / eps)
    rhs = [eps * (1.0 - w0) * pr / CS2 - tau_f * F0 - rho0 * s0,
           *(rho0 * (u - 0.5 * F)), Pi[0, 0], Pi[0, 1], Pi[1, 1]]
    fs = _solve_with_null(np.array(rows), np.array(rhs), rng)
    # --- thermal populations: sum g and sum c g
    M = ((-eps * pr / (2.0 * rho0) + CS2 * sigma * (B - tau_T)) * np.eye(2)
         - 0.5 * (1.0 / eps - 1.0 / sigma) * np.outer(u, u))
    N = M @ gT
    n1 = T * u + N - 0.5 * (T * F + u * Q / sigma)
    rows = [np.ones(9), c[:, 0], c[:, 1]]
    rhs = [sigma * T - 0.5 * Q, *n1]
    gs = _solve_with_null(np.array(rows), np.array(rhs), rng)
    return fs, gs, dict(u=u, p=pr, T=T, S=S, gradT=gT, F=F, N=N)


@pytest.mark.parametrize("seed", range(8))
def test_local_schemes_round_trip(seed):
    rng = np.random.Generator(np.random.PCG64(100 + seed))
    eps = rng.uniform(0.3, 1.0)
    sigma = rng.uniform(0.6, 1.8)
    pb = _problem(rng, eps, sigma)
    fs, gs, ref = _build(pb, rng, eps, sigma)
    m = oracle.cell_moments(pb, eps, fs, gs)
    assert m["T"] == pytest.approx(ref["T"], abs=1e-14)
    assert np.allclose(m["u"], ref["u"], atol=1e-15, rtol=1e-12)
    assert np.allclose(m["F"], ref["F"], atol=1e-18, rtol=1e-12)
    assert m["p"] == pytest.approx(ref["p"], abs=1e-14)
    assert np.allclose(m["S"], ref["S"], atol=1e-13)
    assert np.allclose(m["gradT"], ref["gradT"], atol=1e-13)


@pytest.mark.parametrize("seed", range(4))
def test_gradT_shortcut_when_eps_equals_sigma(seed):
    """With eps = sigma the uu term of M vanishes and grad T follows from N
    alone (Sec. 3.3, last equation)."""
    rng = np.random.Generator(np.random.PCG64(200 + seed))
    eps = rng.uniform(0.3, 1.0)
    pb = _problem(rng, eps, eps)
    fs, gs, ref = _build(pb, rng, eps, eps)
    m = oracle.cell_moments(pb, eps, fs, gs)
    den = CS2 * eps * (pb["B"] - pb["tau_T"]) - eps * m["p"] / (2.0 * pb["rho0"])
    assert np.allclose(m["gradT"], ref["N"] / den, atol=1e-13)
