"""Pins of the oracle's complex-step derivatives (the same C source compiled
over complex numbers): they must equal central finite differences of the
real oracle, and the closed-form sensitivities of pure conduction.  These
derivatives are the reference for the GPU adjoint."""
import numpy as np
import pytest

import oracle
from paper_1505_02976_gb300 import workloads as W


def _nu(p, steps, eps, Th=None, Tc=None):
    q = dict(p)
    tb = list(q["T_bc"])
    if Th is not None:
        tb[0] = Th
    if Tc is not None:
        tb[1] = Tc
    q["T_bc"] = tuple(tb)
    return oracle.Oracle(q, eps_field=eps).run(steps).nusselt("W")[0]


def test_complex_step_equals_central_differences():
    p = W.cavity(14, 1e5, 1e-3, 0.6)
    eps = W.gaussian_random_field(14, corr=4.0, seed=3)
    cells = [(4, 6), (1, 1), (0, 5), (13, 13), (7, 0)]
    steps = 150
    g, dt = oracle.nusselt_gradient(p, steps, eps, cells)
    h = 1e-6
    for k, (x, y) in enumerate(cells):
        ep, em = eps.copy(), eps.copy()
        ep[y, x] += h
        em[y, x] -= h
        fd = (_nu(p, steps, ep) - _nu(p, steps, em)) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=1e-4, abs=1e-9)
    fd_h = (_nu(p, steps, eps, Th=1 + h) - _nu(p, steps, eps, Th=1 - h)) / (2 * h)
    fd_c = (_nu(p, steps, eps, Tc=h) - _nu(p, steps, eps, Tc=-h)) / (2 * h)
    assert dt["W"] == pytest.approx(fd_h, rel=1e-6)
    assert dt["E"] == pytest.approx(fd_c, rel=1e-4, abs=1e-9)


def test_pure_conduction_sensitivities():
    """No buoyancy: the steady state is exactly linear, Nu = (Th - Tc)/dT with
    dT held at its nominal value, so dNu/dTh = 1, dNu/dTc = -1 and the
    porosity does not matter."""
    p = W.cavity(10, 1e3, 1e-2, 0.6, gbeta=0.0, nu=0.1, alpha_e=0.1)
    eps = W.gaussian_random_field(10, corr=3.0, seed=2)
    g, dt = oracle.nusselt_gradient(p, 4000, eps, [(3, 4), (0, 0)])
    assert dt["W"] == pytest.approx(1.0, abs=1e-10)
    assert dt["E"] == pytest.approx(-1.0, abs=1e-10)
    assert np.all(np.abs(g) < 1e-12)
