"""Pins of the internal-heat-source scalings (Sec. 4.3 and Sec. 4.4) and of
the stream function (Table 3's psi), against closed forms.

A slab between two isothermal walls, periodic along them, with no buoyancy,
conducts a uniform source Q into the walls: the steady profile is the
parabola T(y) = T_S + (T_N - T_S) y / H + Q y (H - y) / (2 alpha_e).
* Sec. 4.3 scaling (dT = Q H^2 / alpha_e, both walls at T_c): the peak of
  theta = (T - T_c) / dT is exactly 1/8.
* Sec. 4.4 scaling (Q = Ra_I alpha_e dT / (Ra H^2), T_S = T_c, T_N = T_h):
  theta(H/2) = 1/2 + Ra_I / (8 Ra).
"""
import numpy as np
import pytest
from scipy.integrate import cumulative_trapezoid

import oracle
from paper_1505_02976_gb300 import workloads as W

H = 16


def _slab(B, **kw):
    """B given, so alpha_e = sigma c_s^2 (tau_T - B - 1/2) (Eq. EQA&B)."""
    p = W.problem(nx=3, ny=H + 1, bc=("periodic", "periodic", "dirichlet", "dirichlet"),
                  L=float(H), gbeta=0.0, Pr=1.0, eps=0.7, Da=1e-2, forchheimer=0, B=B, **kw)
    o = oracle.Oracle(p)
    d = oracle.derived(p)
    o.run(int(8 * H * H / d["alpha_e"]))
    return d, o.moments()["T"][:, 1]


def _wall_shift(d, B):
    """At B != 0 the whole interior sits B Q / alpha_e below the parabola: a
    Dirichlet wall node takes grad T from x_f (Sec. 3.4), which on a profile
    of curvature -Q / alpha_e differs from the wall's own gradient by
    Q / alpha_e per lattice spacing, and the B grad T term of g^eq turns that
    into a temperature offset.  It is a boundary error of O(dx^2)."""
    return B * d["Q"] / d["alpha_e"]


@pytest.mark.parametrize("B", [0.0, 0.3])
def test_cooled_slab_peak_is_one_eighth_of_QL2_over_alpha(B):
    d, T = _slab(B, Th=10.0, Tc=0.0, T0=0.0, T_init=0.0, T_bc=(0.0, 0.0, 0.0, 0.0),
                 Ra=6.4e5, Ra_I=6.4e5, Q=float("nan"))
    assert d["Q"] * H * H / d["alpha_e"] == pytest.approx(10.0, rel=1e-14)
    y = np.arange(H + 1.0)
    exact = 10.0 * y * (H - y) / (2.0 * H * H)
    exact[1:-1] -= _wall_shift(d, B)
    assert np.abs(T - exact).max() < 1e-11
    if B == 0.0:
        assert T.max() / 10.0 == pytest.approx(0.125, abs=1e-12)


@pytest.mark.parametrize("ratio,B", [(0.1, 0.0), (4.0, 0.0), (4.0, 0.3)])
def test_heated_slab_with_source_follows_the_ra_i_over_ra_scaling(ratio, B):
    Ra = 1e4
    d, T = _slab(B, Th=1.0, Tc=0.0, T_bc=(0.0, 0.0, 0.0, 1.0), Ra=Ra, Ra_I=ratio * Ra,
                 Q=float("nan"))
    y = np.arange(H + 1.0) / H
    exact = y + 0.5 * ratio * y * (1.0 - y)
    exact[1:-1] -= _wall_shift(d, B)
    assert np.abs(T - exact).max() < 1e-11
    # interior second differences carry the source alone: -Q / alpha_e
    assert np.abs(np.diff(T[1:-1], 2) + ratio / H ** 2).max() < 1e-11


def test_stream_function_integrates_linear_profiles_exactly():
    ny, nx = 21, 6
    y = np.arange(ny, dtype=float)[:, None]
    a = np.linspace(-0.3, 0.4, nx)[None, :]
    ux = a + 0.05 * y * (1 + a)
    psi = oracle.stream_function(ux)
    assert np.abs(psi - (a * y + 0.025 * (1 + a) * y * y)).max() < 1e-13


def test_stream_function_is_the_cumulative_trapezoid_rule():
    rng = np.random.Generator(np.random.PCG64(5))
    ux = rng.standard_normal((37, 29))
    assert np.abs(oracle.stream_function(ux) - cumulative_trapezoid(ux, axis=0, initial=0.0)).max() < 1e-12


def test_stream_function_converges_at_second_order_and_recovers_uy():
    """psi_a = sin(pi x / L) sin(pi y / L)^2: u_x = d psi_a / dy,
    u_y = -d psi_a / dx; the integral has O(h^2) error, and the centred x
    difference of psi returns u_y to O(h^2) as well."""
    err, erry = [], []
    for n in (17, 33, 65):
        h = 1.0 / (n - 1)
        x = np.arange(n)[None, :] * h
        y = np.arange(n)[:, None] * h
        psi_a = np.sin(np.pi * x) * np.sin(np.pi * y) ** 2
        ux = np.sin(np.pi * x) * 2.0 * np.pi * np.sin(np.pi * y) * np.cos(np.pi * y) * np.ones_like(x)
        uy = -np.pi * np.cos(np.pi * x) * np.sin(np.pi * y) ** 2
        psi = h * oracle.stream_function(ux)  # the sum runs in units of the spacing
        err.append(np.abs(psi - psi_a).max())
        erry.append(np.abs(-(psi[:, 2:] - psi[:, :-2]) / (2 * h) - uy[:, 1:-1]).max())
    assert err[-1] < 1e-3 and erry[-1] < 5e-3
    for e in (err, erry):
        assert np.log2(e[1] / e[2]) > 1.95
