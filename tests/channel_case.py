"""The mixed-convection porous channel of Sec. 4.1: problem, driving force
profile and the closed-form steady solution (Eqs. EqVelocity, EqTemper).

Channel of height H (ny = H + 1 nodes, walls at y = 0 and y = H), periodic
in x; the top wall (T_h) moves at u0 and both walls let a uniform normal flow
v0 through (injection at the bottom, withdrawal at the top); the bottom wall
is at T_c.  Lattice units: nu = H v0 / Re, alpha_e = nu / Pr, K = Da H^2,
g beta = Ra nu alpha_e / (dT H^3); F_eps = 0 (the closed form neglects the
Forchheimer drag).  The external force a_y(y) = (nu/K) v0 - g beta (T_a(y) - T0)
cancels the Darcy drag on v0 and the buoyancy of the exact temperature
profile (Sec. 4.1, definition of a_y), so u_y = v0 everywhere.  The paper's
temperature profile is written from the bottom wall's temperature, which is
how T_a is read here; T0 = (T_h + T_c)/2 stays the buoyancy reference, which
shifts a_y by a constant only.
"""
import math

import numpy as np

from paper_1505_02976_gb300 import workloads as W


def channel(H=32, Re=5.0, Ra=100.0, Pr=1.0, eps=0.6, Da=0.01, u0=0.01, v0=0.01, tau=1.0, nx=3,
            standard=False, Th=1.0, Tc=0.0):
    nu = H * v0 / Re
    alpha = nu / Pr
    K = Da * H * H
    dT = Th - Tc
    gbeta = Ra * nu * alpha / (dT * H ** 3)
    cs2 = 1.0 / 3.0
    if standard:  # standard LBGK: A = B = 0, relaxation times carry the transport coefficients
        tau_f = 0.5 + nu / cs2
        tau_T = 0.5 + alpha / cs2
        A = B = 0.0
    else:
        tau_f = tau_T = tau
        A = tau - 0.5 - nu / cs2
        B = tau - 0.5 - alpha / cs2
    p = W.problem(nx=nx, ny=H + 1, bc=("periodic", "periodic", "dirichlet", "dirichlet"),
                  eps=eps, Da=Da, L=float(H), nu=nu, alpha_e=alpha, gbeta=gbeta, A=A, B=B,
                  tau_f=tau_f, tau_T=tau_T, forchheimer=0, Th=Th, Tc=Tc, T_init=0.5 * (Th + Tc),
                  T_bc=(0.0, 0.0, Tc, Th), u_bc=((0.0, 0.0), (0.0, 0.0), (0.0, v0), (u0, v0)))
    y = np.arange(H + 1.0)
    T0 = 0.5 * (Th + Tc)
    Ta = Tc + dT * (np.exp(Pr * Re * y / H) - 1.0) / math.expm1(Pr * Re)
    ay = nu / K * v0 - gbeta * (Ta - T0)
    z1 = Re / (2.0 * eps)
    z2 = math.sqrt(Re * Re + 4.0 * eps ** 3 / Da) / (2.0 * eps)
    ux = u0 * np.exp(z1 * (y / H - 1.0)) * np.sinh(z2 * y / H) / math.sinh(z2)
    dux = (u0 / math.sinh(z2) * np.exp(z1 * (y / H - 1.0))
           * (z1 / H * np.sinh(z2 * y / H) + z2 / H * np.cosh(z2 * y / H)))
    dTa = dT * Pr * Re / H * np.exp(Pr * Re * y / H) / math.expm1(Pr * Re)
    return dict(problem=p, ay=ay, ux=ux, uy=np.full_like(y, v0), T=Ta, dux=dux, dT=dTa, nu=nu)


def relerr(a, n):
    """Relative global error of Sec. 4: sum |a - n| / sum |a|."""
    return float(np.abs(a - n).sum() / np.abs(a).sum())
