"""The oracle on the paper's first test problem: mixed convection in a porous
channel with a moving, permeable top wall and injection through the bottom
(Sec. 4.1).  The steady solution is known in closed form (Eqs. EqVelocity,
EqTemper, EqSoluVelocity, EqSoluTemper); the paper reports second-order
accuracy for u, T and for the local-scheme gradients (Sec. 4.1 figures).
Refinement here is diffusive (nu fixed, v0 = u0 = Re nu / H)."""
import numpy as np
import pytest

import oracle

from channel_case import channel, relerr


def _steady(c, nu, H):
    o = oracle.Oracle(c["problem"], ay_profile=c["ay"])
    o.run(int(12 * H * H / (np.pi ** 2 * nu)))
    return o


@pytest.mark.parametrize("tau,nu", [(1.0, 1.0 / 6.0), (1.0, 0.1)])
def test_channel_matches_closed_form_and_converges(tau, nu):
    e = {}
    for H in (16, 32, 64):
        v0 = 5.0 * nu / H
        c = channel(H=H, u0=v0, v0=v0, tau=tau)
        o = _steady(c, nu, H)
        m = o.moments()
        g = o.gradients()
        e[H] = dict(u=relerr(c["ux"], m["ux"][:, 0]), T=relerr(c["T"], m["T"][:, 0]),
                    du=relerr(c["dux"][1:-1], g["Sxy"][1:-1, 0]),
                    dT=relerr(c["dT"][1:-1], g["dTdy"][1:-1, 0]),
                    uy=float(np.abs(m["uy"][:, 0] - v0).max() / v0))
    assert e[64]["u"] < 5e-3 and e[64]["T"] < 1e-3 and e[64]["du"] < 1e-2 and e[64]["dT"] < 1e-3
    assert e[64]["uy"] < 1e-3
    for k in ("u", "du"):
        assert np.log2(e[32][k] / e[64][k]) > 1.5, (k, e)
    if e[64]["T"] > 1e-6:  # at tau = 1, B = 0 the temperature error is near round-off
        assert np.log2(e[32]["T"] / e[64]["T"]) > 1.7, e
        assert np.log2(e[32]["dT"] / e[64]["dT"]) > 1.7, e
