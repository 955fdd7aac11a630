"""Numerical stability of the modified model against the standard LBGK form
(Sec. 4.1: at low viscosity the standard model, A = B = 0 with the
relaxation times carrying nu and alpha_e, becomes unstable while the
modified model at tau = 1 stays stable).  Divergence is caught by the
step's non-finite watchdog (LBM_ERR_NONFINITE on the next synchronising
call), so nothing on the GPU faults.

Both models start from the same seeded, perturbed state.  The unperturbed
channel is uniform in x, and the standard form then stays finite at these
viscosities: the instability needs a perturbation to grow from."""
import numpy as np
import pytest

from paper_1505_02976_gb300 import lbm, workloads as W

from channel_case import channel, relerr

pytestmark = pytest.mark.gpu

NONFINITE = -3


def _steps_to_divergence(g, steps, chunk):
    for k in range(steps // chunk):
        g.step(chunk)
        try:
            g.sync()
        except lbm.LbmError as e:
            assert e.status == NONFINITE
            return (k + 1) * chunk
    return None


def _channel_lattice(c, H, nx, v0):
    g = lbm.Lattice(c["problem"], "f64")
    rng = np.random.Generator(np.random.PCG64(7))
    shape = (H + 1, nx)
    g.set_fields(T=0.5 + 1e-2 * rng.uniform(-1, 1, shape), ux=v0 * rng.uniform(-1, 1, shape),
                 uy=v0 + v0 * rng.uniform(-1, 1, shape))
    g.set_force_profile(c["ay"])
    return g


@pytest.mark.parametrize("nu", [3e-4, 3e-5])
def test_channel_standard_lbgk_diverges_where_the_modified_model_is_stable(nu):
    """Sec. 4.1's low-viscosity cases: lattice nu = 3e-4 (tau_f = 0.5009) and
    3e-5 (tau_f = 0.50009), Re = 5, Ra = 100, Pr = 1, eps = 0.6, Da = 0.01,
    32 x 32 nodes across the channel."""
    H = nx = 32
    v0 = 5.0 * nu / H
    std = channel(H=H, u0=v0, v0=v0, standard=True, nx=nx)
    mod = channel(H=H, u0=v0, v0=v0, tau=1.0, nx=nx)
    assert std["problem"]["tau_f"] == pytest.approx(0.5 + 3.0 * nu)
    assert _steps_to_divergence(_channel_lattice(std, H, nx, v0), 20_000, 1000) is not None
    g = _channel_lattice(mod, H, nx, v0)
    assert _steps_to_divergence(g, 200_000, 20_000) is None
    m = g.moments()
    assert np.all(np.isfinite(m["ux"])) and np.all(np.isfinite(m["T"]))
    if nu == 3e-4:  # developed: the x-mean profile is within 4 % of the closed form
        assert relerr(mod["ux"], m["ux"].mean(axis=1)) < 0.04


def test_cavity_standard_lbgk_diverges_at_low_viscosity():
    """The porous cavity (Da 1e-2, eps 0.6, Pr 1, Ma 0.1) on 64 x 64 nodes:
    at Ra 1e8 (lattice nu 3.6e-4) both forms stay finite and agree on Nu
    within 1.5 %; at Ra 1e10 (nu 3.6e-5, tau_f = 0.50011) the standard form
    diverges and the modified one does not."""
    def pair(Ra):
        base = W.cavity(64, Ra, 1e-2, 0.6)
        d = lbm.lbm_derived(base)
        std = dict(base, tau_f=0.5 + 3 * d["nu"], tau_T=0.5 + 3 * d["alpha_e"], A=0.0, B=0.0)
        return lbm.Lattice(std, "f64"), lbm.Lattice(base, "f64")
    s, m = pair(1e8)
    assert _steps_to_divergence(s, 300_000, 50_000) is None
    assert _steps_to_divergence(m, 300_000, 50_000) is None
    assert s.nusselt("W")[0] == pytest.approx(m.nusselt("W")[0], rel=0.015)
    s, m = pair(1e10)
    assert _steps_to_divergence(s, 60_000, 2_000) is not None
    assert _steps_to_divergence(m, 100_000, 20_000) is None
