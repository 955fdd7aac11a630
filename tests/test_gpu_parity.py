"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Both sides start from the same seeded inputs; the GPU never supplies an
oracle input.  Tolerances:
  * FP64 storage and arithmetic: max |a - b| / max |b| <= 1e-10 on u and T
    (per field), and the same bound on every population;
  * FP32: one step from a common state agrees to FP32 rounding (1e-6 relative
    to the population scale); multi-step runs agree to
    max |dT| <= 1e-4, ||du||_2 / ||u||_2 <= 1e-3, |dNu| / Nu <= 1e-4.
"""
import numpy as np
import pytest

import oracle
from paper_1505_02976_gb300 import lbm
from paper_1505_02976_gb300 import workloads as W

from oracle_states import sample_nodes, stored_state

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10


def _rel(a, b):
    d = np.abs(np.asarray(a) - np.asarray(b)).max()
    s = np.abs(np.asarray(b)).max()
    return d / s if s > 0 else d


def _pair(p, precision, fields=None, steps=0):
    T, ux, uy = fields if fields is not None else (None, None, None)
    o = oracle.Oracle(p, T=T, ux=ux, uy=uy)
    g = lbm.Lattice(p, precision)
    g.set_fields(T, ux, uy)
    if steps:
        o.run(steps)
        g.step(steps)
        g.sync()
    return o, g


def _check_fp64(o, g, tol=FP64_TOL):
    """Velocity components are compared relative to the largest speed, the
    pressure relative to max(|p|, |u|^2) (it is round-off noise when the
    flow is uniform), T relative to max |T|."""
    mo, mg = o.moments(), g.moments()
    umax = np.sqrt(mo["ux"] ** 2 + mo["uy"] ** 2).max()
    for k in ("ux", "uy"):
        err = np.abs(mg[k] - mo[k]).max() / umax
        assert err <= tol, (k, err)
    pscale = max(np.abs(mo["p"]).max(), umax ** 2)
    assert np.abs(mg["p"] - mo["p"]).max() <= tol * pscale
    assert _rel(mg["T"], mo["T"]) <= tol
    f, gg = g.get_state()
    assert _rel(f[1:], o.f[1:]) <= tol
    assert _rel(gg, o.g) <= tol
    assert np.all(np.isnan(f[0]))


def test_fp64_cavity_32_20000_steps():
    """32 x 32 porous cavity, Ra 1e3, Da 1e-2, eps 0.6, 20 000 steps."""
    p = W.cavity(32, 1e3, 1e-2, 0.6)
    o, g = _pair(p, "f64", steps=20_000)
    _check_fp64(o, g)
    for side in ("W", "E"):
        a, la = g.nusselt(side)
        b, lb = o.nusselt(side)
        assert abs(a - b) <= FP64_TOL * abs(b)
        assert _rel(la, lb) <= FP64_TOL


def test_fp64_poiseuille_channel():
    p = W.poiseuille(nx=8, ny=64)
    o, g = _pair(p, "f64", steps=3000)
    _check_fp64(o, g)


@pytest.mark.parametrize("shape", [(5, 4), (37, 29), (130, 7), (4, 33)])
def test_fp64_ragged_sizes_random_fields(shape):
    nx, ny = shape
    p = W.cavity(nx, 1e4, 1e-3, 0.5, ny=ny, Pr=0.7, sigma=1.3, tau_f=0.8, tau_T=1.3)
    fields = W.random_fields(p, seed=nx * 1000 + ny, amp_u=2e-3)
    o, g = _pair(p, "f64", fields=fields, steps=200)
    _check_fp64(o, g)


@pytest.mark.parametrize("bc", [
    ("adiabatic", "dirichlet", "dirichlet", "adiabatic"),
    ("dirichlet", "adiabatic", "adiabatic", "dirichlet"),
    ("adiabatic", "adiabatic", "adiabatic", "adiabatic"),
    ("periodic", "periodic", "adiabatic", "dirichlet"),
    ("dirichlet", "dirichlet", "periodic", "periodic"),
    ("periodic", "periodic", "periodic", "periodic"),
])
def test_fp64_boundary_combinations(bc):
    p = W.cavity(23, 1e5, 1e-2, 0.7, ny=19, bc=bc, T_bc=(1.0, 0.0, 0.2, 0.9),
                 u_bc=((0.0, 0.0), (0.0, 0.01), (0.02, 0.0), (-0.01, 0.0)), Q=2e-5)
    fields = W.random_fields(p, seed=11, amp_u=1e-3)
    o, g = _pair(p, "f64", fields=fields, steps=150)
    _check_fp64(o, g)


def test_fp64_one_step_sampled_at_scale():
    """One step of a 640 x 384 lattice from the oracle's state three steps
    after a random start: every sampled node (walls, corners and interior)
    against the oracle's node update."""
    p = W.cavity(640, 1e6, 1e-4, 0.4, ny=384)
    o, f0, g0 = stored_state(p, W.random_fields(p, seed=5, amp_u=5e-3), "f64", steps=3)
    g = lbm.Lattice(p, "f64")
    g.set_state(f0, g0)
    g.step(1)
    f1, g1 = g.get_state()
    xs, ys = sample_nodes(p["nx"], p["ny"], 300, seed=9)
    fo, go = o.update_nodes(xs, ys)
    fg = f1[:, ys, xs].T
    gg = g1[:, ys, xs].T
    assert _rel(fg[:, 1:], fo[:, 1:]) <= FP64_TOL
    assert _rel(gg, go) <= FP64_TOL


def test_fp32_cavity_against_oracle():
    """FP32 storage and arithmetic, 96 x 96 cavity at Ra 1e6, Da 1e-4,
    eps 0.4 (the FP32 benchmark's groups), 2000 steps."""
    p = W.cavity(96, 1e6, 1e-4, 0.4)
    o, g = _pair(p, "f32", steps=2000)
    mo, mg = o.moments(), g.moments()
    assert np.abs(mg["T"] - mo["T"]).max() <= 1e-4
    du = np.sqrt((mg["ux"] - mo["ux"]) ** 2 + (mg["uy"] - mo["uy"]) ** 2)
    un = np.sqrt(mo["ux"] ** 2 + mo["uy"] ** 2)
    assert np.linalg.norm(du) / np.linalg.norm(un) <= 1e-3
    a, _ = g.nusselt("W")
    b, _ = o.nusselt("W")
    assert abs(a - b) <= 1e-4 * abs(b)


def test_fp32_one_step_sampled_at_full_size():
    """The 2048 x 2048 FP32 workload in its benchmark launch configuration:
    one step from the oracle's state one step after a random start, rounded
    to FP32 storage; sampled nodes against the oracle's node update evaluated
    in FP64 on the same stored input."""
    p = W.cavity(2048, 1e6, 1e-4, 0.4)
    o, f0, g0 = stored_state(p, W.random_fields(p, seed=21, amp_u=2e-3, amp_T=0.3), "f32", steps=1)
    g = lbm.Lattice(p, "f32")
    g.set_state(f0, g0)
    g.step(1)
    f1, g1 = g.get_state()
    xs, ys = sample_nodes(p["nx"], p["ny"], 400, seed=10)
    fo, go = o.update_nodes(xs, ys)
    fg = f1[:, ys, xs].T
    gg = g1[:, ys, xs].T
    fscale = np.abs(fo[:, 1:]).max()
    gscale = np.abs(go).max()
    assert np.abs(fg[:, 1:] - fo[:, 1:]).max() <= 1e-6 * fscale
    assert np.abs(gg - go).max() <= 1e-6 * gscale


def test_residual_and_nusselt_reductions_fp64():
    p = W.cavity(48, 1e4, 1e-2, 0.6, ny=40)
    o, g = _pair(p, "f64", steps=500)
    m0 = o.moments()
    g.residual()  # snapshot at step 500
    o.run(100)
    g.step(100)
    m1 = o.moments()
    ru, rT = g.residual()
    eu, eT = oracle.residual(m1["ux"], m1["uy"], m1["T"], m0["ux"], m0["uy"], m0["T"])
    assert ru == pytest.approx(eu, rel=1e-9)
    assert rT == pytest.approx(eT, rel=1e-9)
    for side in ("W", "E", "S", "N"):
        a, la = g.nusselt(side)
        b, lb = o.nusselt(side)
        assert a == pytest.approx(b, rel=1e-10, abs=1e-12)
        assert np.allclose(la, lb, rtol=1e-10, atol=1e-12)


def test_state_round_trip_and_step_counter():
    p = W.cavity(33, 1e4, 1e-2, 0.6)
    g = lbm.Lattice(p, "f64")
    g.step(10)
    f, gg = g.get_state()
    g.step(7)
    assert g.steps == 17
    g.set_state(f, gg)
    f2, g2 = g.get_state()
    assert np.array_equal(f[1:], f2[1:]) and np.array_equal(gg, g2)


def test_nonfinite_input_is_reported():
    p = W.cavity(16, 1e4, 1e-2, 0.6)
    g = lbm.Lattice(p, "f32")
    T = np.full((16, 16), 0.5)
    T[5, 7] = np.nan
    g.set_fields(T)
    g.step(2)
    with pytest.raises(lbm.LbmError) as e:
        g.sync()
    assert e.value.status == -3
    with pytest.raises(lbm.LbmError):
        g.step(1)
    g.set_fields()
    g.step(2)
    g.sync()


def test_fp16_cavity_against_oracle():
    """FP16 storage (stochastic rounding), FP32 arithmetic: 64 x 64 cavity at
    the FP16 benchmark's groups (Ra 1e5, Da 1e-3, eps 0.6), 2000 steps.
    Bounds: max abs dT <= 3e-3, L2(du)/L2(u) <= 3e-3, abs dNu / Nu <= 3e-3."""
    p = W.cavity(64, 1e5, 1e-3, 0.6)
    o, g = _pair(p, "f16", steps=2000)
    mo, mg = o.moments(), g.moments()
    assert np.abs(mg["T"] - mo["T"]).max() <= 3e-3
    du = np.sqrt((mg["ux"] - mo["ux"]) ** 2 + (mg["uy"] - mo["uy"]) ** 2)
    un = np.sqrt(mo["ux"] ** 2 + mo["uy"] ** 2)
    assert np.linalg.norm(du) / np.linalg.norm(un) <= 3e-3
    a, _ = g.nusselt("W")
    b, _ = o.nusselt("W")
    assert abs(a - b) <= 3e-3 * abs(b)


def test_fp16_one_step_sampled_at_full_size():
    """The 8192 x 8192 FP16 workload: one step from a random state rounded to
    FP16 storage, sampled nodes against the oracle's node update on the same
    stored values.  The GPU output is rounded to FP16 stochastically, so each
    value may differ by one FP16 step of its magnitude (2^-10 relative) plus
    FP32 rounding."""
    n = 8192
    p = W.config_problem(W.CONFIG_FP16_CAVITY)
    o, f0, g0 = stored_state(p, W.random_fields(p, seed=31, amp_u=2e-3, amp_T=0.3), "f16")
    g = lbm.Lattice(p, "f16")
    g.set_state(f0, g0)
    del f0, g0
    g.step(1)
    f1, g1 = g.get_state()
    xs, ys = sample_nodes(n, n, 400, seed=12)
    fo, go = o.update_nodes(xs, ys)
    fg = f1[:, ys, xs].T
    gg = g1[:, ys, xs].T
    assert np.all(np.abs(fg[:, 1:] - fo[:, 1:]) <= 2.0 ** -10 * np.abs(fo[:, 1:]) + 1e-6 * np.abs(fo[:, 1:]).max())
    # thermal populations are stored as deviations from w_i sigma T0
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    dev = np.abs(go - w * 0.5)
    assert np.all(np.abs(gg - go) <= 2.0 ** -10 * dev + 1e-6 * dev.max())


def test_fp16_halves_the_population_storage():
    p = W.cavity(1024, 1e5, 1e-3, 0.6)
    n16 = lbm.lbm_workspace_size(p, "f16")
    n32 = lbm.lbm_workspace_size(p, "f32")
    assert n32 - n16 >= 2 * 17 * 1024 * 1024 * 2


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_energy_total_conserved_in_periodic_box(precision):
    """Periodic box, Q = 0: sum of g over the lattice is invariant (Sec. 3.2
    moments), and equals the oracle's total."""
    p = W.problem(nx=40, ny=36, bc=("periodic",) * 4, Ra=1e5, Da=1e-3, eps=0.5, sigma=1.3, tau_T=1.2)
    fields = W.random_fields(p, seed=17, amp_u=2e-3)
    o, g = _pair(p, precision, fields=fields)
    sf0, sg0 = g.totals()
    g.step(400)
    o.run(400)
    sf1, sg1 = g.totals()
    tol = 1e-13 if precision == "f64" else 1e-6
    assert sg1 == pytest.approx(sg0, rel=tol)
    assert sg1 == pytest.approx(o.totals()[1], rel=tol)
    tol_f = 1e-12 if precision == "f64" else 1e-5
    assert abs(sf1 - o.f[1:].sum()) <= tol_f * np.abs(o.f[1:]).sum()
