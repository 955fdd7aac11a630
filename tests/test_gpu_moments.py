"""The moment state (tau_f = tau_T = 1, nine moments stored per node; each
step rebuilds the post-collision populations on chip) against the oracle.

At unit relaxation times the post-collision populations are f^eq + F_i and
g^eq + P_i + Q_i of the state the step computes (Eqs. LBEeq, TEqColli), so
this storage must reproduce the oracle exactly as population storage does:
FP64 within 1e-10 on u, p, T and on the post-collision populations
(lbm_get_state), FP32 within the population kernel's bounds."""
import numpy as np
import pytest

import oracle
from paper_1505_02976_gb300 import lbm
from paper_1505_02976_gb300 import workloads as W

from channel_case import channel
from oracle_states import sample_nodes

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _rel(a, b):
    d = np.abs(np.asarray(a) - np.asarray(b)).max()
    s = np.abs(np.asarray(b)).max()
    return d / s if s > 0 else d


def _pair(p, precision="f64", fields=(None, None, None), steps=0, eps_field=None, ay=None):
    T, ux, uy = fields
    o = oracle.Oracle(p, T=T, ux=ux, uy=uy, eps_field=eps_field, ay_profile=ay)
    g = lbm.Lattice(p, precision, state="moments")
    g.set_fields(T, ux, uy, eps_field=eps_field)
    if ay is not None:
        g.set_force_profile(ay)
    if steps:
        o.run(steps)
        g.step(steps)
        g.sync()
    return o, g


def _check(o, g, tol=TOL):
    mo, mg = o.moments(), g.moments()
    umax = np.sqrt(mo["ux"] ** 2 + mo["uy"] ** 2).max()
    for k in ("ux", "uy"):
        assert np.abs(mg[k] - mo[k]).max() <= tol * umax, k
    pscale = max(np.abs(mo["p"]).max(), umax ** 2)
    assert np.abs(mg["p"] - mo["p"]).max() <= tol * pscale
    assert _rel(mg["T"], mo["T"]) <= tol
    f, gg = g.get_state()
    assert _rel(f[1:], o.f[1:]) <= tol
    assert _rel(gg, o.g) <= tol


def test_cavity_32_20000_steps():
    p = W.cavity(32, 1e3, 1e-2, 0.6)
    o, g = _pair(p, steps=20_000)
    _check(o, g)
    for side in ("W", "E"):
        a, la = g.nusselt(side)
        b, lb = o.nusselt(side)
        assert abs(a - b) <= TOL * abs(b)
        assert _rel(la, lb) <= TOL


def test_first_steps_from_set_fields():
    """Step 1 starts from the equilibria alone (no force or source terms),
    later steps from full post-collision states."""
    p = W.cavity(29, 1e5, 1e-3, 0.5, ny=21, Q=3e-5)
    fields = W.random_fields(p, seed=4, amp_u=3e-3)
    o, g = _pair(p, fields=fields)
    _check(o, g)  # the expansion of the initial state
    for n in (1, 1, 3):
        o.run(n)
        g.step(n)
        _check(o, g)


def test_poiseuille_channel():
    p = W.poiseuille(nx=8, ny=64)
    o, g = _pair(p, steps=3000)
    _check(o, g)


@pytest.mark.parametrize("shape", [(5, 4), (37, 29), (130, 7), (4, 33), (300, 11), (9, 200), (260, 130)])
def test_ragged_sizes_bands_and_segments(shape):
    """Several 126-column bands (300, 260 wide) and many 3-row segments
    (200 tall with one band)."""
    nx, ny = shape
    p = W.cavity(nx, 1e4, 1e-3, 0.5, ny=ny, Pr=0.7, sigma=1.3)
    fields = W.random_fields(p, seed=nx * 1000 + ny, amp_u=2e-3)
    o, g = _pair(p, fields=fields, steps=60)
    _check(o, g)


@pytest.mark.parametrize("bc", [
    ("adiabatic", "dirichlet", "dirichlet", "adiabatic"),
    ("dirichlet", "adiabatic", "adiabatic", "dirichlet"),
    ("adiabatic", "adiabatic", "adiabatic", "adiabatic"),
    ("periodic", "periodic", "adiabatic", "dirichlet"),
    ("dirichlet", "dirichlet", "periodic", "periodic"),
    ("periodic", "periodic", "periodic", "periodic"),
])
def test_boundary_combinations(bc):
    p = W.cavity(150, 1e5, 1e-2, 0.7, ny=19, bc=bc, T_bc=(1.0, 0.0, 0.2, 0.9),
                 u_bc=((0.0, 0.0), (0.0, 0.01), (0.02, 0.0), (-0.01, 0.0)), Q=2e-5)
    fields = W.random_fields(p, seed=11, amp_u=1e-3)
    o, g = _pair(p, fields=fields, steps=150)
    _check(o, g)


def test_porosity_field():
    p = W.cavity(140, 1e5, 1e-3, 0.6, ny=30)
    eps = W.gaussian_random_field(140, corr=6.0, seed=2)[:30]
    o, g = _pair(p, fields=W.random_fields(p, seed=8, amp_u=2e-3), steps=200, eps_field=eps)
    _check(o, g)


def test_channel_with_force_profile():
    c = channel(H=32, u0=0.01, v0=0.01, nx=140)
    o, g = _pair(c["problem"], steps=2000, ay=c["ay"])
    _check(o, g)


def test_heat_generating_cavity():
    p = W.heat_generating_cavity(26, 1e-2, Ra_I=2e4)
    o, g = _pair(p, steps=1500)
    _check(o, g)
    psi, _ = g.stream_function()
    ref = oracle.stream_function(o.moments()["ux"])
    assert np.abs(psi - ref).max() <= TOL * np.abs(ref).max()


def test_640_by_384_two_steps():
    p = W.cavity(640, 1e6, 1e-4, 0.4, ny=384)
    o, g = _pair(p, fields=W.random_fields(p, seed=5, amp_u=5e-3), steps=2)
    _check(o, g)


def test_fp32_cavity_against_oracle():
    """FP32 moments, 96 x 96 cavity at the FP32 benchmark's groups, 2000
    steps: the population kernel's multi-step bounds."""
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


def test_fp32_two_steps_sampled_at_full_size():
    """The 2048 x 2048 FP32 benchmark workload in its launch configuration:
    two steps from a random state; sampled post-collision populations
    against the oracle's second step (its first step taken on the whole
    lattice)."""
    p = W.cavity(2048, 1e6, 1e-4, 0.4)
    fields = W.random_fields(p, seed=21, amp_u=2e-3, amp_T=0.3)
    o = oracle.Oracle(p, *fields).run(1)
    xs, ys = sample_nodes(2048, 2048, 400, seed=10)
    fo, go = o.update_nodes(xs, ys)
    g = lbm.Lattice(p, "f32", state="moments")
    g.set_fields(*fields)
    g.step(2)
    f2, g2 = g.get_state()
    assert np.abs(f2[1:, ys, xs].T - fo[:, 1:]).max() <= 2e-6 * np.abs(fo[:, 1:]).max()
    assert np.abs(g2[:, ys, xs].T - go).max() <= 2e-6 * np.abs(go).max()


def test_moment_and_population_storage_agree():
    """Both storages on the GPU, FP64: same moments, Nusselt numbers,
    residuals, totals and stream function to round-off."""
    p = W.cavity(150, 1e5, 1e-2, 0.6, ny=90)
    fields = W.random_fields(p, seed=6, amp_u=1e-3)
    a = lbm.Lattice(p, "f64")
    b = lbm.Lattice(p, "f64", state="moments")
    for g in (a, b):
        g.set_fields(*fields)
        g.step(300)
        g.residual()
        g.step(100)
    ma, mb = a.moments(), b.moments()
    for k in ("ux", "uy", "T"):
        assert _rel(mb[k], ma[k]) <= 1e-12
    assert b.nusselt("W")[0] == pytest.approx(a.nusselt("W")[0], rel=1e-12)
    ra, rb = a.residual(), b.residual()
    assert rb == pytest.approx(ra, rel=1e-9)
    assert b.totals() == pytest.approx(a.totals(), rel=1e-12)
    assert _rel(b.stream_function()[0], a.stream_function()[0]) <= 1e-12


def test_checkpoint_resumes_bit_for_bit(tmp_path):
    p = W.cavity(64, 1e5, 1e-2, 0.6, ny=40)
    for warm in (0, 25):  # right after set_fields (no source terms yet), and later
        g = lbm.Lattice(p, "f32", state="moments")
        g.set_fields(*W.random_fields(p, seed=3, amp_u=1e-3))
        g.step(warm)
        path = str(tmp_path / f"m{warm}.ckpt")
        g.save(path)
        g.step(40)
        ref = g.get_state()
        h = lbm.Lattice(p, "f32", state="moments")
        h.load_checkpoint(path)
        assert h.steps == warm
        h.step(40)
        got = h.get_state()
        assert np.array_equal(ref[0][1:], got[0][1:]) and np.array_equal(ref[1], got[1])
        pop = lbm.Lattice(p, "f32")
        with pytest.raises(lbm.LbmError):
            pop.load_checkpoint(path)  # a moment-state file is refused by a population handle


def test_refusals():
    p = W.cavity(16, 1e4, 1e-2, 0.6)
    g = lbm.Lattice(p, "f64", state="moments")
    f, gg = g.get_state()
    with pytest.raises(lbm.LbmError) as e:
        g.set_state(f, gg)
    assert e.value.status == -1
    with pytest.raises(lbm.LbmError) as e:
        g.adjoint(10)
    assert e.value.status == -1
    for bad in (dict(p, tau_f=0.8), dict(p, tau_T=1.2)):
        with pytest.raises(lbm.LbmError):
            lbm.Lattice(bad, "f64", state="moments")
    with pytest.raises(lbm.LbmError):
        lbm.Lattice(p, "f16", state="moments")
