"""The FP32 step with TMA-staged rows (lattices walled on all four sides).

A single FP32 lattice walled on every side runs the staged kernel; a batch
runs the same per-node code with plain global loads.  The two must agree
bit for bit on lattices that span several 128-column bands and row segments
with ragged edges at tau = 1; away from tau = 1 (with sources) and with a
porosity field the staged kernel is checked against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_1505_02976_gb300 import lbm
from paper_1505_02976_gb300 import workloads as W

from oracle_states import stored_state

pytestmark = pytest.mark.gpu


def _bitwise_against_batch(p, steps, seed):
    T, ux, uy = W.random_fields(p, seed=seed, amp_u=2e-3, amp_T=0.3)
    g = lbm.Lattice(p, "f32")
    g.set_fields(T, ux, uy)
    g.step(steps)
    g.sync()
    b = lbm.Batch([p], "f32")
    b.set_fields(0, T, ux, uy)
    b.step(steps, "fused")
    b.sync()
    mg, mb = g.moments(), b.moments(0)
    for k in ("ux", "uy", "T", "p"):
        assert np.array_equal(mg[k], mb[k]), k
    assert np.all(np.isfinite(mg["T"]))
    b.close()


@pytest.mark.parametrize("nx,ny", [(300, 250), (129, 517), (4, 4), (131, 5), (517, 9)])
def test_staged_step_matches_global_loads(nx, ny):
    """Several bands and segments, ragged last band and segment, and the
    smallest lattices the staged kernel takes (4 rows, one partial band)."""
    _bitwise_against_batch(W.cavity(nx, 1e5, 1e-3, 0.5, ny=ny), 60, seed=nx + ny)


def test_staged_step_off_tau_one_with_sources():
    """tau_f, tau_T != 1 (the general collision) with an internal heat
    source, a body force and Dirichlet walls on all four sides: one step from
    an oracle-made FP32 state against the oracle on every node, at FP32
    rounding.  (The general collision's products may contract into fused
    multiply-adds differently in the two kernels, so this case is not
    compared bit for bit.)"""
    p = W.cavity(260, 1e5, 1e-3, 0.45, ny=140, tau_f=0.8, tau_T=1.15, Q=1e-4, ax=1e-7,
                 bc=("dirichlet",) * 4, T_bc=(1.0, 0.0, 0.7, 0.2))
    o, f0, g0 = stored_state(p, W.random_fields(p, seed=3, amp_u=2e-3, amp_T=0.3), "f32", steps=1)
    g = lbm.Lattice(p, "f32")
    g.set_state(f0, g0)
    g.step(1)
    f1, g1 = g.get_state()
    o.run(1)
    assert np.abs(f1[1:] - o.f[1:]).max() <= 1e-6 * np.abs(o.f[1:]).max()
    assert np.abs(g1 - o.g).max() <= 1e-6 * np.abs(o.g).max()


def test_staged_step_porosity_field_against_oracle():
    """Porosity field on a 160 x 141 cavity (two bands, ragged), 300 FP32
    steps against the FP64 oracle at the FP32 multi-step tolerances."""
    p = W.cavity(160, 1e5, 1e-3, 0.5, ny=141)
    eps = W.gaussian_random_field(160, corr=8.0, seed=5)[:141, :]
    T, ux, uy = W.random_fields(p, seed=12, amp_u=1e-3, amp_T=0.2)
    o = oracle.Oracle(p, T=T, ux=ux, uy=uy, eps_field=eps)
    o.run(300)
    g = lbm.Lattice(p, "f32")
    g.set_fields(T, ux, uy, eps_field=eps)
    g.step(300)
    g.sync()
    mo, mg = o.moments(), g.moments()
    assert np.abs(mg["T"] - mo["T"]).max() <= 1e-4
    du = np.sqrt((mg["ux"] - mo["ux"]) ** 2 + (mg["uy"] - mo["uy"]) ** 2)
    un = np.sqrt(mo["ux"] ** 2 + mo["uy"] ** 2)
    assert np.linalg.norm(du) / np.linalg.norm(un) <= 1e-3
