"""The paper's own tables reproduced on the GPU (Sec. 4.2-4.4): runs to the
steady state of Sec. 4 (relative change of u and T over 100 steps below
1e-6, or a step cap) and compare with the values the paper prints for its
model (golden files under tests/golden, each citing its table).

Grids: the paper's "N x N" is run with N + 1 nodes per side (walls on
nodes; Table 1's printed locations are multiples of 1/N).  Table 3 is run
at Pr = 7 (the value in Sec. 4.3's text; the caption's Pr = 1.0 gives a
psi_max 2.5 times the tabulated one, checked below)."""
import csv
import math
import os

import numpy as np
import pytest

from paper_1505_02976_gb300 import lbm
from paper_1505_02976_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return [[float(v) for v in line.split(",")] for line in fh
                if line.strip() and not line.startswith("#")]


def _steady(p, precision="f32", cap=2_000_000, tol=1e-6):
    """Step until the Sec. 4 criterion holds or `cap` steps; the lattice
    records whether the criterion was met in `.steady`."""
    g = lbm.Lattice(p, precision)
    g.residual()
    n = 0
    g.steady = False
    while n < cap:
        g.step(100)
        n += 100
        if max(g.residual()) < tol:
            g.steady = True
            break
    return g


@pytest.mark.parametrize("Ra,N,u_max,y_max,v_max,x_max,nu_max,y_nu,nu", _rows("table1_clear_cavity.csv"))
def test_table1_clear_fluid_cavity(Ra, N, u_max, y_max, v_max, x_max, nu_max, y_nu, nu):
    n = int(N) + 1
    p = W.clear_fluid_cavity(n, Ra)
    d = lbm.lbm_derived(p)
    # FP32 does not settle below the 1e-6 criterion at Ra 1e6 (round-off):
    # that case runs in FP64
    g = _steady(p, "f64" if Ra >= 1e6 else "f32", cap=500_000)
    m = g.moments()
    L, scale = d["L"], d["L"] / d["alpha_e"]
    c = (n - 1) // 2
    col, row = m["ux"][:, c] * scale, m["uy"][c, :] * scale
    mean, local = g.nusselt("E")
    assert col.max() == pytest.approx(u_max, rel=0.01)
    assert row.max() == pytest.approx(v_max, rel=0.01)
    assert local.max() == pytest.approx(nu_max, rel=0.015)
    assert mean == pytest.approx(nu, rel=0.005)
    for got, ref in ((col.argmax() / L, y_max), (row.argmax() / L, x_max), (local.argmax() / L, y_nu)):
        assert abs(got - ref) <= 1.01 / N


@pytest.mark.parametrize("Da,psi_max,theta_max", _rows("table3_heat_generating.csv"))
def test_table3_heat_generating_cavity(Da, psi_max, theta_max):
    p = W.heat_generating_cavity(121, Da, Pr=7.0)
    d = lbm.lbm_derived(p)
    g = _steady(p, cap=2_000_000)
    _, (lo, hi) = g.stream_function()
    psi = max(abs(lo), abs(hi)) / (d["L"] * d["U"])
    theta = (g.moments()["T"].max() - d["T0"]) / d["dT"]
    assert psi == pytest.approx(psi_max, rel=0.02)
    assert theta == pytest.approx(theta_max, rel=0.015)


def test_table3_caption_prandtl_number_does_not_fit():
    p = W.heat_generating_cavity(121, math.inf, Pr=1.0)
    d = lbm.lbm_derived(p)
    g = _steady(p, cap=2_000_000)
    _, (lo, hi) = g.stream_function()
    assert max(abs(lo), abs(hi)) / (d["L"] * d["U"]) > 2.0 * 2.83e-3


@pytest.mark.parametrize("Ra,Ra_I,Da,nu,theta_max",
                         [r for r in _rows("table4_heat_source.csv") if r[1] <= 1e5])
def test_table4_heat_source_weak_to_moderate_heating(Ra, Ra_I, Da, nu, theta_max):
    eps = 0.9999 if Da >= 1e8 else 0.4
    p = W.heated_cavity_with_source(151, Ra, Ra_I, Da, eps=eps)
    d = lbm.lbm_derived(p)
    g = _steady(p, cap=600_000)
    assert g.nusselt("W")[0] == pytest.approx(nu, rel=0.01)
    assert (g.moments()["T"].max() - d["T0"]) / d["dT"] == pytest.approx(theta_max, abs=1e-3)


@pytest.mark.parametrize("Ra,Ra_I,Da,nu,theta_max",
                         [r for r in _rows("table4_heat_source.csv") if r[0] == 1e5 and r[1] == 1e7 and r[2] >= 1e-4])
def test_table4_strong_internal_heating(Ra, Ra_I, Da, nu, theta_max):
    """Ra_I / Ra = 100: in FP64 the paper's steady criterion is met after
    1.2-2.2e5 steps.  (Run on far beyond that, a slowly growing mode takes
    over at Ma = 0.1 and the run diverges after about 1e6 steps; smaller
    Mach numbers stay steady.)"""
    p = W.heated_cavity_with_source(151, Ra, Ra_I, Da, eps=0.9999 if Da >= 1e8 else 0.4)
    d = lbm.lbm_derived(p)
    g = _steady(p, "f64", cap=400_000)
    assert g.steady
    assert g.nusselt("W")[0] == pytest.approx(nu, rel=0.015)
    assert (g.moments()["T"].max() - d["T0"]) / d["dT"] == pytest.approx(theta_max, rel=0.015)
