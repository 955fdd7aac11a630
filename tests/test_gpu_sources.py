"""Internal heat generation on the GPU (Sec. 4.3, Sec. 4.4): FP64 parity with
the oracle for the derived source Q and the buoyancy reference T0, and the
stream function entry point against the oracle's."""
import numpy as np
import pytest

import oracle
from paper_1505_02976_gb300 import lbm, workloads as W

pytestmark = pytest.mark.gpu

CASES = {
    "cooled_walls_Da1e-2": lambda: W.heat_generating_cavity(26, 1e-2, Ra_I=2e4),
    "cooled_walls_clear": lambda: W.heat_generating_cavity(19, float("inf"), Ra_I=1e4, Pr=7.0),
    "sidewall_plus_source": lambda: W.heated_cavity_with_source(23, 1e4, 1e6, 1e-3, ny=17),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_fp64_heat_source_cavities_match_the_oracle(case):
    p = CASES[case]()
    steps = 1500
    o = oracle.Oracle(p).run(steps)
    g = lbm.Lattice(p, "f64")
    g.step(steps)
    mo, mg = o.moments(), g.moments()
    umax = np.sqrt(mo["ux"] ** 2 + mo["uy"] ** 2).max()
    assert umax > 0
    assert np.abs(mg["ux"] - mo["ux"]).max() <= 1e-10 * umax
    assert np.abs(mg["uy"] - mo["uy"]).max() <= 1e-10 * umax
    assert np.abs(mg["T"] - mo["T"]).max() <= 1e-10 * np.abs(mo["T"]).max()
    psi, (lo, hi) = g.stream_function()
    ref = oracle.stream_function(mo["ux"])
    scale = np.abs(ref).max()
    assert scale > 0
    assert np.abs(psi - ref).max() <= 1e-10 * scale
    assert lo == psi.min() and hi == psi.max()
    # the same quadrature on the GPU's own velocity agrees to the last bits
    assert np.abs(psi - oracle.stream_function(mg["ux"])).max() <= 1e-14 * scale


def test_stream_function_of_the_fp32_benchmark_lattice_at_full_size():
    """2048 x 2048 after a few steps: psi against the oracle's quadrature of
    the same u_x at sampled columns (the oracle integrates whole columns)."""
    p = W.config_problem(W.CONFIG_FP32_CAVITY)
    g = lbm.Lattice(p, "f32")
    g.set_fields(*W.random_fields(p, seed=3, amp_u=1e-2))
    g.step(3)
    ux = g.moments()["ux"]
    psi, (lo, hi) = g.stream_function()
    cols = np.r_[0, 1, 777, 1024, 2046, 2047]
    ref = oracle.stream_function(np.ascontiguousarray(ux[:, cols]))
    assert np.abs(psi[:, cols] - ref).max() <= 1e-13 * np.abs(ref).max()
    assert lo == psi.min() and hi == psi.max()
