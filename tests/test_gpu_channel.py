"""The mixed-convection porous channel (Sec. 4.1) on the GPU: parity with
the oracle under the height-dependent driving force a_y(y)."""
import numpy as np
import pytest

import oracle
from paper_1505_02976_gb300 import lbm

from channel_case import channel

pytestmark = pytest.mark.gpu


def test_fp64_channel_parity_with_force_profile():
    c = channel(H=32, u0=0.01, v0=0.01)
    o = oracle.Oracle(c["problem"], ay_profile=c["ay"]).run(3000)
    g = lbm.Lattice(c["problem"], "f64")
    g.set_force_profile(c["ay"])
    g.step(3000)
    mo, mg = o.moments(), g.moments()
    umax = np.sqrt(mo["ux"] ** 2 + mo["uy"] ** 2).max()
    assert np.abs(mg["ux"] - mo["ux"]).max() <= 1e-10 * umax
    assert np.abs(mg["uy"] - mo["uy"]).max() <= 1e-10 * umax
    assert np.abs(mg["T"] - mo["T"]).max() <= 1e-10
    f, gg = g.get_state()
    assert np.abs(gg - o.g).max() <= 1e-10 * np.abs(o.g).max()
