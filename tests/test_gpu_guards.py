"""Guard words after every workspace region: no kernel of the step, the
diagnostics, the state transfers or the checkpoints writes past the end of a
region, for every storage, state and kernel choice; a corrupted guard is
reported as LBM_ERR_GUARD."""
import os

import numpy as np
import pytest

from paper_1505_02976_gb300 import lbm
from paper_1505_02976_gb300 import workloads as W

pytestmark = pytest.mark.gpu

LBM_ERR_GUARD = -7


def _exercise(g, tmp_path):
    g.step(30)
    g.sync()
    g.moments()
    walled = "periodic" not in g.problem["bc"]
    if walled:
        for side in ("W", "E", "S", "N"):
            g.nusselt(side)
        g.stream_function()
    g.residual()
    g.step(5)
    g.residual()
    g.totals()
    path = os.path.join(str(tmp_path), "ck.bin")
    g.save(path)
    g.step(3)
    g.load_checkpoint(path)
    if g.state == "populations":
        f, gg = g.get_state()
        g.set_state(f, gg)
    g.step(4)
    g.sync()


CASES = [
    ("f32", "populations", None),
    ("f32", "populations", 0),
    ("f16", "populations", None),
    ("f64", "populations", None),
    ("f32", "moments", None),
    ("f64", "moments", None),
]


@pytest.mark.parametrize("precision,state,staged", CASES)
def test_guards_hold_after_every_operation(precision, state, staged, tmp_path):
    p = W.cavity(131, 1e5, 1e-3, 0.5, ny=77)
    g = lbm.Lattice(p, precision, state=state)
    if staged is not None:
        g.staged = staged
    g.set_fields(*W.random_fields(p, seed=5, amp_u=1e-3),
                 eps_field=W.gaussian_random_field(131, corr=8.0, seed=2)[:77, :])
    _exercise(g, tmp_path)
    g.check_guards()


def test_guards_hold_on_a_periodic_channel(tmp_path):
    p = W.poiseuille(nx=9, ny=40)
    g = lbm.Lattice(p, "f32")
    g.set_force_profile(np.linspace(0.0, 1e-6, 40))
    _exercise(g, tmp_path)
    g.check_guards()


def test_a_corrupted_guard_is_reported():
    p = W.cavity(40, 1e4, 1e-2, 0.6)
    g = lbm.Lattice(p, "f32")
    g.step(10)
    g.check_guards()
    g.workspace[-1] = 0  # the last byte of the last guard word
    with pytest.raises(lbm.LbmError) as e:
        g.check_guards()
    assert e.value.status == LBM_ERR_GUARD


def test_batch_guards_hold_and_a_corrupted_guard_is_reported():
    probs = [W.cavity(20, 1e4, 1e-2, 0.6), W.cavity(300, 1e6, 1e-4, 0.4, ny=131), W.cavity(64, 1e5, 1e-3, 0.5)]
    for staged in (True, False):
        b = lbm.Batch(probs, "f32")
        b.staged = staged
        for mode in ("fused", "graph", "per_case"):
            b.step(50 if mode == "graph" else 7, mode)
        b.sync()
        b.nusselt("W")
        b.moments(1)
        b.check_guards()
        b.close()
    b = lbm.Batch(probs, "f64")
    b.step(9, "fused")
    b.check_guards()
    b.workspace[-1] = 0
    with pytest.raises(lbm.LbmError) as e:
        b.check_guards()
    assert e.value.status == LBM_ERR_GUARD
