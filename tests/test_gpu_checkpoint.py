"""Checkpoint and resume (lbm_checkpoint): bit-for-bit continuation, and
host-side fault injection (a corrupted byte, a different problem) that must
be refused without touching the state."""
import numpy as np
import pytest

from paper_1505_02976_gb300 import lbm
from paper_1505_02976_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["f64", "f32", "f16"])
def test_resume_is_bitwise(tmp_path, precision):
    p = W.cavity(70, 1e5, 1e-3, 0.6, ny=50)
    g = lbm.Lattice(p, precision)
    g.set_fields(*W.random_fields(p, seed=1, amp_u=1e-3),
                 eps_field=W.gaussian_random_field(70, corr=8.0, seed=3)[:50, :70])
    g.step(100)
    path = str(tmp_path / "a.ckpt")
    g.save(path)
    g.step(60)
    ref = g.get_state()
    assert g.steps == 160
    h = lbm.Lattice(p, precision)
    h.load_checkpoint(path)
    assert h.steps == 100
    h.step(60)
    got = h.get_state()
    assert np.array_equal(ref[0][1:], got[0][1:]) and np.array_equal(ref[1], got[1])


def test_corrupted_or_foreign_checkpoint_is_refused(tmp_path):
    p = W.cavity(40, 1e4, 1e-2, 0.6)
    g = lbm.Lattice(p, "f32")
    g.step(10)
    path = tmp_path / "b.ckpt"
    g.save(str(path))
    before = g.get_state()
    data = bytearray(path.read_bytes())
    data[len(data) // 2] ^= 0x40
    bad = tmp_path / "bad.ckpt"
    bad.write_bytes(bytes(data))
    with pytest.raises(lbm.LbmError) as e:
        g.load_checkpoint(str(bad))
    assert e.value.status == -1 and "CRC" in str(e.value)
    after = g.get_state()
    assert np.array_equal(before[1], after[1])
    other = lbm.Lattice(W.cavity(40, 1e5, 1e-2, 0.6), "f32")
    with pytest.raises(lbm.LbmError):
        other.load_checkpoint(str(path))
    with pytest.raises(lbm.LbmError):
        lbm.Lattice(p, "f64").load_checkpoint(str(path))


def test_restore_makes_the_restored_state_the_residual_reference(tmp_path):
    """The residual snapshot is not part of the file: after a restore, the
    next lbm_residual compares against the restored state, so a residual
    taken straight after the restore is zero, and one taken after some steps
    equals the one the saved run reports after the same steps."""
    p = W.cavity(40, 1e5, 1e-2, 0.6)
    g = lbm.Lattice(p, "f64")
    g.step(200)
    path = str(tmp_path / "c.ckpt")
    g.save(path)
    g.residual()          # snapshot = the saved state
    g.step(30)
    ref = g.residual()
    h = lbm.Lattice(p, "f64")
    h.step(500)           # a different state and snapshot before the restore
    h.residual()
    h.load_checkpoint(path)
    assert h.residual() == (0.0, 0.0)
    h.step(30)
    assert h.residual() == ref
