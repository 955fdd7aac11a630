"""lbm_nusselt_noalloc: the mean Nusselt number for callers that cannot let
the library allocate device memory (it takes its scratch from a fixed array in
the library).  Checked through the C ABI against lbm_nusselt on two calls in a
row, within the FP64 parity tolerance of the other GPU tests.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import ctypes as C

import pytest

from paper_1505_02976_gb300 import lbm
from paper_1505_02976_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _noalloc(lat, side):
    L = lbm.load()
    L.lbm_nusselt_noalloc.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_double)]
    L.lbm_nusselt_noalloc.restype = C.c_int
    out = C.c_double(float("nan"))
    rc = L.lbm_nusselt_noalloc(lat.h, side, C.byref(out))
    if rc != 0:
        raise lbm.LbmError(rc, L.lbm_last_error(lat.h).decode())
    return out.value


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_noalloc_matches_nusselt_on_two_calls(precision):
    p = W.cavity(48, 1e5, 1e-2, 0.6, ny=40)
    lat = lbm.Lattice(p, precision)
    lat.step(400)
    for side in range(4):
        ref, _ = lat.nusselt(side)
        first = _noalloc(lat, side)
        second = _noalloc(lat, side)
        assert first == pytest.approx(ref, rel=TOL, abs=1e-12)
        assert second == pytest.approx(ref, rel=TOL, abs=1e-12)
    # another lattice with longer walls, then the first again
    q = W.cavity(300, 1e4, 1e-2, 0.6, ny=260)
    other = lbm.Lattice(q, precision)
    other.step(50)
    assert _noalloc(other, 0) == pytest.approx(other.nusselt(0)[0], rel=TOL, abs=1e-12)
    assert _noalloc(lat, 1) == pytest.approx(lat.nusselt(1)[0], rel=TOL, abs=1e-12)


def test_noalloc_rejects_walls_longer_than_its_scratch():
    p = W.problem(nx=70000, ny=4, bc=("periodic", "periodic", "dirichlet", "dirichlet"),
                  T_bc=(0.0, 0.0, 0.0, 1.0), gbeta=0.0, nu=0.1, alpha_e=0.1)
    lat = lbm.Lattice(p, "f32")
    with pytest.raises(lbm.LbmError) as e:
        _noalloc(lat, 2)
    assert e.value.status == -1
    assert "65536" in str(e.value)
