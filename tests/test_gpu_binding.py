"""The Python binding's remaining paths on the GPU: device-resident fields
in and out, the launch shape of the moment state, and the table runner."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_1505_02976_gb300 import cases, lbm
from paper_1505_02976_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_device_fields_in_and_out_match_the_host_path():
    p = W.cavity(70, 1e5, 1e-2, 0.6, ny=50)
    T, ux, uy = W.random_fields(p, seed=2, amp_u=1e-3)
    eps = W.gaussian_random_field(70, corr=5.0, seed=3)[:50]
    a = lbm.Lattice(p, "f64")
    a.set_fields(T, ux, uy, eps_field=eps)
    b = lbm.Lattice(p, "f64")
    dev = [torch.from_numpy(np.ascontiguousarray(v)).cuda() for v in (T, ux, uy, eps)]
    b.set_fields(*dev[:3], eps_field=dev[3])
    for g in (a, b):
        g.step(50)
    ma = a.moments()
    out = {k: torch.empty((50, 70), dtype=torch.float64, device="cuda") for k in ("p", "ux", "uy", "T")}
    b.moments_device(out)
    b.sync()
    for k in ("p", "ux", "uy", "T"):
        assert np.array_equal(out[k].cpu().numpy(), ma[k]), k


def test_moment_segments_change_nothing_but_the_launch():
    p = W.cavity(300, 1e5, 1e-2, 0.6, ny=90)
    fields = W.random_fields(p, seed=5, amp_u=1e-3)
    ref = None
    for seg in (0, 1, 4, 30):
        g = lbm.Lattice(p, "f32", state="moments")
        g.set_moment_segments(seg)
        g.set_fields(*fields)
        g.step(40)
        f, gg = g.get_state()
        if ref is None:
            ref = (f, gg)
        else:
            assert np.array_equal(f[1:], ref[0][1:]) and np.array_equal(gg, ref[1])
    with pytest.raises(lbm.LbmError):
        lbm.Lattice(p, "f32").set_moment_segments(4)


def test_table_runner_yields_every_case():
    rows = list(cases.table_rows(3, "f32", cap=200))
    assert [r["Da"] for r in rows] == [float("inf"), 1e-2, 1e-4]
    for r in rows:
        assert r["steps"] == 200 and r["psi_max"] > 0 and 0 < r["theta_max"] < 1


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_pinned_host_fields_read_in_place_give_the_same_state(precision):
    """Fields in page-locked host memory are read in place by the kernels
    (no staging copy); the state equals the one set from pageable arrays."""
    p = W.cavity(96, 1e5, 1e-3, 0.6, ny=70)
    T, ux, uy = W.random_fields(p, seed=12, amp_u=1e-3)
    eps = W.gaussian_random_field(96, corr=6.0, seed=2)[:70, :]
    a = lbm.Lattice(p, precision)
    a.set_fields(T, ux, uy, eps_field=eps)
    pin = [torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for v in (T, ux, uy, eps)]
    b = lbm.Lattice(p, precision)
    rc = b.lib.lbm_set_fields(b.h, *(C.c_void_p(t.data_ptr()) for t in pin), 0)
    assert rc == 0
    for g in (a, b):
        g.step(7)
    fa, ga = a.get_state()
    fb, gb = b.get_state()
    assert np.array_equal(fa[1:], fb[1:]) and np.array_equal(ga, gb)
