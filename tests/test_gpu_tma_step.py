"""The step with TMA-staged rows (FP32 and FP16 storage, lattices walled on
all four sides).

The staged kernel and the global-load kernel run the same per-node code: at
tau = 1 they must agree bit for bit in FP32, on lattices that span several
128-column bands and 4-row segments with ragged edges, and on the smallest
lattices the staged kernel takes; the FP32 staged lattice also matches the
batched kernel.  In FP16 storage at tau = 1 the staged kernel updates pairs
of interior nodes with packed FP32 instructions, which may fuse a multiply
into the add that follows it: after one step every stored value agrees with
the global-load kernel's to within one FP16 rounding step plus the FP32
rounding of its cancelling terms (and almost all exactly), and after 60
steps the moments agree to FP16 noise.  With a
porosity field both kernels run the one-node code and agree bit for bit.
Away from tau = 1 (with sources) and with a porosity field the staged kernel
is checked against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_1505_02976_gb300 import lbm
from paper_1505_02976_gb300 import workloads as W

from oracle_states import stored_state

pytestmark = pytest.mark.gpu

SIZES = [(300, 250), (129, 517), (4, 4), (131, 5), (517, 9)]


def _run(p, precision, fields, steps, staged, eps_field=None):
    g = lbm.Lattice(p, precision)
    g.set_fields(*fields, eps_field=eps_field)
    if not staged:
        g.staged = False
    assert g.staged == staged
    g.step(steps)
    g.sync()
    return g


@pytest.mark.parametrize("precision", ["f32", "f16"])
@pytest.mark.parametrize("nx,ny", SIZES)
def test_staged_step_matches_global_loads(precision, nx, ny):
    """Several bands and segments, ragged last band and segment, and the
    smallest lattices the staged kernel takes (4 rows, one partial band)."""
    p = W.cavity(nx, 1e5, 1e-3, 0.5, ny=ny)
    fields = W.random_fields(p, seed=nx + ny, amp_u=2e-3, amp_T=0.3)
    if precision == "f16":
        _fp16_pairs_within_one_rounding_step(p, fields)
    a = _run(p, precision, fields, 60, True)
    b = _run(p, precision, fields, 60, False)
    fa, ga = a.get_state()
    fb, gb = b.get_state()
    ma = a.moments()
    if precision == "f32":
        assert np.array_equal(fa[1:], fb[1:]) and np.array_equal(ga, gb)
    else:
        mb = b.moments()
        # FP16 storage noise: the rare different roundings of the first step
        # spread over 60 steps (the FP16 forms are held to 3e-3 against the
        # oracle over 2000 steps)
        assert np.abs(ma["T"] - mb["T"]).max() <= 1e-3
        du = np.sqrt((ma["ux"] - mb["ux"]) ** 2 + (ma["uy"] - mb["uy"]) ** 2)
        assert np.linalg.norm(du) <= 1e-2 * np.linalg.norm(np.sqrt(mb["ux"] ** 2 + mb["uy"] ** 2))
    assert np.all(np.isfinite(ma["T"]))
    if precision == "f32":
        bt = lbm.Batch([p], "f32")
        bt.set_fields(0, *fields)
        bt.step(60, "fused")
        bt.sync()
        mb = bt.moments(0)
        for k in ("ux", "uy", "T", "p"):
            assert np.array_equal(ma[k], mb[k]), k
        bt.close()


W_I = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


FP16_SCALE = 2.0 ** -10  # stored value = population / scale (lbm_host.h)


def _fp16_step(v):
    """The FP16 rounding step at the magnitude of v in population units:
    2^(floor(log2 |v|) - 10), and the subnormal step 2^-24 below 2^-14
    (both times the storage scale)."""
    a = np.maximum(np.abs(v), 1e-30)
    return np.maximum(np.exp2(np.floor(np.log2(a)) - 10), 2.0 ** -24 * FP16_SCALE)


def _fp16_pairs_within_one_rounding_step(p, fields):
    """One step from the same fields: the stored FP16 values of the staged
    kernel (node pairs, packed arithmetic) and of the global-load kernel
    (one node, scalar arithmetic) differ by at most one rounding step, and
    only where the FP32 values fall on different sides of a random rounding
    threshold (rare)."""
    a = _run(p, "f16", fields, 1, True)
    b = _run(p, "f16", fields, 1, False)
    fa, ga = a.get_state()
    fb, gb = b.get_state()
    # thermal values are stored as deviations from w_i sigma T0
    base = (W_I * p["sigma"] * 0.5 * (p["Th"] + p["Tc"]))[:, None, None]
    sa = np.concatenate([fa[1:], ga - base])
    sb = np.concatenate([fb[1:], gb - base])
    diff = np.abs(sa - sb)
    # one rounding step at the value, plus the FP32 rounding of the terms
    # that cancel in it (a few units in the last place of the plane's
    # largest magnitude)
    plane_max = np.abs(sb).max(axis=(1, 2), keepdims=True)
    bound = _fp16_step(np.maximum(np.abs(sa), np.abs(sb))) + 2.0 ** -20 * plane_max
    assert (diff <= bound).all(), (diff / bound).max()
    assert (diff > 0).mean() <= 1e-2, (diff > 0).mean()


@pytest.mark.parametrize("precision", ["f32", "f16"])
def test_staged_step_with_porosity_field_matches_global_loads(precision):
    """Porosity field (per-node constants from K(eps), F_eps(eps)) on a
    260 x 133 cavity: staged and global-load kernels give the same bits."""
    p = W.cavity(260, 1e5, 1e-3, 0.5, ny=133)
    eps = W.gaussian_random_field(260, corr=8.0, seed=9)[:133, :]
    fields = W.random_fields(p, seed=4, amp_u=2e-3, amp_T=0.3)
    fa, ga = _run(p, precision, fields, 40, True, eps_field=eps).get_state()
    fb, gb = _run(p, precision, fields, 40, False, eps_field=eps).get_state()
    assert np.array_equal(fa[1:], fb[1:]) and np.array_equal(ga, gb)
    assert np.all(np.isfinite(ga))


def test_staging_switch_is_refused_where_unavailable():
    per = lbm.Lattice(W.poiseuille(nx=16, ny=32), "f32")
    assert not per.staged
    with pytest.raises(lbm.LbmError):
        per.staged = True
    f64 = lbm.Lattice(W.cavity(32, 1e4, 1e-2, 0.6), "f64")
    assert not f64.staged
    with pytest.raises(lbm.LbmError):
        f64.staged = True
    g = lbm.Lattice(W.cavity(32, 1e4, 1e-2, 0.6), "f16")
    assert g.staged
    g.staged = False
    g.staged = True
    assert g.staged


def _off_tau_problem():
    return W.cavity(260, 1e5, 1e-3, 0.45, ny=140, tau_f=0.8, tau_T=1.15, Q=1e-4, ax=1e-7,
                    bc=("dirichlet",) * 4, T_bc=(1.0, 0.0, 0.7, 0.2))


def test_staged_step_off_tau_one_matches_global_loads():
    """The general collision (tau != 1) with a heat source and a body force,
    FP32: staged and global-load kernels agree to FP32 rounding after 5 steps
    (their products may contract into fused multiply-adds differently)."""
    p = _off_tau_problem()
    fields = W.random_fields(p, seed=8, amp_u=2e-3, amp_T=0.3)
    fa, ga = _run(p, "f32", fields, 5, True).get_state()
    fb, gb = _run(p, "f32", fields, 5, False).get_state()
    assert np.abs(fa[1:] - fb[1:]).max() <= 1e-6 * np.abs(fb[1:]).max()
    assert np.abs(ga - gb).max() <= 1e-6 * np.abs(gb).max()


@pytest.mark.parametrize("precision", ["f32", "f16"])
def test_staged_step_off_tau_one_against_oracle(precision):
    """tau_f 0.8, tau_T 1.15 with an internal heat source, a body force and
    Dirichlet walls on all four sides: one staged step from an oracle-made
    state in the storage precision against the oracle on every node (FP32:
    1e-6 of the population scale; FP16: one FP16 step of each value, the
    thermal populations as deviations from w_i sigma T0)."""
    p = _off_tau_problem()
    o, f0, g0 = stored_state(p, W.random_fields(p, seed=3, amp_u=2e-3, amp_T=0.3), precision, steps=1)
    g = lbm.Lattice(p, precision)
    assert g.staged
    g.set_state(f0, g0)
    g.step(1)
    f1, g1 = g.get_state()
    o.run(1)
    if precision == "f32":
        assert np.abs(f1[1:] - o.f[1:]).max() <= 1e-6 * np.abs(o.f[1:]).max()
        assert np.abs(g1 - o.g).max() <= 1e-6 * np.abs(o.g).max()
    else:
        fo = o.f[1:]
        assert np.all(np.abs(f1[1:] - fo) <= 2.0 ** -10 * np.abs(fo) + 1e-6 * np.abs(fo).max())
        w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]
        dev = np.abs(o.g - w * p["sigma"] * oracle.derived(p)["T0"])
        assert np.all(np.abs(g1 - o.g) <= 2.0 ** -10 * dev + 1e-6 * dev.max())


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


def test_bounded_wait_gives_up_and_reports_timeout():
    """Failure detection without a fault: a wait on an mbarrier that nothing
    arrives on gives up after its time limit, the host reads LBM_ERR_TIMEOUT
    (sticky), and after lbm_set_fields the same context steps normally and
    matches a fresh lattice bit for bit."""
    p = W.cavity(200, 1e5, 1e-3, 0.5, ny=64)
    g = lbm.Lattice(p, "f32")
    g.step(3)
    g.wait_selftest()
    with pytest.raises(lbm.LbmError) as e:
        g.sync()
    assert e.value.status == -4
    with pytest.raises(lbm.LbmError) as e:
        g.step(1)
    assert e.value.status == -4
    g.set_fields()
    g.step(20)
    g.sync()
    ref = lbm.Lattice(p, "f32")
    ref.step(20)
    ref.sync()
    assert np.array_equal(g.moments()["T"], ref.moments()["T"])
