"""Porosity fields and the discrete adjoint on the GPU, through the C ABI.

* forward with a porosity field against the oracle (FP64, 1e-10);
* adjoint gradients (FP64) against the oracle's complex-step derivatives
  (the exact discrete derivatives of the oracle's own step) on small
  lattices with every kind of wall;
* the differentiation workload at full size: 256 x 256 cavity, Ra 1e5,
  porosity from a seeded Gaussian random field (correlation length 16 cells)
  in [0.3, 0.9], Da 1e-3 at eps 0.6 with Kozeny-Carman scaling, 4000 steps:
  FP64 adjoint against central finite differences (h = 1e-4) on 32 random
  cells and both wall temperatures, within 1e-4 of the gradient's scale;
  FP32 adjoint against the FP64 one;
* the torch.autograd.Function.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1505_02976_gb300 import lbm
from paper_1505_02976_gb300 import workloads as W

from oracle_states import sample_nodes, stored_state

pytestmark = pytest.mark.gpu


def test_fp64_porosity_field_forward_parity():
    p = W.cavity(40, 1e5, 1e-3, 0.6, ny=33)
    eps = W.gaussian_random_field(64, corr=6.0, seed=5)[:33, :40]
    fields = W.random_fields(p, seed=8, amp_u=1e-3)
    o = oracle.Oracle(p, *fields, eps_field=eps).run(300)
    g = lbm.Lattice(p, "f64")
    g.set_fields(*fields, eps_field=eps)
    g.step(300)
    mo, mg = o.moments(), g.moments()
    umax = np.sqrt(mo["ux"] ** 2 + mo["uy"] ** 2).max()
    assert np.abs(mg["ux"] - mo["ux"]).max() <= 1e-10 * umax
    assert np.abs(mg["uy"] - mo["uy"]).max() <= 1e-10 * umax
    assert np.abs(mg["T"] - mo["T"]).max() <= 1e-10
    f, gg = g.get_state()
    assert np.abs(gg - o.g).max() <= 1e-10 * np.abs(o.g).max()


def test_fp32_porosity_field_one_step_sampled():
    n = 256
    p = W.cavity(n, 1e5, 1e-3, 0.6)
    eps = W.gaussian_random_field(n, corr=16.0, seed=1)
    o, f0, g0 = stored_state(p, W.random_fields(p, seed=3, amp_u=2e-3), "f32", steps=10, eps_field=eps)
    g = lbm.Lattice(p, "f32")
    g.set_fields(eps_field=eps)
    g.set_state(f0, g0)
    g.step(1)
    f1, g1 = g.get_state()
    xs, ys = sample_nodes(n, n, 300, seed=2)
    fo, go = o.update_nodes(xs, ys)
    assert np.abs(f1[1:, ys, xs].T - fo[:, 1:]).max() <= 1e-6 * np.abs(fo[:, 1:]).max()
    assert np.abs(g1[:, ys, xs].T - go).max() <= 1e-6 * np.abs(go).max()


CASES = {  # boundary set, wall whose Nusselt number is the loss
    "cavity": (dict(bc=("dirichlet", "dirichlet", "adiabatic", "adiabatic")), "W"),
    "heated_floor": (dict(bc=("adiabatic", "adiabatic", "dirichlet", "dirichlet"), T_bc=(1.0, 0.0, 1.0, 0.0)), "S"),
    "mixed": (dict(bc=("dirichlet", "adiabatic", "dirichlet", "adiabatic"), T_bc=(1.0, 0.0, 0.7, 0.0)), "E"),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_fp64_adjoint_matches_oracle_complex_step(case):
    n, steps = 14, 150
    bcs, side = CASES[case]
    p = W.cavity(n, 1e5, 1e-3, 0.6, ny=12, **bcs)
    eps = W.gaussian_random_field(16, corr=4.0, seed=4)[:12, :n]
    g = lbm.Lattice(p, "f64")
    g.set_fields(eps_field=eps)
    loss, g_eps, g_t = g.adjoint(steps, side=side, segment=7)
    cells = [(0, 0), (0, 5), (1, 1), (2, 6), (6, 0), (13, 11), (7, 5), (12, 2), (5, 10)]
    ref, ref_t = oracle.nusselt_gradient(p, steps, eps, cells, sides=("W", "E", "S", "N"), loss_side=side)
    o = oracle.Oracle(p, eps_field=eps).run(steps)
    assert loss == pytest.approx(o.nusselt(side)[0], rel=1e-12)
    assert np.abs(ref).max() > 1e-6
    scale = np.abs(ref).max()
    for k, (x, y) in enumerate(cells):
        assert g_eps[y, x] == pytest.approx(ref[k], abs=1e-9 * scale), (x, y)
    for s, side in enumerate("WESN"):
        assert g_t[s] == pytest.approx(ref_t[side], rel=1e-9, abs=1e-12), side


def _config5(precision):
    n = 256
    p = W.cavity(n, 1e5, 1e-3, 0.6)
    eps = W.gaussian_random_field(n, corr=16.0, seed=1)
    return p, eps


def _nu64(p, eps, steps, Th=1.0, Tc=0.0):
    q = dict(p, T_bc=(Th, Tc, p["T_bc"][2], p["T_bc"][3]))
    g = lbm.Lattice(q, "f64")
    g.set_fields(eps_field=eps)
    g.step(steps)
    return g.nusselt("W")[0]


def test_fp64_adjoint_against_central_differences_full_size():
    steps = 4000
    p, eps = _config5("f64")
    g = lbm.Lattice(p, "f64")
    g.set_fields(eps_field=eps)
    loss, g_eps, g_t = g.adjoint(steps)
    rng = np.random.Generator(np.random.PCG64(2))
    cells = [(int(x), int(y)) for x, y in zip(rng.integers(0, 256, 32), rng.integers(0, 256, 32))]
    h = 1e-4
    fd = []
    for x, y in cells:
        ep, em = eps.copy(), eps.copy()
        ep[y, x] += h
        em[y, x] -= h
        fd.append((_nu64(p, ep, steps) - _nu64(p, em, steps)) / (2 * h))
    fd = np.array(fd)
    ad = np.array([g_eps[y, x] for x, y in cells])
    # per sampled node: |ad - fd| <= 1e-4 |fd|.  A central difference at
    # h = 1e-4 cannot resolve a derivative below its own round-off: two FP64
    # runs of 4000 steps whose rounding differs move Nu (about 3) by ~1e-14,
    # which is ~1e-10 in (Nu+ - Nu-) / 2h, so the bound has that floor.
    floor = 1e-10
    err = np.abs(ad - fd)
    rel = err / np.maximum(np.abs(fd), 1e-300)
    print("\nnode (x, y)   d Nu / d eps (adjoint)   central difference   relative error")
    for (x, y), a, f, r in zip(cells, ad, fd, rel):
        print(f"({x:3d}, {y:3d})   {a: .10e}   {f: .10e}   {r:.2e}")
    print(f"nodes above the floor (|fd| > {floor / 1e-4:.0e}): {(np.abs(fd) * 1e-4 > floor).sum()} of {len(fd)}; "
          f"largest relative error there {rel[np.abs(fd) * 1e-4 > floor].max():.2e}")
    assert (err <= np.maximum(1e-4 * np.abs(fd), floor)).all(), (rel.max(), err.max())
    # Richardson pair at larger steps: (4 D(h/2) - D(h)) / 3 with h = 2e-3
    # cancels the h^2 truncation term (the remainder, h^4 over (1 - eps)^4 at
    # eps <= 0.9, stays below 1e-6 relative) and divides the round-off floor
    # by 20, so most sampled nodes are checked at 1e-4 relative.
    def central(x, y, hh):
        ep, em = eps.copy(), eps.copy()
        ep[y, x] += hh
        em[y, x] -= hh
        return (_nu64(p, ep, steps) - _nu64(p, em, steps)) / (2 * hh)
    hr = 2e-3
    fdr = np.array([(4 * central(x, y, hr / 2) - central(x, y, hr)) / 3 for x, y in cells])
    floor_r = 1e-11
    err_r = np.abs(ad - fdr)
    rel_r = err_r / np.maximum(np.abs(fdr), 1e-300)
    above = np.abs(fdr) * 1e-4 > floor_r
    print(f"Richardson (h = {hr}, {hr / 2}): nodes above the floor (|fd| > {floor_r / 1e-4:.0e}): "
          f"{above.sum()} of {len(fdr)}; largest relative error there {rel_r[above].max():.2e}; "
          f"all relative errors: {np.array2string(rel_r, precision=1)}")
    assert (err_r <= np.maximum(1e-4 * np.abs(fdr), floor_r)).all(), (rel_r.max(), err_r.max())
    fd_h = (_nu64(p, eps, steps, Th=1 + h) - _nu64(p, eps, steps, Th=1 - h)) / (2 * h)
    fd_c = (_nu64(p, eps, steps, Tc=h) - _nu64(p, eps, steps, Tc=-h)) / (2 * h)
    assert g_t[0] == pytest.approx(fd_h, rel=1e-4)
    assert g_t[1] == pytest.approx(fd_c, rel=1e-4)


def test_fp32_adjoint_against_fp64_full_size():
    """FP32 storage and arithmetic, gradients accumulated in FP64: within
    2 % of the FP64 gradient's scale node by node."""
    steps = 4000
    p, eps = _config5("f32")
    res = {}
    for prec in ("f64", "f32"):
        g = lbm.Lattice(p, prec)
        g.set_fields(eps_field=eps)
        res[prec] = g.adjoint(steps)
    l64, e64, t64 = res["f64"]
    l32, e32, t32 = res["f32"]
    assert l32 == pytest.approx(l64, rel=1e-4)
    assert np.abs(e32 - e64).max() <= 2e-2 * np.abs(e64).max()
    assert np.allclose(t32[:2], t64[:2], rtol=1e-3)


def test_autograd_function_returns_the_adjoint_gradients():
    from paper_1505_02976_gb300.autograd import wall_nusselt

    p = W.cavity(24, 1e5, 1e-3, 0.6)
    eps_np = W.gaussian_random_field(24, corr=5.0, seed=6)
    eps = torch.tensor(eps_np, dtype=torch.float64, device="cuda", requires_grad=True)
    tw = torch.tensor([1.0, 0.0], dtype=torch.float64, device="cuda", requires_grad=True)
    nu = wall_nusselt(eps, tw, p, 200, precision="f64")
    (2.0 * nu).backward()
    g = lbm.Lattice(p, "f64")
    g.set_fields(eps_field=eps_np)
    loss, g_eps, g_t = g.adjoint(200)
    assert nu.device == eps.device
    assert float(nu.detach()) == pytest.approx(loss, rel=1e-12)
    assert np.allclose(eps.grad.cpu().numpy(), 2.0 * g_eps, rtol=1e-12, atol=1e-14)
    assert np.allclose(tw.grad.cpu().numpy(), 2.0 * g_t[:2], rtol=1e-12)
    # a gradient for the wall temperatures only, and a loss with no gradient
    eps2 = torch.tensor(eps_np, dtype=torch.float64, device="cuda")
    tw2 = torch.tensor([1.0, 0.0], dtype=torch.float64, device="cuda", requires_grad=True)
    wall_nusselt(eps2, tw2, p, 200, precision="f64").backward()
    assert eps2.grad is None
    assert np.allclose(tw2.grad.cpu().numpy(), g_t[:2], rtol=1e-12)
    with torch.no_grad():
        nu3 = wall_nusselt(eps2, tw2, p, 200, precision="f64")
    assert float(nu3) == pytest.approx(loss, rel=1e-12)
    with pytest.raises(ValueError):
        wall_nusselt(eps2, tw2, W.problem(nx=24, ny=24, bc=("adiabatic", "dirichlet", "dirichlet",
                                                           "adiabatic")), 10)
