"""Batches of independent cavities (lbm_batch_*) against the oracle and
against the single-lattice path, through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_1505_02976_gb300 import lbm
from paper_1505_02976_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _mixed_problems():
    return [
        W.cavity(20, 1e4, 1e-2, 0.6),
        W.cavity(37, 1e5, 1e-3, 0.4, ny=29),
        W.cavity(64, 1e3, 1e-6, 0.9, Pr=0.7),
        W.cavity(45, 3e5, 1e-4, 0.3, ny=70, bc=("dirichlet", "adiabatic", "dirichlet", "adiabatic"),
                 T_bc=(1.0, 0.0, 0.8, 0.0)),
        W.poiseuille(nx=9, ny=33),
        W.cavity(128, 1e6, 1e-4, 0.4, ny=96),
    ]


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def test_fp64_batch_against_oracle():
    probs = _mixed_problems()
    b = lbm.Batch(probs, "f64")
    rng = np.random.Generator(np.random.PCG64(4))
    fields = []
    for c, p in enumerate(probs):
        f = W.random_fields(p, seed=int(rng.integers(1 << 30)), amp_u=1e-3)
        fields.append(f)
        b.set_fields(c, *f)
    b.step(150, "fused")
    b.sync()
    for c, p in enumerate(probs):
        o = oracle.Oracle(p, *fields[c]).run(150)
        mo, mg = o.moments(), b.moments(c)
        umax = np.sqrt(mo["ux"] ** 2 + mo["uy"] ** 2).max()
        assert np.abs(mg["ux"] - mo["ux"]).max() <= 1e-10 * umax
        assert np.abs(mg["uy"] - mo["uy"]).max() <= 1e-10 * umax
        assert _rel(mg["T"], mo["T"]) <= 1e-10
    nu = b.nusselt("W")
    for c, p in enumerate(probs):
        if p["bc"][0] == "periodic":
            continue
        ref, _ = oracle.Oracle(p, *fields[c]).run(150).nusselt("W")
        assert nu[c] == pytest.approx(ref, rel=1e-10, abs=1e-12)


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_modes_and_launch_shapes_agree_bitwise(precision):
    """Fused, graph and per-case steps, and every tile width, run the same
    per-node code: the results are identical bit for bit, and identical to
    single-lattice runs of each cavity."""
    probs = _mixed_problems()
    runs = {}
    for mode, shape in (("fused", (32, 152)), ("fused", (128, 1000)), ("graph", (64, 300)),
                        ("per_case", None)):
        b = lbm.Batch(probs, precision)
        if shape:
            b.set_launch(*shape)
        b.step(120, mode)
        b.sync()
        runs[(mode, shape)] = [b.moments(c) for c in range(len(probs))]
        assert b.steps == 120
        b.close()
    ref = runs[("per_case", None)]
    for key, res in runs.items():
        for c in range(len(probs)):
            for k in ("ux", "uy", "T", "p"):
                assert np.array_equal(res[c][k], ref[c][k]), (key, c, k)
    for c, p in enumerate(probs):
        g = lbm.Lattice(p, precision)
        g.step(120)
        m = g.moments()
        for k in ("ux", "uy", "T", "p"):
            assert np.array_equal(m[k], ref[c][k]), (c, k)


def test_autotune_keeps_results_and_counts_steps():
    probs = _mixed_problems()
    a = lbm.Batch(probs, "f32")
    tx, grid = a.autotune(2)
    assert tx in (32, 64, 128) and grid >= 1
    n_tuned = a.steps
    assert n_tuned == 3 * 3 * 3  # 3 widths x 3 grids x (2 + 1) steps
    a.step(20, "graph")
    a.sync()
    b = lbm.Batch(probs, "f32")
    b.step(n_tuned + 20, "fused")
    b.sync()
    for c in range(len(probs)):
        assert np.array_equal(a.moments(c)["T"], b.moments(c)["T"])


def test_batch_of_the_benchmark_distribution_runs():
    """A slice of the 512-cavity benchmark batch (sizes 64..512, log-uniform
    Ra and Da, uniform eps): finite after steps, Nusselt numbers sane."""
    probs = W.batch_cavities(48, seed=7)
    b = lbm.Batch(probs, "f32")
    b.step(100, "graph")
    b.sync()
    nu = b.nusselt("W")
    assert np.all(np.isfinite(nu)) and np.all(nu > 0.5)


def _walled_problems():
    return [
        W.cavity(20, 1e4, 1e-2, 0.6),
        W.cavity(37, 1e5, 1e-3, 0.4, ny=29),
        W.cavity(300, 1e6, 1e-4, 0.4, ny=131),
        W.cavity(4, 1e4, 1e-2, 0.5, ny=6),
        W.cavity(45, 3e5, 1e-4, 0.3, ny=70, bc=("dirichlet", "adiabatic", "dirichlet", "adiabatic"),
                 T_bc=(1.0, 0.0, 0.8, 0.0)),
        W.cavity(130, 1e5, 1e-3, 0.5, ny=50, tau_f=0.8, tau_T=1.1),
    ]


def test_staged_batch_matches_global_loads_and_single_lattices():
    """An FP32 batch of walled cavities (one band and several, ragged bands and
    segments, 4 x 6, tau != 1 in the last cavity) takes the staged kernel in
    every mode: fused, graph and per-case runs, the global-load batch and
    single lattices agree bit for bit at tau = 1, and to FP32 rounding for
    the tau != 1 cavity (the kernels' products may contract differently)."""
    probs = _walled_problems()
    rng = np.random.Generator(np.random.PCG64(17))
    fields = [W.random_fields(p, seed=int(rng.integers(1 << 30)), amp_u=2e-3, amp_T=0.3) for p in probs]
    runs = {}
    for mode, staged in (("fused", True), ("graph", True), ("per_case", True), ("fused", False)):
        b = lbm.Batch(probs, "f32")
        assert b.staged
        b.staged = staged
        for c, f in enumerate(fields):
            b.set_fields(c, *f)
        b.step(100, mode)
        b.sync()
        runs[(mode, staged)] = [b.moments(c) for c in range(len(probs))]
        b.close()
    ref = runs[("fused", True)]
    singles = []
    for c, p in enumerate(probs):
        g = lbm.Lattice(p, "f32")
        g.set_fields(*fields[c])
        assert g.staged
        g.step(100)
        singles.append(g.moments())
    for c, p in enumerate(probs):
        tau1 = p["tau_f"] == 1.0 and p["tau_T"] == 1.0
        others = [runs[k][c] for k in runs if k != ("fused", True)] + [singles[c]]
        for m in others:
            for k in ("ux", "uy", "T", "p"):
                if tau1:
                    assert np.array_equal(m[k], ref[c][k]), (c, k)
                else:
                    scale = max(np.abs(ref[c][k]).max(), 1e-12)
                    assert np.abs(m[k] - ref[c][k]).max() <= 1e-5 * scale, (c, k)


def test_staging_is_refused_for_fp64_and_periodic_batches():
    b = lbm.Batch(_mixed_problems(), "f32")  # holds a periodic channel
    assert not b.staged
    with pytest.raises(lbm.LbmError):
        b.staged = True
    b.close()
    b = lbm.Batch(_walled_problems()[:2], "f64")
    assert not b.staged
    with pytest.raises(lbm.LbmError):
        b.staged = True
    b.close()


def test_persistent_batch_matches_the_per_step_launches():
    """The persistent form (every step of a call in one cooperative launch,
    items waiting only on their neighbours' previous step) gives the fused
    staged step's results: bit for bit at tau = 1, to FP32 rounding for the
    tau != 1 cavity; calls of odd and even length keep the buffer parity; the
    workspace guards stay intact; a non-staged batch refuses the mode."""
    probs = _walled_problems()
    rng = np.random.Generator(np.random.PCG64(23))
    fields = [W.random_fields(p, seed=int(rng.integers(1 << 30)), amp_u=2e-3, amp_T=0.3) for p in probs]
    runs = {}
    for mode in ("fused", "persistent"):
        b = lbm.Batch(probs, "f32")
        assert b.staged
        for c, f in enumerate(fields):
            b.set_fields(c, *f)
        for n in (37, 1, 62):
            b.step(n, mode)
        b.sync()
        assert b.steps == 100
        b.check_guards()
        runs[mode] = [b.moments(c) for c in range(len(probs))]
        b.close()
    for c, p in enumerate(probs):
        tau1 = p["tau_f"] == 1.0 and p["tau_T"] == 1.0
        for k in ("ux", "uy", "T", "p"):
            a, r = runs["persistent"][c][k], runs["fused"][c][k]
            if tau1:
                assert np.array_equal(a, r), (c, k)
            else:
                assert np.abs(a - r).max() <= 1e-5 * max(np.abs(r).max(), 1e-12), (c, k)
    b = lbm.Batch(_walled_problems()[:2], "f32")
    b.staged = False
    with pytest.raises(lbm.LbmError):
        b.step(3, "persistent")
    b.close()
