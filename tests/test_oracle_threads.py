"""The oracle's threaded loops give the single-threaded result bit for bit.

Each node of a step is a function of the previous state alone and is written
to its own slots, so sharing the rows among threads must not change any bit
of any population, moment or gradient.  The cases cover walls of every kind,
a periodic side, a porosity field, a body-force profile, a heat source and
the one-node update entry point."""
import numpy as np
import pytest

import oracle
from paper_1505_02976_gb300 import workloads as W


@pytest.fixture(autouse=True)
def _restore_threads():
    yield
    oracle.set_threads(0)


def _run(p, steps, threads, eps_field=None, ay=None, seed=3):
    oracle.set_threads(threads)
    T, ux, uy = W.random_fields(p, seed=seed, amp_u=2e-3)
    o = oracle.Oracle(p, T=T, ux=ux, uy=uy, eps_field=eps_field, ay_profile=ay).run(steps)
    m, gr = o.moments(), o.gradients()
    rng = np.random.default_rng(seed)
    xs = rng.integers(0, p["nx"], 40).astype(np.int32)
    ys = rng.integers(0, p["ny"], 40).astype(np.int32)
    fo, go = o.update_nodes(xs, ys)
    return o.f.copy(), o.g.copy(), m, gr, fo, go


CASES = [
    ("cavity", W.cavity(37, 1e5, 1e-3, 0.5), None, None),
    ("channel", W.problem(nx=13, ny=29, bc=("periodic", "periodic", "dirichlet", "adiabatic"),
                          T_bc=(0.0, 0.0, 1.0, 0.0), nu=0.05, alpha_e=0.04, gbeta=1e-4, Q=1e-5,
                          eps=0.7, Da=1e-2), None, "ay"),
    ("porosity", W.cavity(24, 1e4, 1e-2, 0.6), "eps", None),
]


@pytest.mark.parametrize("name,p,eps_kind,ay_kind", CASES, ids=[c[0] for c in CASES])
def test_threaded_oracle_is_bit_identical(name, p, eps_kind, ay_kind):
    eps = None
    if eps_kind:
        eps = 0.4 + 0.4 * np.random.default_rng(5).random((p["ny"], p["nx"]))
    ay = 1e-6 * np.sin(np.arange(p["ny"])) if ay_kind else None
    ref = _run(p, 40, 1, eps, ay)
    for th in (2, 5):
        got = _run(p, 40, th, eps, ay)
        assert oracle.threads() == th
        assert np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1])
        for k in ref[2]:
            assert np.array_equal(ref[2][k], got[2][k]), k
        for k in ref[3]:
            assert np.array_equal(ref[3][k], got[3][k]), k
        assert np.array_equal(ref[4], got[4]) and np.array_equal(ref[5], got[5])
    oracle.set_ay_profile(None)


def test_thread_count_control():
    assert oracle.set_threads(3) == 3
    assert oracle.set_threads(0) >= 1
