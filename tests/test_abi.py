"""The C-ABI library loads and exports every entry point that include/*.h
declares; its host-side parameter derivation (no GPU involved) agrees with
the oracle's independent derivation.  Runs without a GPU."""
import ctypes as C
import glob
import math
import os
import re

import numpy as np
import pytest

import oracle
from paper_1505_02976_gb300 import lbm
from paper_1505_02976_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(lbm_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    L = lbm.load()
    declared = _declared()
    assert "lbm_step" in declared and "lbm_create" in declared
    for name in sorted(declared):
        assert hasattr(L, name), f"{name} declared in include/ but not exported"
    assert declared >= set(lbm.EXPORTED)


def test_params_struct_layout_matches_header():
    p = lbm.lbm_params()
    assert lbm.load().lbm_params_default(C.byref(p)) == 0
    assert (p.nx, p.ny) == (32, 32)
    assert list(p.bc) == [1, 1, 2, 2]
    assert p.precision == 1 and p.moment_state == 0
    assert (p.Ra, p.Da, p.eps, p.Pr, p.Ma) == (1e3, 1e-2, 0.6, 1.0, 0.1)
    assert math.isnan(p.A) and math.isnan(p.K)
    assert list(p.T_bc) == [1.0, 0.0, 1.0, 0.0]
    assert C.sizeof(lbm.lbm_params) == 10 * 4 + 8 * (7 + 2 + 7 + 7 + 4 + 8 + 2)


PROBLEMS = [
    W.cavity(32, 1e3, 1e-2, 0.6),
    W.cavity(2048, 1e6, 1e-4, 0.4),
    W.cavity(8192, 1e5, 1e-3, 0.6),
    W.cavity(100, 1e4, 1e8, 0.9999, Pr=0.71),
    W.poiseuille(),
    W.poiseuille(ny=49, A=0.2, nu=0.1, forchheimer=1),
    W.problem(nx=16, ny=16, bc=("periodic",) * 4, da_infinite=1, gbeta=0.0, nu=0.1, B=0.2,
              sigma=1.5),
]


@pytest.mark.parametrize("p", PROBLEMS)
def test_parameter_derivation_agrees_with_oracle(p):
    a = lbm.lbm_derived(p)
    b = oracle.derived(p)
    for k in oracle.DERIVED_KEYS:
        if math.isinf(b[k]):
            assert math.isinf(a[k])
        else:
            assert a[k] == pytest.approx(b[k], rel=1e-15, abs=1e-300), k


def test_parameter_range_is_rejected():
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_derived(W.problem(A=0.6))
    assert e.value.status == -5
    with pytest.raises(lbm.LbmError):
        lbm.lbm_derived(W.problem(eps=0.0))
    with pytest.raises(lbm.LbmError):
        lbm.lbm_derived(W.problem(tau_T=0.5))


def test_workspace_size_and_shape_checks():
    n32 = lbm.lbm_workspace_size(W.cavity(2048, 1e6, 1e-4, 0.4), "f32")
    n16 = lbm.lbm_workspace_size(W.cavity(2048, 1e6, 1e-4, 0.4), "f16")
    n64 = lbm.lbm_workspace_size(W.cavity(2048, 1e6, 1e-4, 0.4), "f64")
    assert n16 < n32 < n64
    # two population buffers of 17 planes are the bulk of the workspace
    assert n32 >= 2 * 17 * 2048 * 2048 * 4
    with pytest.raises(lbm.LbmError):
        lbm.lbm_workspace_size(W.cavity(3, 1e3, 1e-2, 0.6))
    with pytest.raises(lbm.LbmError):
        lbm.lbm_workspace_size(W.problem(bc=("periodic", "dirichlet", "adiabatic", "adiabatic")))


def test_no_cpu_fallback_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(lbm.LbmError):
        lbm.Lattice(W.cavity(32, 1e3, 1e-2, 0.6))


def test_moment_state_parameters_are_checked_on_the_host():
    p = W.cavity(256, 1e6, 1e-4, 0.4)
    pop = lbm.lbm_workspace_size(p, "f32")
    mom = lbm.lbm_workspace_size(p, "f32", "moments")
    plane = 256 * 256 * 4
    # one population buffer (17 planes) for the expansion plus two 9-plane moment buffers
    assert mom - pop == pytest.approx(plane, rel=0.05)
    for bad, prec in ((dict(p, tau_f=0.9), "f32"), (dict(p, tau_T=1.1), "f64"), (p, "f16")):
        with pytest.raises(lbm.LbmError):
            lbm.lbm_workspace_size(bad, prec, "moments")
    with pytest.raises(ValueError):
        lbm.params_from_problem(p, "f32", "other")
