"""The reduced-precision storage forms against the FP64 GPU path (itself
within 1e-10 of the oracle), at sizes the oracle cannot run: the 512^2
restriction of the FP16 workload for 20 000 steps, and the 8192^2 FP16
workload itself for 200 steps compared on a 16-stride subsample.

Bounds: FP32 max |dT| <= 1e-4 and ||du||/||u|| <= 1e-3 as in the FP32
parity tests, |dNu|/Nu <= 5e-4 (measured 1.7e-4 after 20 000 steps at 512^2:
the wall gradient of a thin thermal boundary layer is the most sensitive
quantity); FP16 |dNu|/Nu <= 1e-2 with T and u errors below 1e-2 (measured
4.7e-4, 8.3e-4, 1.7e-3: stochastic rounding keeps the stored values exact in
expectation)."""
import numpy as np
import pytest

from paper_1505_02976_gb300 import lbm, precision
from paper_1505_02976_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_fp16_and_fp32_against_fp64_at_512():
    p = W.config_problem(W.CONFIG_FP16_CAVITY, n=512)
    res = precision.compare(p, 20_000)
    f32, f16 = res["f32"], res["f16"]
    print(res)
    assert f32["max_abs_dT"] <= 1e-4 and f32["l2_du_over_l2_u"] <= 1e-3 and f32["rel_dNu"] <= 5e-4
    assert f16["rel_dNu"] <= 1e-2
    assert f16["max_abs_dT"] <= 1e-2 and f16["l2_du_over_l2_u"] <= 1e-2


def test_fp16_against_fp64_at_8192_subsampled():
    p = W.config_problem(W.CONFIG_FP16_CAVITY)
    fields = W.random_fields(p, seed=41, amp_u=2e-3, amp_T=0.3)
    out = {}
    for prec in ("f64", "f16"):
        g = lbm.Lattice(p, prec)
        g.set_fields(*fields)
        g.step(200)
        g.sync()
        m = g.moments()
        out[prec] = {k: m[k][::16, ::16].copy() for k in ("ux", "uy", "T")}
        out[prec]["Nu"] = g.nusselt("W")[0]
        g.close()
        del g, m
    a, b = out["f16"], out["f64"]
    speed = np.sqrt(b["ux"] ** 2 + b["uy"] ** 2)
    du = np.sqrt((a["ux"] - b["ux"]) ** 2 + (a["uy"] - b["uy"]) ** 2)
    assert np.abs(a["T"] - b["T"]).max() <= 1e-2
    assert np.linalg.norm(du) / np.linalg.norm(speed) <= 1e-2
    assert abs(a["Nu"] - b["Nu"]) <= 1e-2 * abs(b["Nu"])
