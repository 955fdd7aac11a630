"""Error of the reduced-precision storage forms against the FP64 path.

``compare(problem, steps)`` advances the same lattice with FP64, FP32 and
FP16 population storage on the GPU and reports, for each reduced form, the
errors of T, u and the hot-wall Nusselt number against the FP64 run.  The
FP64 GPU path itself agrees with the FP64 CPU oracle to 1e-10 (the parity
tests), so these errors are the storage precision's own.
"""
from __future__ import annotations

import numpy as np

from . import lbm


def field_errors(m: dict, ref: dict, nu: float, nu_ref: float) -> dict:
    speed = np.sqrt(ref["ux"] ** 2 + ref["uy"] ** 2)
    du = np.sqrt((m["ux"] - ref["ux"]) ** 2 + (m["uy"] - ref["uy"]) ** 2)
    return {
        "max_abs_dT": float(np.abs(m["T"] - ref["T"]).max()),
        "l2_du_over_l2_u": float(np.linalg.norm(du) / np.linalg.norm(speed)),
        "max_du_over_max_u": float(du.max() / speed.max()),
        "rel_dNu": float(abs(nu - nu_ref) / abs(nu_ref)),
        "Nu": float(nu),
        "Nu_ref": float(nu_ref),
    }


def run(problem: dict, precision: str, steps: int, device: int = 0):
    lat = lbm.Lattice(problem, precision, device=device)
    lat.step(steps)
    lat.sync()
    m = lat.moments()
    nu, _ = lat.nusselt("W")
    lat.close()
    return m, nu


def compare(problem: dict, steps: int, precisions=("f32", "f16"), device: int = 0) -> dict:
    ref, nu_ref = run(problem, "f64", steps, device)
    out = {}
    for p in precisions:
        m, nu = run(problem, p, steps, device)
        out[p] = field_errors(m, ref, nu, nu_ref)
    return out
