"""Run one of the measured workloads from the command line (used for
profiling captures and quick timings).

  python -m paper_1505_02976_gb300.cases step    --n 2048 --precision f32 --steps 10
  python -m paper_1505_02976_gb300.cases batch   --count 128 --steps 10
  python -m paper_1505_02976_gb300.cases adjoint --n 256 --steps 200
  python -m paper_1505_02976_gb300.cases table   --table 4 --cap 8000000

Prints one line with the achieved MLUPS (CUDA events on the workload's
stream).  Workloads: the porous cavity of Sec. 4.2 (``step``: Ra 1e6,
Da 1e-4, eps 0.4 for FP32/FP64, Ra 1e5, Da 1e-3, eps 0.6 for FP16), the
benchmark's batch of uneven cavities (``batch``), and the differentiation
workload with a random porosity field (``adjoint``).  ``table`` runs the
cases of the paper's Table 1, 3 or 4 to the steady state of Sec. 4 (or
--cap steps) and prints the tabulated quantities, one JSON line per case.
"""
from __future__ import annotations

import argparse
import json
import time

import torch

from . import lbm
from . import workloads as W


def _timed(stream, fn):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / 1e3


def _steady(p, precision, cap, tol=1e-6):
    g = lbm.Lattice(p, precision)
    g.residual()
    n, r = 0, (1.0, 1.0)
    while n < cap:
        g.step(100)
        n += 100
        r = g.residual()
        if max(r) < tol:
            break
    return g, n, r


def table_rows(which: int, precision: str, cap: int):
    """Yield one dict per case of Table `which` (1, 3 or 4): the steady
    quantities the paper tabulates for it ("N x N" grids are N + 1 nodes)."""
    if which == 1:
        for Ra, N in ((1e3, 100), (1e4, 150), (1e5, 200), (1e6, 200)):
            n = N + 1
            p = W.clear_fluid_cavity(n, Ra)
            d = lbm.lbm_derived(p)
            g, steps, r = _steady(p, precision, cap)
            m = g.moments()
            c, sc = (n - 1) // 2, d["L"] / d["alpha_e"]
            col, row = m["ux"][:, c] * sc, m["uy"][c, :] * sc
            nu, loc = g.nusselt("E")
            yield dict(table=1, Ra=Ra, N=N, steps=steps, residual=r, u_max=float(col.max()),
                       y_max=float(col.argmax() / d["L"]), v_max=float(row.max()),
                       x_max=float(row.argmax() / d["L"]), Nu_max=float(loc.max()),
                       y_Nu=float(loc.argmax() / d["L"]), Nu=nu)
    elif which == 3:
        for Da in (float("inf"), 1e-2, 1e-4):
            p = W.heat_generating_cavity(121, Da, Pr=7.0)
            d = lbm.lbm_derived(p)
            g, steps, r = _steady(p, precision, cap)
            _, (lo, hi) = g.stream_function()
            yield dict(table=3, Da=Da, steps=steps, residual=r,
                       psi_max=max(abs(lo), abs(hi)) / (d["L"] * d["U"]),
                       theta_max=float((g.moments()["T"].max() - d["T0"]) / d["dT"]))
    else:
        for Ra, Ra_I in ((1e5, 1e3), (1e5, 1e5), (1e5, 1e7), (1e6, 1e7)):
            for Da in (1e8, 1e-2, 1e-4, 1e-6):
                p = W.heated_cavity_with_source(151 if Ra == 1e5 else 201, Ra, Ra_I, Da,
                                                eps=0.9999 if Da >= 1e8 else 0.4)
                d = lbm.lbm_derived(p)
                try:
                    g, steps, r = _steady(p, precision, cap)
                    g.sync()
                except lbm.LbmError as e:
                    yield dict(table=4, Ra=Ra, Ra_I=Ra_I, Da=Da, diverged=str(e))
                    continue
                yield dict(table=4, Ra=Ra, Ra_I=Ra_I, Da=Da, steps=steps, residual=r,
                           Nu=g.nusselt("W")[0],
                           theta_max=float((g.moments()["T"].max() - d["T0"]) / d["dT"]))


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("case", choices=("step", "batch", "adjoint", "table"))
    ap.add_argument("--table", type=int, default=1, choices=(1, 3, 4))
    ap.add_argument("--cap", type=int, default=2_000_000, help="step cap of a table case")
    ap.add_argument("--state", default="populations", choices=lbm.STATES)
    ap.add_argument("--n", type=int, default=2048)
    ap.add_argument("--precision", default="f32", choices=("f64", "f32", "f16"))
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--count", type=int, default=128)
    a = ap.parse_args(argv)
    if a.case == "table":
        for row in table_rows(a.table, a.precision, a.cap):
            print(json.dumps(row), flush=True)
        return 0
    stream = torch.cuda.Stream()
    if a.case == "step":
        p = (W.cavity(a.n, 1e5, 1e-3, 0.6) if a.precision == "f16" else W.cavity(a.n, 1e6, 1e-4, 0.4))
        lat = lbm.Lattice(p, a.precision, stream=stream, state=a.state)
        lat.step(a.warmup)
        sec = _timed(stream, lambda: lat.step(a.steps))
        out = dict(case="step", n=a.n, precision=a.precision, state=a.state,
                   MLUPS=a.n * a.n * a.steps / sec / 1e6)
    elif a.case == "batch":
        b = lbm.Batch(W.batch_cavities(a.count), "f32", stream=stream)
        b.step(a.warmup, "fused")
        sec = _timed(stream, lambda: b.step(a.steps, "fused"))
        out = dict(case="batch", cavities=a.count, nodes=b.cells, MLUPS=b.cells * a.steps / sec / 1e6)
    else:
        p = W.cavity(a.n, 1e5, 1e-3, 0.6)
        lat = lbm.Lattice(p, a.precision if a.precision != "f16" else "f32", stream=stream)
        lat.set_fields(eps_field=W.gaussian_random_field(a.n, corr=16.0, seed=1))
        t0 = time.perf_counter()
        loss, _, _ = lat.adjoint(a.steps)
        sec = time.perf_counter() - t0
        out = dict(case="adjoint", n=a.n, steps=a.steps, seconds=sec, loss=loss,
                   MLUPS=a.n * a.n * a.steps / sec / 1e6)
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
