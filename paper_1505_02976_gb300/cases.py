"""Run one of the measured workloads from the command line (used for
profiling captures and quick timings).

  python -m paper_1505_02976_gb300.cases step    --n 2048 --precision f32 --steps 10
  python -m paper_1505_02976_gb300.cases batch   --count 128 --steps 10
  python -m paper_1505_02976_gb300.cases adjoint --n 256 --steps 200

Prints one line with the achieved MLUPS (CUDA events on the workload's
stream).  Workloads: the porous cavity of Sec. 4.2 (``step``: Ra 1e6,
Da 1e-4, eps 0.4 for FP32/FP64, Ra 1e5, Da 1e-3, eps 0.6 for FP16), the
benchmark's batch of uneven cavities (``batch``), and the differentiation
workload with a random porosity field (``adjoint``).
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


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("case", choices=("step", "batch", "adjoint"))
    ap.add_argument("--n", type=int, default=2048)
    ap.add_argument("--precision", default="f32", choices=("f64", "f32", "f16"))
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--count", type=int, default=128)
    a = ap.parse_args(argv)
    stream = torch.cuda.Stream()
    if a.case == "step":
        p = (W.cavity(a.n, 1e5, 1e-3, 0.6) if a.precision == "f16" else W.cavity(a.n, 1e6, 1e-4, 0.4))
        lat = lbm.Lattice(p, a.precision, stream=stream)
        lat.step(a.warmup)
        sec = _timed(stream, lambda: lat.step(a.steps))
        out = dict(case="step", n=a.n, precision=a.precision, MLUPS=a.n * a.n * a.steps / sec / 1e6)
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
