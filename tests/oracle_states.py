"""Common input states for the one-step GPU-vs-oracle checks.

The oracle advances its own state from seeded fields; the test then rounds
that state to the GPU's storage type (FP32, or FP16 of value / 2^-10 with the
thermal populations stored as deviations g_i - w_i sigma T0), hands the
rounded populations to lbm_set_state and builds a second oracle on exactly
the same values.  Both sides then take one step from identical stored
inputs, and every input comes from the oracle."""
import numpy as np

import oracle

W_D2Q9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
FP16_SCALE = 2.0 ** -10


def stored_state(p, fields, storage="f64", steps=0, eps_field=None):
    """(oracle on the rounded state, f, g) after `steps` oracle steps."""
    T, ux, uy = fields
    o = oracle.Oracle(p, T=T, ux=ux, uy=uy, eps_field=eps_field)
    if steps:
        o.run(steps)
    f, g = o.f, o.g
    if storage != "f64":
        sT0 = p["sigma"] * oracle.derived(p)["T0"]
        rest = W_D2Q9[:, None, None] * sT0
        if storage == "f32":
            f = f.astype(np.float32).astype(np.float64)
            g = (g - rest).astype(np.float32).astype(np.float64) + rest
        else:
            f = (f / FP16_SCALE).astype(np.float16).astype(np.float64) * FP16_SCALE
            g = ((g - rest) / FP16_SCALE).astype(np.float16).astype(np.float64) * FP16_SCALE + rest
    f = np.ascontiguousarray(f)
    g = np.ascontiguousarray(g)
    f[0] = 0.0  # f_0 is never read (the GPU does not store it)
    return oracle.Oracle.from_state(p, f, g, eps_field=eps_field, copy=False), f, g


def sample_nodes(nx, ny, count, seed):
    """Random nodes plus every corner and a few nodes next to the walls."""
    rng = np.random.Generator(np.random.PCG64(seed))
    xs = np.r_[rng.integers(0, nx, count), 0, 0, nx - 1, nx - 1, 1, 2, nx - 2].astype(np.int32)
    ys = np.r_[rng.integers(0, ny, count), 0, ny - 1, 0, ny - 1, 0, ny - 1, 1].astype(np.int32)
    return xs, ys
