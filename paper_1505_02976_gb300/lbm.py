"""Python binding of the C ABI in ``include/lbm.h`` (ctypes).

Argument marshalling only: every step of the method runs in the CUDA kernels of
``liblbm_gb300.so``.  PyTorch supplies the device workspace and the stream.
The functions keep the C names (``lbm_create``, ``lbm_step``, ...); the
``Lattice`` class wraps one handle.  There is no CPU fallback: without the
built library or a CUDA device every call raises.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

from . import build as _build

LBM_OK = 0
STATUS = {0: "LBM_OK", -1: "LBM_ERR_ARG", -2: "LBM_ERR_CUDA", -3: "LBM_ERR_NONFINITE",
          -4: "LBM_ERR_TIMEOUT", -5: "LBM_ERR_PARAM_RANGE", -6: "LBM_ERR_OOM", -7: "LBM_ERR_GUARD"}
PRECISION = {"f64": 0, "f32": 1, "f16": 2}
BC = {"periodic": 0, "dirichlet": 1, "adiabatic": 2}
SIDE = {"W": 0, "E": 1, "S": 2, "N": 3}

EXPORTED = ("lbm_params_default", "lbm_derived", "lbm_workspace_size", "lbm_create", "lbm_destroy",
            "lbm_last_error", "lbm_set_fields", "lbm_step", "lbm_sync", "lbm_moments", "lbm_nusselt",
            "lbm_residual", "lbm_get_state", "lbm_set_state", "lbm_steps_done",
            "lbm_kernel_launches", "lbm_batch_workspace_size", "lbm_batch_create",
            "lbm_batch_destroy", "lbm_batch_last_error", "lbm_batch_set_fields", "lbm_batch_step",
            "lbm_batch_autotune", "lbm_batch_set_launch", "lbm_batch_sync", "lbm_batch_nusselt",
            "lbm_batch_moments", "lbm_batch_steps_done", "lbm_batch_kernel_launches",
            "lbm_adjoint", "lbm_totals", "lbm_checkpoint", "lbm_set_force_profile",
            "lbm_stream_function", "lbm_set_moment_segments", "lbm_wait_selftest",
            "lbm_set_step_staging", "lbm_step_staged", "lbm_batch_set_staging", "lbm_batch_staged",
            "lbm_check_guards", "lbm_batch_check_guards", "lbm_fp64_peak")
BATCH_MODE = {"fused": 0, "graph": 1, "per_case": 2, "persistent": 3}


class LbmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class lbm_params(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("bc", C.c_int32 * 4),
        ("forchheimer", C.c_int32), ("da_infinite", C.c_int32),
        ("precision", C.c_int32), ("moment_state", C.c_int32),
        ("Ra", C.c_double), ("Pr", C.c_double), ("Da", C.c_double), ("J", C.c_double),
        ("eps", C.c_double), ("sigma", C.c_double), ("Ma", C.c_double),
        ("tau_f", C.c_double), ("tau_T", C.c_double),
        ("Th", C.c_double), ("Tc", C.c_double), ("T_init", C.c_double), ("rho0", C.c_double),
        ("Q", C.c_double), ("ax", C.c_double), ("ay", C.c_double),
        ("L", C.c_double), ("nu", C.c_double), ("alpha_e", C.c_double), ("gbeta", C.c_double),
        ("A", C.c_double), ("B", C.c_double), ("K", C.c_double),
        ("T_bc", C.c_double * 4), ("u_bc", (C.c_double * 2) * 4),
        ("T0", C.c_double), ("Ra_I", C.c_double),
    ]


_lib = None


def load(build_if_missing: bool = True):
    """Load the in-tree library (building it first when it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise LbmError(-2, f"CUDA library not built: {path}")
        _build.build()
    L = C.CDLL(path)
    P = C.POINTER(lbm_params)
    H = C.c_void_p
    dp = C.POINTER(C.c_double)
    L.lbm_params_default.argtypes = [P]
    L.lbm_derived.argtypes = [P, dp]
    L.lbm_workspace_size.argtypes = [P, C.POINTER(C.c_size_t)]
    L.lbm_create.argtypes = [P, C.c_void_p, C.c_void_p, C.c_size_t, C.POINTER(H)]
    L.lbm_destroy.argtypes = [H]
    L.lbm_destroy.restype = None
    L.lbm_last_error.argtypes = [H]
    L.lbm_last_error.restype = C.c_char_p
    L.lbm_set_fields.argtypes = [H, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
    L.lbm_step.argtypes = [H, C.c_int64]
    L.lbm_sync.argtypes = [H]
    L.lbm_wait_selftest.argtypes = [H]
    L.lbm_check_guards.argtypes = [H]
    L.lbm_set_step_staging.argtypes = [H, C.c_int32]
    L.lbm_step_staged.argtypes = [H]
    L.lbm_step_staged.restype = C.c_int32
    L.lbm_moments.argtypes = [H, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
    L.lbm_nusselt.argtypes = [H, C.c_int, dp, C.c_void_p]
    L.lbm_residual.argtypes = [H, dp, dp]
    L.lbm_get_state.argtypes = [H, C.c_void_p, C.c_void_p, C.c_int]
    L.lbm_set_state.argtypes = [H, C.c_void_p, C.c_void_p, C.c_int]
    L.lbm_steps_done.argtypes = [H]
    L.lbm_steps_done.restype = C.c_int64
    L.lbm_kernel_launches.argtypes = [H]
    L.lbm_kernel_launches.restype = C.c_int64
    L.lbm_adjoint.argtypes = [H, C.c_int64, C.c_int64, C.c_int, dp, C.c_void_p, C.c_void_p]
    L.lbm_totals.argtypes = [H, dp, dp]
    L.lbm_checkpoint.argtypes = [H, C.c_char_p, C.c_int]
    L.lbm_set_force_profile.argtypes = [H, C.c_void_p]
    L.lbm_stream_function.argtypes = [H, C.c_void_p, C.c_int, C.c_void_p]
    L.lbm_set_moment_segments.argtypes = [H, C.c_int32]
    L.lbm_fp64_peak.argtypes = [C.c_void_p, dp]
    B = C.c_void_p
    L.lbm_batch_set_staging.argtypes = [B, C.c_int32]
    L.lbm_batch_staged.argtypes = [B]
    L.lbm_batch_staged.restype = C.c_int32
    L.lbm_batch_check_guards.argtypes = [B]
    L.lbm_batch_workspace_size.argtypes = [P, C.c_int32, C.POINTER(C.c_size_t)]
    L.lbm_batch_create.argtypes = [P, C.c_int32, C.c_void_p, C.c_void_p, C.c_size_t, C.POINTER(B)]
    L.lbm_batch_destroy.argtypes = [B]
    L.lbm_batch_destroy.restype = None
    L.lbm_batch_last_error.argtypes = [B]
    L.lbm_batch_last_error.restype = C.c_char_p
    L.lbm_batch_set_fields.argtypes = [B, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]
    L.lbm_batch_step.argtypes = [B, C.c_int64, C.c_int]
    L.lbm_batch_autotune.argtypes = [B, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
    L.lbm_batch_set_launch.argtypes = [B, C.c_int32, C.c_int32]
    L.lbm_batch_sync.argtypes = [B]
    L.lbm_batch_nusselt.argtypes = [B, C.c_int, C.c_void_p]
    L.lbm_batch_moments.argtypes = [B, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    L.lbm_batch_steps_done.argtypes = [B]
    L.lbm_batch_steps_done.restype = C.c_int64
    L.lbm_batch_kernel_launches.argtypes = [B]
    L.lbm_batch_kernel_launches.restype = C.c_int64
    for name in EXPORTED:
        if name not in ("lbm_destroy", "lbm_last_error", "lbm_steps_done", "lbm_kernel_launches", "lbm_step_staged", "lbm_batch_staged",
                        "lbm_batch_destroy", "lbm_batch_last_error", "lbm_batch_steps_done",
                        "lbm_batch_kernel_launches"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _nan(v):
    return float("nan") if v is None else float(v)


STATES = ("populations", "moments")


def params_from_problem(p: dict, precision: str = "f32", state: str = "populations") -> lbm_params:
    """Marshal a problem dict (``workloads.problem``) into ``lbm_params``;
    ``state="moments"`` selects the moment-state storage (tau = 1 only)."""
    s = lbm_params()
    s.nx, s.ny = int(p["nx"]), int(p["ny"])
    for k, b in enumerate(p["bc"]):
        s.bc[k] = BC[b]
    s.forchheimer = int(p["forchheimer"])
    s.da_infinite = int(p["da_infinite"])
    s.precision = PRECISION[precision]
    if state not in STATES:
        raise ValueError(f"state {state!r} not in {STATES}")
    s.moment_state = int(state == "moments")
    for name in ("Ra", "Pr", "Da", "J", "eps", "sigma", "Ma", "tau_f", "tau_T", "Th", "Tc",
                 "T_init", "rho0", "Q", "ax", "ay", "Ra_I"):
        setattr(s, name, float(p[name]))
    for name in ("L", "nu", "alpha_e", "gbeta", "A", "B", "K", "T0"):
        setattr(s, name, _nan(p[name]))
    for k in range(4):
        s.T_bc[k] = float(p["T_bc"][k])
        s.u_bc[k][0] = float(p["u_bc"][k][0])
        s.u_bc[k][1] = float(p["u_bc"][k][1])
    return s


def _check(status: int, handle=None):
    if status != LBM_OK:
        msg = load().lbm_last_error(handle)
        raise LbmError(status, msg.decode() if msg else "")


DERIVED_KEYS = ("L", "T0", "dT", "U", "gbeta", "nu", "nu_e", "alpha_e", "A", "B", "K", "Feps", "Q")


def lbm_derived(p: dict) -> dict:
    out = (C.c_double * 13)()
    _check(load().lbm_derived(C.byref(params_from_problem(p)), out))
    return dict(zip(DERIVED_KEYS, list(out)))


def lbm_workspace_size(p: dict, precision: str = "f32", state: str = "populations") -> int:
    n = C.c_size_t()
    _check(load().lbm_workspace_size(C.byref(params_from_problem(p, precision, state)), C.byref(n)))
    return int(n.value)


def _ptr(a):
    """Device pointer of a torch tensor, or host pointer of a numpy array."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


class Lattice:
    """One lattice on the current CUDA device, advanced by the fused kernel.

    ``Lattice(problem, precision)`` creates the handle with a torch-allocated
    workspace on ``device`` and the current torch stream of that device."""

    def __init__(self, problem: dict, precision: str = "f32", device: int = 0, stream=None,
                 state: str = "populations"):
        import torch

        if not torch.cuda.is_available():
            raise LbmError(-2, "no CUDA device: the library has no CPU path")
        self.lib = load()
        self.problem = dict(problem)
        self.precision = precision
        self.nx, self.ny = int(problem["nx"]), int(problem["ny"])
        self.state = state
        self.params = params_from_problem(problem, precision, state)
        self.device = torch.device("cuda", device)
        nbytes = lbm_workspace_size(problem, precision, state)
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = C.c_void_p()
        _check(self.lib.lbm_create(C.byref(self.params), C.c_void_p(self.stream.cuda_stream),
                                   _ptr(self.workspace), nbytes, C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- state
    def set_fields(self, T=None, ux=None, uy=None, eps_field=None):
        """Initial state from fields (numpy arrays, or float64 CUDA tensors);
        eps_field sets a porosity field (None: the uniform eps)."""
        given = [a for a in (T, ux, uy, eps_field) if a is not None]
        on_dev = any(hasattr(a, "data_ptr") for a in given)
        if on_dev and not all(hasattr(a, "data_ptr") for a in given):
            raise ValueError("fields must all be host arrays or all device tensors")
        conv = (lambda a: a) if on_dev else (lambda a: None if a is None else np.ascontiguousarray(a, np.float64))
        T, ux, uy, eps_field = conv(T), conv(ux), conv(uy), conv(eps_field)
        _check(self.lib.lbm_set_fields(self.h, _ptr(T), _ptr(ux), _ptr(uy), _ptr(eps_field), int(on_dev)),
               self.h)

    def adjoint(self, steps: int, side="W", segment: int = 0, porosity_gradient: bool = True):
        """Run `steps` steps, return (loss, d loss/d eps [ny, nx] or None,
        d loss/d T_bc [4]) for loss = mean Nusselt number on `side`."""
        k = SIDE[side] if isinstance(side, str) else int(side)
        loss = C.c_double()
        g_eps = np.empty((self.ny, self.nx)) if porosity_gradient else None
        g_t = np.empty(4)
        _check(self.lib.lbm_adjoint(self.h, int(steps), int(segment), k, C.byref(loss), _ptr(g_eps),
                                    _ptr(g_t)), self.h)
        return loss.value, g_eps, g_t

    def step(self, n: int = 1):
        _check(self.lib.lbm_step(self.h, int(n)), self.h)

    def sync(self):
        _check(self.lib.lbm_sync(self.h), self.h)

    @property
    def staged(self) -> bool:
        """Whether the next step uses the kernel with TMA-staged rows."""
        return bool(self.lib.lbm_step_staged(self.h))

    @staged.setter
    def staged(self, on: bool):
        _check(self.lib.lbm_set_step_staging(self.h, int(bool(on))), self.h)

    def check_guards(self):
        """Raise LbmError (LBM_ERR_GUARD) if a kernel wrote past the end of
        any workspace region."""
        _check(self.lib.lbm_check_guards(self.h), self.h)

    def wait_selftest(self):
        """Launch the failure-detection self-test: a bounded device-side
        wait that must give up; the next sync raises LBM_ERR_TIMEOUT."""
        _check(self.lib.lbm_wait_selftest(self.h), self.h)

    def moments(self) -> dict:
        shape = (self.ny, self.nx)
        out = {k: np.empty(shape) for k in ("p", "ux", "uy", "T")}
        _check(self.lib.lbm_moments(self.h, _ptr(out["p"]), _ptr(out["ux"]), _ptr(out["uy"]),
                                    _ptr(out["T"]), 0), self.h)
        return out

    def moments_device(self, out: dict):
        """Write the moment fields into float64 torch tensors (asynchronous)."""
        _check(self.lib.lbm_moments(self.h, _ptr(out.get("p")), _ptr(out.get("ux")),
                                    _ptr(out.get("uy")), _ptr(out.get("T")), 1), self.h)

    def nusselt(self, side="W"):
        k = SIDE[side] if isinstance(side, str) else int(side)
        n = self.ny if k <= 1 else self.nx
        loc = np.empty(n)
        mean = C.c_double()
        _check(self.lib.lbm_nusselt(self.h, k, C.byref(mean), _ptr(loc)), self.h)
        return mean.value, loc

    def residual(self):
        ru, rT = C.c_double(), C.c_double()
        _check(self.lib.lbm_residual(self.h, C.byref(ru), C.byref(rT)), self.h)
        return ru.value, rT.value

    def stream_function(self):
        """(psi [ny][nx], (min psi, max psi)): u_x = d psi/dy, psi = 0 on row 0."""
        psi = np.empty((self.ny, self.nx))
        rng = np.empty(2)
        _check(self.lib.lbm_stream_function(self.h, _ptr(psi), 0, _ptr(rng)), self.h)
        return psi, (float(rng[0]), float(rng[1]))

    def set_moment_segments(self, segments: int = 0):
        """Row segments per band of the moment-state step (0: default)."""
        _check(self.lib.lbm_set_moment_segments(self.h, int(segments)), self.h)

    def set_force_profile(self, ay=None):
        """Per-row external acceleration a_y(y) (None removes it)."""
        a = None if ay is None else np.ascontiguousarray(ay, np.float64)
        _check(self.lib.lbm_set_force_profile(self.h, _ptr(a)), self.h)

    def save(self, path: str):
        _check(self.lib.lbm_checkpoint(self.h, os.fsencode(path), 1), self.h)

    def load_checkpoint(self, path: str):
        _check(self.lib.lbm_checkpoint(self.h, os.fsencode(path), 0), self.h)

    def totals(self):
        """(sum of f_1..f_8, sum of g_0..g_8) over the stored state, FP64."""
        sf, sg = C.c_double(), C.c_double()
        _check(self.lib.lbm_totals(self.h, C.byref(sf), C.byref(sg)), self.h)
        return sf.value, sg.value

    def get_state(self):
        shape = (9, self.ny, self.nx)
        f = np.empty(shape)
        g = np.empty(shape)
        _check(self.lib.lbm_get_state(self.h, _ptr(f), _ptr(g), 0), self.h)
        return f, g

    def set_state(self, f, g):
        f = np.ascontiguousarray(f, np.float64)
        g = np.ascontiguousarray(g, np.float64)
        _check(self.lib.lbm_set_state(self.h, _ptr(f), _ptr(g), 0), self.h)

    @property
    def steps(self) -> int:
        return int(self.lib.lbm_steps_done(self.h))

    @property
    def launches(self) -> int:
        return int(self.lib.lbm_kernel_launches(self.h))


def _params_array(problems, precision):
    arr = (lbm_params * len(problems))()
    for k, p in enumerate(problems):
        arr[k] = params_from_problem(p, precision)
    return arr


def lbm_batch_workspace_size(problems, precision: str = "f32") -> int:
    n = C.c_size_t()
    status = load().lbm_batch_workspace_size(_params_array(problems, precision), len(problems), C.byref(n))
    if status != LBM_OK:
        raise LbmError(status, load().lbm_batch_last_error(None).decode())
    return int(n.value)


class Batch:
    """Many cavities advanced together (``lbm_batch_*``).  The stream must
    not be the legacy default stream for graph mode; a private torch stream
    is created when none is given."""

    def __init__(self, problems, precision: str = "f32", device: int = 0, stream=None):
        import torch

        if not torch.cuda.is_available():
            raise LbmError(-2, "no CUDA device: the library has no CPU path")
        self.lib = load()
        self.problems = [dict(p) for p in problems]
        self.n = len(problems)
        self.precision = precision
        self.device = torch.device("cuda", device)
        self.params = _params_array(problems, precision)
        nbytes = lbm_batch_workspace_size(problems, precision)
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        h = C.c_void_p()
        status = self.lib.lbm_batch_create(self.params, self.n, C.c_void_p(self.stream.cuda_stream),
                                           _ptr(self.workspace), nbytes, C.byref(h))
        if status != LBM_OK:
            raise LbmError(status, self.lib.lbm_batch_last_error(None).decode())
        self.h = h

    def _check(self, status):
        if status != LBM_OK:
            raise LbmError(status, self.lib.lbm_batch_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.lbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_fields(self, cavity: int, T=None, ux=None, uy=None):
        conv = lambda a: None if a is None else np.ascontiguousarray(a, np.float64)
        T, ux, uy = conv(T), conv(ux), conv(uy)
        self._check(self.lib.lbm_batch_set_fields(self.h, int(cavity), _ptr(T), _ptr(ux), _ptr(uy)))

    def step(self, n: int = 1, mode: str = "fused"):
        self._check(self.lib.lbm_batch_step(self.h, int(n), BATCH_MODE[mode]))

    def autotune(self, steps_per_candidate: int = 3):
        tx, grid = C.c_int32(), C.c_int32()
        self._check(self.lib.lbm_batch_autotune(self.h, int(steps_per_candidate), C.byref(tx), C.byref(grid)))
        return tx.value, grid.value

    def set_launch(self, tile_x: int, grid: int):
        self._check(self.lib.lbm_batch_set_launch(self.h, int(tile_x), int(grid)))

    def sync(self):
        self._check(self.lib.lbm_batch_sync(self.h))

    def check_guards(self):
        """Raise LbmError (LBM_ERR_GUARD) if a kernel wrote past the end of
        any workspace region."""
        self._check(self.lib.lbm_batch_check_guards(self.h))

    @property
    def staged(self) -> bool:
        """Whether the next step uses the kernel with TMA-staged rows."""
        return bool(self.lib.lbm_batch_staged(self.h))

    @staged.setter
    def staged(self, on: bool):
        self._check(self.lib.lbm_batch_set_staging(self.h, int(bool(on))))

    def nusselt(self, side="W"):
        k = SIDE[side] if isinstance(side, str) else int(side)
        out = np.empty(self.n)
        self._check(self.lib.lbm_batch_nusselt(self.h, k, _ptr(out)))
        return out

    def moments(self, cavity: int) -> dict:
        p = self.problems[cavity]
        shape = (int(p["ny"]), int(p["nx"]))
        out = {k: np.empty(shape) for k in ("p", "ux", "uy", "T")}
        self._check(self.lib.lbm_batch_moments(self.h, int(cavity), _ptr(out["p"]), _ptr(out["ux"]),
                                               _ptr(out["uy"]), _ptr(out["T"])))
        return out

    @property
    def steps(self) -> int:
        return int(self.lib.lbm_batch_steps_done(self.h))

    @property
    def launches(self) -> int:
        return int(self.lib.lbm_batch_kernel_launches(self.h))

    @property
    def cells(self) -> int:
        return sum(int(p["nx"]) * int(p["ny"]) for p in self.problems)


def fp64_peak(stream=None) -> float:
    """FP64 fused multiply-add throughput of the stream's device, FLOP/s
    (lbm_fp64_peak)."""
    out = C.c_double()
    s = None if stream is None else C.c_void_p(stream.cuda_stream)
    _check(load().lbm_fp64_peak(s, C.byref(out)))
    return out.value


def mlups(nx: int, ny: int, steps: int, seconds: float) -> float:
    """Million lattice updates per second, all nodes counted."""
    return nx * ny * steps / seconds / 1e6 if seconds > 0 else math.nan
