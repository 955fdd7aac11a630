"""Python access to the FP64 CPU oracle (``lbm_oracle.c``).

TEST INFRASTRUCTURE.  The oracle is the independent, plain and slow
implementation of the paper's evolution equations that the CUDA path is
checked against.  Only the test suite, the smoke check and the CPU-baseline
leg of the benchmark may import this package.  It never imports the CUDA
library or its binding, and the library never imports it.

Problems are the plain dicts of ``paper_1505_02976_gb300.workloads``; they are
marshalled here into the oracle's own C struct.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_CS_LIB_PATH = os.path.join(_OUT_DIR, "liboracle_cs.so")
_lock = threading.Lock()
_lib = None
_cs_lib = None

_BC = {"periodic": 0, "dirichlet": 1, "adiabatic": 2}
SIDE = {"W": 0, "E": 1, "S": 2, "N": 3}


class _Problem(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("bc", C.c_int32 * 4),
        ("forchheimer", C.c_int32), ("da_infinite", C.c_int32),
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


def _compile(out: str, extra=()) -> str:
    if os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(_OUT_DIR, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-std=c99",
                    *extra, "-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library (plain gcc, -O2, no FMA
    contraction, no target-specific flags, OpenMP over the rows of a step),
    and its complex-step twin."""
    with _lock:
        if force:
            for f in (_LIB_PATH, _CS_LIB_PATH):
                if os.path.exists(f):
                    os.remove(f)
        _compile(_CS_LIB_PATH, ("-DORC_COMPLEX",))
        return _compile(_LIB_PATH)


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
        ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
        P = C.POINTER(_Problem)
        vp = C.c_void_p
        L.orc_lattice.argtypes = [ip, ip, dp, dp]
        L.orc_derived_values.argtypes = [P, dp]
        L.orc_cell_eval.argtypes = [P, C.c_int, C.c_double, C.c_double, dp, C.c_double, dp, dp, dp, dp]
        L.orc_cell_moments.argtypes = [P, C.c_double, dp, dp, dp]
        L.orc_cell_velocity.argtypes = [P, C.c_double, dp, dp, dp]
        L.orc_init.argtypes = [P, vp, vp, vp, vp, dp, dp]
        L.orc_run.argtypes = [P, vp, dp, dp, C.c_int64]
        L.orc_update_nodes.argtypes = [P, vp, dp, dp, C.c_int64, ip, ip, dp, dp]
        L.orc_moments.argtypes = [P, vp, dp, dp, vp, vp, vp, vp]
        L.orc_gradients.argtypes = [P, vp, dp, dp, dp, dp, dp, dp, dp]
        L.orc_nusselt.argtypes = [P, dp, C.c_int, vp, C.POINTER(C.c_double)]
        L.orc_residual.argtypes = [C.c_int64, dp, dp, dp, dp, dp, dp, dp]
        L.orc_stream_function.argtypes = [C.c_int, C.c_int, dp, dp]
        L.orc_totals.argtypes = [P, dp, dp, dp]
        L.orc_set_ay_profile.argtypes = [vp, C.c_int]
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_get_threads.argtypes = []
        _lib = L
    return _lib


def cs_lib():
    """The oracle compiled over complex numbers (complex-step derivatives)."""
    global _cs_lib
    if _cs_lib is None:
        build()
        L = C.CDLL(_CS_LIB_PATH)
        cp = np.ctypeslib.ndpointer(dtype=np.complex128, flags="C_CONTIGUOUS")
        dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
        P = C.POINTER(_Problem)
        vp = C.c_void_p
        L.orc_cs_set_tbc_imag.argtypes = [dp]
        L.orc_init.argtypes = [P, vp, vp, vp, vp, cp, cp]
        L.orc_run.argtypes = [P, vp, cp, cp, C.c_int64]
        L.orc_moments.argtypes = [P, vp, cp, cp, vp, vp, vp, vp]
        L.orc_nusselt.argtypes = [P, cp, C.c_int, vp, vp]
        L.orc_set_ay_profile.argtypes = [vp, C.c_int]
        L.orc_set_threads.argtypes = [C.c_int]
        _cs_lib = L
    return _cs_lib


def complex_step_nusselt(p: dict, steps: int, eps_field=None, tbc_imag=(0.0, 0.0, 0.0, 0.0),
                         T=None, ux=None, uy=None, side: str = "W"):
    """Mean Nusselt number on `side` after `steps` steps, evaluated in
    complex arithmetic.  eps_field may be complex (a perturbed cell carries
    i h); tbc_imag adds i h to Dirichlet wall temperatures.  Returns the
    complex Nu: its imaginary part / h is the exact discrete derivative."""
    L = cs_lib()
    s = problem_struct(p)
    nx, ny = int(p["nx"]), int(p["ny"])
    c = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.complex128)
    eps_c = c(eps_field)
    L.orc_cs_set_tbc_imag(np.ascontiguousarray(tbc_imag, dtype=np.float64))
    f = np.zeros((9, ny, nx), np.complex128)
    g = np.zeros((9, ny, nx), np.complex128)
    rc = L.orc_init(C.byref(s), _ptr(c(T)), _ptr(c(ux)), _ptr(c(uy)), _ptr(eps_c), f, g)
    if rc:
        raise ValueError(f"oracle rejected the problem (code {rc})")
    rc = L.orc_run(C.byref(s), _ptr(eps_c), f, g, int(steps))
    if rc:
        raise RuntimeError(f"oracle run failed (code {rc})")
    Tf = np.zeros((ny, nx), np.complex128)
    L.orc_moments(C.byref(s), _ptr(eps_c), f, g, None, None, None, _ptr(Tf))
    mean = np.zeros(1, np.complex128)
    L.orc_nusselt(C.byref(s), Tf, SIDE[side], None, _ptr(mean))
    L.orc_cs_set_tbc_imag(np.zeros(4))
    return complex(mean[0])


def nusselt_gradient(p: dict, steps: int, eps_field, cells, sides=("W", "E"), h: float = 1e-30,
                     T=None, ux=None, uy=None, loss_side: str = "W"):
    """Exact discrete derivatives of the mean Nusselt number on `loss_side`
    after `steps` steps with respect to eps at each (x, y) in `cells` and to
    the Dirichlet temperature of each side in `sides`, by the complex-step
    method (one complex run per derivative)."""
    base = np.asarray(eps_field, dtype=np.float64)
    d_eps = []
    for (x, y) in cells:
        e = base.astype(np.complex128)
        e[y, x] += 1j * h
        d_eps.append(complex_step_nusselt(p, steps, e, T=T, ux=ux, uy=uy, side=loss_side).imag / h)
    d_t = {}
    for side in sides:
        im = [0.0, 0.0, 0.0, 0.0]
        im[SIDE[side]] = h
        d_t[side] = complex_step_nusselt(p, steps, base, tuple(im), T=T, ux=ux, uy=uy,
                                         side=loss_side).imag / h
    return np.array(d_eps), d_t


def set_threads(n: int = 0) -> int:
    """Threads for the oracle's loops over nodes (0: one per processor, the
    default); returns the count now in use.  The result of every call is the
    same bit for bit whatever the count (each node of a step depends on the
    previous state alone; sums stay single-threaded)."""
    lib().orc_set_threads(int(n))
    cs_lib().orc_set_threads(int(n))
    return int(lib().orc_get_threads())


def threads() -> int:
    return int(lib().orc_get_threads())


def set_ay_profile(ay, complex_build: bool = False):
    """External acceleration a_y(y) per row (None: none) for the next calls."""
    L = cs_lib() if complex_build else lib()
    if ay is None:
        L.orc_set_ay_profile(None, 0)
    else:
        a = np.ascontiguousarray(ay, dtype=np.float64)
        L.orc_set_ay_profile(a.ctypes.data_as(C.c_void_p), a.size)


def _nan_or(v):
    return float("nan") if v is None else float(v)


def problem_struct(p: dict) -> _Problem:
    s = _Problem()
    s.nx, s.ny = int(p["nx"]), int(p["ny"])
    for k, b in enumerate(p["bc"]):
        s.bc[k] = _BC[b]
    s.forchheimer = int(p["forchheimer"])
    s.da_infinite = int(p["da_infinite"])
    for name in ("Ra", "Pr", "Da", "J", "eps", "sigma", "Ma", "tau_f", "tau_T", "Th", "Tc",
                 "T_init", "rho0", "Q", "ax", "ay", "Ra_I"):
        setattr(s, name, float(p[name]))
    for name in ("L", "nu", "alpha_e", "gbeta", "A", "B", "K", "T0"):
        setattr(s, name, _nan_or(p[name]))
    for k in range(4):
        s.T_bc[k] = float(p["T_bc"][k])
        s.u_bc[k][0] = float(p["u_bc"][k][0])
        s.u_bc[k][1] = float(p["u_bc"][k][1])
    return s


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def lattice():
    cx = np.zeros(9, np.int32); cy = np.zeros(9, np.int32)
    w = np.zeros(9); varpi = np.zeros(9)
    lib().orc_lattice(cx, cy, w, varpi)
    return cx, cy, w, varpi


DERIVED_KEYS = ("L", "T0", "dT", "U", "gbeta", "nu", "nu_e", "alpha_e", "A", "B", "K", "Feps", "Q")


def derived(p: dict) -> dict:
    out = np.zeros(13)
    s = problem_struct(p)
    rc = lib().orc_derived_values(C.byref(s), out)
    if rc:
        raise ValueError(f"oracle rejected the problem (code {rc})")
    return dict(zip(DERIVED_KEYS, out.tolist()))


CELL_FUNCS = {"feq0": 0, "feq": 1, "F": 2, "geq0": 3, "geq": 4, "P": 5, "Q": 6}


def cell_eval(p: dict, which: str, eps: float, T=0.0, u=(0.0, 0.0), pr=0.0,
              S=((0.0, 0.0), (0.0, 0.0)), F=(0.0, 0.0), gradT=(0.0, 0.0)) -> np.ndarray:
    out = np.zeros(9)
    s = problem_struct(p)
    rc = lib().orc_cell_eval(C.byref(s), CELL_FUNCS[which], float(eps), float(T),
                             np.asarray(u, float), float(pr), np.asarray(S, float).reshape(4).copy(),
                             np.asarray(F, float), np.asarray(gradT, float), out)
    if rc:
        raise ValueError(f"oracle rejected the problem (code {rc})")
    return out


def cell_moments(p: dict, eps: float, fs, gs) -> dict:
    out = np.zeros(12)
    s = problem_struct(p)
    rc = lib().orc_cell_moments(C.byref(s), float(eps), _c64(fs), _c64(gs), out)
    if rc:
        raise ValueError(f"oracle rejected the problem (code {rc})")
    return dict(T=out[0], u=out[1:3].copy(), F=out[3:5].copy(), p=out[5],
                S=out[6:10].reshape(2, 2).copy(), gradT=out[10:12].copy())


def cell_velocity(p: dict, eps: float, v):
    out = np.zeros(2); c01 = np.zeros(2)
    s = problem_struct(p)
    lib().orc_cell_velocity(C.byref(s), float(eps), np.asarray(v, float), out, c01)
    return out, c01[0], c01[1]


def residual(ux, uy, T, ux0, uy0, T0):
    out = np.zeros(2)
    a = [_c64(np.ravel(v)) for v in (ux, uy, T, ux0, uy0, T0)]
    lib().orc_residual(a[0].size, *a, out)
    return float(out[0]), float(out[1])


def stream_function(ux):
    """psi [ny][nx] of u_x [ny][nx] (zero on row 0, trapezoid rule up the columns)."""
    u = _c64(ux)
    ny, nx = u.shape
    psi = np.zeros((ny, nx))
    lib().orc_stream_function(nx, ny, u, psi)
    return psi


class Oracle:
    """A lattice advanced by the oracle.  State: post-collision populations
    f[9][ny][nx], g[9][ny][nx] (float64)."""

    def __init__(self, p: dict, T=None, ux=None, uy=None, eps_field=None, ay_profile=None):
        self.ay_profile = None if ay_profile is None else np.ascontiguousarray(ay_profile, np.float64)
        self.p = dict(p)
        self.s = problem_struct(p)
        self.nx, self.ny = int(p["nx"]), int(p["ny"])
        self.eps_field = _c64(eps_field)
        shape = (9, self.ny, self.nx)
        self.f = np.zeros(shape)
        self.g = np.zeros(shape)
        rc = lib().orc_init(C.byref(self.s), _ptr(_c64(T)), _ptr(_c64(ux)), _ptr(_c64(uy)),
                            _ptr(self.eps_field), self.f, self.g)
        if rc:
            raise ValueError(f"oracle rejected the problem (code {rc})")
        self.steps = 0

    @classmethod
    def from_state(cls, p: dict, f, g, eps_field=None, copy: bool = True):
        """An oracle lattice holding the given post-collision populations
        (copy=False adopts contiguous float64 arrays without copying)."""
        o = cls.__new__(cls)
        o.p = dict(p)
        o.s = problem_struct(p)
        o.nx, o.ny = int(p["nx"]), int(p["ny"])
        o.eps_field = _c64(eps_field)
        o.ay_profile = None
        o.steps = 0
        derived(p)  # validates the problem
        if copy:
            o.set_state(f, g)
        else:
            o.f = np.ascontiguousarray(f, dtype=np.float64)
            o.g = np.ascontiguousarray(g, dtype=np.float64)
        return o

    def set_state(self, f, g):
        self.f = np.ascontiguousarray(f, dtype=np.float64).copy()
        self.g = np.ascontiguousarray(g, dtype=np.float64).copy()

    def run(self, n: int):
        set_ay_profile(self.ay_profile)
        rc = lib().orc_run(C.byref(self.s), _ptr(self.eps_field), self.f, self.g, int(n))
        if rc:
            raise RuntimeError(f"oracle run failed (code {rc})")
        self.steps += int(n)
        return self

    def update_nodes(self, xs, ys):
        set_ay_profile(self.ay_profile)
        xs = np.ascontiguousarray(xs, np.int32); ys = np.ascontiguousarray(ys, np.int32)
        fo = np.zeros((xs.size, 9)); go = np.zeros((xs.size, 9))
        lib().orc_update_nodes(C.byref(self.s), _ptr(self.eps_field), self.f, self.g,
                               xs.size, xs, ys, fo, go)
        return fo, go

    def moments(self):
        set_ay_profile(self.ay_profile)
        shape = (self.ny, self.nx)
        p = np.zeros(shape); ux = np.zeros(shape); uy = np.zeros(shape); T = np.zeros(shape)
        lib().orc_moments(C.byref(self.s), _ptr(self.eps_field), self.f, self.g,
                          _ptr(p), _ptr(ux), _ptr(uy), _ptr(T))
        return dict(p=p, ux=ux, uy=uy, T=T)

    def gradients(self):
        set_ay_profile(self.ay_profile)
        shape = (self.ny, self.nx)
        out = [np.zeros(shape) for _ in range(5)]
        lib().orc_gradients(C.byref(self.s), _ptr(self.eps_field), self.f, self.g, *out)
        return dict(Sxx=out[0], Sxy=out[1], Syy=out[2], dTdx=out[3], dTdy=out[4])

    def nusselt(self, side="W", T=None):
        if T is None:
            T = self.moments()["T"]
        T = _c64(T)
        k = SIDE[side] if isinstance(side, str) else int(side)
        n = self.ny if k <= 1 else self.nx
        loc = np.zeros(n)
        mean = C.c_double()
        rc = lib().orc_nusselt(C.byref(self.s), T, k, _ptr(loc), C.byref(mean))
        if rc:
            raise ValueError(f"oracle rejected the problem (code {rc})")
        return mean.value, loc

    def totals(self):
        out = np.zeros(2)
        lib().orc_totals(C.byref(self.s), self.f, self.g, out)
        return float(out[0]), float(out[1])
