"""FP64 CPU oracle for the RD-CNN FitzHugh-Nagumo update (arXiv 2102.10340).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import this package.
The CUDA product path never imports, links or calls it, and the two share no
code: this package holds its own C source (``rdcnn_oracle.c``), its own
ctypes loader and a second, independent numpy formulation.

Functions and the passages they follow:

* :func:`step`, :func:`run` -- Eq. 1 with Eq. 2-3, Jacobi update, toroidal
  boundary (Sec. II.A-II.C); plain C loops in FP64.
* :func:`step_numpy`, :func:`run_numpy` -- the same model restated as whole-
  array numpy code with ``np.roll`` for the periodic neighbours (the array
  form of Sec. II.D).  A second formulation used to cross-check the C loops.
* ``boundary=ZEROFLUX`` -- no flux across the grid edge (the ghost cell
  beyond an edge holds the edge cell's value); ``reaction=CENN`` -- the
  Chua-Yang cellular neural network cell (output y = (|x+1| - |x-1|)/2,
  feedback centre c, arms Du, offset plane w held in v).  Sec. I and II.A
  present the framework as a template for such models without fixing one;
  both are readings, written out in ``rdcnn_oracle.c``.
* :func:`run_storage`, :func:`step_f32`, :func:`round_to_storage` -- the
  reduced-precision storage variant (16-bit planes, FP32 arithmetic, the
  state rounded to the storage format after every k-step block); not in the
  paper, the arithmetic is Eq. 1-3 in FP32 in their literal order.
* :func:`scalar_map` -- Eq. 1 for an isolated cell (no diffusion term).
* :func:`adjoint` -- exact discrete adjoint of Eq. 1-3 (not in the paper;
  derivation in ``rdcnn_oracle.c``).
* :func:`init_state` -- u = v = k_a x (Eq. 1, first line).
* :func:`summary` -- per-state statistics used to rank the instances of a
  parameter search (Sec. III.A-III.B): plain definitions (mean, population
  variance, min, max, wrapped forward-difference gradient sum, fraction of
  cells above a threshold).

Parity status: every function above is pinned by ``tests/test_oracle_pins.py``
(fixed point, linearisation, Fourier decay, mass conservation, symmetries,
hand-expanded tiny grids, finite differences; :func:`init_state` by products
worked by hand for k_a = 0.75 and -2.5 and by the uncoupled-cell map from
k_a x).  None is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rdcnn_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

FHN = 0
NONE = 1
CENN = 2

PERIODIC = 0
ZEROFLUX = 1

# Sec. II.A: get_init_state() defaults  a=-0.3, b=1.3, eps=-0.1, c=1, Du=0.06, Dv=1, dt=0.1
PARAM_ORDER = ("dt", "a", "b", "eps", "c", "Du", "Dv")

_lock = threading.Lock()
_default = None


def compile_source(src_path: str, out_path: str) -> str:
    """gcc the oracle C source into a shared object (FP contraction off, OpenMP rows)."""
    tmp = out_path + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           "-std=c11", "-o", tmp, src_path, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out_path)
    return out_path


def build(force: bool = False) -> str:
    """Compile ``rdcnn_oracle.c`` into ``liboracle.so`` (skipped when up to date)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    return compile_source(_SRC, _LIB)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def pvec(params: dict) -> np.ndarray:
    """The gene + step as the 7-vector {dt, a, b, eps, c, Du, Dv} (Sec. II.B "Pars")."""
    return np.array([float(params[k]) for k in PARAM_ORDER], dtype=np.float64)


def _plane(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def init_state(x, ka: float = 1.0):
    """u = v = k_a x (Eq. 1, first line)."""
    x = _plane(x)
    u = ka * x
    return u.copy(), u.copy()


class Oracle:
    """ctypes view of one compiled copy of ``rdcnn_oracle.c``."""

    FHN = FHN
    NONE = NONE
    CENN = CENN
    PERIODIC = PERIODIC
    ZEROFLUX = ZEROFLUX

    def __init__(self, lib_path: str):
        lib = ctypes.CDLL(lib_path)
        dp = ctypes.POINTER(ctypes.c_double)
        i64 = ctypes.c_int64
        lib.oracle_step.argtypes = [i64, i64, dp, dp, dp, dp, dp, ctypes.c_int, ctypes.c_int]
        lib.oracle_step.restype = None
        lib.oracle_run.argtypes = [i64, i64, dp, dp, dp, ctypes.c_int, i64, ctypes.c_int]
        lib.oracle_run.restype = ctypes.c_int
        lib.oracle_step_bc.argtypes = [i64, i64, dp, dp, dp, dp, dp, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int]
        lib.oracle_step_bc.restype = None
        lib.oracle_run_bc.argtypes = [i64, i64, dp, dp, dp, ctypes.c_int, ctypes.c_int, i64, ctypes.c_int]
        lib.oracle_run_bc.restype = ctypes.c_int
        lib.oracle_scalar_map.argtypes = [ctypes.c_double, ctypes.c_double, dp, i64, dp, dp, dp, dp]
        lib.oracle_scalar_map.restype = None
        lib.oracle_adjoint.argtypes = [i64, i64, dp, dp, dp, ctypes.c_int, i64, dp, dp, i64,
                                       dp, dp, dp, ctypes.c_int]
        lib.oracle_adjoint.restype = ctypes.c_int
        lib.oracle_adjoint_bc.argtypes = [i64, i64, dp, dp, dp, ctypes.c_int, ctypes.c_int, i64, dp, dp,
                                          i64, dp, dp, dp, ctypes.c_int]
        lib.oracle_adjoint_bc.restype = ctypes.c_int
        lib.oracle_max_threads.argtypes = []
        lib.oracle_max_threads.restype = ctypes.c_int
        self.lib = lib
        self.path = lib_path

    init_state = staticmethod(init_state)

    def max_threads(self) -> int:
        return int(self.lib.oracle_max_threads())

    def step(self, u, v, params: dict, reaction: int = FHN, nthreads: int = 1,
             boundary: int = PERIODIC):
        """One Jacobi application of Eq. 1 on the whole grid (C loops, FP64)."""
        u = _plane(u); v = _plane(v)
        nn, nm = u.shape
        un = np.empty_like(u); vn = np.empty_like(v)
        p = pvec(params)
        if boundary == PERIODIC:
            self.lib.oracle_step(nn, nm, _ptr(u), _ptr(v), _ptr(un), _ptr(vn), _ptr(p), reaction,
                                 nthreads)
        else:
            self.lib.oracle_step_bc(nn, nm, _ptr(u), _ptr(v), _ptr(un), _ptr(vn), _ptr(p), reaction,
                                    boundary, nthreads)
        return un, vn

    def run(self, u, v, params: dict, T: int, reaction: int = FHN, nthreads: int = 1,
            boundary: int = PERIODIC):
        """T applications of Eq. 1 (t = 1..T); returns new arrays (u_T, v_T)."""
        u = _plane(u).copy(); v = _plane(v).copy()
        if u.ndim != 2 or u.shape != v.shape:
            raise ValueError("u and v must be 2-D planes of the same shape")
        nn, nm = u.shape
        p = pvec(params)
        if boundary == PERIODIC:
            rc = self.lib.oracle_run(nn, nm, _ptr(u), _ptr(v), _ptr(p), reaction, int(T), nthreads)
        else:
            rc = self.lib.oracle_run_bc(nn, nm, _ptr(u), _ptr(v), _ptr(p), reaction, boundary, int(T),
                                        nthreads)
        if rc != 0:
            raise RuntimeError("oracle_run failed")
        return u, v

    def scalar_map(self, u0: float, v0: float, params: dict, T: int):
        """Trajectory of one isolated cell under Eq. 1 without diffusion; arrays of length T+1."""
        tu = np.empty(T + 1); tv = np.empty(T + 1)
        ou = ctypes.c_double(); ov = ctypes.c_double()
        p = pvec(params)
        self.lib.oracle_scalar_map(float(u0), float(v0), _ptr(p), int(T), _ptr(tu), _ptr(tv),
                                   ctypes.byref(ou), ctypes.byref(ov))
        return tu, tv

    def adjoint(self, u0, v0, params: dict, T: int, lu_T, lv_T, n_checkpoints: int = 0,
                reaction: int = FHN, nthreads: int = 1, boundary: int = PERIODIC):
        """Reverse-mode derivative of T steps of Eq. 1 (derivation in rdcnn_oracle.c).

        Returns (dL/du0, dL/dv0, grad) with grad = dL/d[Du, Dv, a, b, eps, c], given the
        co-state (lu_T, lv_T) = dL/d(u_T, v_T).  boundary: PERIODIC (the paper's torus) or
        ZEROFLUX.
        """
        u0 = _plane(u0); v0 = _plane(v0); lu_T = _plane(lu_T); lv_T = _plane(lv_T)
        nn, nm = u0.shape
        lu0 = np.empty_like(u0); lv0 = np.empty_like(v0); g = np.zeros(6)
        p = pvec(params)
        rc = self.lib.oracle_adjoint_bc(nn, nm, _ptr(u0), _ptr(v0), _ptr(p), reaction, int(boundary), int(T),
                                        _ptr(lu_T), _ptr(lv_T), int(n_checkpoints), _ptr(lu0), _ptr(lv0),
                                        _ptr(g), nthreads)
        if rc != 0:
            raise RuntimeError("oracle_adjoint failed")
        return lu0, lv0, g

    def step_numpy(self, u, v, params: dict, reaction: int = FHN, boundary: int = PERIODIC):
        return step_numpy(u, v, params, reaction, boundary)

    def run_numpy(self, u, v, params: dict, T: int, reaction: int = FHN, boundary: int = PERIODIC):
        return run_numpy(u, v, params, T, reaction, boundary)

    def summary(self, u, v, threshold: float, precision=np.float64):
        return summary(u, v, threshold, precision)

    def round_to_storage(self, x, storage: str):
        return round_to_storage(x, storage)

    def step_f32(self, u, v, params: dict, reaction: int = FHN, boundary: int = PERIODIC):
        return step_f32(u, v, params, reaction, boundary)

    def run_storage(self, u, v, params: dict, T: int, k: int, storage: str, reaction: int = FHN,
                    boundary: int = PERIODIC):
        return run_storage(u, v, params, T, k, storage, reaction, boundary)


def _get() -> Oracle:
    global _default
    with _lock:
        if _default is None:
            build()
            _default = Oracle(_LIB)
        return _default


def max_threads() -> int:
    return _get().max_threads()


def step(u, v, params: dict, reaction: int = FHN, nthreads: int = 1, boundary: int = PERIODIC):
    return _get().step(u, v, params, reaction, nthreads, boundary)


def run(u, v, params: dict, T: int, reaction: int = FHN, nthreads: int = 1,
        boundary: int = PERIODIC):
    return _get().run(u, v, params, T, reaction, nthreads, boundary)


def scalar_map(u0: float, v0: float, params: dict, T: int):
    return _get().scalar_map(u0, v0, params, T)


def adjoint(u0, v0, params: dict, T: int, lu_T, lv_T, n_checkpoints: int = 0,
            reaction: int = FHN, nthreads: int = 1, boundary: int = PERIODIC):
    return _get().adjoint(u0, v0, params, T, lu_T, lv_T, n_checkpoints, reaction, nthreads, boundary)


# ---------------------------------------------------------------------------
# Second formulation: whole-array numpy (Sec. II.D style, np.roll neighbours).
# Written independently of the C loops above; used only as a cross-check.
# ---------------------------------------------------------------------------

def _neighbours(f: np.ndarray, boundary: int = PERIODIC):
    """(north, south, west, east) neighbour planes: values at rows i-1 / i+1 and
    columns j-1 / j+1.  Periodic: np.roll; zero flux: edge-replicated padding."""
    if boundary == PERIODIC:
        return np.roll(f, 1, axis=0), np.roll(f, -1, axis=0), np.roll(f, 1, axis=1), np.roll(f, -1, axis=1)
    g = np.pad(f, 1, mode="edge")
    return g[:-2, 1:-1], g[2:, 1:-1], g[1:-1, :-2], g[1:-1, 2:]


def _lap_roll(f: np.ndarray, boundary: int = PERIODIC) -> np.ndarray:
    north, south, west, east = _neighbours(f, boundary)
    return north + south + west + east - 4.0 * f


def step_numpy(u, v, params: dict, reaction: int = FHN, boundary: int = PERIODIC):
    u = _plane(u); v = _plane(v)
    dt, a, b, eps, c, Du, Dv = pvec(params)
    if reaction == CENN:
        y = np.clip(u, -1.0, 1.0)                 # the saturating output, as a clamp
        return u + dt * (-u + c * y + Du * sum(_neighbours(y, boundary)) + v), v.copy()
    if reaction == FHN:
        f1 = c * u - u ** 3 / 3.0 - v
        f2 = -eps * (u - b * v + a)
    else:
        f1 = np.zeros_like(u); f2 = np.zeros_like(v)
    return (u + dt * (f1 + Du * _lap_roll(u, boundary)),
            v + dt * (f2 + Dv * _lap_roll(v, boundary)))


def run_numpy(u, v, params: dict, T: int, reaction: int = FHN, boundary: int = PERIODIC):
    for _ in range(int(T)):
        u, v = step_numpy(u, v, params, reaction, boundary)
    return _plane(u), _plane(v)


# ---------------------------------------------------------------------------
# Reduced-precision storage: the state planes are held in a 16-bit format,
# the arithmetic is FP32, and the state is rounded to the storage format at
# the end of every block of k steps (one HBM round trip of a k-step launch).
# Not in the paper (its listings use float32 throughout); the rounding is a
# quantisation, so it is decided on FP32 values as the kernels decide it.
# ---------------------------------------------------------------------------

STORAGE_FORMATS = ("f32", "f16", "bf16")


def round_to_storage(x, storage: str) -> np.ndarray:
    """Round FP32 values to the storage format (nearest, ties to even); returns float32.

    bf16 = the upper 16 bits of an IEEE single (8 exponent bits, 7 fraction bits): add
    0x7FFF plus the lowest kept bit to the 32-bit pattern and clear the low 16 bits.
    f16 = IEEE half (numpy's conversion).  Finite inputs within range only."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    if storage == "f32":
        return x.copy()
    if storage == "f16":
        return x.astype(np.float16).astype(np.float32)
    if storage == "bf16":
        bits = x.view(np.uint32).astype(np.uint64)
        keep_lsb = (bits >> 16) & 1
        rounded = ((bits + 0x7FFF + keep_lsb) & 0xFFFF0000).astype(np.uint32)
        return rounded.view(np.float32)
    raise ValueError(f"storage must be one of {STORAGE_FORMATS}")


def step_f32(u, v, params: dict, reaction: int = FHN, boundary: int = PERIODIC):
    """One application of the update in FP32 (numpy float32 arrays: every operation rounded
    to single precision as written, no fused multiply-add), in the literal form of Eq. 1-3:
    neighbour sum ((n + s) + (w + e)) - 4 centre, f1 = c u - u^3/3 - v, f2 = -eps (u - b v + a);
    the CeNN cell as in step_numpy."""
    u = np.asarray(u, dtype=np.float32)
    v = np.asarray(v, dtype=np.float32)
    dt, a, b, eps, c, Du, Dv = (np.float32(x) for x in pvec(params))
    four, three = np.float32(4.0), np.float32(3.0)
    if reaction == CENN:
        y = np.clip(u, np.float32(-1.0), np.float32(1.0))
        n, s_, w, e = _neighbours(y, boundary)
        feedback = c * y + Du * ((n + s_) + (w + e))
        return u + dt * ((-u + feedback) + v), v.copy()

    def lap(f):
        n, s_, w, e = _neighbours(f, boundary)
        return ((n + s_) + (w + e)) - four * f

    if reaction == FHN:
        f1 = c * u - (u * u * u) / three - v
        f2 = -eps * (u - b * v + a)
    else:
        f1 = np.zeros_like(u)
        f2 = np.zeros_like(v)
    return u + dt * (f1 + Du * lap(u)), v + dt * (f2 + Dv * lap(v))


def run_storage(u, v, params: dict, T: int, k: int, storage: str, reaction: int = FHN,
                boundary: int = PERIODIC):
    """T steps with the state stored in `storage`: the start state is rounded to the format,
    then each block of k steps (the last block may be shorter) runs in FP32 and ends with
    both planes rounded to the format.  Returns float32 arrays."""
    if k < 1:
        raise ValueError("k must be >= 1")
    u = round_to_storage(u, storage)
    v = round_to_storage(v, storage)
    left = int(T)
    while left > 0:
        kk = min(k, left)
        for _ in range(kk):
            u, v = step_f32(u, v, params, reaction, boundary)
        u, v = round_to_storage(u, storage), round_to_storage(v, storage)
        left -= kk
    return u, v


# ---------------------------------------------------------------------------
# Statistics of a state for ranking the instances of a parameter search
# (Sec. III.A sorts (Du, Dv) into slow growth / patterns / dull states).
# ---------------------------------------------------------------------------

SUMMARY_FIELDS = ("mean_u", "var_u", "min_u", "max_u", "mean_v", "var_v", "grad_u", "edge_frac")


def summary(u, v, threshold: float, precision=np.float64) -> np.ndarray:
    """The 8 statistics of (u, v): mean(u), var(u), min(u), max(u), mean(v), var(v),
    mean over cells of g = |u(i+1,j) - u(i,j)| + |u(i,j+1) - u(i,j)| (indices wrap), and
    the fraction of cells with g > threshold.  Sums in FP64; g and the threshold test are
    evaluated in `precision` (the precision the state was computed in), because that test
    turns floating point into a count."""
    u64 = np.asarray(u, dtype=np.float64)
    v64 = np.asarray(v, dtype=np.float64)
    up = np.asarray(u, dtype=precision)
    g = np.abs(np.roll(up, -1, axis=0) - up) + np.abs(np.roll(up, -1, axis=1) - up)
    n = u64.size
    mu, mv = u64.sum() / n, v64.sum() / n
    return np.array([mu, np.sum((u64 - mu) ** 2) / n, u64.min(), u64.max(),
                     mv, np.sum((v64 - mv) ** 2) / n,
                     np.asarray(g, dtype=np.float64).sum() / n,
                     np.count_nonzero(g > np.asarray(threshold, dtype=precision)) / n])
