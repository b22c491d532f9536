"""FP64 CPU oracle for the 4D GSUBSURF segmentation scheme (arXiv 2111.11866).

TEST INFRASTRUCTURE ONLY.  This package may be imported by ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` -- nothing in the product path may use it.  It shares no
code with the CUDA implementation: the arithmetic lives in
``seg4d_oracle.c`` (plain C, double precision, built with gcc
``-ffp-contract=off``); this module only builds it and marshals numpy arrays.

Array conventions: compact interior arrays of shape (n4, n3, n2, n1) (C order,
so x is fastest, as the 4D->1D map of Section 3.7); face arrays carry a last
axis of 8 faces ordered f = 2*d + (side > 0) for axes d = x1..x4.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "seg4d_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libseg4d_oracle.so")
_LIB_OMP = os.path.join(_BUILD, "libseg4d_oracle_omp.so")
_lock = threading.Lock()
_libs = {}

OR_OK = 0
OR_NOT_CONVERGED = 1


def build(force: bool = False, omp: bool = False) -> str:
    """Compile the oracle shared library (a few seconds, gcc only).  omp: the
    separate OpenMP build whose sweeps follow the paper's frame-split
    red-black scheme -- a timed CPU baseline only; the tests use the plain
    build."""
    os.makedirs(_BUILD, exist_ok=True)
    out = _LIB_OMP if omp else _LIB
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-std=c99", "-Wall", "-o", tmp, _SRC, "-lm"]
        if omp:
            cmd[1:1] = ["-fopenmp", "-DSEG4D_ORACLE_OMP"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return out


class Params(C.Structure):
    _fields_ = [("h", C.c_double * 4), ("tau", C.c_double), ("eps", C.c_double),
                ("K", C.c_double), ("delta", C.c_double), ("vartheta", C.c_double),
                ("lambda_th", C.c_double), ("r_ball", C.c_double), ("R_init", C.c_double),
                ("v_init", C.c_double), ("sigma_t", C.c_double), ("omega", C.c_double),
                ("tol", C.c_double), ("omega_smooth", C.c_double),
                ("max_iters", C.c_int), ("check_every", C.c_int)]


@dataclass
class OracleParams:
    """Parameters of one segmentation run (Section 4 lists the paper's values:
    delta = vartheta = 0.5, h = 0.01, tau = 0.01, eps = 1, sigma = h^2/8, R = 12,
    and 0.87 / 0.13 read as lambda and 1 - lambda)."""
    h: tuple = (0.01, 0.01, 0.01, 0.01)
    tau: float = 0.01
    eps: float = 1.0
    K: float = 1.0
    delta: float = 0.5
    vartheta: float = 0.5
    lambda_th: float = 0.87
    r_ball: float = 12.0
    R_init: float = 12.0
    v_init: float = 1.0
    sigma_t: float = 0.01 ** 2 / 8.0
    omega: float = 1.8
    tol: float = 1e-12
    omega_smooth: float = 1.0
    max_iters: int = 100000
    check_every: int = 4

    def c_struct(self) -> Params:
        p = Params()
        p.h = (C.c_double * 4)(*[float(x) for x in self.h])
        for name in ("tau", "eps", "K", "delta", "vartheta", "lambda_th", "r_ball", "R_init",
                     "v_init", "sigma_t", "omega", "tol", "omega_smooth"):
            setattr(p, name, float(getattr(self, name)))
        p.max_iters = int(self.max_iters)
        p.check_every = int(self.check_every)
        return p


def lib(omp: bool = False):
    with _lock:
        if omp not in _libs:
            L = C.CDLL(build(omp=omp))
            D = C.POINTER(C.c_double)
            I = C.POINTER(C.c_int)
            sig = {
                "or_face_grad_sq": [I, D, D, C.c_int, D],
                "or_owner": [I, D, I, C.c_int, C.c_double, I],
                "or_threshold": [I, D, D, I, C.c_int, C.c_double, C.c_double, D],
                "or_solve": [I, D, D, D, D, C.c_double, C.c_double, C.c_int, C.c_int, I, D],
                "or_residual": [I, D, D, D, D, D],
                "or_presmooth": [I, D, D, C.c_double, C.c_double, C.c_double, C.c_int, C.c_int,
                                 D, I, D],
                "or_face_G": [I, D, D, D, C.c_double, C.c_double, C.c_double, D],
                "or_init_u": [I, D, I, C.c_int, C.c_double, C.c_double, D],
                "or_rescale": [I, D, D, I, C.c_int, C.c_double],
                "or_assemble": [I, D, D, D, C.c_double, C.c_double, D, D],
                "or_segment": [I, D, D, I, C.c_int, C.POINTER(Params), C.c_int, D, I, D],
                "or_eoc": [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double,
                           C.c_double, C.c_double, C.c_double, C.c_int, D, D, I],
            }
            for name, args in sig.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = C.c_int
            L.or_threads.argtypes = []
            L.or_threads.restype = C.c_int
            _libs[omp] = L
    return _libs[omp]


def threads(omp: bool = False) -> int:
    """Threads the sweeps of that build use."""
    return int(lib(omp).or_threads())


# --------------------------------------------------------------------------
# marshalling helpers
# --------------------------------------------------------------------------

def _dims(shape) -> C.Array:
    if len(shape) != 4:
        raise ValueError("expected a 4D array of shape (n4, n3, n2, n1)")
    n4, n3, n2, n1 = shape
    return (C.c_int * 4)(n1, n2, n3, n4)


def _d(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _seeds(seeds):
    """seeds: sequence of (x, y, z, frame) in 0-based interior voxel units."""
    s = np.asarray(seeds, dtype=np.float64).reshape(-1, 4)
    xyz = np.ascontiguousarray(s[:, :3])
    fr = np.ascontiguousarray(s[:, 3].astype(np.int32))
    if xyz.shape[0] == 0:
        xyz = np.zeros((1, 3))
        fr = np.full(1, -1, dtype=np.int32)
        return xyz, fr, 0
    return xyz, fr, int(s.shape[0])


def _hv(h) -> np.ndarray:
    if np.isscalar(h):
        h = (h, h, h, h)
    return _f64(np.asarray(h, dtype=np.float64).reshape(4))


# --------------------------------------------------------------------------
# public functions (each wraps one C routine)
# --------------------------------------------------------------------------

def face_grad_sq(u, h, mode: str = "dirichlet") -> np.ndarray:
    """|grad^f u|^2 on the 8 faces of every voxel (reduced diamond cell)."""
    u = _f64(u)
    out = np.empty(u.shape + (8,))
    lib().or_face_grad_sq(_dims(u.shape), _d(u), _d(_hv(h)), 0 if mode == "dirichlet" else 1, _d(out))
    return out


def owner(shape, seeds, r) -> np.ndarray:
    xyz, fr, n = _seeds(seeds)
    out = np.empty(shape, dtype=np.int32)
    lib().or_owner(_dims(shape), _d(xyz), _i(fr), n, float(r), _i(out))
    return out


def threshold(I0, seeds, r, lam) -> np.ndarray:
    I0 = _f64(I0)
    xyz, fr, n = _seeds(seeds)
    out = np.empty_like(I0)
    lib().or_threshold(_dims(I0.shape), _d(I0), _d(xyz), _i(fr), n, float(r), float(lam), _d(out))
    return out


def presmooth(I, h, sigma_t, omega=1.0, tol=1e-12, max_iters=100000, check_every=4):
    I = _f64(I)
    out = np.empty_like(I)
    it = C.c_int(0)
    rr = C.c_double(0)
    st = lib().or_presmooth(_dims(I.shape), _d(I), _d(_hv(h)), float(sigma_t), float(omega),
                            float(tol), int(max_iters), int(check_every), _d(out), C.byref(it),
                            C.byref(rr))
    return out, {"status": st, "iters": it.value, "res_rel": rr.value}


def face_G(Is0, IsTH, h, K, delta, vartheta) -> np.ndarray:
    Is0 = _f64(Is0)
    IsTH = _f64(IsTH)
    out = np.empty(Is0.shape + (8,))
    lib().or_face_G(_dims(Is0.shape), _d(Is0), _d(IsTH), _d(_hv(h)), float(K), float(delta),
                    float(vartheta), _d(out))
    return out


def init_u(shape, seeds, R, v) -> np.ndarray:
    xyz, fr, n = _seeds(seeds)
    out = np.empty(shape)
    lib().or_init_u(_dims(shape), _d(xyz), _i(fr), n, float(R), float(v), _d(out))
    return out


def rescale(u, seeds, r) -> np.ndarray:
    out = _f64(u).copy()
    xyz, fr, n = _seeds(seeds)
    lib().or_rescale(_dims(out.shape), _d(out), _d(xyz), _i(fr), n, float(r))
    return out


def assemble(u, G, h, tau, eps):
    """Returns (diag, off) of the step system built from u (zero Dirichlet)."""
    u = _f64(u)
    G = _f64(G) if G is not None else None
    diag = np.empty_like(u)
    off = np.empty(u.shape + (8,))
    lib().or_assemble(_dims(u.shape), _d(u), _d(G) if G is not None else None, _d(_hv(h)),
                      float(tau), float(eps), _d(diag), _d(off))
    return diag, off


def solve(diag, off, b, u0=None, omega=1.8, tol=1e-12, max_iters=100000, check_every=4):
    diag = _f64(diag)
    off = _f64(off)
    b = _f64(b)
    u = _f64(b if u0 is None else u0).copy()
    it = C.c_int(0)
    rr = C.c_double(0)
    st = lib().or_solve(_dims(b.shape), _d(diag), _d(off), _d(b), _d(u), float(omega), float(tol),
                        int(max_iters), int(check_every), C.byref(it), C.byref(rr))
    return u, {"status": st, "iters": it.value, "res_rel": rr.value}


def residual(diag, off, b, u) -> np.ndarray:
    diag, off, b, u = _f64(diag), _f64(off), _f64(b), _f64(u)
    r = np.empty_like(b)
    lib().or_residual(_dims(b.shape), _d(diag), _d(off), _d(b), _d(u), _d(r))
    return r


def segment(I0, seeds, params: OracleParams | None = None, nsteps: int = 10,
            omp: bool = False):
    """The whole pipeline; returns (u, info) with per-step sweeps and residuals.
    omp: run it on the OpenMP build (the timed CPU baseline, and the reference
    of the full-size parity test, where the plain build would take too long;
    solved to 1e-12 both builds reach the same solutions)."""
    params = params or OracleParams()
    I0 = _f64(I0)
    xyz, fr, n = _seeds(seeds)
    u = np.empty_like(I0)
    iters = np.zeros(max(nsteps, 1), dtype=np.int32)
    res = np.zeros(max(nsteps, 1))
    P = params.c_struct()
    st = lib(omp).or_segment(_dims(I0.shape), _d(I0), _d(xyz), _i(fr), n, C.byref(P), int(nsteps),
                          _d(u), _i(iters), _d(res))
    return u, {"status": st, "iters": iters[:nsteps].tolist(), "res_rel": res[:nsteps].tolist()}


def eoc(n, nsteps, T=0.0625, L=1.25, hdiv=0.0, xoff=-0.5, eps_factor=1.0, omega=1.5,
        tol=1e-12, max_iters=100000):
    """EOC run of Section 3.4: h = 2L/(n + hdiv), x(a) = -L + (a + xoff) h for
    padded index a = 0..n+1.  Returns (error, info)."""
    err = C.c_double(0)
    it = C.c_int(0)
    steps = np.zeros(max(int(nsteps), 1))
    st = lib().or_eoc(int(n), int(nsteps), float(T), float(L), float(hdiv), float(xoff),
                      float(eps_factor), float(omega), float(tol), int(max_iters), C.byref(err),
                      _d(steps), C.byref(it))
    return err.value, {"status": st, "iters": it.value, "err_steps": steps[:nsteps].tolist()}
