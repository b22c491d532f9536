"""ctypes binding of libseg4d (include/seg4d.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts numpy arrays
(host memory) and torch CUDA tensors (device memory) into pointers and status
codes into exceptions.  There is no CPU fallback: if the shared library is
missing, importing the handle class raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass, fields

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libseg4d.so")
_lock = threading.Lock()
_lib = None

OK, ERR_INVALID, ERR_OOM, ERR_STATE, ERR_NOT_CONVERGED, ERR_CUDA, ERR_TIMEOUT = 0, -1, -2, -3, -4, -5, -6
STATUS_NAMES = {0: "OK", -1: "INVALID", -2: "OOM", -3: "STATE", -4: "NOT_CONVERGED", -5: "CUDA",
                -6: "TIMEOUT"}

CREATE_LEAN = 1   # seg4d_create_ex flag (seg4d.h)
FIELDS = {"u": 0, "I0": 1, "ITH": 2, "Isig0": 3, "IsigTH": 4, "G": 5, "owner": 6, "diag": 7,
          "off": 8}
FACE_FIELDS = {"G", "off"}


class Seg4DError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"seg4d {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class CDims(C.Structure):
    _fields_ = [("n1", C.c_int), ("n2", C.c_int), ("n3", C.c_int), ("n4", C.c_int)]


class CParams(C.Structure):
    _fields_ = [("h", C.c_double * 4), ("tau", C.c_double), ("eps", C.c_double),
                ("K", C.c_double), ("delta", C.c_double), ("vartheta", C.c_double),
                ("lambda_th", C.c_double), ("r_ball", C.c_double), ("R_init", C.c_double),
                ("v_init", C.c_double), ("sigma_t", C.c_double), ("omega", C.c_double),
                ("omega_smooth", C.c_double), ("tol", C.c_double), ("tol_smooth", C.c_double),
                ("max_iters", C.c_int), ("check_every", C.c_int), ("precision", C.c_int),
                ("sweep_variant", C.c_int), ("ctas_per_sm", C.c_int), ("wait_test", C.c_int),
                ("tol_inf", C.c_double), ("omega_adapt", C.c_int)]


class CSeed(C.Structure):
    _fields_ = [("x", C.c_double), ("y", C.c_double), ("z", C.c_double), ("frame", C.c_int),
                ("reserved", C.c_int)]


class CInfo(C.Structure):
    _fields_ = [("iters", C.c_int), ("status", C.c_int), ("res_l2", C.c_double),
                ("res_rel", C.c_double), ("bnorm", C.c_double), ("umin", C.c_double),
                ("umax", C.c_double), ("sweeps_total", C.c_longlong), ("steps_done", C.c_int),
                ("ms", C.c_float), ("sweep_ms", C.c_double), ("launches", C.c_longlong),
                ("sweep_launches", C.c_longlong), ("res_inf", C.c_double), ("bmax", C.c_double)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


# exported entry points: name -> (restype, argtypes)
_P = C.c_void_p
SIGNATURES = {
    "seg4d_default_params": (None, [C.POINTER(CParams)]),
    "seg4d_create": (C.c_int, [C.POINTER(CDims), _P, C.POINTER(_P)]),
    "seg4d_create_ex": (C.c_int, [C.POINTER(CDims), _P, C.c_int, C.POINTER(_P)]),
    "seg4d_device_bytes_ex": (C.c_size_t, [C.POINTER(CDims), C.c_int]),
    "seg4d_destroy": (C.c_int, [_P]),
    "seg4d_set_params": (C.c_int, [_P, C.POINTER(CParams)]),
    "seg4d_set_image": (C.c_int, [_P, _P, C.c_size_t, C.c_int]),
    "seg4d_set_seed": (C.c_int, [_P, C.POINTER(CSeed), C.c_int]),
    "seg4d_set_u": (C.c_int, [_P, _P, C.c_size_t, C.c_int]),
    "seg4d_dirichlet_count": (C.c_size_t, [C.POINTER(CDims)]),
    "seg4d_set_dirichlet": (C.c_int, [_P, _P, _P, C.c_size_t, C.c_int]),
    "seg4d_setup": (C.c_int, [_P, C.POINTER(CInfo)]),
    "seg4d_solve": (C.c_int, [_P, C.POINTER(CInfo)]),
    "seg4d_step": (C.c_int, [_P, C.c_int, C.POINTER(CInfo)]),
    "seg4d_read_u": (C.c_int, [_P, _P, C.c_size_t, C.c_int]),
    "seg4d_read_field": (C.c_int, [_P, C.c_int, _P, C.c_size_t, C.c_int]),
    "seg4d_device_bytes": (C.c_size_t, [C.POINTER(CDims)]),
    "seg4d_last_error": (C.c_char_p, [_P]),
    "seg4d_residual_norms_noalloc": (C.c_int, [C.POINTER(CDims), _P, _P, _P, _P, _P, _P]),
}


def residual_norms_noalloc(dims, u, b, diag, off, result, stream=None):
    """Binding of seg4d_residual_norms_noalloc: all arguments are CUDA tensors
    (float32 u, b, diag of n voxels, off of 8n; float64 result of 2)."""
    lib = load()
    n1, n2, n3, n4 = dims
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    ptrs = [C.c_void_p(t.data_ptr()) for t in (u, b, diag, off, result)]
    st = lib.seg4d_residual_norms_noalloc(C.byref(CDims(n1, n2, n3, n4)), *ptrs,
                                          C.c_void_p(stream or 0))
    if st != OK:
        raise Seg4DError(st, lib.seg4d_last_error(None).decode())


def load(path: str | None = None):
    """Load the shared library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise ImportError(f"libseg4d is not built ({p} missing); run "
                                  "`python -c 'import __graft_entry__ as g; g.build()'`")
            lib = C.CDLL(p)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


@dataclass
class Params:
    """Mirror of seg4d_params; defaults come from seg4d_default_params()."""
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
    omega: float = 1.6
    omega_smooth: float = 1.0
    tol: float = 1e-5
    tol_smooth: float = 1e-6
    max_iters: int = 20000
    check_every: int = 10
    precision: int = 0
    sweep_variant: int = 1
    ctas_per_sm: int = 0
    wait_test: int = 0
    tol_inf: float = 1e-5
    omega_adapt: int = 1

    @classmethod
    def defaults(cls) -> "Params":
        cp = CParams()
        load().seg4d_default_params(C.byref(cp))
        kw = {}
        for f in fields(cls):
            v = getattr(cp, f.name)
            kw[f.name] = tuple(v) if f.name == "h" else v
        return cls(**kw)

    def to_c(self) -> CParams:
        cp = CParams()
        h = self.h if not np.isscalar(self.h) else (self.h,) * 4
        cp.h = (C.c_double * 4)(*[float(x) for x in h])
        for f in fields(self):
            if f.name == "h":
                continue
            setattr(cp, f.name, getattr(self, f.name))
        return cp


def _ptr(a, n_expected):
    """(pointer, on_device, keepalive) for a numpy array or a torch tensor."""
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        import torch
        if a.dtype != torch.float32:
            raise TypeError("expected a float32 tensor")
        if not a.is_contiguous():
            raise ValueError("expected a contiguous tensor")
        if a.numel() != n_expected:
            raise ValueError(f"expected {n_expected} elements, got {a.numel()}")
        # device tensors stay on the device; CPU tensors (pinned or not) are
        # host memory, read or written in place
        return C.c_void_p(a.data_ptr()), (1 if a.is_cuda else 0), a
    arr = np.ascontiguousarray(a, dtype=np.float32)
    if arr.size != n_expected:
        raise ValueError(f"expected {n_expected} elements, got {arr.size}")
    return C.c_void_p(arr.ctypes.data), 0, arr


class Seg4D:
    """One segmentation problem on the current CUDA device (see seg4d.h).

    dims = (n1, n2, n3, n4) with n1 the fastest (x) axis and n4 the frames;
    arrays are shaped (n4, n3, n2, n1)."""

    def __init__(self, dims, stream=None, params: Params | None = None, lean: bool = False):
        self.lib = load()
        self.dims = tuple(int(x) for x in dims)
        n1, n2, n3, n4 = self.dims
        self.shape = (n4, n3, n2, n1)
        self.nvox = n1 * n2 * n3 * n4
        cd = CDims(n1, n2, n3, n4)
        h = C.c_void_p()
        if stream is not None and hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        st = self.lib.seg4d_create_ex(C.byref(cd), C.c_void_p(stream or 0),
                                      CREATE_LEAN if lean else 0, C.byref(h))
        if st != OK:
            raise Seg4DError(st, self.lib.seg4d_last_error(None).decode())
        self.h = h
        self.params = params or Params.defaults()
        self.set_params(self.params)

    # ------------------------------------------------------------------
    def _check(self, st, allow=()):
        if st != OK and st not in allow:
            raise Seg4DError(st, self.lib.seg4d_last_error(self.h).decode())
        return st

    def close(self):
        if getattr(self, "h", None):
            self.lib.seg4d_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------------
    def set_params(self, params: Params | None = None, **kw):
        if params is None:
            params = self.params
        for k, v in kw.items():
            if not hasattr(params, k):
                raise AttributeError(k)
            setattr(params, k, v)
        self.params = params
        cp = params.to_c()
        self._check(self.lib.seg4d_set_params(self.h, C.byref(cp)))

    def set_image(self, image):
        p, dev, keep = _ptr(image, self.nvox)
        self._check(self.lib.seg4d_set_image(self.h, p, self.nvox, dev))

    def set_seeds(self, seeds):
        s = np.asarray(seeds, dtype=np.float64).reshape(-1, 4)
        arr = (CSeed * max(len(s), 1))()
        for m, (x, y, z, f) in enumerate(s):
            arr[m] = CSeed(float(x), float(y), float(z), int(f), 0)
        self._check(self.lib.seg4d_set_seed(self.h, arr, len(s)))

    def set_u(self, u):
        p, dev, keep = _ptr(u, self.nvox)
        self._check(self.lib.seg4d_set_u(self.h, p, self.nvox, dev))

    @staticmethod
    def dirichlet_count(dims) -> int:
        n1, n2, n3, n4 = dims
        return int(load().seg4d_dirichlet_count(C.byref(CDims(n1, n2, n3, n4))))

    def set_dirichlet(self, g_prev=None, g_now=None):
        """Ghost-ring Dirichlet data (seg4d_set_dirichlet); None, None = zero."""
        if g_prev is None and g_now is None:
            self._check(self.lib.seg4d_set_dirichlet(self.h, None, None, 0, 0))
            return
        n = self.dirichlet_count(self.dims)
        p0, dev0, k0 = _ptr(g_prev, n)
        p1, dev1, k1 = _ptr(g_now, n)
        if dev0 != dev1:
            raise ValueError("both ghost arrays on the host or both on the device")
        self._check(self.lib.seg4d_set_dirichlet(self.h, p0, p1, n, dev0))

    def setup(self, allow_not_converged=False):
        info = CInfo()
        self._check(self.lib.seg4d_setup(self.h, C.byref(info)),
                    (ERR_NOT_CONVERGED,) if allow_not_converged else ())
        return info.as_dict()

    def solve(self, allow_not_converged=False):
        info = CInfo()
        self._check(self.lib.seg4d_solve(self.h, C.byref(info)),
                    (ERR_NOT_CONVERGED,) if allow_not_converged else ())
        return info.as_dict()

    def step(self, nsteps=1, allow_not_converged=False):
        info = CInfo()
        self._check(self.lib.seg4d_step(self.h, int(nsteps), C.byref(info)),
                    (ERR_NOT_CONVERGED,) if allow_not_converged else ())
        return info.as_dict()

    def read_u(self, out=None):
        return self.read_field("u", out)

    def read_field(self, name: str, out=None):
        nf = 8 if name in FACE_FIELDS else 1
        shape = self.shape + ((8,) if nf == 8 else ())
        if out is None:
            out = np.empty(shape, dtype=np.float32)
        p, dev, keep = _ptr(out, self.nvox * nf)
        if not dev and keep is not out:
            raise ValueError("host output must be a contiguous float32 numpy array")
        self._check(self.lib.seg4d_read_field(self.h, FIELDS[name], p, self.nvox * nf, dev))
        return out

    @staticmethod
    def device_bytes(dims, lean: bool = False) -> int:
        n1, n2, n3, n4 = dims
        return int(load().seg4d_device_bytes_ex(C.byref(CDims(n1, n2, n3, n4)),
                                                CREATE_LEAN if lean else 0))


# ----------------------------------------------------------------- batches

class CBatchInfo(C.Structure):
    _fields_ = [("setup_windows", C.c_int), ("stepped_windows", C.c_int),
                ("active_windows", C.c_int), ("done_windows", C.c_int),
                ("failed_windows", C.c_int), ("status", C.c_int), ("window_sweeps", C.c_longlong),
                ("launches", C.c_longlong), ("arena_used", C.c_longlong), ("ms", C.c_float),
                ("pad", C.c_float), ("sweep_ms", C.c_double)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_ if name != "pad"}


class CWindowInfo(C.Structure):
    _fields_ = [("state", C.c_int), ("steps_done", C.c_int), ("nsteps", C.c_int),
                ("last_iters", C.c_int), ("sweeps", C.c_longlong), ("device_bytes", C.c_longlong),
                ("last_res_rel", C.c_double)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


SIGNATURES.update({
    "seg4d_batch_create": (C.c_int, [C.c_size_t, C.c_int, _P, C.POINTER(_P)]),
    "seg4d_batch_destroy": (C.c_int, [_P]),
    "seg4d_batch_set_params": (C.c_int, [_P, C.POINTER(CParams)]),
    "seg4d_batch_add": (C.c_int, [_P, C.POINTER(CDims), _P, C.c_int, C.POINTER(CSeed), C.c_int,
                                  C.c_int, C.POINTER(C.c_int)]),
    "seg4d_batch_advance": (C.c_int, [_P, C.POINTER(CBatchInfo)]),
    "seg4d_batch_poll": (C.c_int, [_P, C.c_int, C.POINTER(CWindowInfo)]),
    "seg4d_batch_read_u": (C.c_int, [_P, C.c_int, _P, C.c_size_t, C.c_int]),
    "seg4d_batch_remove": (C.c_int, [_P, C.c_int]),
    "seg4d_batch_window_bytes": (C.c_size_t, [C.POINTER(CDims), C.c_int, C.c_int]),
    "seg4d_batch_last_error": (C.c_char_p, [_P]),
})

WINDOW_STATES = {0: "pending", 1: "active", 2: "done", 3: "failed"}


def _seed_array(seeds):
    s = np.asarray(seeds, dtype=np.float64).reshape(-1, 4)
    arr = (CSeed * max(len(s), 1))()
    for m, (x, y, z, f) in enumerate(s):
        arr[m] = CSeed(float(x), float(y), float(z), int(f), 0)
    return arr, len(s)


class Batch:
    """Many windows advanced together (seg4d_batch_* in seg4d.h)."""

    def __init__(self, arena_bytes: int, max_windows: int = 4096, stream=None,
                 params: Params | None = None):
        self.lib = load()
        if stream is not None and hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        h = C.c_void_p()
        st = self.lib.seg4d_batch_create(int(arena_bytes), int(max_windows),
                                         C.c_void_p(stream or 0), C.byref(h))
        if st != OK:
            raise Seg4DError(st, self.lib.seg4d_batch_last_error(None).decode())
        self.h = h
        self.shapes = {}
        self.params = params or Params.defaults()
        self.set_params(self.params)

    def _check(self, st, allow=()):
        if st != OK and st not in allow:
            raise Seg4DError(st, self.lib.seg4d_batch_last_error(self.h).decode())
        return st

    def close(self):
        if getattr(self, "h", None):
            self.lib.seg4d_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_params(self, params: Params | None = None, **kw):
        params = params or self.params
        for k, v in kw.items():
            setattr(params, k, v)
        self.params = params
        cp = params.to_c()
        self._check(self.lib.seg4d_batch_set_params(self.h, C.byref(cp)))

    def add(self, image, seeds, nsteps: int):
        """Admit a window; returns its id, or None when the arena has no room."""
        if hasattr(image, "shape"):
            n4, n3, n2, n1 = image.shape
        else:
            raise ValueError("image must be a 4D array (n4, n3, n2, n1)")
        p, dev, keep = _ptr(image, n1 * n2 * n3 * n4)
        arr, ns = _seed_array(seeds)
        wid = C.c_int(0)
        st = self.lib.seg4d_batch_add(self.h, C.byref(CDims(n1, n2, n3, n4)), p, dev, arr, ns,
                                      int(nsteps), C.byref(wid))
        if st == ERR_OOM:
            return None
        self._check(st)
        self.shapes[wid.value] = (n4, n3, n2, n1)
        return wid.value

    def advance(self):
        info = CBatchInfo()
        self._check(self.lib.seg4d_batch_advance(self.h, C.byref(info)))
        return info.as_dict()

    def poll(self, wid: int):
        wi = CWindowInfo()
        self._check(self.lib.seg4d_batch_poll(self.h, int(wid), C.byref(wi)))
        d = wi.as_dict()
        d["state"] = WINDOW_STATES.get(d["state"], d["state"])
        return d

    def read_u(self, wid: int, out=None):
        shape = self.shapes[wid]
        if out is None:
            out = np.empty(shape, dtype=np.float32)
        n = int(np.prod(shape))
        p, dev, keep = _ptr(out, n)
        self._check(self.lib.seg4d_batch_read_u(self.h, int(wid), p, n, dev))
        return out

    def remove(self, wid: int):
        self._check(self.lib.seg4d_batch_remove(self.h, int(wid)))
        self.shapes.pop(wid, None)

    @staticmethod
    def window_bytes(dims, nseeds=1, precision=0) -> int:
        n1, n2, n3, n4 = dims
        return int(load().seg4d_batch_window_bytes(C.byref(CDims(n1, n2, n3, n4)), int(nseeds),
                                                   int(precision)))
