"""Python binding of libfblisa, the GB300 (sm_103a) FB-LISA hot path.

Argument marshalling only: every computation runs in the CUDA kernels behind
the C ABI declared in include/fblisa.h; the names here are the C names.
Arrays may be torch tensors (CUDA or CPU) or numpy arrays; CPU/numpy buffers
are staged to the device by the library itself.  There is no CPU fallback:
importing this package fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfblisa.so")

F32, BF16, F16 = 0, 1, 2
REG_L1, REG_TV = 0, 1
STATUS = {0: "FBL_OK", 1: "FBL_E_INVAL", 2: "FBL_E_NOMEM", 3: "FBL_E_CUDA",
          4: "FBL_E_UNSUPPORTED", 5: "FBL_E_LINESEARCH", 6: "FBL_E_NONFINITE", 7: "FBL_E_TIMEOUT"}


class FblError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class fbl_geometry_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("vx", ctypes.c_double), ("vy", ctypes.c_double), ("vz", ctypes.c_double),
                ("n_views", ctypes.c_int32), ("angles", ctypes.POINTER(ctypes.c_double)),
                ("sod", ctypes.c_double), ("sdd", ctypes.c_double),
                ("nu", ctypes.c_int32), ("nv", ctypes.c_int32),
                ("du", ctypes.c_double), ("dv", ctypes.c_double)]


class fbl_params(ctypes.Structure):
    _fields_ = [("alpha0", ctypes.c_double), ("beta", ctypes.c_double), ("mu", ctypes.c_double),
                ("C", ctypes.c_double), ("eps_base", ctypes.c_double),
                ("N0", ctypes.c_int32), ("n_max", ctypes.c_int32),
                ("max_backtracks", ctypes.c_int32), ("proposal", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("x_dtype", ctypes.c_int32),
                ("b_dtype", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("force_reject", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("fixed_step", ctypes.c_int32), ("reg", ctypes.c_int32), ("tv_iters", ctypes.c_int32),
                ("tv_warm", ctypes.c_int32), ("x_max", ctypes.c_double)]


class fbl_step_stats(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int64), ("epoch", ctypes.c_int32), ("N_t", ctypes.c_int32),
                ("backtracks", ctypes.c_int32), ("status", ctypes.c_int32),
                ("alpha", ctypes.c_double), ("alpha_init", ctypes.c_double),
                ("rho0", ctypes.c_double), ("f_x", ctypes.c_double),
                ("f_xbar", ctypes.c_double), ("gTd", ctypes.c_double),
                ("dnorm2", ctypes.c_double), ("margin", ctypes.c_double),
                ("grad_norm2", ctypes.c_double), ("j_start", ctypes.c_int32),
                ("pred", ctypes.c_float), ("features", ctypes.c_float * 8)]

    def as_dict(self):
        d = {name: getattr(self, name) for name, _ in self._fields_}
        d["features"] = list(self.features)
        return d


class fbl_tune_report(ctypes.Structure):
    _fields_ = [("k1_ms", ctypes.c_float * 5), ("k2_ms", ctypes.c_float * 6),
                ("k1_cols", ctypes.c_int32), ("k1_split", ctypes.c_int32),
                ("k2_vpl", ctypes.c_int32)]


class fbl_profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 6), ("launches", ctypes.c_int64 * 6)]


PROFILE_CLASSES = ("residual_projection", "objective_projection", "gradient_backprojection",
                   "prox_reduce", "final_reduce", "pack")

EXPORTS = ["fbl_params_default", "fblisa_profile", "geometry_create", "geometry_destroy", "project", "backproject",
           "residual_norm", "prox_reduce", "fblisa_create", "fblisa_destroy", "fblisa_step",
           "fblisa_run", "fblisa_last_batch", "fbl_last_error", "fbl_schedule",
           "fbl_epoch_batches", "prox_reduce_static", "geometry_autotune",
           "geometry_set_launch", "evaluate", "mlp_forward", "mlp_gradient", "mlp_train",
           "fblisa_set_proposal", "fblisa_batch_create", "fblisa_batch_destroy",
           "fblisa_batch_set_proposal", "fblisa_batch_step", "fblisa_batch_run",
           "fblisa_batch_info", "fblisa_batch_last_batch", "fdk", "prox_tv", "tv_norm"]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libfblisa.so is not built (%s); run __graft_entry__.build() or "
                          "python -m paper_2605_12085_gb300.build" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    P, vp, i32, i64, dbl = ctypes.POINTER, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    st = ctypes.c_int
    sig = {
        "fbl_params_default": (None, [P(fbl_params)]),
        "geometry_create": (st, [P(fbl_geometry_desc), P(vp)]),
        "geometry_destroy": (None, [vp]),
        "geometry_autotune": (st, [vp, i32, i32, vp, P(fbl_tune_report)]),
        "geometry_set_launch": (st, [vp, i32, i32, i32]),
        "project": (st, [vp, vp, i32, P(i32), i32, vp, i32, vp]),
        "backproject": (st, [vp, vp, i32, P(i32), i32, vp, i32, vp]),
        "residual_norm": (st, [vp, vp, i32, P(i32), i32, vp, i32, P(dbl), vp]),
        "prox_reduce": (st, [vp, i32, vp, i64, dbl, dbl, vp, P(dbl), vp]),
        "prox_reduce_static": (st, [vp, i32, vp, i64, dbl, dbl, vp, P(dbl), vp]),
        "evaluate": (st, [vp, vp, i32, vp, i32, dbl, vp, P(dbl), vp]),
        "mlp_forward": (st, [vp, vp, i32, vp, vp]),
        "mlp_gradient": (st, [vp, vp, vp, i32, vp, P(dbl), vp]),
        "mlp_train": (st, [vp, vp, vp, vp, vp, vp, i32, i32, i32, ctypes.c_float, P(dbl), vp]),
        "fblisa_create": (st, [vp, P(fbl_params), P(vp)]),
        "fblisa_destroy": (None, [vp]),
        "fblisa_step": (st, [vp, vp, vp, P(fbl_step_stats), vp]),
        "fblisa_run": (st, [vp, vp, vp, i32, P(fbl_step_stats), i64, P(i64), vp]),
        "fblisa_last_batch": (st, [vp, P(i32), i32, P(i32)]),
        "fblisa_profile": (st, [vp, i32, P(fbl_profile)]),
        "fblisa_set_proposal": (st, [vp, vp, ctypes.c_float, i32]),
        "fblisa_batch_create": (st, [P(vp), P(fbl_params), i32, P(vp)]),
        "fblisa_batch_destroy": (None, [vp]),
        "fblisa_batch_set_proposal": (st, [vp, vp, ctypes.c_float, i32]),
        "fblisa_batch_step": (st, [vp, P(vp), P(vp), P(fbl_step_stats), vp]),
        "fblisa_batch_run": (st, [vp, P(vp), P(vp), i32, P(fbl_step_stats), i64, P(i64), vp]),
        "fblisa_batch_info": (st, [vp, P(i32), P(i64)]),
        "fblisa_batch_last_batch": (st, [vp, i32, P(i32), i32, P(i32)]),
        "fdk": (st, [vp, vp, i32, P(i32), i32, vp, vp]),
        "prox_tv": (st, [P(i32), vp, dbl, dbl, i32, vp, i32, vp, vp]),
        "tv_norm": (st, [P(i32), vp, P(dbl), vp]),
        "fbl_last_error": (ctypes.c_char_p, []),
        "fbl_schedule": (st, [i32, i32, i32, dbl, dbl, i32, P(i32), P(i32)]),
        "fbl_epoch_batches": (st, [ctypes.c_uint64, i32, i32, i32, P(i32)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def _check(status: int):
    if status != 0:
        raise FblError(status, lib.fbl_last_error().decode())


# ---------------------------------------------------------------------------
# Buffers: torch tensors (any device) or numpy arrays
# ---------------------------------------------------------------------------
def _dtype_code(a) -> int:
    try:
        import torch
        if isinstance(a, torch.Tensor):
            m = {torch.float32: F32, torch.bfloat16: BF16, torch.float16: F16}
            if a.dtype not in m:
                raise TypeError("unsupported dtype %s" % a.dtype)
            return m[a.dtype]
    except ImportError:  # pragma: no cover
        pass
    a = np.asarray(a)
    m = {np.dtype(np.float32): F32, np.dtype(np.float16): F16}
    if a.dtype not in m:
        raise TypeError("unsupported dtype %s" % a.dtype)
    return m[a.dtype]


def _ptr(a) -> int:
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if not a.is_contiguous():
                raise ValueError("tensor must be contiguous")
            return a.data_ptr()
    except ImportError:  # pragma: no cover
        pass
    if not (isinstance(a, np.ndarray) and a.flags["C_CONTIGUOUS"]):
        raise ValueError("array must be a C-contiguous numpy array")
    return a.ctypes.data


def _stream(*arrays, stream=None) -> Optional[int]:
    if stream is not None:
        return int(stream)
    try:
        import torch
        for a in arrays:
            if isinstance(a, torch.Tensor) and a.is_cuda:
                return torch.cuda.current_stream(a.device).cuda_stream
    except ImportError:  # pragma: no cover
        pass
    return None


def _views(views) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(list(views), dtype=np.int32))


def _like(template, shape, dtype_code):
    try:
        import torch
        if isinstance(template, torch.Tensor):
            td = {F32: torch.float32, BF16: torch.bfloat16, F16: torch.float16}[dtype_code]
            return torch.empty(shape, dtype=td, device=template.device)
    except ImportError:  # pragma: no cover
        pass
    if dtype_code == BF16:
        raise TypeError("numpy has no bfloat16: pass torch tensors")
    return np.empty(shape, dtype=np.float32 if dtype_code == F32 else np.float16)


# ---------------------------------------------------------------------------
# API
# ---------------------------------------------------------------------------
class Geometry:
    """Handle of a fbl_geometry (cone-beam geometry + device tables)."""

    def __init__(self, desc):
        self.desc = desc
        self._angles = None
        d = fbl_geometry_desc()
        for f in ("nx", "ny", "nz", "vx", "vy", "vz", "n_views", "sod", "sdd", "nu", "nv", "du", "dv"):
            setattr(d, f, getattr(desc, f))
        ang = getattr(desc, "angles", None)
        if ang is not None:
            self._angles = np.ascontiguousarray(np.asarray(ang, dtype=np.float64))
            d.angles = self._angles.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        self._c = d
        h = ctypes.c_void_p()
        _check(lib.geometry_create(ctypes.byref(d), ctypes.byref(h)))
        self.handle = h

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            lib.geometry_destroy(h)
            self.handle = None

    @property
    def vol_shape(self):
        return (self.desc.nz, self.desc.ny, self.desc.nx)

    @property
    def n_views(self):
        return self.desc.n_views


def geometry_create(desc) -> Geometry:
    return Geometry(desc)


def geometry_set_launch(geom: Geometry, k1_cols: int, k1_split: int, k2_vpl: int) -> None:
    _check(lib.geometry_set_launch(geom.handle, k1_cols, k1_split, k2_vpl))


def geometry_autotune(geom: Geometry, x_dtype: int = F32, n_sel: int = 8, stream=None) -> dict:
    rep = fbl_tune_report()
    _check(lib.geometry_autotune(geom.handle, x_dtype, n_sel, stream, ctypes.byref(rep)))
    return {"k1_ms": list(rep.k1_ms), "k2_ms": list(rep.k2_ms), "k1_cols": rep.k1_cols,
            "k1_split": rep.k1_split, "k2_vpl": rep.k2_vpl}


def project(geom: Geometry, x, views: Sequence[int], y=None, y_dtype: Optional[int] = None,
            stream=None):
    v = _views(views)
    xd = _dtype_code(x)
    if y is None:
        y = _like(x, (v.size, geom.desc.nv, geom.desc.nu), F32 if y_dtype is None else y_dtype)
    _check(lib.project(geom.handle, _ptr(x), xd, v.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                       v.size, _ptr(y), _dtype_code(y), _stream(x, y, stream=stream)))
    return y


def backproject(geom: Geometry, y, views: Sequence[int], x=None, accumulate: bool = False,
                stream=None):
    v = _views(views)
    if x is None:
        x = _like(y, geom.vol_shape, F32)
    if _dtype_code(x) != F32:
        raise TypeError("backproject output must be float32")
    _check(lib.backproject(geom.handle, _ptr(y), _dtype_code(y),
                           v.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), v.size, _ptr(x),
                           int(bool(accumulate)), _stream(x, y, stream=stream)))
    return x


def fdk(geom: Geometry, y, views: Sequence[int], x=None, stream=None):
    """FDK reconstruction from the projections y[len(views)][nv][nu] of the
    listed views; returns x [nz][ny][nx] float32 (allocated like y if None)."""
    v = _views(views)
    if x is None:
        x = _like(y, geom.vol_shape, F32)
    if _dtype_code(x) != F32:
        raise TypeError("fdk output must be float32")
    _check(lib.fdk(geom.handle, _ptr(y), _dtype_code(y), v.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                   v.size, _ptr(x), _stream(x, y, stream=stream)))
    return x


def residual_norm(geom: Geometry, x, views: Sequence[int], b, stream=None) -> float:
    v = _views(views)
    rho = ctypes.c_double()
    _check(lib.residual_norm(geom.handle, _ptr(x), _dtype_code(x),
                             v.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), v.size, _ptr(b),
                             _dtype_code(b), ctypes.byref(rho), _stream(x, b, stream=stream)))
    return rho.value


def evaluate(geom: Geometry, x, b, mu: float, x_true=None, stream=None):
    """(F(x), 1/2||Ax-b||^2, RE) over all views (RE = 0 without x_true);
    x_true must have x's dtype."""
    if x_true is not None and _dtype_code(x_true) != _dtype_code(x):
        raise ValueError("evaluate: x_true must have the dtype of x")
    out = (ctypes.c_double * 3)()
    _check(lib.evaluate(geom.handle, _ptr(x), _dtype_code(x), _ptr(b), _dtype_code(b), float(mu),
                        None if x_true is None else _ptr(x_true), out,
                        _stream(x, b, stream=stream)))
    return out[0], out[1], out[2]


def _prox_args(x, g, xbar, need_cuda: bool):
    """Checks shared by the prox calls: g float32 with x's element count, xbar
    (when given) of x's dtype and size; with need_cuda, all three CUDA tensors
    of one device.  The C side cannot check buffer sizes itself."""
    n = int(np.prod(tuple(x.shape)))
    if need_cuda:
        import torch
        for name, a in (("x", x), ("g", g), ("xbar", xbar)):
            if not (isinstance(a, torch.Tensor) and a.is_cuda):
                raise TypeError("prox_reduce_static: %s must be a CUDA tensor" % name)
        if not (x.device == g.device == xbar.device):
            raise ValueError("prox_reduce_static: x, g and xbar must be on one device")
    if _dtype_code(g) != F32:
        raise TypeError("prox: g must be float32")
    if int(np.prod(tuple(g.shape))) != n:
        raise ValueError("prox: g must have x's %d elements" % n)
    if xbar is not None:
        if _dtype_code(xbar) != _dtype_code(x):
            raise TypeError("prox: xbar must have x's dtype")
        if int(np.prod(tuple(xbar.shape))) != n:
            raise ValueError("prox: xbar must have x's %d elements" % n)
    return n


def prox_reduce(x, g, alpha: float, mu: float, xbar=None, stream=None):
    n = _prox_args(x, g, xbar, need_cuda=False)
    if xbar is None:
        xbar = _like(x, tuple(x.shape), _dtype_code(x))
    out = (ctypes.c_double * 3)()
    _check(lib.prox_reduce(_ptr(x), _dtype_code(x), _ptr(g), n, float(alpha), float(mu),
                           _ptr(xbar), out, _stream(x, g, xbar, stream=stream)))
    return xbar, (out[0], out[1], out[2])


def prox_reduce_static(x, g, alpha: float, mu: float, xbar, stream=None):
    """prox_reduce without any allocation: x, g and xbar must be CUDA tensors
    (xbar caller-provided) of the current device; n <= 2^27.  Calls that
    overlap on the GPU race."""
    n = _prox_args(x, g, xbar, need_cuda=True)
    out = (ctypes.c_double * 3)()
    _check(lib.prox_reduce_static(_ptr(x), _dtype_code(x), _ptr(g), n, float(alpha), float(mu),
                                  _ptr(xbar), out, _stream(x, g, xbar, stream=stream)))
    return xbar, (out[0], out[1], out[2])


def prox_tv(v, lam: float, iters: int, x_max: float = float("inf"), q=None, q_in: bool = False, x=None,
            stream=None):
    """prox of lam TV + indicator{0 <= x <= x_max} at v [nz][ny][nx] float32 by
    ``iters`` FGP iterations; q [3][nz][ny][nx] float32: the start (q_in) and
    the last dual on return.  Returns x."""
    if _dtype_code(v) != F32 or (x is not None and _dtype_code(x) != F32) or (q is not None and _dtype_code(q) != F32):
        raise TypeError("prox_tv works on float32 volumes")
    nz, ny, nx = (int(t) for t in v.shape)
    if x is None:
        x = _like(v, (nz, ny, nx), F32)
    dims = (ctypes.c_int32 * 3)(nx, ny, nz)
    _check(lib.prox_tv(dims, _ptr(v), float(lam), float(x_max), int(iters), _ptr(q) if q is not None else None,
                       1 if q_in else 0, _ptr(x), _stream(v, x, stream=stream)))
    return x


def tv_norm(x, stream=None) -> float:
    """Isotropic TV of x [nz][ny][nx] float32 (forward differences, FP64 sum)."""
    if _dtype_code(x) != F32:
        raise TypeError("tv_norm works on float32 volumes")
    nz, ny, nx = (int(t) for t in x.shape)
    dims = (ctypes.c_int32 * 3)(nx, ny, nz)
    out = ctypes.c_double()
    _check(lib.tv_norm(dims, _ptr(x), ctypes.byref(out), _stream(x, stream=stream)))
    return out.value


MLP_PARAMS = 4801


def mlp_forward(params, X, y=None, stream=None):
    """y = net(X) for X [n][8] (CUDA tensors)."""
    n = int(X.shape[0])
    if y is None:
        y = _like(X, (n,), F32)
    _check(lib.mlp_forward(_ptr(params), _ptr(X), n, _ptr(y), _stream(params, X, stream=stream)))
    return y


def mlp_gradient(params, X, t, stream=None):
    """(full-batch gradient of 1/(2n) sum (y - t)^2, loss) for CUDA tensors."""
    n = int(X.shape[0])
    g = _like(params, (MLP_PARAMS,), F32)
    loss = ctypes.c_double()
    _check(lib.mlp_gradient(_ptr(params), _ptr(X), _ptr(t), n, _ptr(g), ctypes.byref(loss),
                            _stream(params, X, stream=stream)))
    return g, loss.value


class MlpTrainer:
    """Adam state for training a parameter vector in place on the GPU."""

    def __init__(self, params):
        import torch
        self.params = params
        self.m = torch.zeros_like(params)
        self.v = torch.zeros_like(params)
        self.step = torch.zeros(1, dtype=torch.int32, device=params.device)

    def train(self, X, t, batch=256, epochs=1, lr=1e-3, stream=None) -> float:
        loss = ctypes.c_double()
        _check(lib.mlp_train(_ptr(self.params), _ptr(self.m), _ptr(self.v), _ptr(self.step),
                             _ptr(X), _ptr(t), int(X.shape[0]), int(batch), int(epochs),
                             float(lr), ctypes.byref(loss),
                             _stream(self.params, X, stream=stream)))
        return loss.value


def params_default(**kw) -> fbl_params:
    p = fbl_params()
    lib.fbl_params_default(ctypes.byref(p))
    for k, val in kw.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, val)
    return p


class Solver:
    """Handle of a fbl_solver (Algorithm 1 state and scratch)."""

    def __init__(self, geom: Geometry, params: fbl_params):
        self.geom = geom
        self.params = params
        h = ctypes.c_void_p()
        _check(lib.fblisa_create(geom.handle, ctypes.byref(params), ctypes.byref(h)))
        self.handle = h

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            lib.fblisa_destroy(h)
            self.handle = None

    def step(self, x, b, stream=None) -> dict:
        st = fbl_step_stats()
        _check(lib.fblisa_step(self.handle, _ptr(x), _ptr(b), ctypes.byref(st),
                               _stream(x, b, stream=stream)))
        return st.as_dict()

    def step_raw(self, x, b, stream=None):
        """Like step() but returns (status, stats) instead of raising."""
        st = fbl_step_stats()
        rc = lib.fblisa_step(self.handle, _ptr(x), _ptr(b), ctypes.byref(st),
                             _stream(x, b, stream=stream))
        return rc, st.as_dict()

    def run(self, x, b, epochs: int, trace_cap: int = 100000, stream=None):
        trace = (fbl_step_stats * max(1, trace_cap))()
        n = ctypes.c_int64()
        _check(lib.fblisa_run(self.handle, _ptr(x), _ptr(b), int(epochs), trace, trace_cap,
                              ctypes.byref(n), _stream(x, b, stream=stream)))
        return [trace[q].as_dict() for q in range(min(n.value, trace_cap))]

    def profile(self, enable: bool = True):
        """Return {class: (ms, launches)} accumulated so far (then reset) and
        switch event timing on or off."""
        pr = fbl_profile()
        _check(lib.fblisa_profile(self.handle, int(bool(enable)), ctypes.byref(pr)))
        return {name: (pr.ms[c], pr.launches[c]) for c, name in enumerate(PROFILE_CLASSES)}

    def set_proposal(self, params, margin: float = 0.25, enable: bool = True):
        """Install the step-proposal network (4801 floats, tensor or array)."""
        if params is None:
            _check(lib.fblisa_set_proposal(self.handle, None, float(margin), int(bool(enable))))
        else:
            _check(lib.fblisa_set_proposal(self.handle, _ptr(params), float(margin),
                                           int(bool(enable))))

    def last_batch(self):
        n = ctypes.c_int32()
        _check(lib.fblisa_last_batch(self.handle, None, 0, ctypes.byref(n)))
        buf = (ctypes.c_int32 * max(1, n.value))()
        _check(lib.fblisa_last_batch(self.handle, buf, n.value, ctypes.byref(n)))
        return list(buf[:n.value])


def fblisa_create(geom: Geometry, params: fbl_params) -> Solver:
    return Solver(geom, params)


class Batch:
    """Handle of a fbl_batch: one Algorithm 1 per volume, every phase of an
    iteration of all volumes in one persistent launch (fblisa_batch_*)."""

    def __init__(self, geoms: Sequence[Geometry], params: Sequence[fbl_params]):
        if len(geoms) != len(params) or not geoms:
            raise ValueError("one parameter record per geometry")
        self.geoms = list(geoms)  # keep the geometries alive
        self.n = len(geoms)
        gh = (ctypes.c_void_p * self.n)(*[g.handle.value for g in geoms])
        pa = (fbl_params * self.n)(*params)
        h = ctypes.c_void_p()
        _check(lib.fblisa_batch_create(gh, pa, self.n, ctypes.byref(h)))
        self.handle = h

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            lib.fblisa_batch_destroy(h)
            self.handle = None

    def _arrays(self, xs, bs):
        if len(xs) != self.n or len(bs) != self.n:
            raise ValueError("one x and one b per volume")
        xp = (ctypes.c_void_p * self.n)(*[_ptr(x) for x in xs])
        bp = (ctypes.c_void_p * self.n)(*[_ptr(b) for b in bs])
        return xp, bp

    def set_proposal(self, params, margin: float = 0.25, enable: bool = True):
        _check(lib.fblisa_batch_set_proposal(self.handle, None if params is None else _ptr(params),
                                             float(margin), int(bool(enable))))

    def step_raw(self, xs, bs, stream=None):
        """One iteration of every volume: (status, [stats per volume])."""
        xp, bp = self._arrays(xs, bs)
        st = (fbl_step_stats * self.n)()
        rc = lib.fblisa_batch_step(self.handle, xp, bp, st, _stream(*xs, *bs, stream=stream))
        return rc, [st[v].as_dict() for v in range(self.n)]

    def step(self, xs, bs, stream=None):
        rc, st = self.step_raw(xs, bs, stream=stream)
        _check(rc)
        return st

    def run(self, xs, bs, iterations: int, stream=None):
        """`iterations` batched steps; returns [[stats per volume] per step]."""
        xp, bp = self._arrays(xs, bs)
        cap = max(1, iterations)
        trace = (fbl_step_stats * (cap * self.n))()
        n = ctypes.c_int64()
        _check(lib.fblisa_batch_run(self.handle, xp, bp, int(iterations), trace, cap, ctypes.byref(n),
                                    _stream(*xs, *bs, stream=stream)))
        return [[trace[q * self.n + v].as_dict() for v in range(self.n)] for q in range(n.value)]

    def info(self):
        cfg = (ctypes.c_int32 * 4)()
        n = ctypes.c_int64()
        _check(lib.fblisa_batch_info(self.handle, cfg, ctypes.byref(n)))
        return {"k1_cols": cfg[0], "k1_split": cfg[1], "k2_vpl": cfg[2], "ntap": cfg[3],
                "launches": n.value}

    def last_batch(self, v: int):
        n = ctypes.c_int32()
        _check(lib.fblisa_batch_last_batch(self.handle, v, None, 0, ctypes.byref(n)))
        buf = (ctypes.c_int32 * max(1, n.value))()
        _check(lib.fblisa_batch_last_batch(self.handle, v, buf, n.value, ctypes.byref(n)))
        return list(buf[:n.value])


def fblisa_batch_create(geoms, params) -> Batch:
    return Batch(geoms, params)


def fbl_schedule(n_theta, N0, n_max, C, eps_base, epochs):
    N = (ctypes.c_int32 * max(1, epochs))()
    it = (ctypes.c_int32 * max(1, epochs))()
    _check(lib.fbl_schedule(n_theta, N0, n_max, C, eps_base, epochs, N, it))
    return [(N[t], it[t]) for t in range(epochs)]


def fbl_epoch_batches(seed, epoch, n_theta, N_t):
    iters = -(-n_theta // N_t)
    out = (ctypes.c_int32 * (iters * N_t))()
    _check(lib.fbl_epoch_batches(seed, epoch, n_theta, N_t, out))
    flat = list(out)
    return [flat[q * N_t:(q + 1) * N_t] for q in range(iters)]
