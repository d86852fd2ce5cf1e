"""Python binding of libgrav (argument marshalling only).

Every operator step runs in the CUDA kernels of ``libgrav.so`` (built
in-tree by ``paper_2602_03857_b300.build``); this module only converts torch
tensors and numpy arrays into the pointers and sizes of the C ABI declared
in ``include/grav.h`` and raises on error codes.  There is no CPU fallback:
if the shared library is missing, importing this package fails.

Notation follows the paper: d = G m (Section 2.1, Eq. 5-6), G^T r, and the
data-space inversion m = m_ref + W^-2 G^T (G W^-2 G^T + lambda I)^-1 (d - G m_ref)
(Section 2.2, Eq. 10-11).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgrav.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"libgrav.so not found at {LIB_PATH}: build it with `python paper_2602_03857_b300/build.py` "
        "(the CUDA library is required; there is no CPU fallback)")

_lib = ctypes.CDLL(LIB_PATH)

GRAV_OK = 0
GRAV_EINVAL = -1
GRAV_ENOMEM = -2
GRAV_ENOTCONVERGED = -3
GRAV_ETIMEDOUT = -4
GRAV_EDEVICE = -5
GRAV_ECANCELED = -6
GRAV_ENOTFOUND = -7
GRAV_EBUSY = -8
GRAV_FP64 = 0
GRAV_MIXED = 1
GRAV_MIXED_CORNER = 2
GRAV_JOB_FORWARD, GRAV_JOB_INVERT = 0, 1
JOB_STATES = {0: "queued", 1: "running", 2: "done", 3: "failed", 4: "canceled"}
PRECISIONS = {"fp64": GRAV_FP64, "mixed": GRAV_MIXED, "mixed_corner": GRAV_MIXED_CORNER}

_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)


class grav_mesh(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("xe", _D), ("ye", _D), ("ze", _D)]


class grav_survey(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("x", _P), ("y", _P), ("z", _P)]


class grav_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("z0", ctypes.c_double), ("lambda_scale", ctypes.c_double),
                ("lambda_", ctypes.c_double), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("check_every", ctypes.c_int), ("near_cells", ctypes.c_double), ("timeout_s", ctypes.c_double),
                ("precond", ctypes.c_int), ("cache_g", ctypes.c_int), ("outer_max", ctypes.c_int),
                ("inner_max", ctypes.c_int), ("reorth", ctypes.c_int), ("check_stations", ctypes.c_int),
                ("nys_rank", ctypes.c_int), ("nys_coarsen", ctypes.c_int), ("refine", ctypes.c_int),
                ("near_fp64", ctypes.c_int),
                ("diag_fp64", ctypes.c_int)]


class grav_job(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("mesh", grav_mesh), ("survey", grav_survey), ("input", _P),
                ("m_ref", _P), ("output", _P), ("opt", grav_options)]


class grav_solve_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("converged", ctypes.c_int), ("rel_res", ctypes.c_double),
                ("true_rel_res", ctypes.c_double), ("lambda_", ctypes.c_double), ("trace", ctypes.c_double),
                ("seconds", ctypes.c_double), ("outer", ctypes.c_int), ("alpha_min", ctypes.c_double),
                ("restarts", ctypes.c_int), ("fp64_rel_err", ctypes.c_double), ("nys_shift", ctypes.c_double),
                ("nys_setup_s", ctypes.c_double)]


def _sig(name, res, args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = args
    return f


_i, _vp = ctypes.c_int, ctypes.c_void_p
_sig("grav_options_default", None, [ctypes.POINTER(grav_options)])
_sig("grav_version", ctypes.c_char_p, [])
_sig("grav_ctx_create", _i, [ctypes.POINTER(_vp), _i, ctypes.c_size_t])
_sig("grav_ctx_destroy", _i, [_vp])
_sig("grav_last_error", ctypes.c_char_p, [_vp])
_sig("grav_ctx_sync", _i, [_vp, _vp, ctypes.c_double])
_sig("grav_forward", _i, [_vp, ctypes.POINTER(grav_mesh), ctypes.POINTER(grav_survey), _vp, _vp,
                          ctypes.POINTER(grav_options), _vp])
_sig("grav_adjoint", _i, [_vp, ctypes.POINTER(grav_mesh), ctypes.POINTER(grav_survey), _vp, _vp, _i,
                          ctypes.POINTER(grav_options), _vp])
_sig("grav_diag", _i, [_vp, ctypes.POINTER(grav_mesh), ctypes.POINTER(grav_survey), _vp, _D,
                       ctypes.POINTER(grav_options), _vp])
_sig("grav_datainv_solve", _i, [_vp, ctypes.POINTER(grav_mesh), ctypes.POINTER(grav_survey), _vp, _vp, _vp,
                                _vp, ctypes.POINTER(grav_solve_info), ctypes.POINTER(grav_options), _vp])
_sig("grav_plan_create", _i, [_vp, ctypes.POINTER(grav_mesh), ctypes.POINTER(grav_survey),
                              ctypes.POINTER(grav_options), ctypes.POINTER(_vp), _vp])
_sig("grav_plan_forward", _i, [_vp, _vp, _vp, _vp])
_sig("grav_plan_adjoint", _i, [_vp, _vp, _vp, _i, _vp])
_sig("grav_plan_bytes", ctypes.c_size_t, [_vp])
_sig("grav_plan_destroy", _i, [_vp, _vp])
_sig("grav_launch_count", ctypes.c_uint64, [])
_sig("grav_plan_timing", _i, [_vp, _i, _D, ctypes.POINTER(ctypes.c_int64)])
_sig("grav_bench_pipes", _i, [_i, _D])
_sig("grav_plan_describe", _i, [_vp, ctypes.c_char_p, ctypes.c_size_t])
_sig("grav_serve_config", _i, [_vp, _i])
_sig("grav_submit", _i, [_vp, ctypes.POINTER(grav_job), ctypes.POINTER(ctypes.c_uint64)])
_sig("grav_poll", _i, [_vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(grav_solve_info)])
_sig("grav_wait", _i, [_vp, ctypes.c_uint64, ctypes.c_double])
_sig("grav_cancel", _i, [_vp, ctypes.c_uint64])
_sig("grav_job_times", _i, [_vp, ctypes.c_uint64, _D, _D, _D])
_sig("grav_job_release", _i, [_vp, ctypes.c_uint64])
_sig("grav_job_plan", _i, [_vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int), _D, ctypes.POINTER(ctypes.c_size_t)])
_sig("grav_serve_plan_cache", _i, [_vp, _i])
_sig("grav_serve_stats", _i, [_vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                              ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_size_t)])
_sig("grav_eval_fn64", _i, [_vp, _i, _vp, _vp, _vp, ctypes.c_int64, _vp])
_sig("grav_plan_check_fp64", _i, [_vp, _vp, _vp, _i, _D, _D, _vp])
_sig("grav_selftest_wait", _i, [_vp, ctypes.c_double, _vp])
_sig("grav_nystrom_coarse_apply", _i, [_vp, ctypes.POINTER(grav_mesh), ctypes.POINTER(grav_survey), _i, _vp, _i,
                                       _vp, ctypes.POINTER(grav_options), _vp])
_sig("grav_dense_check", _i, [_vp, _i, _i, _i, _i, _vp, ctypes.c_int64, _vp, ctypes.c_int64, _vp, ctypes.c_int64, _i,
                             _vp])
_sig("grav_datainv_solve_ex", _i, [_vp, ctypes.POINTER(grav_mesh), ctypes.POINTER(grav_survey), _vp, _vp, _vp,
                                   _vp, ctypes.POINTER(grav_solve_info), ctypes.POINTER(grav_options), _vp,
                                   _vp, _vp, _i])

EXPORTED = [
    "grav_options_default", "grav_version", "grav_ctx_create", "grav_ctx_destroy", "grav_last_error",
    "grav_ctx_sync", "grav_forward", "grav_adjoint", "grav_diag", "grav_datainv_solve", "grav_plan_create",
    "grav_plan_forward", "grav_plan_adjoint", "grav_plan_bytes", "grav_plan_destroy",
    "grav_launch_count", "grav_plan_timing", "grav_bench_pipes", "grav_plan_describe",
    "grav_serve_config", "grav_submit", "grav_poll", "grav_wait", "grav_cancel", "grav_job_times",
    "grav_job_release", "grav_job_plan", "grav_serve_plan_cache", "grav_serve_stats", "grav_eval_fn64", "grav_plan_check_fp64", "grav_datainv_solve_ex", "grav_selftest_wait",
    "grav_nystrom_coarse_apply", "grav_dense_check",
]

STAGES = ("fwd_main", "adj_main", "fwd_near", "adj_near")


def eval_fn64(fn: str, a, b=None, stream=None, ctx: Optional["Context"] = None):
    """Self-check hook: the library's FP64 log(a) / atan(a / b) ("log", "atan"),
    CUDA's ("cuda_log", "cuda_atan"), or the double-float forms of the
    near-field set-up ("df_log", "df_atan", and "df_psi" with a = (x, z)
    concatenated, b = y) on CUDA float64 tensors."""
    torch = _torch()
    ctx = ctx or context()
    code = {"log": 0, "atan": 1, "cuda_log": 2, "cuda_atan": 3, "df_log": 4, "df_atan": 5, "df_psi": 6}[fn]
    n = a.numel() // 2 if code == 6 else a.numel()
    a = _f64(a, a.numel(), "a")
    b = _f64(b, n, "b") if b is not None else None
    out = torch.empty(n, dtype=torch.float64, device=a.device)
    ctx.check(_lib.grav_eval_fn64(ctx.h, code, a.data_ptr(), b.data_ptr() if b is not None else None,
                                  out.data_ptr(), n, _stream(stream)))
    return out


def launch_count() -> int:
    """Kernels launched by libgrav so far in this process."""
    return int(_lib.grav_launch_count())


def bench_pipes(device: int = 0) -> dict:
    """Measured unit throughputs (per second) and SM clocks of the B300 pipes."""
    out = (ctypes.c_double * 27)()
    rc = _lib.grav_bench_pipes(int(device), out)
    if rc != GRAV_OK:
        raise GravError(rc, _lib.grav_last_error(None).decode())
    sms = out[10]
    r = {"sm_count": int(sms)}
    slots = [(name, 2 * k) for k, name in enumerate(("rsqrt", "lg2", "ffma", "dfma", "ffma_f32x2"))]
    slots += [(name, 11 + 2 * k) for k, name in enumerate(("log_f64", "atan_f64", "sqrt_f64", "div_f64",
                                                            "log64_table", "atan_ratio64_table", "rcp", "ex2"))]
    for name, i in slots:
        r[name + "_per_s"] = out[i]
        r[name + "_mhz"] = out[i + 1]
        r[name + "_per_clk_sm"] = out[i] / (out[i + 1] * 1e6 * sms) if out[i + 1] > 0 else 0.0
    return r


class GravError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libgrav error {code}: {msg}")
        self.code = code


def version() -> str:
    return _lib.grav_version().decode()


def _torch():
    import torch
    return torch


class Context:
    """A libgrav context on one CUDA device (owns scratch memory pool)."""

    def __init__(self, device: int = 0, hbm_budget: int = 0):
        h = _vp()
        rc = _lib.grav_ctx_create(ctypes.byref(h), int(device), int(hbm_budget))
        if rc != GRAV_OK:
            raise GravError(rc, _lib.grav_last_error(None).decode())
        self.h = h
        self.device = device

    def check(self, rc: int):
        if rc != GRAV_OK and rc != GRAV_ENOTCONVERGED:
            raise GravError(rc, _lib.grav_last_error(self.h).decode())
        return rc

    def sync(self, stream=None, timeout_s: float = 600.0):
        self.check(_lib.grav_ctx_sync(self.h, _stream(stream), timeout_s))

    def close(self):
        if getattr(self, "h", None):
            _lib.grav_ctx_destroy(self.h)
            self.h = None
            self._jobs = {}

    # ---- serving -----------------------------------------------------------
    def serve_config(self, slots: int):
        self.check(_lib.grav_serve_config(self.h, int(slots)))

    def submit(self, kind: str, mesh, survey, inp, out, m_ref=None, **opts) -> int:
        """Queue a job ("forward": out = G inp; "invert": out = m from data inp).
        The tensors are kept alive by the context until the job is released."""
        mesh, survey = Mesh.of(mesh), Survey.of(survey)
        j = grav_job()
        j.kind = GRAV_JOB_FORWARD if kind == "forward" else GRAV_JOB_INVERT
        j.mesh, j.survey = mesh.c, survey.c
        j.input, j.output = inp.data_ptr(), out.data_ptr()
        j.m_ref = m_ref.data_ptr() if m_ref is not None else None
        j.opt = options(**opts)
        jid = ctypes.c_uint64(0)
        self.check(_lib.grav_submit(self.h, ctypes.byref(j), ctypes.byref(jid)))
        if not hasattr(self, "_jobs"):
            self._jobs = {}
        self._jobs[jid.value] = (mesh, survey, inp, out, m_ref)
        return jid.value

    def poll(self, job_id: int):
        st = ctypes.c_int(0)
        info = grav_solve_info()
        self.check(_lib.grav_poll(self.h, ctypes.c_uint64(job_id), ctypes.byref(st), ctypes.byref(info)))
        return JOB_STATES[st.value], {"iters": info.iters, "converged": bool(info.converged),
                                       "true_rel_res": info.true_rel_res, "lambda": info.lambda_,
                                       "fp64_rel_err": info.fp64_rel_err, "nys_setup_s": info.nys_setup_s}

    def wait(self, job_id: int, timeout_s: float = 600.0) -> int:
        """Job result code (GRAV_OK, GRAV_ENOTCONVERGED, GRAV_ECANCELED, ...) or GRAV_ETIMEDOUT."""
        return int(_lib.grav_wait(self.h, ctypes.c_uint64(job_id), float(timeout_s)))

    def cancel(self, job_id: int):
        self.check(_lib.grav_cancel(self.h, ctypes.c_uint64(job_id)))

    def job_times(self, job_id: int):
        a, b, c = ctypes.c_double(0), ctypes.c_double(0), ctypes.c_double(0)
        self.check(_lib.grav_job_times(self.h, ctypes.c_uint64(job_id), ctypes.byref(a), ctypes.byref(b),
                                       ctypes.byref(c)))
        return a.value, b.value, c.value

    def job_plan(self, job_id: int) -> dict:
        """Whether the job ran on a resident plan, its plan set-up time and its reserved footprint."""
        r, t, b = ctypes.c_int(0), ctypes.c_double(0), ctypes.c_size_t(0)
        self.check(_lib.grav_job_plan(self.h, ctypes.c_uint64(job_id), ctypes.byref(r), ctypes.byref(t),
                                      ctypes.byref(b)))
        return {"plan_reused": bool(r.value), "setup_s": t.value, "footprint": int(b.value)}

    def plan_cache(self, max_plans: int):
        """At most max_plans idle plans stay resident (0 turns the plan cache off)."""
        self.check(_lib.grav_serve_plan_cache(self.h, int(max_plans)))

    def serve_stats(self) -> dict:
        a, b, c, d = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int(0), ctypes.c_size_t(0)
        self.check(_lib.grav_serve_stats(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)))
        return {"plans_built": a.value, "plans_reused": b.value, "plans_resident": c.value,
                "bytes_resident": int(d.value)}

    def release(self, job_id: int):
        self.check(_lib.grav_job_release(self.h, ctypes.c_uint64(job_id)))
        getattr(self, "_jobs", {}).pop(job_id, None)


_contexts = {}


def context(device: Optional[int] = None) -> Context:
    torch = _torch()
    if device is None:
        device = torch.cuda.current_device()
    if device not in _contexts:
        _contexts[device] = Context(device)
    return _contexts[device]


def _stream(stream):
    if stream is None:
        return _vp(_torch().cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return _vp(stream)
    return _vp(stream.cuda_stream)


class Mesh:
    """Rectilinear mesh: host float64 edge arrays (m); ze is depth, positive down."""

    def __init__(self, xe, ye, ze):
        self.xe = np.ascontiguousarray(xe, dtype=np.float64)
        self.ye = np.ascontiguousarray(ye, dtype=np.float64)
        self.ze = np.ascontiguousarray(ze, dtype=np.float64)
        self.c = grav_mesh(len(self.xe) - 1, len(self.ye) - 1, len(self.ze) - 1,
                           self.xe.ctypes.data_as(_D), self.ye.ctypes.data_as(_D), self.ze.ctypes.data_as(_D))

    @classmethod
    def of(cls, m) -> "Mesh":
        return m if isinstance(m, Mesh) else cls(m.xe, m.ye, m.ze)

    @property
    def ncells(self) -> int:
        return self.c.nx * self.c.ny * self.c.nz


class Survey:
    """Stations as device float64 tensors (x, y, z = -height)."""

    def __init__(self, x, y, z, device=None):
        torch = _torch()
        dev = torch.device("cuda", device if device is not None else torch.cuda.current_device())
        self.x = torch.as_tensor(x, dtype=torch.float64, device=dev).contiguous()
        self.y = torch.as_tensor(y, dtype=torch.float64, device=dev).contiguous()
        self.z = torch.as_tensor(z, dtype=torch.float64, device=dev).contiguous()
        self.c = grav_survey(self.x.numel(), self.x.data_ptr(), self.y.data_ptr(), self.z.data_ptr())

    @classmethod
    def of(cls, s) -> "Survey":
        return s if isinstance(s, Survey) else cls(s.x, s.y, s.z)

    @property
    def n(self) -> int:
        return int(self.c.n)


def options(precision="fp64", z0=50.0, lambda_scale=1e-2, lam=0.0, tol=1e-6, max_iter=1000,
            check_every=0, near_cells=8.0, timeout_s=3600.0, precond="none", cache_g=False, outer_max=0,
            inner_max=20, reorth=1000, check_stations=0, nys_rank=0, nys_coarsen=0, refine=0,
            near_fp64=False, diag_fp64=False) -> grav_options:
    o = grav_options()
    _lib.grav_options_default(ctypes.byref(o))
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.z0, o.lambda_scale, o.lambda_ = float(z0), float(lambda_scale), float(lam)
    o.tol, o.max_iter, o.check_every = float(tol), int(max_iter), int(check_every)
    o.near_cells, o.timeout_s = float(near_cells), float(timeout_s)
    o.precond = {"none": 0, "jacobi": 1, "nystrom": 2}[precond] if isinstance(precond, str) else int(precond)
    o.cache_g = int(bool(cache_g))
    o.outer_max, o.inner_max = int(outer_max), int(inner_max)
    o.reorth = int(reorth)
    o.check_stations = int(check_stations)
    o.nys_rank, o.nys_coarsen = int(nys_rank), int(nys_coarsen)
    o.refine = int(refine)
    o.near_fp64 = int(bool(near_fp64))
    o.diag_fp64 = int(bool(diag_fp64))
    return o


def _f64(t, n, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor):
        t = torch.as_tensor(np.asarray(t), dtype=torch.float64, device="cuda")
    if t.dtype != torch.float64 or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA float64 tensor")
    t = t.contiguous()
    if t.numel() != n:
        raise ValueError(f"{name} has {t.numel()} entries, expected {n}")
    return t


def forward(m, mesh, survey, stream=None, ctx: Optional[Context] = None, **opts):
    """d = G m (mGal) for density contrast m (kg/m^3), k = i + nx*(j + ny*l)."""
    torch = _torch()
    ctx = ctx or context()
    mesh, survey = Mesh.of(mesh), Survey.of(survey)
    m = _f64(m, mesh.ncells, "m")
    d = torch.empty(survey.n, dtype=torch.float64, device=m.device)
    o = options(**opts)
    ctx.check(_lib.grav_forward(ctx.h, ctypes.byref(mesh.c), ctypes.byref(survey.c), m.data_ptr(), d.data_ptr(),
                                ctypes.byref(o), _stream(stream)))
    return d


def adjoint(r, mesh, survey, depth_weighted=False, stream=None, ctx: Optional[Context] = None, **opts):
    """G^T r (times W^-2 = (zc + z0)^2 when depth_weighted)."""
    torch = _torch()
    ctx = ctx or context()
    mesh, survey = Mesh.of(mesh), Survey.of(survey)
    r = _f64(r, survey.n, "r")
    out = torch.empty(mesh.ncells, dtype=torch.float64, device=r.device)
    o = options(**opts)
    ctx.check(_lib.grav_adjoint(ctx.h, ctypes.byref(mesh.c), ctypes.byref(survey.c), r.data_ptr(), out.data_ptr(),
                                int(bool(depth_weighted)), ctypes.byref(o), _stream(stream)))
    return out


def diag(mesh, survey, stream=None, ctx: Optional[Context] = None, **opts):
    """(diag(G W^-2 G^T), trace)."""
    torch = _torch()
    ctx = ctx or context()
    mesh, survey = Mesh.of(mesh), Survey.of(survey)
    out = torch.empty(survey.n, dtype=torch.float64, device="cuda")
    tr = ctypes.c_double(0.0)
    o = options(**opts)
    ctx.check(_lib.grav_diag(ctx.h, ctypes.byref(mesh.c), ctypes.byref(survey.c), out.data_ptr(), ctypes.byref(tr),
                             ctypes.byref(o), _stream(stream)))
    return out, tr.value


def nystrom_coarse_apply(X, mesh, survey, coarsen, stream=None, ctx: Optional[Context] = None, **opts):
    """K_c X (n x k) with the explicit coarse operator of the Nystrom sketch
    (mesh coarsened `coarsen` times per axis); X: (n, k) or (n,) float64."""
    torch = _torch()
    ctx = ctx or context()
    mesh, survey = Mesh.of(mesh), Survey.of(survey)
    X = torch.as_tensor(X, dtype=torch.float64, device="cuda")
    vec = X.dim() == 1
    Xc = X.reshape(survey.n, -1).t().contiguous()   # column-major n x k = row-major k x n
    Y = torch.empty_like(Xc)
    o = options(**opts)
    ctx.check(_lib.grav_nystrom_coarse_apply(ctx.h, ctypes.byref(mesh.c), ctypes.byref(survey.c), int(coarsen),
                                             Xc.data_ptr(), Xc.shape[0], Y.data_ptr(), ctypes.byref(o),
                                             _stream(stream)))
    Y = Y.t()
    return Y.reshape(-1) if vec else Y


def datainv(d, mesh, survey, m_ref=None, return_y=False, stream=None, ctx: Optional[Context] = None, y0=None,
            res_hist=False, **opts):
    """Data-space inversion (Eq. 10-11) by CG.  Returns (m, info) or (m, y, info).
    y0: start CG from this y (e.g. an earlier call's y; resume).  res_hist:
    info["res_hist"] holds the recurrence relative residual per iteration."""
    torch = _torch()
    ctx = ctx or context()
    mesh, survey = Mesh.of(mesh), Survey.of(survey)
    d = _f64(d, survey.n, "d")
    mr = _f64(m_ref, mesh.ncells, "m_ref") if m_ref is not None else None
    yi = _f64(y0, survey.n, "y0") if y0 is not None else None
    m = torch.empty(mesh.ncells, dtype=torch.float64, device=d.device)
    y = torch.empty(survey.n, dtype=torch.float64, device=d.device) if return_y else None
    info = grav_solve_info()
    o = options(**opts)
    hist = torch.empty(max(1, o.max_iter), dtype=torch.float64, device=d.device) if res_hist else None
    rc = ctx.check(_lib.grav_datainv_solve_ex(ctx.h, ctypes.byref(mesh.c), ctypes.byref(survey.c), d.data_ptr(),
                                              mr.data_ptr() if mr is not None else None, m.data_ptr(),
                                              y.data_ptr() if y is not None else None, ctypes.byref(info),
                                              ctypes.byref(o), _stream(stream),
                                              yi.data_ptr() if yi is not None else None,
                                              hist.data_ptr() if hist is not None else None,
                                              hist.numel() if hist is not None else 0))
    inf = {"iters": info.iters, "converged": bool(info.converged), "rel_res": info.rel_res,
           "true_rel_res": info.true_rel_res, "lambda": info.lambda_, "trace": info.trace,
           "seconds": info.seconds, "status": rc, "outer": info.outer, "alpha_min": info.alpha_min,
           "restarts": info.restarts, "fp64_rel_err": info.fp64_rel_err, "nys_shift": info.nys_shift,
           "nys_setup_s": info.nys_setup_s}
    if hist is not None:
        h = hist.cpu().numpy()
        inf["res_hist"] = h[h >= 0]
    return (m, y, inf) if return_y else (m, inf)


class Plan:
    """One (mesh, survey, options) problem resident on the device."""

    def __init__(self, mesh, survey, stream=None, ctx: Optional[Context] = None, **opts):
        self.ctx = ctx or context()
        self.mesh, self.survey = Mesh.of(mesh), Survey.of(survey)
        self.opts = opts
        o = options(**opts)
        h = _vp()
        self.ctx.check(_lib.grav_plan_create(self.ctx.h, ctypes.byref(self.mesh.c), ctypes.byref(self.survey.c),
                                             ctypes.byref(o), ctypes.byref(h), _stream(stream)))
        self.h = h

    @property
    def nbytes(self) -> int:
        return int(_lib.grav_plan_bytes(self.h))

    def forward(self, m, out=None, stream=None):
        torch = _torch()
        m = _f64(m, self.mesh.ncells, "m")
        d = out if out is not None else torch.empty(self.survey.n, dtype=torch.float64, device=m.device)
        self.ctx.check(_lib.grav_plan_forward(self.h, m.data_ptr(), d.data_ptr(), _stream(stream)))
        return d

    def adjoint(self, r, depth_weighted=False, out=None, stream=None):
        torch = _torch()
        r = _f64(r, self.survey.n, "r")
        g = out if out is not None else torch.empty(self.mesh.ncells, dtype=torch.float64, device=r.device)
        self.ctx.check(_lib.grav_plan_adjoint(self.h, r.data_ptr(), g.data_ptr(), int(bool(depth_weighted)),
                                              _stream(stream)))
        return g

    def check_fp64(self, m, d, n_check=64, stream=None):
        """(max |d - d64|, that / max |d64|) at n_check evenly spaced stations,
        d64 = G m from the FP64 operator; d is this plan's product G m."""
        m = _f64(m, self.mesh.ncells, "m")
        d = _f64(d, self.survey.n, "d")
        ea, er = ctypes.c_double(0.0), ctypes.c_double(0.0)
        self.ctx.check(_lib.grav_plan_check_fp64(self.h, m.data_ptr(), d.data_ptr(), int(n_check), ctypes.byref(ea),
                                                 ctypes.byref(er), _stream(stream)))
        return ea.value, er.value

    def describe(self) -> dict:
        """Launch configuration chosen for this plan (kernels, chunking, bytes)."""
        import json
        buf = ctypes.create_string_buffer(1024)
        rc = _lib.grav_plan_describe(self.h, buf, 1024)
        if rc < 0:
            raise GravError(rc, _lib.grav_last_error(None).decode())
        return json.loads(buf.value.decode())

    def timing(self, enable: bool = True, read: bool = True):
        """Start/stop stage timing; returns {stage: (ms, count)} recorded since the last read."""
        ms = (ctypes.c_double * 4)()
        cnt = (ctypes.c_int64 * 4)()
        self.ctx.check(_lib.grav_plan_timing(self.h, int(enable), ms if read else None, cnt if read else None))
        return {STAGES[k]: (ms[k], int(cnt[k])) for k in range(4)} if read else None

    def close(self, stream=None):
        if getattr(self, "h", None):
            _lib.grav_plan_destroy(self.h, _stream(stream))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _make_autograd():
    torch = _torch()

    class GravForward(torch.autograd.Function):
        """d = G m with backward grad_m = G^T grad_d (the hand-written adjoint kernel)."""

        @staticmethod
        def forward(ctx_, m, plan: Plan):
            ctx_.plan = plan
            return plan.forward(m.detach())

        @staticmethod
        def backward(ctx_, grad_d):
            return ctx_.plan.adjoint(grad_d.contiguous()), None

    return GravForward


_GravForward = None


def GravForwardFn():
    global _GravForward
    if _GravForward is None:
        _GravForward = _make_autograd()
    return _GravForward


def gravity(m, plan: Plan):
    """Differentiable d = G m through ``plan`` (torch.autograd)."""
    return GravForwardFn().apply(m, plan)
