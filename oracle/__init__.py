"""CPU ORACLE for the prism-gravity operator and the data-space inversion.

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / --impl reference leg may import this package; the CUDA
library (paper_2602_03857_b300) never does, and this package never imports
it.  The two share only the seeded input generators in ``synth``.

Contents
  * oracle.c (built to liboracle.so by ``build()``): FP64 per-prism operator,
    one prism at a time, Eq. 1-6 (forward d = G m, adjoint G^T r, explicit G,
    diag of G W^-2 G^T).
  * numpy solvers written in the paper's order and notation:
      - ``lambda_from_trace``: W_d = lambda*I with lambda = 1e-2 * trace(G W_m G^T)/N
        (the data weighting is diagonal with one value, Section 2.2; the
        1e-2 * trace / N rule is the reading adopted for that value).
      - ``modelspace_solve``: Eq. 8, (G^T W_d^-1 G + W_m^-1)(m - m_ref) = G^T W_d^-1 (d - G m_ref).
      - ``dataspace_solve``: Eq. 10-11, dm = W_m G^T (G W_m G^T + W_d)^-1 dd,
        dd = d - G m_ref, with a dense LU (numpy.linalg.solve).
      - ``dataspace_cg``: the same N x N system by plain conjugate gradients
        (Section 3.1 and Section 2.2: iterative CG, no factorisation).
    W_m = W^-2 = diag((zc + z0)^2), the depth weighting read as
    w(z) = (z + z0)^-1 with zc the cell-centre depth below the mesh top.

Parity status: every function here is pinned by tests/test_oracle_pins.py
against closed forms, an independent quadrature or algebraic identities;
nothing is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Callable, Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

GAMMA = 6.67430e-11          # m^3 kg^-1 s^-2 (CODATA 2018)
SI_TO_MGAL = 1.0e5


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc -O2 -fopenmp into liboracle.so (in-tree)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99",
               "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", _LIB_PATH, "-lm"]
        subprocess.check_call(cmd)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    P = ctypes.POINTER(ctypes.c_double)
    i, d = ctypes.c_int, ctypes.c_double
    lib.oracle_psi.restype = d
    lib.oracle_psi.argtypes = [d, d, d]
    lib.oracle_prism.restype = d
    lib.oracle_prism.argtypes = [d] * 6
    lib.oracle_gamma.restype = d
    geo = [i, i, i, P, P, P, i, P, P, P]
    lib.oracle_forward.argtypes = geo + [P, P]
    lib.oracle_adjoint.argtypes = geo + [P, P, i, d]
    lib.oracle_G.argtypes = geo + [P]
    lib.oracle_diag.argtypes = geo + [d, P]
    lib.oracle_set_threads.argtypes = [i]
    lib.oracle_get_threads.restype = i
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def get_threads() -> int:
    return int(_load().oracle_get_threads())


def psi(x: float, y: float, z: float) -> float:
    """Eq. 2 corner function (station at the origin, z positive down)."""
    return float(_load().oracle_psi(x, y, z))


def prism(x1, x2, y1, y2, z1, z2) -> float:
    """Eq. 1 parity sum without gamma*rho."""
    return float(_load().oracle_prism(x1, x2, y1, y2, z1, z2))


def _geo(mesh, survey):
    xe, ye, ze = _c(mesh.xe), _c(mesh.ye), _c(mesh.ze)
    sx, sy, sz = _c(survey.x), _c(survey.y), _c(survey.z)
    keep = (xe, ye, ze, sx, sy, sz)
    args = [len(xe) - 1, len(ye) - 1, len(ze) - 1, _ptr(xe), _ptr(ye), _ptr(ze),
            len(sx), _ptr(sx), _ptr(sy), _ptr(sz)]
    return args, keep


def forward(mesh, survey, m) -> np.ndarray:
    """d = G m in mGal (Eq. 5-6)."""
    lib = _load()
    args, keep = _geo(mesh, survey)
    m = _c(m)
    d = np.zeros(survey.n)
    lib.oracle_forward(*args, _ptr(m), _ptr(d))
    return d


def adjoint(mesh, survey, r, depth_weighted: bool = False, z0: float = 50.0) -> np.ndarray:
    """G^T r, optionally times W^-2 = (zc + z0)^2."""
    lib = _load()
    args, keep = _geo(mesh, survey)
    r = _c(r)
    out = np.zeros(mesh.ncells)
    lib.oracle_adjoint(*args, _ptr(r), _ptr(out), int(bool(depth_weighted)), float(z0))
    return out


def G_explicit(mesh, survey) -> np.ndarray:
    """Dense G [N, M] in mGal per (kg/m^3)."""
    lib = _load()
    args, keep = _geo(mesh, survey)
    G = np.zeros((survey.n, mesh.ncells))
    lib.oracle_G(*args, _ptr(G))
    return G


def diag_GWG(mesh, survey, z0: float) -> np.ndarray:
    """diag(G W^-2 G^T)_i = sum_k G_ik^2 (zc_k + z0)^2."""
    lib = _load()
    args, keep = _geo(mesh, survey)
    out = np.zeros(survey.n)
    lib.oracle_diag(*args, float(z0), _ptr(out))
    return out


def depth_w2(mesh, z0: float) -> np.ndarray:
    """W_m = W^-2 = diag((zc + z0)^2) per cell, k = i + nx*(j + ny*l)."""
    zc = 0.5 * (mesh.ze[:-1] + mesh.ze[1:]) - mesh.ze[0]
    w2 = (zc + z0) ** 2
    return np.repeat(w2, mesh.nx * mesh.ny)


def lambda_from_trace(trace: float, n: int, scale: float = 1e-2) -> float:
    return scale * trace / n


def dataspace_solve(G: np.ndarray, d: np.ndarray, m_ref: np.ndarray, wm: np.ndarray,
                    lam: float) -> Tuple[np.ndarray, np.ndarray]:
    """Eq. 10-11 with a dense LU: returns (m, y) with
    y = (G W_m G^T + lam I)^-1 (d - G m_ref) and m = m_ref + W_m G^T y."""
    dd = d - G @ m_ref
    A = (G * wm[None, :]) @ G.T + lam * np.eye(G.shape[0])
    y = np.linalg.solve(A, dd)
    return m_ref + wm * (G.T @ y), y


def modelspace_solve(G: np.ndarray, d: np.ndarray, m_ref: np.ndarray, wm: np.ndarray,
                     lam: float) -> np.ndarray:
    """Eq. 8 with W_d = lam I: (G^T G / lam + W_m^-1)(m - m_ref) = G^T (d - G m_ref) / lam."""
    dd = d - G @ m_ref
    A = G.T @ G / lam + np.diag(1.0 / wm)
    return m_ref + np.linalg.solve(A, G.T @ dd / lam)


def dataspace_cg(apply_A: Callable[[np.ndarray], np.ndarray], b: np.ndarray, tol: float,
                 max_iter: int) -> Tuple[np.ndarray, int, float]:
    """Plain CG on A y = b from y0 = 0; stops when ||r|| <= tol ||b||.
    Returns (y, iterations, final relative recurrence residual)."""
    y = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = float(r @ r)
    bnorm = float(np.sqrt(b @ b))
    it = 0
    if bnorm == 0.0:
        return y, 0, 0.0
    while it < max_iter and np.sqrt(rr) > tol * bnorm:
        Ap = apply_A(p)
        alpha = rr / float(p @ Ap)
        y += alpha * p
        r -= alpha * Ap
        rr_new = float(r @ r)
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return y, it, float(np.sqrt(rr) / bnorm)


def invert_dense(mesh, survey, d: np.ndarray, m_ref: Optional[np.ndarray] = None,
                 z0: float = 50.0, lam_scale: float = 1e-2):
    """Full data-space inversion on a small problem with explicit G and dense LU.
    Returns dict(m, y, lam, G)."""
    G = G_explicit(mesh, survey)
    wm = depth_w2(mesh, z0)
    if m_ref is None:
        m_ref = np.zeros(mesh.ncells)
    trace = float(np.sum((G * G) @ wm))
    lam = lambda_from_trace(trace, survey.n, lam_scale)
    m, y = dataspace_solve(G, d, m_ref, wm, lam)
    return {"m": m, "y": y, "lam": lam, "G": G, "wm": wm}
