"""Plant plausible mistakes in a COPY of the oracle's C source (on the CPU)
and check that the independent pins catch every one of them.

Each mutant is compiled to a temporary shared library and evaluated on a
handful of pin checks (Newton-kernel derivative, Gauss-Legendre Newton
integral, on-axis solid angle, 50-digit far field, depth weighting).  A
mutant that survives all of them would mean the pins cannot see that kind of
error.
"""
import ctypes
import math
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from tests.test_oracle_pins import (ASYM_ST, ASYM_XE, ASYM_YE, ASYM_ZE, _newton_gl, _on_axis, _prism_mp,
                                    asym_expected)

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

MUTANTS = {
    "atan_sign": ("if (z != 0.0) t_atan = z * atan((x * y) / (z * R));",
                  "if (z != 0.0) t_atan = -z * atan((x * y) / (z * R));"),
    "drop_x_log": ("if (x != 0.0) t_lx = x * log_R_plus(R, y, x2 + z2);",
                   "t_lx = 0.0;"),
    "swap_log_args": ("if (x != 0.0) t_lx = x * log_R_plus(R, y, x2 + z2);",
                      "if (x != 0.0) t_lx = x * log_R_plus(R, x, y2 + z2);"),
    "parity_sign": ("double sigma = ((p + q + r) % 2 == 0) ? 1.0 : -1.0;",
                    "double sigma = ((p + q) % 2 == 0) ? 1.0 : -1.0;"),
    "naive_log": ("if (a >= 0.0) return log(R + a);", "return log(R + a);"),
    "robust_log_wrong_b2": ("if (x != 0.0) t_lx = x * log_R_plus(R, y, x2 + z2);",
                            "if (x != 0.0) t_lx = x * log_R_plus(R, y, x2 + y2);"),
    "depth_weight_top_edge": ("double zc = 0.5 * (ze[l] + ze[l + 1]) - ze[0];",
                              "double zc = ze[l] - ze[0];"),
    "z_index_shift": ("ze[l] - sz, ze[l + 1] - sz);", "ze[l] - sz, ze[l] + (ze[1] - ze[0]) - sz);"),
    # the edge arrays swapped, the station's coordinates not (swapping both is
    # no mistake: Psi and hence g_z are symmetric under x <-> y)
    "swap_xy_edges": ("oracle_prism(xe[i] - sx, xe[i + 1] - sx,\n                        ye[j] - sy, ye[j + 1] - sy,",
                      "oracle_prism(ye[j] - sx, ye[j + 1] - sx,\n                        xe[i] - sy, xe[i + 1] - sy,"),
    "swap_station_xy": ("oracle_prism(xe[i] - sx, xe[i + 1] - sx,\n                        ye[j] - sy, ye[j + 1] - sy,",
                        "oracle_prism(xe[i] - sy, xe[i + 1] - sy,\n                        ye[j] - sx, ye[j + 1] - sx,"),
    "forward_cell_order_y_fastest": ("size_t k = (size_t)i + (size_t)nx * ((size_t)j + (size_t)ny * l);",
                                     "size_t k = (size_t)j + (size_t)ny * ((size_t)i + (size_t)nx * l);"),
    "adjoint_cell_order_y_fastest": ("int i = (int)(k % nx);\n        int j = (int)((k / nx) % ny);",
                                     "int j = (int)(k % ny);\n        int i = (int)((k / ny) % nx);"),
}


def _build(src_text, tmpdir, name):
    c = os.path.join(tmpdir, name + ".c")
    so = os.path.join(tmpdir, name + ".so")
    with open(c, "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c99", c, "-o", so, "-lm"])
    lib = ctypes.CDLL(so)
    d = ctypes.c_double
    lib.oracle_psi.restype = d
    lib.oracle_psi.argtypes = [d, d, d]
    lib.oracle_prism.restype = d
    lib.oracle_prism.argtypes = [d] * 6
    P = ctypes.POINTER(d)
    lib.oracle_adjoint.argtypes = [ctypes.c_int] * 3 + [P] * 3 + [ctypes.c_int] + [P] * 3 + [P, P, ctypes.c_int, d]
    lib.oracle_forward.argtypes = [ctypes.c_int] * 3 + [P] * 3 + [ctypes.c_int] + [P] * 3 + [P, P]
    return lib


def _pins_fail(lib):
    """Return the list of pin checks the library fails."""
    failed = []
    # Newton-kernel mixed derivative
    x, y, z = 3.0, -2.0, 1.5
    def mixed(h):
        return sum(sx * sy * sz * lib.oracle_psi(x + sx * h, y + sy * h, z + sz * h)
                   for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)) / (8 * h ** 3)
    d1, d2 = mixed(0.02), mixed(0.01)
    R = math.sqrt(x * x + y * y + z * z)
    if abs((d2 + (d2 - d1) / 3) / (z / R ** 3) - 1) > 2e-6:
        failed.append("derivative")
    for box in [(150.0, 250.0, -50.0, 50.0, 30.0, 130.0), (-50.0, 50.0, -350.0, -250.0, 10.0, 110.0)]:
        if abs(lib.oracle_prism(*box) / _newton_gl(*box) - 1) > 1e-11:
            failed.append("gauss_legendre")
            break
    if abs(lib.oracle_prism(-50.0, 50.0, -80.0, 80.0, 25.0, 125.0) / _on_axis(50.0, 80.0, 25.0, 125.0) - 1) > 1e-11:
        failed.append("on_axis")
    for c in ((0.0, -20000.0, 1.0), (-9000.0, 10.0, 5.0)):
        box = (c[0] - 50, c[0] + 50, c[1] - 50, c[1] + 50, c[2], c[2] + 100)
        ref = _prism_mp(*box)
        zc = c[2] + 50.0
        R = math.sqrt(c[0] ** 2 + c[1] ** 2 + zc ** 2)
        bound = 6 * 2.2e-16 * (R / 100.0) ** 3 * (R / zc) * math.log(R)
        if abs(lib.oracle_prism(*box) - ref) / abs(ref) > bound:
            failed.append("far_field_50_digit")
            break
    # depth weighting and z indexing through the adjoint of a 1x1x3 column
    xe = np.array([0.0, 10.0]); ye = np.array([0.0, 10.0]); ze = np.array([0.0, 10.0, 30.0, 70.0])
    sx = np.array([5.0]); sy = np.array([5.0]); sz = np.array([-2.0]); r = np.array([1.0])
    out = np.zeros(3)
    P = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    lib.oracle_adjoint(1, 1, 3, P(xe), P(ye), P(ze), 1, P(sx), P(sy), P(sz), P(r), P(out), 1, 50.0)
    expect = []
    for l in range(3):
        g = oracle.GAMMA * 1e5 * _newton_gl(-5.0, 5.0, -5.0, 5.0, ze[l] + 2.0, ze[l + 1] + 2.0)
        expect.append(g * (0.5 * (ze[l] + ze[l + 1]) + 50.0) ** 2)
    if not np.allclose(out, expect, rtol=1e-9):
        failed.append("depth_weighted_adjoint")
    # x/y edge assignment and cell ordering: one cell at a time (forward) and
    # one station at a time (adjoint) on the asymmetric 3 x 2 x 2 mesh
    ref = asym_expected()
    xe, ye, ze = ASYM_XE.copy(), ASYM_YE.copy(), ASYM_ZE.copy()
    sx, sy, sz = (np.ascontiguousarray(ASYM_ST[:, c]) for c in range(3))
    ns, M = ref.shape
    G_fwd = np.zeros((ns, M))
    for k in range(M):
        m = np.zeros(M); m[k] = 1.0
        d = np.zeros(ns)
        lib.oracle_forward(3, 2, 2, P(xe), P(ye), P(ze), ns, P(sx), P(sy), P(sz), P(m), P(d))
        G_fwd[:, k] = d
    if not np.allclose(G_fwd, ref, rtol=1e-11, atol=0):
        failed.append("horizontal_geometry_forward")
    G_adj = np.zeros((ns, M))
    for s in range(ns):
        r = np.zeros(ns); r[s] = 1.0
        out = np.zeros(M)
        lib.oracle_adjoint(3, 2, 2, P(xe), P(ye), P(ze), ns, P(sx), P(sy), P(sz), P(r), P(out), 0, 50.0)
        G_adj[s] = out
    if not np.allclose(G_adj, ref, rtol=1e-11, atol=0):
        failed.append("horizontal_geometry_adjoint")
    return failed


def test_unmutated_oracle_passes_mutation_pins():
    with tempfile.TemporaryDirectory() as td:
        lib = _build(open(SRC).read(), td, "orig")
        assert _pins_fail(lib) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name):
    before, after = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(before) == 1, f"mutation anchor not found for {name}"
    with tempfile.TemporaryDirectory() as td:
        lib = _build(text.replace(before, after), td, name)
        assert _pins_fail(lib), f"mutant {name} survived every pin"
