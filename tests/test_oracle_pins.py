"""Pins that tie the CPU oracle to results it does not share code with.

Each test names what fixes the expected value: a closed form, an independent
quadrature of Newton's integral, an algebraic identity of the paper
(Eq. 9), or a symmetry of the field.  A plausible mistake in the oracle (a
dropped term of Eq. 2, a wrong parity sign in Eq. 1, a swapped coordinate, a
wrong depth-weight index, a transposed G) fails at least one of them.
"""
import functools
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
GAMMA = 6.67430e-11


def prism_g(x1, x2, y1, y2, z1, z2):
    return oracle.prism(x1, x2, y1, y2, z1, z2)


# --- Eq. 2-3: the corner function is a triple antiderivative of z/R^3 -------

@pytest.mark.parametrize("pt", [(3.0, 2.0, 1.5), (-4.0, 1.0, 2.0), (0.7, -2.5, 0.9),
                                (-1.3, -0.4, 3.3), (12.0, -7.0, 4.0)])
def test_psi_mixed_third_derivative_is_newton_kernel(pt):
    """d^3 Psi / dx dy dz = z / R^3 (Newton kernel of g_z, z down): central
    mixed difference with Richardson extrapolation.  Fixes the sign and every
    term of Eq. 2 (dropping or flipping any term changes the derivative)."""
    x, y, z = pt

    def mixed(h):
        s = 0.0
        for sx in (-1, 1):
            for sy in (-1, 1):
                for sz in (-1, 1):
                    s += sx * sy * sz * oracle.psi(x + sx * h, y + sy * h, z + sz * h)
        return s / (8 * h ** 3)

    h = 0.02
    d1, d2 = mixed(h), mixed(h / 2)
    est = d2 + (d2 - d1) / 3.0          # Richardson: O(h^4)
    R = math.sqrt(x * x + y * y + z * z)
    assert est == pytest.approx(z / R ** 3, rel=2e-6)


# --- Eq. 1: point-mass limit ----------------------------------------------

@pytest.mark.parametrize("direction", [(0, 0, 1), (1, 0, 1), (1, -2, 1.5), (-3, 1, 0.5)])
def test_point_mass_limit_fourth_order(direction):
    """A cube of side a seen from distance R tends to the point mass
    a^3 dz / R^3; its quadrupole vanishes, so the relative error falls as
    (a/R)^4: the error ratio between R and 2R is 16 (within 3 %)."""
    u = np.array(direction, float)
    u /= np.linalg.norm(u)
    a = 1.0
    errs = []
    for R in (15.0, 30.0):
        c = R * u
        v = prism_g(c[0] - a / 2, c[0] + a / 2, c[1] - a / 2, c[1] + a / 2, c[2] - a / 2, c[2] + a / 2)
        pm = a ** 3 * c[2] / R ** 3
        errs.append((v - pm) / pm)
        assert abs(v - pm) / pm < 2.0 * (a / R) ** 4 + 1e-12
    if abs(errs[1]) > 1e-11:
        assert errs[0] / errs[1] == pytest.approx(16.0, rel=0.03)


# --- Eq. 1: independent Newton integral by tensor Gauss-Legendre ------------

def _newton_gl(x1, x2, y1, y2, z1, z2, n=24, sub=4):
    """g_z/(gamma rho) = int z / r^3 dV by an n-point Gauss-Legendre rule on a
    sub^3 split of the box (no use of Psi)."""
    t, w = np.polynomial.legendre.leggauss(n)
    tot = 0.0
    xs = np.linspace(x1, x2, sub + 1)
    ys = np.linspace(y1, y2, sub + 1)
    zs = np.linspace(z1, z2, sub + 1)
    for a in range(sub):
        X = 0.5 * (xs[a + 1] - xs[a]) * t + 0.5 * (xs[a + 1] + xs[a]); wx = 0.5 * (xs[a + 1] - xs[a]) * w
        for b in range(sub):
            Y = 0.5 * (ys[b + 1] - ys[b]) * t + 0.5 * (ys[b + 1] + ys[b]); wy = 0.5 * (ys[b + 1] - ys[b]) * w
            for c in range(sub):
                Z = 0.5 * (zs[c + 1] - zs[c]) * t + 0.5 * (zs[c + 1] + zs[c]); wz = 0.5 * (zs[c + 1] - zs[c]) * w
                XX, YY, ZZ = np.meshgrid(X, Y, Z, indexing="ij")
                W = wx[:, None, None] * wy[None, :, None] * wz[None, None, :]
                R2 = XX ** 2 + YY ** 2 + ZZ ** 2
                tot += float(np.sum(W * ZZ / R2 ** 1.5))
    return tot


@pytest.mark.parametrize("box", [
    (150.0, 250.0, -50.0, 50.0, 30.0, 130.0),       # beside, shallow
    (-320.0, -220.0, 80.0, 180.0, 100.0, 200.0),    # x < 0, y > 0
    (-50.0, 50.0, -350.0, -250.0, 10.0, 110.0),     # y < 0
    (40.0, 140.0, 40.0, 140.0, 60.0, 160.0),        # diagonal
    (-20.0, 180.0, -260.0, -60.0, 120.0, 170.0),    # non-cubic, straddles x = 0
])
def test_newton_integral_gauss_legendre(box):
    v = prism_g(*box)
    ref = _newton_gl(*box)
    assert v == pytest.approx(ref, rel=1e-11)


# --- on-axis closed form via the solid angle; Bouguer slab limit -----------

def _on_axis(a, b, z1, z2):
    """Station on the vertical axis of a prism with half-sides a, b: a thin
    horizontal lamina at depth z attracts with gamma*sigma*Omega(z), Omega the
    solid angle 4*atan(a b / (z sqrt(a^2 + b^2 + z^2))); integrate over z."""
    from scipy.integrate import quad
    f = lambda z: 4.0 * math.atan(a * b / (z * math.sqrt(a * a + b * b + z * z)))
    v, err = quad(f, z1, z2, epsabs=0, epsrel=1e-13, limit=400)
    return v


@pytest.mark.parametrize("a,b,z1,z2", [(50.0, 50.0, 1.0, 101.0), (50.0, 80.0, 25.0, 125.0),
                                       (500.0, 20.0, 5.0, 300.0), (10.0, 10.0, 1000.0, 1010.0)])
def test_on_axis_solid_angle(a, b, z1, z2):
    assert prism_g(-a, a, -b, b, z1, z2) == pytest.approx(_on_axis(a, b, z1, z2), rel=1e-11)


def test_bouguer_slab_limit():
    """Laterally infinite slab of thickness t: g = 2 pi gamma rho t."""
    t, h = 100.0, 10.0
    vals = []
    for L in (1e4, 1e5, 1e6):
        v = prism_g(-L, L, -L, L, h, h + t)
        vals.append(abs(v / (2 * math.pi * t) - 1.0))
        assert v == pytest.approx(_on_axis(L, L, h, h + t), rel=1e-10)
    assert vals[0] < 1e-2 and vals[1] < 1e-3 and vals[2] < 1e-4
    assert vals[0] > vals[1] > vals[2]


# --- superposition, symmetry, mirror, translation ---------------------------

def test_superposition_eight_subprisms():
    rng = np.random.Generator(np.random.PCG64(3))
    for _ in range(20):
        x1, y1 = rng.uniform(-200, 200, 2)
        z1 = rng.uniform(0.5, 100)
        dx, dy, dz = rng.uniform(5, 150, 3)
        x2, y2, z2 = x1 + dx, y1 + dy, z1 + dz
        xm, ym, zm = rng.uniform(x1, x2), rng.uniform(y1, y2), rng.uniform(z1, z2)
        whole = prism_g(x1, x2, y1, y2, z1, z2)
        parts = 0.0
        for xa, xb in ((x1, xm), (xm, x2)):
            for ya, yb in ((y1, ym), (ym, y2)):
                for za, zb in ((z1, zm), (zm, z2)):
                    parts += prism_g(xa, xb, ya, yb, za, zb)
        assert parts == pytest.approx(whole, rel=1e-11, abs=1e-13 * abs(whole) + 1e-14)


def test_symmetry_centred_body():
    """Field of a centred square body is invariant under x->-x, y->-y, x<->y."""
    mesh = synth.uniform_mesh(10, 10, 5, 20.0, 20.0, 20.0, x0=-100.0, y0=-100.0)
    m = np.zeros((5, 10, 10)); m[1:4, 3:7, 3:7] = 250.0; m = m.ravel()
    xs = np.linspace(-150, 150, 7)
    X, Y = np.meshgrid(xs, xs, indexing="xy")
    sv = synth.Survey(X.ravel(), Y.ravel(), np.full(X.size, -7.0))
    d = oracle.forward(mesh, sv, m).reshape(7, 7)     # [y, x]
    scale = np.abs(d).max()
    assert np.allclose(d, d[:, ::-1], rtol=0, atol=1e-12 * scale)
    assert np.allclose(d, d[::-1, :], rtol=0, atol=1e-12 * scale)
    assert np.allclose(d, d.T, rtol=0, atol=1e-12 * scale)
    assert d[3, 3] == d.max() and d.min() > 0


def test_z_mirror_and_translation():
    """Station at height h above a body vs station at h below the mirrored
    body: g_z flips sign.  Joint translation of station and prism: unchanged."""
    rng = np.random.Generator(np.random.PCG64(5))
    for _ in range(10):
        x1, y1 = rng.uniform(-100, 100, 2)
        z1 = rng.uniform(1, 50)
        x2, y2, z2 = x1 + rng.uniform(5, 60), y1 + rng.uniform(5, 60), z1 + rng.uniform(5, 60)
        g = prism_g(x1, x2, y1, y2, z1, z2)
        g_mirror = prism_g(x1, x2, y1, y2, -z2, -z1)
        assert g_mirror == pytest.approx(-g, rel=1e-12)
        sx, sy, sz = rng.uniform(-1e4, 1e4, 3)
        g_t = oracle.prism((x1 + sx) - sx, (x2 + sx) - sx, (y1 + sy) - sy, (y2 + sy) - sy,
                           (z1 + sz) - sz, (z2 + sz) - sz)
        assert g_t == pytest.approx(g, rel=1e-9)


# --- high-precision check of the cancellation-free evaluation ---------------

def _prism_mp(x1, x2, y1, y2, z1, z2, dps=50):
    import mpmath as mp
    mp.mp.dps = dps

    def psi(x, y, z):
        x, y, z = mp.mpf(x), mp.mpf(y), mp.mpf(z)
        R = mp.sqrt(x * x + y * y + z * z)
        t = z * mp.atan(x * y / (z * R))
        if x != 0:
            t -= x * mp.log(R + y)
        if y != 0:
            t -= y * mp.log(R + x)
        return t
    s = mp.mpf(0)
    for p, xv in ((1, x1), (2, x2)):
        for q, yv in ((1, y1), (2, y2)):
            for r, zv in ((1, z1), (2, z2)):
                s += (-1) ** (p + q + r) * psi(xv, yv, zv)
    return float(s)


@pytest.mark.parametrize("c", [(3000.0, 0.0, 50.0), (-9000.0, 10.0, 5.0), (20.0, -12000.0, 30.0),
                               (-2500.0, -2500.0, 400.0), (0.0, -20000.0, 1.0), (-15000.0, 30.0, 2.0)])
def test_far_field_rounding_vs_50_digit(c):
    """At R/a = 30-120 the FP64 corner sum keeps the relative error of a
    rounding-limited evaluation: |Psi| ~ R ln R against a result of
    a^3 zc / R^3, i.e. eps * (R/a)^3 * (R/zc) * ln R (grazing geometries,
    zc << R, lose the extra R/zc).  The constant 6 leaves a 2x margin over
    the worst case seen; the naive ln(R+y) for y << 0 exceeds it 2-17x on
    the far-side geometries (-9000,10,5), (20,-12000,30), (0,-20000,1),
    (-15000,30,2)."""
    a = 100.0
    box = (c[0] - a / 2, c[0] + a / 2, c[1] - a / 2, c[1] + a / 2, c[2], c[2] + a)
    v = prism_g(*box)
    ref = _prism_mp(*box)
    zc = c[2] + a / 2
    R = math.sqrt(c[0] ** 2 + c[1] ** 2 + zc ** 2)
    bound = 6 * 2.2e-16 * (R / a) ** 3 * (R / zc) * math.log(R)
    assert abs(v - ref) / abs(ref) < bound


# --- operator-level consistency: transpose, dot test, diag -----------------

def test_transpose_and_dot():
    mesh, sv, m = synth.small_random_problem(5, 4, 3, 17, seed=1, irregular=True)
    G = oracle.G_explicit(mesh, sv)
    d = oracle.forward(mesh, sv, m)
    assert np.allclose(d, G @ m, rtol=1e-12, atol=1e-12 * np.abs(d).max())
    r = synth.random_vector(sv.n, 2)
    gtr = oracle.adjoint(mesh, sv, r)
    assert np.allclose(gtr, G.T @ r, rtol=1e-12, atol=1e-12 * np.abs(gtr).max())
    lhs, rhs = float(d @ r), float(m @ gtr)
    assert lhs == pytest.approx(rhs, rel=1e-12)
    wm = oracle.depth_w2(mesh, 50.0)
    gtrw = oracle.adjoint(mesh, sv, r, depth_weighted=True, z0=50.0)
    assert np.allclose(gtrw, wm * (G.T @ r), rtol=1e-12, atol=1e-12 * np.abs(gtrw).max())
    diag = oracle.diag_GWG(mesh, sv, 50.0)
    assert np.allclose(diag, (G * G) @ wm, rtol=1e-12)


# --- horizontal geometry: x/y edge assignment and the cell ordering --------

# A mesh with nx != ny, unequal x, y and z spacings and x0 != y0, seen from
# stations that sit off every axis of symmetry: swapping the x and y edges,
# the station's x and y, or the order of i and j in k changes every value.
ASYM_XE = -37.0 + np.array([0.0, 10.0, 20.0, 30.0])
ASYM_YE = 112.0 + np.array([0.0, 25.0, 50.0])
ASYM_ZE = np.array([0.0, 15.0, 35.0])
ASYM_ST = np.array([[-57.0, 172.0, -30.0], [8.0, 97.0, -40.0], [-32.0, 122.0, -25.0], [-9.0, 149.0, -33.0]])


@functools.lru_cache(maxsize=1)
def asym_expected():
    """G[s, k] of the asymmetric mesh from the Newton integral of each cell's
    explicit box [xe_i, xe_i+1] x [ye_j, ye_j+1] x [ze_l, ze_l+1], with
    k = i + nx (j + ny l) (x fastest), by Gauss-Legendre (no Psi)."""
    nx, ny, nz = len(ASYM_XE) - 1, len(ASYM_YE) - 1, len(ASYM_ZE) - 1
    G = np.zeros((len(ASYM_ST), nx * ny * nz))
    for s, (sx, sy, sz) in enumerate(ASYM_ST):
        for l in range(nz):
            for j in range(ny):
                for i in range(nx):
                    k = i + nx * (j + ny * l)
                    G[s, k] = GAMMA * 1e5 * _newton_gl(ASYM_XE[i] - sx, ASYM_XE[i + 1] - sx,
                                                       ASYM_YE[j] - sy, ASYM_YE[j + 1] - sy,
                                                       ASYM_ZE[l] - sz, ASYM_ZE[l + 1] - sz)
    return G


def test_horizontal_geometry_and_cell_order_one_cell_at_a_time():
    """One non-zero cell at a time: the oracle's forward, adjoint and explicit
    G reproduce the Newton integral of that cell's own box at off-axis
    stations (Eq. 1 and Eq. 4-6, cell k = i + nx (j + ny l)).  This fixes the
    x/y edge assignment and the (i, j, l) -> k ordering, which the symmetric
    pins above cannot see."""
    mesh = synth.Mesh(ASYM_XE.copy(), ASYM_YE.copy(), ASYM_ZE.copy())
    sv = synth.Survey(ASYM_ST[:, 0].copy(), ASYM_ST[:, 1].copy(), ASYM_ST[:, 2].copy())
    ref = asym_expected()
    assert mesh.ncells == ref.shape[1] == 12
    for k in range(mesh.ncells):
        m = np.zeros(mesh.ncells)
        m[k] = 1.0
        d = oracle.forward(mesh, sv, m)
        assert np.allclose(d, ref[:, k], rtol=1e-11, atol=0), k
    for s in range(sv.n):
        r = np.zeros(sv.n)
        r[s] = 1.0
        assert np.allclose(oracle.adjoint(mesh, sv, r), ref[s], rtol=1e-11, atol=0), s
    assert np.allclose(oracle.G_explicit(mesh, sv), ref, rtol=1e-11, atol=0)
    # the values really differ under the mistakes this pin is for
    swapped = ref.reshape(sv.n, 2, 2, 3).transpose(0, 1, 3, 2).reshape(sv.n, -1)
    assert np.abs(swapped - ref).max() > 1e-3 * np.abs(ref).max()


def test_depth_weight_indexing():
    """W^-2 = (zc + z0)^2 with zc the cell-centre depth below the mesh top,
    constant over each layer (k = i + nx*(j + ny*l))."""
    mesh = synth.Mesh(np.array([0.0, 1.0, 3.0]), np.array([0.0, 2.0]), np.array([0.0, 10.0, 30.0, 70.0]))
    w = oracle.depth_w2(mesh, 50.0)
    assert list(w) == [55.0 ** 2] * 2 + [70.0 ** 2] * 2 + [100.0 ** 2] * 2


def test_units_mgal():
    """1000 kg/m^3 cube of 100 m with centre 1 km below: point mass
    gamma * 1e9 kg / (1e3 m)^2 = 6.6743e-5 m/s^2 = 6.6743 mGal (within 1e-5)."""
    mesh = synth.uniform_mesh(1, 1, 1, 100.0, 100.0, 100.0, x0=-50.0, y0=-50.0)
    mesh.ze = mesh.ze + 950.0
    sv = synth.Survey(np.array([0.0]), np.array([0.0]), np.array([0.0]))
    d = oracle.forward(mesh, sv, np.array([1000.0]))
    assert d[0] == pytest.approx(GAMMA * 1e9 / 1e6 * 1e5, rel=1e-5)


# --- Eq. 8 vs Eq. 10-11 through the push-through identity Eq. 9; CG ---------

def test_dataspace_equals_modelspace_and_cg():
    mesh, sv, m_true = synth.small_random_problem(6, 5, 4, 23, seed=4)
    G = oracle.G_explicit(mesh, sv)
    d = G @ m_true + synth.random_vector(sv.n, 5, 0.01)
    wm = oracle.depth_w2(mesh, 50.0)
    lam = oracle.lambda_from_trace(float(np.sum((G * G) @ wm)), sv.n)
    m_ref = np.full(mesh.ncells, 0.1)
    m_ds, y = oracle.dataspace_solve(G, d, m_ref, wm, lam)
    m_ms = oracle.modelspace_solve(G, d, m_ref, wm, lam)
    assert np.allclose(m_ds, m_ms, rtol=1e-8, atol=1e-9 * np.abs(m_ds).max())
    A = lambda p: G @ (wm * (G.T @ p)) + lam * p
    y_cg, it, rel = oracle.dataspace_cg(A, d - G @ m_ref, 1e-12, 500)
    assert rel <= 1e-12
    assert np.allclose(y_cg, y, rtol=1e-8, atol=1e-9 * np.abs(y).max())
    # the data-space minimiser makes the gradient of Eq. 7 vanish
    grad = -G.T @ (d - G @ m_ds) / lam + (m_ds - m_ref) / wm
    assert np.abs(grad).max() < 1e-8 * np.abs(G.T @ d / lam).max()


# --- the paper's printed shape arithmetic (tests/golden) --------------------

def test_paper_dense_G_sizes():
    with open(os.path.join(GOLDEN, "paper_dense_G_sizes.json")) as f:
        rows = json.load(f)["rows"]
    for row in rows:
        gb = row["cells"] * row["obs"] * 4 / 1e9
        assert gb == pytest.approx(row["gb"], abs=row.get("abs_tol", 0.01)), row["cite"]
    # the mesh shape of the regional sections matches their cell counts
    assert 322 * 187 * 10 == 602_140 and 322 * 186 * 10 == 598_920


def test_golden_block_forward_regression():
    """The block workload's forward data, written by tests/golden/make_golden.py
    (which calls only the oracle), is reproduced bit-for-bit-close."""
    gold = np.loadtxt(os.path.join(GOLDEN, "block_20x20x10_forward.txt"))
    wl = synth.make_workload("block_20x20x10")
    d = oracle.forward(wl.mesh, wl.survey, wl.m)
    assert np.allclose(d, gold, rtol=1e-13, atol=1e-15)
