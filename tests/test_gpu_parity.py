"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs.

Tolerances of the product's accuracy requirement:
  FP64 mode:  |d_gpu - d_oracle| <= 1e-10 * max|d_oracle|   (same for G^T r)
  mixed mode: |d_gpu - d_oracle| <= 1e-5  * max|d_oracle|
Sizes span several CTA tiles with ragged tails; edge cases cover n = 1,
one-cell-wide meshes, stations above nodes and edges, and stations outside
the mesh footprint.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOLMIX = 1e-5


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_03857_b300 as g
    return g


def _rel(a, b):
    a = np.asarray(a); b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _dev(x):
    return torch.as_tensor(np.asarray(x, dtype=np.float64), device="cuda")


# ---------------------------------------------------------------- FP64 -----

@pytest.mark.parametrize("shape,ns,irregular,seed", [
    ((5, 4, 3), 17, True, 1), ((1, 1, 1), 1, False, 2), ((1, 7, 2), 33, True, 3),
    ((9, 1, 4), 40, False, 4), ((13, 11, 7), 300, True, 5), ((24, 19, 9), 700, False, 6),
])
def test_forward_adjoint_fp64_small(g, shape, ns, irregular, seed):
    mesh, sv, m = synth.small_random_problem(*shape, ns, seed=seed, irregular=irregular)
    d_ref = oracle.forward(mesh, sv, m)
    d = g.forward(_dev(m), mesh, g.Survey(sv.x, sv.y, sv.z)).cpu().numpy()
    assert _rel(d, d_ref) <= TOL64
    r = synth.random_vector(sv.n, seed)
    for dw in (False, True):
        a_ref = oracle.adjoint(mesh, sv, r, depth_weighted=dw, z0=50.0)
        a = g.adjoint(_dev(r), mesh, g.Survey(sv.x, sv.y, sv.z), depth_weighted=dw).cpu().numpy()
        assert _rel(a, a_ref) <= TOL64


def test_stations_above_nodes_edges_and_outside(g):
    mesh = synth.uniform_mesh(6, 5, 4, 10.0, 10.0, 10.0)
    xs = np.array([0.0, 10.0, 30.0, 35.0, 60.0, -25.0, 95.0, 30.0, 0.0])
    ys = np.array([0.0, 20.0, 25.0, 50.0, 50.0, 10.0, -40.0, 0.0, 50.0])
    zs = -np.array([1.0, 0.5, 2.0, 3.0, 1e-3, 4.0, 7.0, 20.0, 0.25])
    sv = synth.Survey(xs, ys, zs)
    m = synth.random_vector(mesh.ncells, 9, 200.0)
    d_ref = oracle.forward(mesh, sv, m)
    d = g.forward(_dev(m), mesh, g.Survey(xs, ys, zs)).cpu().numpy()
    assert _rel(d, d_ref) <= TOL64
    r = synth.random_vector(sv.n, 10)
    a_ref = oracle.adjoint(mesh, sv, r)
    a = g.adjoint(_dev(r), mesh, g.Survey(xs, ys, zs)).cpu().numpy()
    assert _rel(a, a_ref) <= TOL64


@pytest.mark.parametrize("diag_fp64", [False, True])
def test_diag_fp64(g, diag_fp64):
    mesh, sv, _ = synth.small_random_problem(11, 9, 6, 150, seed=12, irregular=True)
    ref = oracle.diag_GWG(mesh, sv, 50.0)
    dg, tr = g.diag(mesh, g.Survey(sv.x, sv.y, sv.z), diag_fp64=diag_fp64)
    dg = dg.cpu().numpy()
    assert _rel(dg, ref) <= TOL64
    assert float(np.max(np.abs(dg - ref) / ref)) <= TOL64   # every entry, relative to itself
    assert tr == pytest.approx(ref.sum(), rel=1e-10)


@pytest.mark.parametrize("shape,ns,seed", [
    ((1, 1, 1), 5, 41), ((31, 2, 16), 40, 42), ((32, 3, 17), 60, 43), ((62, 5, 33), 90, 44),
    ((63, 1, 2), 33, 45), ((5, 70, 3), 70, 46), ((2, 2, 48), 200, 47),
])
def test_diag_double_float_shapes(g, shape, ns, seed):
    """The double-float diagonal at the edges of its layout: one cell; x
    segments of exactly 31 and 32 cells and one past two segments; layer
    groups of exactly 16 layers, one layer over, several groups with a
    ragged last one; long y (more rows than a 32-row broadcast block); many
    stations over a thin column (several row chunks)."""
    mesh, sv, _ = synth.small_random_problem(*shape, ns, seed=seed, irregular=True)
    ref = oracle.diag_GWG(mesh, sv, 50.0)
    dg, tr = g.diag(mesh, g.Survey(sv.x, sv.y, sv.z))
    dg = dg.cpu().numpy()
    assert float(np.max(np.abs(dg - ref) / ref)) <= TOL64
    assert tr == pytest.approx(ref.sum(), rel=1e-12)


def test_diag_double_float_against_fp64(g):
    """The default diagonal (corner function in double-float) against the FP64
    kernel's, entry by entry: several 31-cell x segments with a ragged last
    one, layer groups with a ragged last one, several row chunks, irregular
    spacing, stations above nodes and edges and outside the footprint; then
    every station of the 80 x 80 x 40 slab workload.  A diagonal entry is a
    sum of squares, so the double-float corner function's ~2^-45 per node
    stays near 1e-13 of the entry; stations far outside the footprint, whose
    entries are all far field (large corner values, small differences), lose
    most (1.1e-11 measured for the station 300 m off this mesh's edge)."""
    mesh, sv, _ = synth.small_random_problem(70, 45, 37, 1500, seed=31, irregular=True)
    xs = np.concatenate([sv.x, mesh.xe[[0, 5, 70]], [mesh.xe[0] - 300.0, mesh.xe[-1] + 50.0]])
    ys = np.concatenate([sv.y, mesh.ye[[0, 20, 45]], [mesh.ye[-1] + 10.0, mesh.ye[0] - 400.0]])
    zs = np.concatenate([sv.z, -np.array([0.5, 2.0, 1e-3, 5.0, 30.0])])
    S = g.Survey(xs, ys, zs)
    ddf, tdf = g.diag(mesh, S)
    d64, t64 = g.diag(mesh, S, diag_fp64=True)
    ddf, d64 = ddf.cpu().numpy(), d64.cpu().numpy()
    assert np.all(d64 > 0)
    assert float(np.max(np.abs(ddf - d64) / d64)) <= TOL64
    assert float(np.max(np.abs(ddf - d64)[:1500] / d64[:1500])) <= 1e-11   # stations over or near the mesh
    assert tdf == pytest.approx(t64, rel=1e-12)
    w = synth.vslab_80x80x40()
    S = g.Survey(w.survey.x, w.survey.y, w.survey.z)
    ddf, tdf = g.diag(w.mesh, S)
    d64, t64 = g.diag(w.mesh, S, diag_fp64=True)
    ddf, d64 = ddf.cpu().numpy(), d64.cpu().numpy()
    assert float(np.max(np.abs(ddf - d64) / d64)) <= 1e-11
    assert tdf == pytest.approx(t64, rel=1e-13)


def test_dot_test_and_determinism(g):
    mesh, sv, m = synth.small_random_problem(20, 17, 8, 500, seed=13)
    S = g.Survey(sv.x, sv.y, sv.z)
    plan = g.Plan(mesh, S)
    mt = _dev(m)
    r = _dev(synth.random_vector(sv.n, 14))
    d1 = plan.forward(mt)
    d2 = plan.forward(mt)
    assert torch.equal(d1, d2)
    gt = plan.adjoint(r)
    assert torch.equal(gt, plan.adjoint(r))
    lhs = float(torch.dot(d1, r)); rhs = float(torch.dot(mt, gt))
    assert lhs == pytest.approx(rhs, rel=1e-11)
    plan.close()


def test_block_workload_golden(g):
    """Full-size 20x20x10 block workload against the oracle values stored by
    tests/golden/make_golden.py."""
    import os
    gold = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "block_20x20x10_forward.txt"))
    wl = synth.make_workload("block_20x20x10")
    d = g.forward(_dev(wl.m), wl.mesh, g.Survey(wl.survey.x, wl.survey.y, wl.survey.z)).cpu().numpy()
    assert _rel(d, gold) <= TOL64


def test_vslab_full_size_sampled(g):
    """80x80x40 vertical-slab workload at full size (the launch configuration of
    the bench); the oracle checks 48 sampled stations and 64 sampled cells."""
    wl = synth.make_workload("vslab_80x80x40")
    S = g.Survey(wl.survey.x, wl.survey.y, wl.survey.z)
    plan = g.Plan(wl.mesh, S)
    d = plan.forward(_dev(wl.m)).cpu().numpy()
    rng = np.random.Generator(np.random.PCG64(21))
    idx = np.sort(rng.choice(wl.survey.n, 48, replace=False))
    d_ref = oracle.forward(wl.mesh, wl.survey.subset(idx), wl.m)
    assert np.abs(d[idx] - d_ref).max() <= TOL64 * np.abs(d_ref).max()
    # adjoint: sampled cells, via explicit rows of G^T restricted to those cells
    r = synth.random_vector(wl.survey.n, 22)
    a = plan.adjoint(_dev(r)).cpu().numpy()
    cells = np.sort(rng.choice(wl.mesh.ncells, 64, replace=False))
    a_ref = _adjoint_cells(wl.mesh, wl.survey, r, cells)
    assert np.abs(a[cells] - a_ref).max() <= TOL64 * np.abs(a_ref).max()
    plan.close()


def _adjoint_cells(mesh, sv, r, cells):
    """(G^T r)_k for selected cells with the oracle: one single-cell mesh per cell."""
    out = []
    nx, ny = mesh.nx, mesh.ny
    for k in cells:
        i, j, l = k % nx, (k // nx) % ny, k // (nx * ny)
        sub = synth.Mesh(mesh.xe[i:i + 2].copy(), mesh.ye[j:j + 2].copy(), mesh.ze[l:l + 2].copy())
        out.append(oracle.adjoint(sub, sv, r)[0])
    return np.array(out)


@pytest.mark.parametrize("precond", ["none", "jacobi"])
def test_datainv_fp64_block_vs_dense_lu(g, precond):
    """20x20x10 block workload: CG or Jacobi-preconditioned CG (tol 1e-8)
    against the oracle's dense LU of Eq. 11; the difference must stay inside
    the bound implied by the CG residual,
    ||y - y*|| <= ||dd - A y|| / lambda_min(A) <= ||dd - A y|| / lambda."""
    wl = synth.make_workload("block_20x20x10")
    G = oracle.G_explicit(wl.mesh, wl.survey)
    d = synth.add_noise(G @ wl.m, wl.noise_abs, wl.noise_rel, 0)
    ref = oracle.invert_dense(wl.mesh, wl.survey, d, z0=50.0)
    S = g.Survey(wl.survey.x, wl.survey.y, wl.survey.z)
    m, y, info = g.datainv(_dev(d), wl.mesh, S, return_y=True, tol=1e-8, max_iter=2000, precond=precond)
    assert info["converged"], info
    assert info["lambda"] == pytest.approx(ref["lam"], rel=1e-10)
    y = y.cpu().numpy(); m = m.cpu().numpy()
    A = (G * ref["wm"]) @ G.T + ref["lam"] * np.eye(len(d))
    res = np.linalg.norm(d - A @ y)
    assert res <= 1.5e-8 * np.linalg.norm(d)
    assert np.linalg.norm(y - ref["y"]) <= 1.01 * res / ref["lam"]
    m_from_y = ref["wm"] * (G.T @ y)
    # G^T y cancels heavily for the CG solution; the adjoint's rounding error
    # scales with W^-2 |G|^T |y|, so that is the reference magnitude here
    scale = np.max(ref["wm"] * (np.abs(G).T @ np.abs(y)))
    assert np.abs(m - m_from_y).max() <= 1e-10 * scale
    assert info["true_rel_res"] <= 1.5e-8


@pytest.mark.parametrize("opts", [dict(precision="fp64"), dict(precision="mixed"),
                                  dict(precision="fp64", refine=8), dict(precision="fp64", cache_g=True),
                                  dict(precision="fp64", outer_max=5)])
def test_inversion_of_zero_data(g, opts):
    """Data that the reference model already explains (dd = d - G m_ref = 0,
    exactly: d is zero with no m_ref, or the same path's own forward of m_ref)
    make y = 0 the solution: every inversion path (FP64, mixed, refinement,
    stored G, outer loop) returns y = 0 and the reference model bit for bit,
    converged.  The model comes from the adjoint of the final y that the last
    residual already took, or from zero when no step ran."""
    mesh, sv, _ = synth.small_random_problem(9, 7, 5, 60, seed=51)   # uniform: mixed and refine need it
    S = g.Survey(sv.x, sv.y, sv.z)
    m, y, info = g.datainv(_dev(np.zeros(sv.n)), mesh, S, return_y=True, tol=1e-6, max_iter=200, **opts)
    assert info["converged"], info
    assert float(m.abs().max()) == 0.0 and float(y.abs().max()) == 0.0
    m_ref = _dev(synth.random_vector(mesh.ncells, 52, 50.0))
    fwd = {k: v for k, v in opts.items() if k in ("precision", "cache_g")}
    d = g.forward(m_ref, mesh, S, **fwd)
    m2, y2, info2 = g.datainv(d, mesh, S, m_ref=m_ref, return_y=True, tol=1e-6, max_iter=200, **opts)
    assert info2["converged"], info2
    assert float(y2.abs().max()) == 0.0
    assert torch.equal(m2, m_ref)


@pytest.mark.parametrize("tol,precond", [(1e-6, "none"), (1e-8, "none"), (1e-8, "nystrom")])
def test_fp64_inversion_by_mixed_refinement(g, tol, precond):
    """FP64 inversion with refine: mixed-precision CG solves of the current
    residual, which is recomputed with the FP64 operator after each step.  On
    the block workload the reported residual is the FP64 one (recomputed here
    from the oracle's explicit G) and meets tol, lambda is the FP64 trace
    rule's, and the model is the oracle's dense-LU minimiser of Eq. 11 within
    the bound the residual implies, ||y - y*|| <= ||dd - A y|| / lambda, also
    with a reference model; the mixed inner solves take the Nystrom
    preconditioner as well."""
    wl = synth.make_workload("block_20x20x10")
    G = oracle.G_explicit(wl.mesh, wl.survey)
    d = synth.add_noise(G @ wl.m, wl.noise_abs, wl.noise_rel, 0)
    m_ref = np.full(wl.mesh.ncells, 0.1)
    ref = oracle.invert_dense(wl.mesh, wl.survey, d, m_ref=m_ref, z0=50.0)
    S = g.Survey(wl.survey.x, wl.survey.y, wl.survey.z)
    m, y, info = g.datainv(_dev(d), wl.mesh, S, m_ref=_dev(m_ref), return_y=True, tol=tol, max_iter=2000,
                           refine=8, precond=precond)
    assert info["converged"], info
    assert 1 <= info["outer"] <= 8 and info["iters"] > 0
    assert info["lambda"] == pytest.approx(ref["lam"], rel=1e-10)
    y = y.cpu().numpy(); m = m.cpu().numpy()
    A = (G * ref["wm"]) @ G.T + ref["lam"] * np.eye(len(d))
    dd = d - G @ m_ref
    res = np.linalg.norm(dd - A @ y)
    assert res <= tol * np.linalg.norm(dd)
    assert info["true_rel_res"] == pytest.approx(res / np.linalg.norm(dd), rel=1e-6, abs=1e-12)
    assert np.linalg.norm(y - ref["y"]) <= 1.01 * res / ref["lam"]
    m_from_y = m_ref + ref["wm"] * (G.T @ y)
    scale = np.max(ref["wm"] * (np.abs(G).T @ np.abs(y)))
    assert np.abs(m - m_from_y).max() <= 1e-10 * scale


def test_refine_is_refused_where_it_does_not_apply(g):
    """refine needs precision fp64 (mixed is refused), and serving jobs refuse it."""
    wl = synth.make_workload("block_20x20x10")
    S = g.Survey(wl.survey.x, wl.survey.y, wl.survey.z)
    d = _dev(np.ones(wl.survey.n))
    with pytest.raises(g.GravError):
        g.datainv(d, wl.mesh, S, precision="mixed", refine=4)
    ctx = g.Context(0)
    out = torch.empty(wl.mesh.ncells, dtype=torch.float64, device="cuda")
    with pytest.raises(g.GravError):
        ctx.submit("invert", wl.mesh, S, d, out, refine=4)
    ctx.close()


def test_datainv_with_reference_model(g):
    mesh, sv, m_true = synth.small_random_problem(8, 7, 5, 60, seed=31)
    G = oracle.G_explicit(mesh, sv)
    d = G @ m_true
    m_ref = np.full(mesh.ncells, 0.1)     # the paper's 0.0001 g/cm^3 reference model
    wm = oracle.depth_w2(mesh, 50.0)
    lam = oracle.lambda_from_trace(float(np.sum((G * G) @ wm)), sv.n)
    m_star, y_star = oracle.dataspace_solve(G, d, m_ref, wm, lam)
    m, info = g.datainv(_dev(d), mesh, g.Survey(sv.x, sv.y, sv.z), m_ref=_dev(m_ref), tol=1e-12,
                        max_iter=5000)
    assert info["converged"]
    assert _rel(m.cpu().numpy(), m_star) <= 1e-6


# ---------------------------------------------------------------- mixed ----

@pytest.fixture(params=["shuffle", "broadcast"])
def adjoint_layout(request, monkeypatch):
    """Both mixed far-field adjoint layouts (lanes split stations + warp-shuffle
    reduction; lanes own cells + broadcast stations), chosen at plan creation."""
    monkeypatch.setenv("GRAV_ADJOINT_LAYOUT", request.param)
    return request.param


@pytest.mark.parametrize("shape,cell,h,seed", [((30, 26, 12), 40.0, 10.0, 1), ((17, 23, 9), 25.0, 3.0, 2),
                                               ((41, 37, 15), 100.0, 30.0, 3)])
def test_mixed_forward_adjoint_vs_oracle(g, shape, cell, h, seed, adjoint_layout):
    nx, ny, nz = shape
    mesh = synth.uniform_mesh(nx, ny, nz, cell, cell, cell)
    rng = np.random.Generator(np.random.PCG64(40 + seed))
    m = synth.lognormal_background(mesh.ncells, 20.0, rng).reshape(nz, ny, nx)
    m[2:6, ny // 4: 3 * ny // 4, nx // 3: nx // 3 + 3] += 350.0
    m = m.ravel()
    n = 500
    sv = synth.Survey(rng.uniform(-cell, nx * cell + cell, n), rng.uniform(-cell, ny * cell + cell, n),
                      -rng.uniform(0.5, h, n))
    S = g.Survey(sv.x, sv.y, sv.z)
    G = oracle.G_explicit(mesh, sv)
    d_ref = G @ m
    r = synth.random_vector(n, seed)
    a_ref = oracle.depth_w2(mesh, 50.0) * (G.T @ r)
    # accuracy of the mixed operator against the exact FP64 oracle: the forward
    # meets 1e-5 from a 6-cell window on, the adjoint of white-noise r from the
    # default 8-cell window on (relative to max |G^T r|)
    for k in (6.0, 8.0):
        d = g.forward(_dev(m), mesh, S, precision="mixed", near_cells=k).cpu().numpy()
        assert _rel(d, d_ref) <= TOLMIX, k
    a = g.adjoint(_dev(r), mesh, S, depth_weighted=True, precision="mixed").cpu().numpy()
    assert _rel(a, a_ref) <= TOLMIX
    # the kernels implement the definition of the mixed operator at any window:
    # exact prism inside the window, point mass gamma V dz / R^3 outside
    for k in (3.0, 4.5):
        Gk = _mixed_definition(mesh, sv, G, cell, k)
        d = g.forward(_dev(m), mesh, S, precision="mixed", near_cells=k).cpu().numpy()
        assert np.abs(d - Gk @ m).max() <= 1e-6 * np.abs(Gk @ m).max(), k
        a = g.adjoint(_dev(r), mesh, S, precision="mixed", near_cells=k).cpu().numpy()
        assert np.abs(a - Gk.T @ r).max() <= 1e-6 * np.abs(Gk.T @ r).max(), k


@pytest.mark.parametrize("near_cells", [8.0, 3.0, 5.0])
def test_near_adjoint_forms_agree_and_match_oracle(g, near_cells, monkeypatch):
    """The near-field adjoint in its four forms: layer-split (warp w owns
    the region's layers w, w + 8, ... of one shared FP32 accumulator and
    streams that layer's segment of every station's row; the default),
    warp-private (each warp streams its stations' table rows into its own
    FP32 region accumulator; GRAV_NEAR_ADJ=warp), station-streaming (whole rows by TMA bulk copy into one
    shared accumulator, a barrier per station; GRAV_NEAR_ADJ=rows) and
    cell-tiled (GRAV_NEAR_ADJ=tiles).  Windows 3 and 5 give 147- and
    605-slot boxes, not multiples of 4, so the table rows carry padding that
    the forward's 16-byte fast path and the streaming adjoint read.  Each form
    is within 1e-6 of the definition of the approximation (exact prism inside
    the window, point mass outside), 1e-5 of the exact oracle at the default
    window, bitwise repeatable, and the forms agree to FP32 rounding."""
    mesh = synth.uniform_mesh(45, 38, 14, 30.0, 30.0, 30.0)
    rng = np.random.Generator(np.random.PCG64(211))
    n = 1500
    sv = synth.Survey(rng.uniform(-60, 45 * 30 + 60, n), rng.uniform(-60, 38 * 30 + 60, n), -rng.uniform(0.5, 15, n))
    S = g.Survey(sv.x, sv.y, sv.z)
    G = oracle.G_explicit(mesh, sv)
    r = synth.random_vector(n, 212)
    m = rng.normal(0.0, 100.0, mesh.ncells)
    Gk = _mixed_definition(mesh, sv, G, 30.0, near_cells)
    out = {}
    for form in ("layer", "warp", "rows", "tiles"):
        monkeypatch.setenv("GRAV_NEAR_ADJ", form)
        plan = g.Plan(mesh, S, precision="mixed", near_cells=near_cells)
        a = plan.adjoint(_dev(r))
        assert torch.equal(plan.adjoint(_dev(r)), a), form
        a = a.cpu().numpy()
        assert np.abs(a - Gk.T @ r).max() <= 1e-6 * np.abs(Gk.T @ r).max(), form
        d = plan.forward(_dev(m)).cpu().numpy()
        assert np.abs(d - Gk @ m).max() <= 1e-6 * np.abs(Gk @ m).max(), form
        if near_cells == 8.0:
            assert _rel(a, G.T @ r) <= TOLMIX, form
        out[form] = a
        plan.close()
    for form in ("layer", "warp", "rows"):
        assert np.abs(out[form] - out["tiles"]).max() <= 1e-7 * np.abs(out["tiles"]).max(), form


@pytest.mark.parametrize("near_cells", [8.0, 3.0])
def test_near_table_double_float_against_fp64(g, near_cells):
    """The near-field table formed from the corner function in double-float
    (the default) against the same table formed in FP64 (near_fp64): forward
    and adjoint products agree within 1e-8 of max (the double-float corner
    values carry ~2^-45 of R (|ln R| + 1)), and both implement the definition
    of the mixed operator within 1e-6 of max (exact prism inside the window,
    point mass outside), on stations inside and outside the footprint."""
    mesh = synth.uniform_mesh(33, 29, 14, 40.0, 40.0, 40.0)
    rng = np.random.Generator(np.random.PCG64(219))
    n = 900
    sv = synth.Survey(rng.uniform(-300, 33 * 40 + 300, n), rng.uniform(-300, 29 * 40 + 300, n),
                      -rng.uniform(0.5, 20, n))
    S = g.Survey(sv.x, sv.y, sv.z)
    G = oracle.G_explicit(mesh, sv)
    Gk = _mixed_definition(mesh, sv, G, 40.0, near_cells)
    m = rng.normal(0.0, 100.0, mesh.ncells) + 20.0
    r = synth.random_vector(n, 220)
    out = {}
    for f64 in (False, True):
        plan = g.Plan(mesh, S, precision="mixed", near_cells=near_cells, near_fp64=f64)
        d = plan.forward(_dev(m)).cpu().numpy()
        a = plan.adjoint(_dev(r)).cpu().numpy()
        plan.close()
        assert np.abs(d - Gk @ m).max() <= 1e-6 * np.abs(Gk @ m).max(), f64
        assert np.abs(a - Gk.T @ r).max() <= 1e-6 * np.abs(Gk.T @ r).max(), f64
        out[f64] = (d, a)
    for k in (0, 1):
        assert np.abs(out[False][k] - out[True][k]).max() <= 1e-8 * np.abs(out[True][k]).max(), k


@pytest.mark.parametrize("near_cells", [8.0, 3.0, 5.0])
def test_near_forward_forms_agree_and_match_oracle(g, near_cells, monkeypatch):
    """The near-field forward in its two forms: per tile of station bins with
    the tile's q and slot offsets in shared memory (the default) and one warp
    per station gathering q from global memory (GRAV_NEAR_FWD=warp).  Stations
    lie inside, on the edges of and outside the mesh footprint, some with
    windows that miss the mesh.  Each form is within 1e-6 of the definition of
    the approximation, 1e-5 of the exact oracle at the default window, bitwise
    repeatable, and the two agree to FP32 rounding."""
    mesh = synth.uniform_mesh(41, 36, 13, 30.0, 30.0, 30.0)
    rng = np.random.Generator(np.random.PCG64(215))
    n = 1400
    sv = synth.Survey(rng.uniform(-400, 41 * 30 + 400, n), rng.uniform(-400, 36 * 30 + 400, n),
                      -rng.uniform(0.5, 15, n))
    S = g.Survey(sv.x, sv.y, sv.z)
    G = oracle.G_explicit(mesh, sv)
    m = rng.normal(0.0, 100.0, mesh.ncells) + 30.0
    Gk = _mixed_definition(mesh, sv, G, 30.0, near_cells)
    out = {}
    for form in ("tile", "warp"):
        monkeypatch.setenv("GRAV_NEAR_FWD", form)
        plan = g.Plan(mesh, S, precision="mixed", near_cells=near_cells)
        d = plan.forward(_dev(m))
        assert torch.equal(plan.forward(_dev(m)), d), form
        d = d.cpu().numpy()
        assert np.abs(d - Gk @ m).max() <= 1e-6 * np.abs(Gk @ m).max(), form
        if near_cells == 8.0:
            assert _rel(d, G @ m) <= TOLMIX, form
        out[form] = d
        plan.close()
    assert np.abs(out["tile"] - out["warp"]).max() <= 1e-7 * np.abs(out["warp"]).max()


@pytest.mark.parametrize("shape,cells", [((1, 1, 1), (20.0, 20.0, 20.0)), ((7, 1, 1), (20.0, 20.0, 20.0)),
                                         ((1, 9, 3), (15.0, 15.0, 15.0)), ((23, 19, 1), (30.0, 30.0, 30.0)),
                                         ((9, 11, 2), (25.0, 10.0, 40.0)), ((13, 12, 17), (20.0, 20.0, 20.0)),
                                         ((64, 1, 5), (10.0, 30.0, 10.0))])
def test_mixed_degenerate_meshes_and_far_stations(g, shape, cells, adjoint_layout):
    """Mixed mode on one-cell-wide, single-layer and ragged-layer meshes (nz = 1,
    2, 17 against the 16-layer adjoint groups), rectangular cells, and stations
    both above the mesh and far outside its footprint (empty near windows):
    forward and depth-weighted adjoint within 1e-5 of max against the oracle."""
    nx, ny, nz = shape
    a, b, c = cells
    mesh = synth.uniform_mesh(nx, ny, nz, a, b, c)
    rng = np.random.Generator(np.random.PCG64(160 + nx + 7 * ny + 31 * nz))
    m = rng.normal(0.0, 100.0, mesh.ncells) + 50.0
    n = 97
    X, Y = nx * a, ny * b
    far = np.stack([rng.uniform(-20 * X - 500, 21 * X + 500, 24), rng.uniform(-20 * Y - 500, 21 * Y + 500, 24)])
    sv = synth.Survey(np.concatenate([rng.uniform(-a, X + a, n - 24), far[0]]),
                      np.concatenate([rng.uniform(-b, Y + b, n - 24), far[1]]),
                      -rng.uniform(0.5, 12.0, n))
    S = g.Survey(sv.x, sv.y, sv.z)
    G = oracle.G_explicit(mesh, sv)
    d = g.forward(_dev(m), mesh, S, precision="mixed").cpu().numpy()
    assert _rel(d, G @ m) <= TOLMIX
    r = synth.random_vector(n, 161)
    at = g.adjoint(_dev(r), mesh, S, depth_weighted=True, precision="mixed").cpu().numpy()
    assert _rel(at, oracle.depth_w2(mesh, 50.0) * (G.T @ r)) <= TOLMIX


@pytest.mark.parametrize("cells", [(20.0, 20.0, 20.0), (30.0, 20.0, 25.0)])
def test_mixed_products_scale_exactly(g, cells, adjoint_layout):
    """The mixed products divide their input by its largest magnitude before
    the FP32 arithmetic and multiply the FP64 result back, so an input scaled
    by 2^k gives the output scaled by exactly 2^k, also far outside the range
    in which FP32 products of the raw input would stay normal (2^-110 ~ 8e-34
    times a density of ~100 flushed to zero before); zero entries and an
    all-zero input are exact, and the scaled results still match the oracle."""
    mesh = synth.uniform_mesh(23, 19, 18, *cells)
    rng = np.random.Generator(np.random.PCG64(171))
    m = rng.normal(0.0, 100.0, mesh.ncells)
    m[::7] = 0.0
    n = 300
    sv = synth.Survey(rng.uniform(0, 23 * cells[0], n), rng.uniform(0, 19 * cells[1], n), -rng.uniform(0.5, 8.0, n))
    sv.x[0], sv.y[0] = 11.5 * cells[0], 9.5 * cells[1]   # above a column centre, with r = 0 below
    r = synth.random_vector(n, 172)
    r[::5] = 0.0
    plan = g.Plan(mesh, g.Survey(sv.x, sv.y, sv.z), precision="mixed")
    d = plan.forward(_dev(m))
    a = plan.adjoint(_dev(r), depth_weighted=True)
    for k in (-110, -60, 60, 110):
        s = 2.0 ** k
        assert torch.equal(plan.forward(_dev(m * s)), d * s), k
        assert torch.equal(plan.adjoint(_dev(r * s), depth_weighted=True), a * s), k
    z = plan.forward(_dev(np.zeros(mesh.ncells)))
    assert bool((z == 0).all())
    z = plan.adjoint(_dev(np.zeros(n)), depth_weighted=True)
    assert bool((z == 0).all())
    G = oracle.G_explicit(mesh, sv)
    s = 2.0 ** -110
    assert _rel(plan.forward(_dev(m * s)).cpu().numpy(), G @ (m * s)) <= TOLMIX
    a_ref = oracle.depth_w2(mesh, 50.0) * (G.T @ (r * s))
    assert _rel(plan.adjoint(_dev(r * s), depth_weighted=True).cpu().numpy(), a_ref) <= TOLMIX
    plan.close()


def _mixed_definition(mesh, sv, G, cell, k):
    """Dense matrix of the mixed approximation: G_ik from the oracle when the
    cell centre lies within k cell widths of station i, else the point mass
    gamma * 1e5 * V * dz / R^3 (mGal per kg/m^3)."""
    xc = 0.5 * (mesh.xe[:-1] + mesh.xe[1:]); yc = 0.5 * (mesh.ye[:-1] + mesh.ye[1:])
    zc = 0.5 * (mesh.ze[:-1] + mesh.ze[1:])
    Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")
    DX = X.ravel()[None, :] - sv.x[:, None]; DY = Y.ravel()[None, :] - sv.y[:, None]
    DZ = Z.ravel()[None, :] - sv.z[:, None]
    R = np.sqrt(DX ** 2 + DY ** 2 + DZ ** 2)
    far = 6.67430e-11 * 1e5 * cell ** 3 * DZ / R ** 3
    return np.where(R < k * cell, G, far)


@pytest.mark.parametrize("shape,a,b,c,h,seed", [((30, 26, 14), 40.0, 40.0, 20.0, 6.0, 11),
                                                ((21, 19, 9), 20.0, 20.0, 30.0, 4.0, 12),
                                                ((26, 35, 10), 30.0, 20.0, 25.0, 5.0, 13),
                                                ((12, 48, 8), 50.0, 12.5, 20.0, 3.0, 14)])
def test_mixed_noncubic_prisms_vs_oracle(g, shape, a, b, c, h, seed, adjoint_layout):
    """Non-cubic a x b x c cells: the far field carries the box's quadrupole
    factor 1 + (A dx^2 + B dy^2 + C dz^2) / R^4 (second moments a^2/12, b^2/12,
    c^2/12 of the box in the Taylor expansion of dz / R^3), so the mixed
    operator still meets 1e-5 of max against the oracle, and the kernels
    implement that definition (exact inside the window of k * max(a, b, c),
    corrected point mass outside) at 1e-6."""
    nx, ny, nz = shape
    mesh = synth.uniform_mesh(nx, ny, nz, a, b, c)
    rng = np.random.Generator(np.random.PCG64(60 + seed))
    m = synth.lognormal_background(mesh.ncells, 20.0, rng).reshape(nz, ny, nx)
    m[2:7, ny // 4: 3 * ny // 4, nx // 3: nx // 3 + 3] += 400.0
    m = m.ravel()
    n = 400
    sv = synth.Survey(rng.uniform(0, nx * a, n), rng.uniform(0, ny * b, n), -rng.uniform(0.5, h, n))
    S = g.Survey(sv.x, sv.y, sv.z)
    G = oracle.G_explicit(mesh, sv)
    d = g.forward(_dev(m), mesh, S, precision="mixed").cpu().numpy()
    assert _rel(d, G @ m) <= TOLMIX
    r = synth.random_vector(n, seed)
    at = g.adjoint(_dev(r), mesh, S, precision="mixed").cpu().numpy()
    assert _rel(at, G.T @ r) <= TOLMIX
    L = max(a, b, c)
    xc = 0.5 * (mesh.xe[:-1] + mesh.xe[1:]); yc = 0.5 * (mesh.ye[:-1] + mesh.ye[1:])
    zc = 0.5 * (mesh.ze[:-1] + mesh.ze[1:])
    Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")
    DX = X.ravel()[None, :] - sv.x[:, None]; DY = Y.ravel()[None, :] - sv.y[:, None]
    DZ = Z.ravel()[None, :] - sv.z[:, None]
    R2 = DX ** 2 + DY ** 2 + DZ ** 2
    qa = (12 * a * a - 3 * b * b - 9 * c * c) / 24
    qb = (12 * b * b - 3 * a * a - 9 * c * c) / 24
    qg = (6 * c * c - 3 * a * a - 3 * b * b) / 24
    far = 6.67430e-11 * 1e5 * a * b * c * DZ / R2 ** 1.5 * (1 + (qa * DX ** 2 + qb * DY ** 2 + qg * DZ ** 2) / R2 ** 2)
    for k in (3.0, 5.0):
        Gk = np.where(R2 < (k * L) ** 2, G, far)
        dk = g.forward(_dev(m), mesh, S, precision="mixed", near_cells=k).cpu().numpy()
        assert np.abs(dk - Gk @ m).max() <= 1e-6 * np.abs(Gk @ m).max(), k


@pytest.mark.parametrize("name", ["two_body_160x160x80", "tube_slab_100x100x50", "dipdyke_150x150x60"])
def test_mixed_paper_shaped_workloads_sampled(g, name):
    """Full-size paper-shaped workloads in mixed mode (tube_slab: square-based
    200 x 200 x 100 m prisms, so the quadrupole far-field term is active): 48
    sampled stations of G m and 192 sampled cells of G^T r (white-noise r;
    128 of the cells in the top layer, where |G^T r| peaks) against the oracle."""
    wl = synth.make_workload(name)
    S = g.Survey(wl.survey.x, wl.survey.y, wl.survey.z)
    plan = g.Plan(wl.mesh, S, precision="mixed")
    rng = np.random.Generator(np.random.PCG64(150))
    d = plan.forward(_dev(wl.m)).cpu().numpy()
    idx = np.sort(rng.choice(wl.survey.n, 48, replace=False))
    d_ref = oracle.forward(wl.mesh, wl.survey.subset(idx), wl.m)
    assert _rel(d[idx], d_ref) <= TOLMIX
    r = synth.random_vector(wl.survey.n, 151)
    a = plan.adjoint(_dev(r)).cpu().numpy()
    ncol = wl.mesh.nx * wl.mesh.ny
    cells = np.unique(np.concatenate([rng.choice(ncol, 128, replace=False),
                                      rng.choice(wl.mesh.ncells, 64, replace=False)]))
    a_ref = _adjoint_cells(wl.mesh, wl.survey, r, cells)
    assert _rel(a[cells], a_ref) <= TOLMIX
    plan.close()


def test_paper_scale_sampled_in_bench_configuration(g):
    """The benchmarked workload at full size (210 x 210 x 75 = 3,307,500 cells,
    178,797 stations scattered at 1-50 m height) in the launch configuration
    bench.py times (mixed, default 8-cell window, broadcast adjoint, 12 station
    chunks): 48 sampled stations of G m and 160 sampled cells of G^T r against
    the oracle (1e-5 of the sample's max).  The FP64 mode at the same size is
    checked through row and column restrictions of the operator, which are
    exact: G m at 16 stations from a plan over those stations, and G^T r at 8
    cells from one-cell meshes over all stations (1e-10 of the output's max)."""
    wl = synth.make_workload("paper_210x210x75")
    S = g.Survey(wl.survey.x, wl.survey.y, wl.survey.z)
    plan = g.Plan(wl.mesh, S, precision="mixed")
    desc = plan.describe()
    assert desc["adj_kernel"].startswith("k_madj_bc"), desc
    rng = np.random.Generator(np.random.PCG64(190))
    d = plan.forward(_dev(wl.m)).cpu().numpy()
    idx = np.sort(rng.choice(wl.survey.n, 48, replace=False))
    d_ref = oracle.forward(wl.mesh, wl.survey.subset(idx), wl.m)
    assert _rel(d[idx], d_ref) <= TOLMIX
    r = synth.random_vector(wl.survey.n, 191)
    a = plan.adjoint(_dev(r)).cpu().numpy()
    ncol = wl.mesh.nx * wl.mesh.ny
    cells = np.unique(np.concatenate([rng.choice(ncol, 96, replace=False),
                                      rng.choice(wl.mesh.ncells, 64, replace=False)]))
    a_ref = _adjoint_cells(wl.mesh, wl.survey, r, cells)
    assert _rel(a[cells], a_ref) <= TOLMIX
    plan.close()
    # FP64 mode: rows (stations) and columns (cells) of the full-size operator
    i16 = idx[::3]
    sub = wl.survey.subset(i16)
    d64 = g.forward(_dev(wl.m), wl.mesh, g.Survey(sub.x, sub.y, sub.z), precision="fp64").cpu().numpy()
    assert _rel(d64, d_ref[::3]) <= TOL64
    c8 = cells[::20]
    a64 = []
    nx, ny = wl.mesh.nx, wl.mesh.ny
    for k in c8:
        i, j, l = k % nx, (k // nx) % ny, k // (nx * ny)
        one = synth.Mesh(wl.mesh.xe[i:i + 2].copy(), wl.mesh.ye[j:j + 2].copy(), wl.mesh.ze[l:l + 2].copy())
        a64.append(float(g.adjoint(_dev(r), one, S, precision="fp64").cpu().numpy()[0]))
    # relative to max |G^T r| over the whole output (the FP64 criterion); a deep
    # cell 10 km from most stations loses ~(R/a)^3 to the corner-sum cancellation
    # in both the oracle and the kernel, ~4e-13 absolute against max ~3e-3
    assert np.abs(np.array(a64) - a_ref[::20]).max() <= TOL64 * np.abs(a).max()


def test_mixed_with_window_covering_mesh_is_exact(g, adjoint_layout):
    """If every cell lies inside every station's window the mixed operator is
    the exact FP64 operator up to the FP32 rounding of the far-field terms,
    which still run for every cell and cancel against their FP64 correction
    only up to fl32(gamma V rho) and the FP32 accumulation (~1e-7 relative)."""
    mesh = synth.uniform_mesh(4, 5, 3, 10.0, 10.0, 10.0)
    rng = np.random.Generator(np.random.PCG64(50))
    sv = synth.Survey(rng.uniform(5, 35, 40), rng.uniform(5, 45, 40), -rng.uniform(0.5, 3, 40))
    m = rng.normal(0, 100, mesh.ncells)
    d_ref = oracle.forward(mesh, sv, m)
    d = g.forward(_dev(m), mesh, g.Survey(sv.x, sv.y, sv.z), precision="mixed", near_cells=16.0).cpu().numpy()
    assert _rel(d, d_ref) <= 1e-6
    r = rng.normal(0, 1, sv.n)
    a_ref = oracle.adjoint(mesh, sv, r)
    a = g.adjoint(_dev(r), mesh, g.Survey(sv.x, sv.y, sv.z), precision="mixed", near_cells=16.0).cpu().numpy()
    assert _rel(a, a_ref) <= 1e-6


def test_mixed_diag_and_dot(g, adjoint_layout):
    mesh = synth.uniform_mesh(25, 21, 10, 50.0, 50.0, 50.0)
    rng = np.random.Generator(np.random.PCG64(60))
    sv = synth.Survey(rng.uniform(0, 1250, 300), rng.uniform(0, 1050, 300), -rng.uniform(1, 20, 300))
    S = g.Survey(sv.x, sv.y, sv.z)
    ref = oracle.diag_GWG(mesh, sv, 50.0)
    dg, tr = g.diag(mesh, S, precision="mixed")
    assert _rel(dg.cpu().numpy(), ref) <= TOLMIX
    plan = g.Plan(mesh, S, precision="mixed")
    m = _dev(rng.normal(0, 50, mesh.ncells)); r = _dev(rng.normal(0, 1, sv.n))
    Gm = plan.forward(m)
    lhs = float(torch.dot(Gm, r)); rhs = float(torch.dot(m, plan.adjoint(r)))
    # the mixed forward and adjoint are transposes of one approximate operator
    # up to FP32 rounding, which scales with ||G m|| ||r||
    assert abs(lhs - rhs) <= 1e-6 * float(torch.linalg.norm(Gm) * torch.linalg.norm(r))
    plan.close()


# ------------------------------------------------- literal FP32 corners ---

def _node_weights(mesh, m):
    """w = D m: each cell adds -(-1)^(da+db+dc) m to its vertex (i+da, j+db, l+dc)."""
    nx, ny, nz = mesh.nx, mesh.ny, mesh.nz
    mc = m.reshape(nz, ny, nx)
    w = np.zeros((nz + 1, ny + 1, nx + 1))
    for dc in (0, 1):
        for db in (0, 1):
            for da in (0, 1):
                w[dc:dc + nz, db:db + ny, da:da + nx] += (1 if (da + db + dc) % 2 else -1) * mc
    return w


def test_mixed_corner_equals_exact_up_to_fp32_accumulation(g):
    """GRAV_MIXED_CORNER with a window that covers every cell: every corner
    difference is replaced by its FP64 value, so only the FP32 accumulation of
    w_n Psi32_n over a row of nx+1 nodes remains.  The standard bound for a
    recursive sum, (nx + 1) u sum_n |w_n Psi_n| (u = 2^-24; integer m keeps
    the FP32 node weights exact), holds station by station."""
    # 16 cell widths (160 m) exceed the farthest cell centre (~154 m) from any station
    mesh = synth.uniform_mesh(12, 10, 4, 10.0, 10.0, 10.0, x0=512_345.0, y0=7_301_234.0)
    rng = np.random.Generator(np.random.PCG64(140))
    n = 700
    sv = synth.Survey(512_345.0 + rng.uniform(0, 120, n), 7_301_234.0 + rng.uniform(0, 100, n),
                      -rng.uniform(0.5, 5, n))
    m = rng.integers(-300, 301, mesh.ncells).astype(np.float64)
    d_ref = oracle.forward(mesh, sv, m)
    d = g.forward(_dev(m), mesh, g.Survey(sv.x, sv.y, sv.z), precision="mixed_corner",
                  near_cells=16.0).cpu().numpy()
    w = _node_weights(mesh, m).ravel()
    Z, Y, X = np.meshgrid(mesh.ze, mesh.ye, mesh.xe, indexing="ij")
    X, Y, Z = X.ravel(), Y.ravel(), Z.ravel()
    bound = np.empty(n)
    for s in range(n):
        x, y, z = X - sv.x[s], Y - sv.y[s], Z - sv.z[s]
        R = np.sqrt(x * x + y * y + z * z)
        psi_abs = np.abs(z * np.arctan(x * y / (z * R))) + np.abs(x * np.log(R + y)) + np.abs(y * np.log(R + x))
        bound[s] = (mesh.nx + 3) * 2.0 ** -24 * np.sum(np.abs(w) * psi_abs)
    bound = 6.6743e-6 * bound + 1e-12 * np.abs(d_ref).max()
    assert np.all(np.abs(d - d_ref) <= bound), float(np.max(np.abs(d - d_ref) / bound))
    # the bound is far below the signal here, so a wrong weight, sign or term would show
    assert np.median(bound) < 0.05 * np.median(np.abs(d_ref))


def test_mixed_corner_error_at_default_window(g):
    """The literal reading (FP32 corner terms everywhere outside the 8-cell
    window) against the FP64 oracle; this reports the error (printed), and the
    proposed scheme on the same inputs meets 1e-5 of max."""
    wl = synth.make_workload("vslab_80x80x40")
    idx = np.random.Generator(np.random.PCG64(141)).choice(wl.survey.n, 64, replace=False)
    S = g.Survey(wl.survey.x, wl.survey.y, wl.survey.z)
    d_ref = oracle.forward(wl.mesh, wl.survey.subset(idx), wl.m)
    dc = g.forward(_dev(wl.m), wl.mesh, S, precision="mixed_corner").cpu().numpy()[idx]
    dm = g.forward(_dev(wl.m), wl.mesh, S, precision="mixed").cpu().numpy()[idx]
    ec, em = _rel(dc, d_ref), _rel(dm, d_ref)
    print(f"vslab_80x80x40: mixed_corner max error {ec:.3e} of max|d|, mixed {em:.3e}")
    assert np.all(np.isfinite(dc)) and em <= TOLMIX


def test_mixed_corner_is_forward_only(g):
    mesh, sv, m = synth.small_random_problem(6, 5, 4, 30, seed=142)
    S = g.Survey(sv.x, sv.y, sv.z)
    r = _dev(np.ones(sv.n))
    with pytest.raises(g.GravError) as e:
        g.adjoint(r, mesh, S, precision="mixed_corner")
    assert e.value.code == g.GRAV_EINVAL
    with pytest.raises(g.GravError) as e:
        g.diag(mesh, S, precision="mixed_corner")
    assert e.value.code == g.GRAV_EINVAL
    with pytest.raises(g.GravError) as e:
        g.datainv(_dev(np.ones(sv.n)), mesh, S, precision="mixed_corner")
    assert e.value.code == g.GRAV_EINVAL
    with pytest.raises(g.GravError) as e:
        g.Plan(mesh, S, precision="mixed_corner").adjoint(r)
    assert e.value.code == g.GRAV_EINVAL


# ---------------------------------------------------------------- errors ---

def test_error_paths(g):
    mesh, sv, m = synth.small_random_problem(4, 4, 3, 10, seed=70)
    S = g.Survey(sv.x, sv.y, sv.z)
    with pytest.raises(g.GravError) as e:
        g.forward(_dev(m), synth.Mesh(mesh.xe[::-1].copy(), mesh.ye, mesh.ze), S)
    assert e.value.code == g.GRAV_EINVAL
    irregular, sv2, m2 = synth.small_random_problem(4, 4, 3, 10, seed=71, irregular=True)
    with pytest.raises(g.GravError) as e:
        g.forward(_dev(m2), irregular, g.Survey(sv2.x, sv2.y, sv2.z), precision="mixed")
    assert e.value.code == g.GRAV_EINVAL and "uniform mesh" in str(e.value)
    with pytest.raises(g.GravError):
        g.forward(_dev(m), mesh, S, near_cells=0.2, precision="mixed")
    # host pointer for a device argument
    import ctypes
    ctx = g.context()
    d = torch.empty(sv.n, dtype=torch.float64, device="cuda")
    host = np.zeros(mesh.ncells)
    rc = g._lib.grav_forward(ctx.h, ctypes.byref(g.Mesh.of(mesh).c), ctypes.byref(S.c), host.ctypes.data,
                             d.data_ptr(), None, g._stream(None))
    assert rc == g.GRAV_EINVAL


# ------------------------------------------------------------ stored G -----

def test_stored_g_matches_oracle(g):
    """cache_g: G built once in FP64 (node-shared differencing) and streamed for
    every product; forward, adjoint (plain and depth-weighted) and diag match
    the oracle at the FP64 tolerance."""
    mesh, sv, m = synth.small_random_problem(17, 13, 9, 333, seed=101, irregular=True)
    S = g.Survey(sv.x, sv.y, sv.z)
    plan = g.Plan(mesh, S, cache_g=True)
    assert plan.describe()["stored_g"] is True
    d = plan.forward(_dev(m)).cpu().numpy()
    assert _rel(d, oracle.forward(mesh, sv, m)) <= TOL64
    r = synth.random_vector(sv.n, 102)
    for dw in (False, True):
        a = plan.adjoint(_dev(r), depth_weighted=dw).cpu().numpy()
        assert _rel(a, oracle.adjoint(mesh, sv, r, depth_weighted=dw, z0=50.0)) <= TOL64
    dg, tr = g.diag(mesh, S, cache_g=True)
    assert _rel(dg.cpu().numpy(), oracle.diag_GWG(mesh, sv, 50.0)) <= TOL64
    plan.close()


def test_stored_g_inversion_equals_matrix_free(g):
    wl = synth.make_workload("block_20x20x10")
    S = g.Survey(wl.survey.x, wl.survey.y, wl.survey.z)
    d = g.forward(_dev(wl.m), wl.mesh, S)
    m1, i1 = g.datainv(d, wl.mesh, S, tol=1e-10, max_iter=3000)
    m2, i2 = g.datainv(d, wl.mesh, S, tol=1e-10, max_iter=3000, cache_g=True)
    assert i1["converged"] and i2["converged"]
    assert i2["lambda"] == pytest.approx(i1["lambda"], rel=1e-12)
    assert _rel(m2.cpu().numpy(), m1.cpu().numpy()) <= 1e-6


def test_stored_g_vslab_full_size_sampled(g):
    wl = synth.make_workload("vslab_80x80x40")
    S = g.Survey(wl.survey.x, wl.survey.y, wl.survey.z)
    plan = g.Plan(wl.mesh, S, cache_g=True)
    assert plan.describe()["stored_g"] is True
    d = plan.forward(_dev(wl.m)).cpu().numpy()
    rng = np.random.Generator(np.random.PCG64(103))
    idx = np.sort(rng.choice(wl.survey.n, 32, replace=False))
    d_ref = oracle.forward(wl.mesh, wl.survey.subset(idx), wl.m)
    assert np.abs(d[idx] - d_ref).max() <= TOL64 * np.abs(d_ref).max()
    plan.close()


@pytest.mark.parametrize("precond", ["none", "jacobi"])
def test_outer_loop_reaches_dense_lu_minimiser(g, precond):
    """The paper's outer model-update loop (<= 20 inner CG iterations per
    update, step length by backtracking on the objective of Eq. 7) converges to
    the same minimiser as the dense LU of Eq. 11."""
    wl = synth.make_workload("block_20x20x10")
    G = oracle.G_explicit(wl.mesh, wl.survey)
    d = synth.add_noise(G @ wl.m, wl.noise_abs, wl.noise_rel, 0)
    ref = oracle.invert_dense(wl.mesh, wl.survey, d, z0=50.0)
    S = g.Survey(wl.survey.x, wl.survey.y, wl.survey.z)
    m, y, info = g.datainv(_dev(d), wl.mesh, S, return_y=True, tol=1e-8, max_iter=5000, outer_max=100,
                           inner_max=20, precond=precond)
    assert info["converged"] and info["outer"] >= 2, info
    y = y.cpu().numpy()
    A = (G * ref["wm"]) @ G.T + ref["lam"] * np.eye(len(d))
    res = np.linalg.norm(d - A @ y)
    assert res <= 1.5e-8 * np.linalg.norm(d)
    assert np.linalg.norm(y - ref["y"]) <= 1.01 * res / ref["lam"]
    assert info["true_rel_res"] <= 1e-8


def test_empty_survey_one_shot_calls(g):
    """n = 0 stations: forward is a no-op, G^T r = 0, the inversion returns
    m_ref (the minimiser of Eq. 7 with no data term), and a plan is refused."""
    mesh = synth.uniform_mesh(5, 4, 3, 10.0, 10.0, 10.0)
    S = g.Survey(np.zeros(0), np.zeros(0), np.zeros(0))
    empty = torch.zeros(0, dtype=torch.float64, device="cuda")
    m = _dev(np.arange(mesh.ncells, dtype=np.float64))
    for prec in ("fp64", "mixed"):
        assert g.forward(m, mesh, S, precision=prec).numel() == 0
        a = g.adjoint(empty, mesh, S, precision=prec)
        assert a.shape == (mesh.ncells,) and not a.any()
        mo, info = g.datainv(empty, mesh, S, precision=prec, m_ref=m)
        assert torch.equal(mo, m) and info["converged"] and info["iters"] == 0
        mo, info = g.datainv(empty, mesh, S, precision=prec)
        assert not mo.any()
    with pytest.raises(g.GravError) as e:
        g.Plan(mesh, S)
    assert e.value.code == g.GRAV_EINVAL


def test_fp64_error_statement(g):
    """check_fp64 / check_stations: the error a mixed result states against the
    FP64 operator equals its error against the oracle at the same stations
    (the FP64 operator matches the oracle to 1e-10), and is within 1e-5."""
    wl = synth.make_workload("vslab_80x80x40")
    S = g.Survey(wl.survey.x, wl.survey.y, wl.survey.z)
    plan = g.Plan(wl.mesh, S, precision="mixed")
    m = _dev(wl.m)
    d = plan.forward(m)
    n_check = 48
    ea, er = plan.check_fp64(m, d, n_check)
    idx = (np.arange(n_check) * wl.survey.n) // n_check
    d_ref = oracle.forward(wl.mesh, wl.survey.subset(idx), wl.m)
    dd = d.cpu().numpy()[idx]
    assert abs(ea - np.abs(dd - d_ref).max()) <= 1e-10 * np.abs(d_ref).max()
    assert 0 < er <= TOLMIX
    # relative to max |g|: the larger of the checked stations' FP64 values and
    # the product's largest magnitude over every station
    scale = max(np.abs(d_ref).max(), np.abs(d.cpu().numpy()).max())
    assert abs(er - ea / scale) <= 1e-12 * er
    plan.close()
    p64 = g.Plan(wl.mesh, S)
    assert p64.check_fp64(m, p64.forward(m), 16)[1] <= 1e-13
    p64.close()
    with pytest.raises(g.GravError):
        plan2 = g.Plan(wl.mesh, S, precision="mixed")
        try:
            plan2.check_fp64(m, d, wl.survey.n + 1)
        finally:
            plan2.close()
    # inversions state the error of their predicted data
    blk = synth.make_workload("block_20x20x10")
    S1 = g.Survey(blk.survey.x, blk.survey.y, blk.survey.z)
    d1 = g.forward(_dev(blk.m), blk.mesh, S1)
    _, info = g.datainv(d1, blk.mesh, S1, precision="mixed", tol=1e-6, check_stations=32)
    assert 0 < info["fp64_rel_err"] <= TOLMIX
    _, info = g.datainv(d1, blk.mesh, S1, precision="fp64", tol=1e-6, check_stations=32)
    assert info["fp64_rel_err"] == -1.0


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_reorthogonalised_cg(g, prec):
    """Full reorthogonalisation of the CG residuals (the default) reaches the
    minimiser of Eq. 7 like plain CG (reorth = 0), in fewer iterations: for
    either solve ||y - y*|| <= ||dd - A y|| / lambda with A and y* from the
    oracle's explicit G and dense LU."""
    wl = synth.make_workload("block_20x20x10")
    G = oracle.G_explicit(wl.mesh, wl.survey)
    d = synth.add_noise(G @ wl.m, wl.noise_abs, wl.noise_rel, 5)
    ref = oracle.invert_dense(wl.mesh, wl.survey, d, z0=50.0)
    A = (G * ref["wm"]) @ G.T + ref["lam"] * np.eye(len(d))
    S = g.Survey(wl.survey.x, wl.survey.y, wl.survey.z)
    tol = 1e-8 if prec == "fp64" else 1e-6
    its = {}
    for reorth in (1000, 0):
        m, y, info = g.datainv(_dev(d), wl.mesh, S, precision=prec, tol=tol, max_iter=5000, reorth=reorth,
                               return_y=True)
        assert info["converged"], (reorth, info)
        y = y.cpu().numpy()
        res = np.linalg.norm(d - A @ y)
        assert res <= (1.5e-8 if prec == "fp64" else 1e-5) * np.linalg.norm(d)
        assert np.linalg.norm(y - ref["y"]) <= 1.01 * res / ref["lam"]
        its[reorth] = info["iters"]
    assert its[1000] < its[0], its


def test_resume_from_y0_and_residual_history(g):
    """grav_datainv_solve_ex: a solve stopped at max_iter resumes from its y
    (checkpoint/resume) and reaches the same minimiser; a converged y needs no
    iteration; res_hist records the recurrence residual of every iteration."""
    wl = synth.make_workload("block_20x20x10")
    G = oracle.G_explicit(wl.mesh, wl.survey)
    d = synth.add_noise(G @ wl.m, wl.noise_abs, wl.noise_rel, 3)
    ref = oracle.invert_dense(wl.mesh, wl.survey, d, z0=50.0)
    A = (G * ref["wm"]) @ G.T + ref["lam"] * np.eye(len(d))
    S = g.Survey(wl.survey.x, wl.survey.y, wl.survey.z)
    dd = _dev(d)
    m1, y1, info1 = g.datainv(dd, wl.mesh, S, tol=1e-8, max_iter=15, return_y=True, res_hist=True)
    assert info1["status"] == g.GRAV_ENOTCONVERGED and info1["iters"] == 15
    h = info1["res_hist"]
    assert len(h) == 15 and h[-1] < h[0]
    m2, y2, info2 = g.datainv(dd, wl.mesh, S, tol=1e-8, max_iter=2000, return_y=True, y0=y1, res_hist=True)
    assert info2["converged"]
    y2n = y2.cpu().numpy()
    res = np.linalg.norm(d - A @ y2n)
    assert res <= 1.5e-8 * np.linalg.norm(d)
    assert np.linalg.norm(y2n - ref["y"]) <= 1.01 * res / ref["lam"]
    assert abs(info2["res_hist"][-1] - info2["rel_res"]) <= 1e-12 + 1e-6 * info2["rel_res"]
    m3, info3 = g.datainv(dd, wl.mesh, S, tol=1e-6, max_iter=100, y0=y2)
    assert info3["converged"] and info3["iters"] == 0
    assert torch.allclose(m3, m2, rtol=0, atol=1e-9 * float(m2.abs().max()))


def test_restarted_cg_counts_iterations_and_history(g):
    """Mixed inversion on noisy data that needs restarts from the true
    residual (vertical slab, 80 x 80 x 40 cells, 1 % + 0.01 mGal noise): the
    CG batches run one ahead of the host's convergence check, yet the
    reported iterations are those that updated y, res_hist holds one entry
    per such iteration (no gaps after a restart), the true residual meets
    tol, and the predicted data match the FP64 operator."""
    wl = synth.make_workload("vslab_80x80x40")
    S = g.Survey(wl.survey.x, wl.survey.y, wl.survey.z)
    d = g.forward(_dev(wl.m), wl.mesh, S, precision="fp64").cpu().numpy()
    d = synth.add_noise(d, wl.noise_abs, wl.noise_rel, 7)
    m, info = g.datainv(_dev(d), wl.mesh, S, precision="mixed", tol=1e-6, max_iter=3000, res_hist=True)
    assert info["converged"] and info["true_rel_res"] <= 1e-6
    assert info["restarts"] >= 1, info
    h = info["res_hist"]
    assert len(h) == info["iters"]
    assert np.all(h > 0) and h[-1] <= 1e-6 * (1 + 1e-9)
    dm = g.forward(m, wl.mesh, S, precision="mixed").cpu().numpy()
    d64 = g.forward(m, wl.mesh, S, precision="fp64").cpu().numpy()
    assert _rel(dm, d64) <= TOLMIX


@pytest.mark.parametrize("cf", [1, 2])
def test_nystrom_coarse_operator_matches_oracle_and_matrix_free(g, cf):
    """The sketch operator of the Nystrom preconditioner, K_c X with explicit
    FP32 blocks of G_c W_c^-1 / cf^1.5 and two FP32 GEMMs, against
    (a) K_c = G_c W_c^-2 G_c^T / cf^3 from the oracle's explicit G of the
    coarsened mesh (exact prisms; the sketch's point-mass term beyond 3 coarse
    cells is off by at most 6e-5 of max |K_c X| on this geometry, computed in
    FP64 on the CPU), and (b) the matrix-free mixed products on the coarse
    mesh with the same near window (identical entries: FP32 rounding only)."""
    wl = synth.make_workload("block_20x20x10")
    cm = synth.Mesh(wl.mesh.xe[::cf], wl.mesh.ye[::cf], wl.mesh.ze[::cf])
    G = oracle.G_explicit(cm, wl.survey)
    K = (G * oracle.depth_w2(cm, 50.0)) @ G.T / cf ** 3
    X = np.stack([synth.random_vector(wl.survey.n, 5 + j) for j in range(4)], axis=1)
    S = g.Survey(wl.survey.x, wl.survey.y, wl.survey.z)
    Y = g.nystrom_coarse_apply(torch.tensor(X, device="cuda"), wl.mesh, S, cf).cpu().numpy()
    ref = K @ X
    for j in range(X.shape[1]):
        scale = np.abs(ref[:, j]).max()
        assert np.abs(Y[:, j] - ref[:, j]).max() <= 2e-4 * scale, j
        q = g.adjoint(torch.tensor(X[:, j], device="cuda"), cm, S, depth_weighted=True, precision="mixed",
                      near_cells=3)
        ymf = g.forward(q, cm, S, precision="mixed", near_cells=3).cpu().numpy() / cf ** 3
        assert np.abs(Y[:, j] - ymf).max() <= 1e-5 * scale, j
    # a vector input gives the same column
    y0 = g.nystrom_coarse_apply(torch.tensor(X[:, 0], device="cuda"), wl.mesh, S, cf).cpu().numpy()
    assert np.abs(y0 - Y[:, 0]).max() <= 1e-6 * np.abs(ref[:, 0]).max()


@pytest.mark.parametrize("prec,rank,cf", [("fp64", 120, 0), ("mixed", 120, 0), ("mixed", 120, 2), ("fp64", 0, 0)])
def test_nystrom_pcg_reaches_dense_lu_minimiser(g, prec, rank, cf):
    """precond = 2: CG preconditioned by a randomized Nystrom approximation of
    G W^-2 G^T, sketched with the explicit operator (automatic coarsening: 1
    on this 20 x 20 x 10 mesh; also 2 x 2 x 2), and reorthogonalised in the
    preconditioner's inner product, reaches the minimiser of Eq. 7 from the
    oracle's explicit G and dense LU (||y - y*|| <= ||dd - A y|| / lambda), in
    fewer iterations than Jacobi PCG.  Rank 0 (automatic, N / 2 in FP64)
    sketches half the spectrum, far below the FP32 rounding of the products."""
    wl = synth.make_workload("block_20x20x10")
    G = oracle.G_explicit(wl.mesh, wl.survey)
    d = synth.add_noise(G @ wl.m, wl.noise_abs, wl.noise_rel, 9)
    ref = oracle.invert_dense(wl.mesh, wl.survey, d, z0=50.0)
    A = (G * ref["wm"]) @ G.T + ref["lam"] * np.eye(len(d))
    S = g.Survey(wl.survey.x, wl.survey.y, wl.survey.z)
    tol = 1e-8 if prec == "fp64" else 1e-6
    its = {}
    for pc in ("nystrom", "jacobi"):
        m, y, info = g.datainv(_dev(d), wl.mesh, S, precision=prec, tol=tol, max_iter=3000, precond=pc,
                               nys_rank=rank, nys_coarsen=cf, return_y=True)
        assert info["converged"], (pc, info)
        y = y.cpu().numpy()
        res = np.linalg.norm(d - A @ y)
        assert res <= (1.5e-8 if prec == "fp64" else 1e-5) * np.linalg.norm(d), pc
        assert np.linalg.norm(y - ref["y"]) <= 1.01 * res / ref["lam"], pc
        its[pc] = info["iters"]
    assert its["nystrom"] < its["jacobi"], its


# ------------------------------------------------ dense kernels (Nystrom) ---

def test_dense_kernels_sgemm_and_gram(g):
    """The preconditioner's dense kernels against float64 products of the same
    FP32 inputs, on ragged sizes (partial 128 x 128 / 64 x 64 tiles, K not a
    multiple of the 16-deep slices).  SGEMM (FP32 sums of K terms): within the
    recursive-summation bound (K + 2) u (|A| |B|), u = 2^-24.  Gram (exact
    products, double-float runs of 128 products added into FP64): within
    min(K, 128) 2^-48 + K 2^-53 of (|X|^T |X|), the runs' bound plus an FP64
    recursive sum's, also at K = 60,000 where one double-float run over all of
    K would be 400 times worse; dropping the low word or the products'
    rounding errors misses it by orders of magnitude.  Accumulation adds to
    C; a leading dimension that is not a multiple of 4 is refused."""
    ctx = g.context()
    rng = np.random.default_rng(31)
    u = 2.0 ** -24

    def run(op, M, N, K, A, lda, B, ldb, C, ldc, acc):
        rc = g._lib.grav_dense_check(ctx.h, op, M, N, K, A.data_ptr(), lda,
                                     B.data_ptr() if B is not None else None, ldb, C.data_ptr(), ldc, acc,
                                     g._stream(None))
        return rc

    for op, M, N, K in ((0, 132, 77, 1000), (1, 260, 130, 52), (0, 4, 1, 4), (1, 388, 257, 1028)):
        lda = K + 4 if op == 0 else M + 8
        a_cols = M if op == 0 else K
        A = rng.standard_normal((a_cols, lda)).astype(np.float32)   # row = one column of the col-major array
        ldb = K + 8
        B = rng.standard_normal((N, ldb)).astype(np.float32)
        ldc = M + 4
        C0 = rng.standard_normal((N, ldc)).astype(np.float32)
        Am = A[:, :K].astype(np.float64) if op == 0 else A[:, :M].T.astype(np.float64)   # Am[m, k]
        Bm = B[:, :K].T.astype(np.float64)                                             # Bm[k, n]
        ref = Am @ Bm
        bound = (K + 2) * u * (np.abs(Am) @ np.abs(Bm))
        for acc in (0, 1):
            At, Bt, Ct = (torch.tensor(x, device="cuda") for x in (A, B, C0))
            assert run(op, M, N, K, At, lda, Bt, ldb, Ct, ldc, acc) == g.GRAV_OK
            got = Ct.cpu().numpy()[:, :M].T.astype(np.float64)
            want = ref + (C0[:, :M].T.astype(np.float64) if acc else 0.0)
            assert np.all(np.abs(got - want) <= bound + (np.abs(C0[:, :M].T) * u * 2 if acc else 0.0)), (op, M, N, K)
            # untouched padding columns of C
            assert np.array_equal(Ct.cpu().numpy()[:, M:], C0[:, M:])
    # Gram: G = X^T X, lower triangle
    for n, K in ((150, 1004), (64, 16), (5, 4), (70, 60000)):
        ldx = K + 4
        X = rng.standard_normal((n, ldx)).astype(np.float32)
        Xm = X[:, :K].T.astype(np.float64)
        ref = Xm.T @ Xm
        scale = np.abs(Xm).T @ np.abs(Xm)
        Gt = torch.full((n, n), 7.0, dtype=torch.float64, device="cuda")   # G[i + n j] -> row j, column i
        Xt = torch.tensor(X, device="cuda")
        assert run(2, 0, n, K, Xt, ldx, None, 0, Gt, n, 0) == g.GRAV_OK
        got = Gt.cpu().numpy().T           # got[i, j]
        low = np.tril(np.ones((n, n), bool))
        tol = min(K, 128) * 2.0 ** -48 + K * 2.0 ** -53
        assert np.all(np.abs(got - ref)[low] <= tol * scale[low]), (n, K)
        assert np.all(got[~low] == 7.0)    # the upper triangle is not written
        assert run(2, 0, n, K, Xt, ldx, None, 0, Gt, n, 1) == g.GRAV_OK
        got2 = Gt.cpu().numpy().T
        assert np.all(np.abs(got2 - 2 * ref)[low] <= 2 * tol * scale[low])
    # k-slow layouts (no transposed tiles): op 3 / 4 take B(k, n) = B[n + ldb k]
    # (op 3 also writes C(m, n) = C[n + ldc m]), op 5 the Gram of X(k, i) = X[i + ldx k];
    # N not a multiple of 4, rows padded to a multiple of 4
    for op, M, N, K in ((3, 260, 77, 1000), (4, 132, 130, 52), (3, 4, 1, 4), (4, 388, 257, 1028)):
        lda = M + 8
        A = rng.standard_normal((K, lda)).astype(np.float32)            # A(m, k) = A[k, m]
        ldb = (N + 3) // 4 * 4 + 4
        B = rng.standard_normal((K, ldb)).astype(np.float32)            # B(k, n) = B[k, n]
        Am, Bm = A[:, :M].T.astype(np.float64), B[:, :N].astype(np.float64)
        ref = Am @ Bm
        bound = (K + 2) * u * (np.abs(Am) @ np.abs(Bm))
        if op == 3:
            ldc = (N + 3) // 4 * 4
            C0 = rng.standard_normal((M, ldc)).astype(np.float32)       # C(m, n) = C[m, n]
        else:
            ldc = M + 4
            C0 = rng.standard_normal((N, ldc)).astype(np.float32)       # C(m, n) = C[n, m]
        for acc in (0, 1):
            At, Bt, Ct = (torch.tensor(x, device="cuda") for x in (A, B, C0))
            assert run(op, M, N, K, At, lda, Bt, ldb, Ct, ldc, acc) == g.GRAV_OK
            c = Ct.cpu().numpy()
            got = c[:, :N].astype(np.float64) if op == 3 else c[:, :M].T.astype(np.float64)
            c0 = C0[:, :N] if op == 3 else C0[:, :M].T
            want = ref + (c0.astype(np.float64) if acc else 0.0)
            assert np.all(np.abs(got - want) <= bound + (np.abs(c0) * u * 2 if acc else 0.0)), (op, M, N, K)
    for n, K in ((150, 1004), (63, 16), (5, 4)):
        ldx = (n + 3) // 4 * 4 + 4
        X = rng.standard_normal((K, ldx)).astype(np.float32)            # X(k, i) = X[k, i]
        Xm = X[:, :n].astype(np.float64)
        ref = Xm.T @ Xm
        scale = np.abs(Xm).T @ np.abs(Xm)
        tol = min(K, 128) * 2.0 ** -48 + K * 2.0 ** -53
        Gt = torch.full((n, n), 7.0, dtype=torch.float64, device="cuda")
        assert run(5, 0, n, K, torch.tensor(X, device="cuda"), ldx, None, 0, Gt, n, 0) == g.GRAV_OK
        got = Gt.cpu().numpy().T
        low = np.tril(np.ones((n, n), bool))
        assert np.all(np.abs(got - ref)[low] <= tol * scale[low]), (n, K)
        assert np.all(got[~low] == 7.0)
    # refused layouts: nothing launched
    A = torch.zeros((8, 10), dtype=torch.float32, device="cuda")
    C = torch.zeros((8, 8), dtype=torch.float32, device="cuda")
    assert run(0, 8, 8, 8, A, 10, A, 10, C, 8, 0) == g.GRAV_EINVAL
    assert run(1, 6, 8, 8, A, 8, A, 8, C, 8, 0) == g.GRAV_EINVAL
    assert run(3, 8, 9, 8, A, 8, A, 8, C, 12, 0) == g.GRAV_EINVAL      # n-major B rows shorter than 12


def test_fp64_widest_node_row_and_the_cap(g):
    """The FP64 forward stages one row of nx+1 node weights (rounded up to
    even) in shared memory with two stage buffers: nx + 1 = 8527 fills the
    200 KB limit exactly (128 + 24 * 8528 bytes) and still matches the oracle
    (forward, and the adjoint on the cells near the stations, 1e-10 of max);
    one node more is refused with GRAV_EINVAL before anything runs."""
    nx = 8526
    xe = np.linspace(0.0, 10.0 * nx, nx + 1)
    mesh = synth.Mesh(xe, np.array([0.0, 10.0]), np.array([0.0, 10.0, 25.0]))
    rng = np.random.Generator(np.random.PCG64(213))
    n = 300
    # stations over x in [40, 45] km and densities only in cells 3500..4999
    # (35-50 km): every node row is staged (zero node weights are skipped, not
    # left out), while no station sees a non-zero cell more than ~1,000 cells
    # away -- at 8,500 cells of 10 m the FP64 corner formula itself (oracle
    # and kernel alike) loses ~1e-10 of max |d| to its far-field rounding
    # (relative error ~ eps (R/a)^3 (R/z) ln R per prism)
    sv = synth.Survey(rng.uniform(40000.0, 45000.0, n), rng.uniform(-20, 30, n), -rng.uniform(0.5, 10, n))
    m = np.zeros(mesh.ncells)
    for layer in (0, 1):
        m[layer * nx + 3500:layer * nx + 5000] = rng.normal(0.0, 5.0, 1500)
    for c0 in rng.integers(3500, 4700, 6):
        m[c0:c0 + 300] += 250.0
    S = g.Survey(sv.x, sv.y, sv.z)
    d = g.forward(_dev(m), mesh, S).cpu().numpy()
    assert _rel(d, oracle.forward(mesh, sv, m)) <= TOL64
    r = synth.random_vector(n, 214)
    a = g.adjoint(_dev(r), mesh, S).cpu().numpy()
    a_ref = oracle.adjoint(mesh, sv, r)
    # G^T r of the cells within 500 cells of the stations: further out the
    # corner formula's rounding grows like eps (R/a)^3 (R/z) ln R in any FP64
    # evaluation (a node-shared FP64 sum in numpy differs from the oracle by
    # 6e-11 of max over these cells, 1.6e-10 over cells within 1,500)
    near = np.zeros(mesh.ncells, bool)
    for layer in (0, 1):
        near[layer * nx + 3500:layer * nx + 5000] = True
    assert _rel(a[near], a_ref[near]) <= TOL64
    wide = synth.Mesh(np.linspace(0.0, 10.0 * (nx + 2), nx + 3), mesh.ye, mesh.ze)
    with pytest.raises(g.GravError) as e:
        g.forward(_dev(np.zeros(wide.ncells)), wide, S)
    assert e.value.code == g.GRAV_EINVAL and "nx+1 must be <=" in str(e.value)


def test_dense_cholesky_and_triangular_inverse(g):
    """The device factorisation of the Nystrom matrix (blocked FP64 Cholesky
    and explicit inverse of the factor): on SPD matrices of sizes around the
    32-wide blocks and the 64-wide update tiles, L L^T reproduces A to the
    backward-error scale n 2^-53 |L| |L|^T, L equals numpy's Cholesky factor on
    a well-conditioned matrix, and L^-1 L = I to n 2^-53 |L^-1| |L|; a matrix
    that is not positive definite is reported as GRAV_EDEVICE."""
    ctx = g.context()
    rng = np.random.default_rng(77)
    u = 2.0 ** -53

    def factor(A):
        n = A.shape[0]
        At = torch.tensor(np.asfortranarray(A).ravel(order="F"), device="cuda")
        Ct = torch.zeros(2 * n * n, dtype=torch.float64, device="cuda")
        rc = g._lib.grav_dense_check(ctx.h, 6, 0, n, 0, At.data_ptr(), 0, None, 0, Ct.data_ptr(), 0, 0,
                                     g._stream(None))
        C = Ct.cpu().numpy()
        return rc, np.tril(C[:n * n].reshape(n, n, order="F")), C[n * n:].reshape(n, n, order="F")

    for n in (1, 5, 31, 32, 33, 64, 100, 257, 1000):
        X = rng.standard_normal((n, n + 3))
        A = X @ X.T + n * np.eye(n)
        rc, L, Li = factor(A)
        assert rc == g.GRAV_OK, n
        assert np.all(np.abs(L @ L.T - A) <= 4 * n * u * (np.abs(L) @ np.abs(L).T) + 1e-300), n
        Lnp = np.linalg.cholesky(A)
        assert np.abs(L - Lnp).max() <= 1e-12 * np.abs(Lnp).max(), n
        assert np.array_equal(np.triu(Li, 1), np.zeros((n, n))), n
        assert np.all(np.abs(Li @ L - np.eye(n)) <= 4 * n * u * (np.abs(Li) @ np.abs(L)) + 1e-300), n
    # ill-conditioned, shaped like the preconditioner's T (a Gram matrix plus a small shift)
    n = 300
    Y = rng.standard_normal((2000, n)) * np.logspace(0, -5, n)
    A = Y.T @ Y + 1e-9 * np.eye(n)
    rc, L, Li = factor(A)
    assert rc == g.GRAV_OK
    assert np.all(np.abs(L @ L.T - A) <= 4 * n * u * (np.abs(L) @ np.abs(L).T))
    assert np.all(np.abs(Li @ L - np.eye(n)) <= 4 * n * u * (np.abs(Li) @ np.abs(L)))
    # not positive definite
    A = np.eye(40)
    A[20, 20] = -1.0
    rc, _, _ = factor(A)
    assert rc == g.GRAV_EDEVICE
