"""GPU tests of the serving scheduler (grav_submit / poll / wait / cancel).

* A mix of forward and inversion jobs (FP64 and mixed precision, different
  mesh and survey sizes) submitted together to a 3-slot scheduler gives, for
  every job, bitwise the same output as the same job run alone through the
  one-shot calls, and at least two jobs overlap in time.
* Nystrom-preconditioned inversion jobs (precond = 2) in such a mix give the
  results they give alone, within 1e-9 of max |m|.
* Host-side failure paths, none of which faults the GPU: cancelling a queued
  and a running job, a bounded wait that times out, an unknown job id, a job
  larger than the context's HBM budget, and CG stopping at max_iter.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_03857_b300 as g
    return g


def _problem(seed, nx, ny, nz, ns, cell):
    rng = np.random.Generator(np.random.PCG64(500 + seed))
    mesh = synth.uniform_mesh(nx, ny, nz, cell, cell, cell)
    sv = synth.Survey(rng.uniform(0, nx * cell, ns), rng.uniform(0, ny * cell, ns), -rng.uniform(1, 20, ns))
    m = np.zeros((nz, ny, nx))
    m[1:nz // 2, ny // 4:ny // 2, nx // 3:nx // 3 + 3] = rng.uniform(100, 400)
    m = m.ravel() + rng.normal(0, 5, m.size)
    return mesh, sv, m


def _dev(x):
    return torch.as_tensor(np.asarray(x, dtype=np.float64), device="cuda")


def test_mixed_batch_matches_solo_runs(g):
    solo_ctx = g.context()
    specs = [("forward", "fp64", (20, 18, 8, 300, 25.0)), ("invert", "mixed", (40, 36, 12, 900, 50.0)),
             ("forward", "mixed", (60, 50, 20, 2000, 40.0)), ("invert", "fp64", (16, 14, 6, 200, 30.0)),
             ("invert", "mixed", (30, 30, 10, 600, 20.0)), ("forward", "fp64", (12, 40, 9, 350, 35.0)),
             ("invert", "mixed", (50, 20, 16, 700, 45.0)), ("forward", "mixed", (24, 24, 24, 1200, 30.0))]
    jobs = []
    for q, (kind, prec, shape) in enumerate(specs):
        mesh, sv, m = _problem(q, *shape)
        S = g.Survey(sv.x, sv.y, sv.z)
        opts = dict(precision=prec, tol=1e-8 if prec == "fp64" else 1e-5, max_iter=3000)
        if kind == "forward":
            inp = _dev(m)
            solo = g.forward(inp, mesh, S, ctx=solo_ctx, **opts)
            out = torch.full((sv.n,), float("nan"), dtype=torch.float64, device="cuda")
        else:
            inp = g.forward(_dev(m), mesh, S, ctx=solo_ctx, precision="fp64")
            solo, info = g.datainv(inp, mesh, S, ctx=solo_ctx, **opts)
            out = torch.full((mesh.ncells,), float("nan"), dtype=torch.float64, device="cuda")
        jobs.append((kind, mesh, S, inp, out, solo, opts))
    torch.cuda.synchronize()
    ctx = g.Context(0)
    try:
        ctx.serve_config(3)
        ids = [ctx.submit(kind, mesh, S, inp, out, **opts) for kind, mesh, S, inp, out, solo, opts in jobs]
        for jid in ids:
            assert ctx.wait(jid, 600.0) == g.GRAV_OK
        for jid, (kind, mesh, S, inp, out, solo, opts) in zip(ids, jobs):
            assert torch.equal(out, solo), (kind, opts["precision"])
            assert ctx.poll(jid)[0] == "done"
        # a mixed forward job asked to state its error against the FP64 operator
        mesh, sv, m = _problem(20, 40, 30, 12, 800, 25.0)
        S = g.Survey(sv.x, sv.y, sv.z)
        out = torch.empty(sv.n, dtype=torch.float64, device="cuda")
        jid = ctx.submit("forward", mesh, S, _dev(m), out, precision="mixed", check_stations=24)
        assert ctx.wait(jid, 600.0) == g.GRAV_OK
        err = ctx.poll(jid)[1]["fp64_rel_err"]
        assert 0 < err <= 1e-5
        times = [ctx.job_times(j) for j in ids]
        assert all(t0 <= t1 <= t2 for t0, t1, t2 in times)
        overlaps = sum(1 for a in times for b in times if a is not b and a[1] < b[2] and b[1] < a[2])
        assert overlaps > 0, "no two jobs ran at the same time"
    finally:
        ctx.close()


def test_nystrom_inversions_in_the_mix_match_solo_runs(g):
    """precond = 2 inversion jobs (each builds its own sketch, cuBLAS handle and
    host Cholesky factor in its worker thread) submitted with a forward job to a
    3-slot scheduler: each result equals the same job run alone within 1e-9 of
    max |m| (the set-up is deterministic: counter-based Omega, fixed-order
    factorisation), and the preconditioned jobs converge."""
    solo_ctx = g.context()
    specs = [("invert", "mixed", (40, 36, 12, 900, 50.0)), ("invert", "fp64", (16, 14, 8, 200, 30.0)),
             ("forward", "mixed", (60, 50, 20, 2000, 40.0)), ("invert", "mixed", (30, 30, 16, 600, 20.0))]
    jobs = []
    for q, (kind, prec, shape) in enumerate(specs):
        mesh, sv, m = _problem(40 + q, *shape)
        S = g.Survey(sv.x, sv.y, sv.z)
        if kind == "forward":
            opts = dict(precision=prec)
            inp = _dev(m)
            solo = g.forward(inp, mesh, S, ctx=solo_ctx, **opts)
            out = torch.full((sv.n,), float("nan"), dtype=torch.float64, device="cuda")
        else:
            opts = dict(precision=prec, tol=1e-8 if prec == "fp64" else 1e-5, max_iter=3000, precond="nystrom")
            inp = g.forward(_dev(m), mesh, S, ctx=solo_ctx, precision="fp64")
            solo, info = g.datainv(inp, mesh, S, ctx=solo_ctx, **opts)
            assert info["converged"], info
            out = torch.full((mesh.ncells,), float("nan"), dtype=torch.float64, device="cuda")
        jobs.append((kind, mesh, S, inp, out, solo, opts))
    torch.cuda.synchronize()
    ctx = g.Context(0)
    try:
        ctx.serve_config(3)
        ids = [ctx.submit(kind, mesh, S, inp, out, **opts) for kind, mesh, S, inp, out, solo, opts in jobs]
        for jid in ids:
            assert ctx.wait(jid, 600.0) == g.GRAV_OK
        for jid, (kind, mesh, S, inp, out, solo, opts) in zip(ids, jobs):
            state, info = ctx.poll(jid)
            assert state == "done"
            scale = float(solo.abs().max())
            assert float((out - solo).abs().max()) <= 1e-9 * scale, (kind, opts["precision"])
    finally:
        ctx.close()


def test_cancel_timeout_and_errors(g):
    ctx = g.Context(0)
    try:
        ctx.serve_config(1)
        wl = synth.make_workload("dipdyke_150x150x60")
        S = g.Survey(wl.survey.x, wl.survey.y, wl.survey.z)
        d = g.forward(_dev(wl.m), wl.mesh, S, precision="mixed", near_cells=3.0)
        out_a = torch.empty(wl.mesh.ncells, dtype=torch.float64, device="cuda")
        out_b = torch.empty(wl.mesh.ncells, dtype=torch.float64, device="cuda")
        slow = dict(precision="mixed", near_cells=3.0, tol=1e-14, max_iter=100000)
        a = ctx.submit("invert", wl.mesh, S, d, out_a, **slow)
        b = ctx.submit("invert", wl.mesh, S, d, out_b, **slow)
        assert ctx.poll(b)[0] == "queued"
        ctx.cancel(b)
        assert ctx.wait(b, 5.0) == g.GRAV_ECANCELED
        assert ctx.poll(b)[0] == "canceled"
        assert ctx.wait(a, 1e-3) == g.GRAV_ETIMEDOUT
        ctx.cancel(a)                                     # running inversion: stops at its next CG check
        assert ctx.wait(a, 120.0) == g.GRAV_ECANCELED
        with pytest.raises(g.GravError) as e:
            ctx.poll(987654321)
        assert e.value.code == g.GRAV_ENOTFOUND
        # CG stopping at max_iter finishes the job with GRAV_ENOTCONVERGED and writes the iterate
        c = ctx.submit("invert", wl.mesh, S, d, out_a, precision="mixed", near_cells=3.0, tol=1e-12, max_iter=2)
        assert ctx.wait(c, 120.0) == g.GRAV_ENOTCONVERGED
        assert torch.isfinite(out_a).all()
    finally:
        ctx.close()
    small = g.Context(0, hbm_budget=1 << 20)           # 1 MiB budget: admission must refuse
    try:
        mesh, sv, m = _problem(9, 40, 40, 20, 500, 25.0)
        S = g.Survey(sv.x, sv.y, sv.z)
        out = torch.empty(sv.n, dtype=torch.float64, device="cuda")
        with pytest.raises(g.GravError) as e:
            small.submit("forward", mesh, S, _dev(m), out)
        assert e.value.code == g.GRAV_ENOMEM
    finally:
        small.close()
