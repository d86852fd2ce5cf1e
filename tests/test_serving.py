"""GPU tests of the serving scheduler (grav_submit / poll / wait / cancel).

* A mix of forward and inversion jobs (FP64 and mixed precision, different
  mesh and survey sizes, one inversion with the paper's non-zero reference
  model) submitted together to a 3-slot scheduler gives, for every job,
  bitwise the same output as the same job run alone through the one-shot
  calls, and at least two jobs overlap in time.  Every job's output is also
  checked against the CPU oracle (see _oracle_check).
* Nystrom-preconditioned inversion jobs (precond = 2) in such a mix give the
  results they give alone, within 1e-9 of max |m|, and pass the same oracle
  check.
* Host-side failure paths, none of which faults the GPU: cancelling a queued
  and a running job, a bounded wait that times out, an unknown job id, a job
  larger than the context's HBM budget, and CG stopping at max_iter.
"""
import numpy as np
import pytest

import oracle
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


TOL64, TOLMIX = 1e-10, 1e-5
# The mixed operator's own exact minimiser (exact prisms inside the window,
# point masses outside, solved by dense LU on the CPU) lies 1.8e-10 to 2.3e-10
# of the minimum above the exact one on the 600-900-station meshes of these
# tests; this allowance keeps a 40x margin.
MIXED_EXCESS = 1e-8


def _oracle_check(kind, prec, mesh, sv, inp, out, tol=None, m_ref=None):
    """A serving job's output against the CPU oracle.

    forward: d at up to 256 evenly spaced stations against oracle.forward,
    within 1e-10 (FP64) or 1e-5 (mixed) of max |d|.

    invert: the Eq. 7 objective phi(m) = |d - G m|^2 / lam + |m - m_ref|^2_{W^2}
    with the oracle's explicit G and lam = 1e-2 trace / N, against its exact
    minimiser m* (dense LU of Eq. 10-11).  For m = m_ref + W^-2 G^T y and
    r = dd - A y (A = G W^-2 G^T + lam I, dd = d - G m_ref):
    phi(m) - phi(m*) = r^T A^-1 K r / lam <= |r|^2 / lam and
    phi(m*) = dd^T A^-1 dd >= |dd|^2 / |A|, so a solve converged to a
    relative residual <= tol has a relative excess <= tol^2 |A|_2 / lam."""
    inp = inp.cpu().numpy()
    out = out.cpu().numpy()
    if kind == "forward":
        idx = np.linspace(0, sv.n - 1, min(sv.n, 256)).astype(int)
        ref = oracle.forward(mesh, sv.subset(idx), inp)
        err = np.abs(out[idx] - ref).max() / np.abs(ref).max()
        assert err <= (TOL64 if prec == "fp64" else TOLMIX), (kind, prec, err)
        return err
    mr = np.zeros(mesh.ncells) if m_ref is None else m_ref
    ref = oracle.invert_dense(mesh, sv, inp, m_ref=mr)
    G, wm, lam = ref["G"], ref["wm"], ref["lam"]
    A = (G * wm[None, :]) @ G.T + lam * np.eye(sv.n)
    norm_a = float(np.linalg.eigvalsh(A)[-1])

    def phi(x):
        return float(np.sum((inp - G @ x) ** 2) / lam + np.sum((x - mr) ** 2 / wm))

    excess = (phi(out) - phi(ref["m"])) / phi(ref["m"])
    bound = tol ** 2 * norm_a / lam + (1e-11 if prec == "fp64" else MIXED_EXCESS)
    assert -1e-11 <= excess <= bound, (kind, prec, excess, bound)
    return excess


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
        m_ref = None
        if kind == "forward":
            inp = _dev(m)
            solo = g.forward(inp, mesh, S, ctx=solo_ctx, **opts)
            out = torch.full((sv.n,), float("nan"), dtype=torch.float64, device="cuda")
        else:
            inp = _dev(oracle.forward(mesh, sv, m))          # data from the oracle
            if q == 4:                                        # the paper's reference model, 0.1 kg/m^3
                m_ref = np.full(mesh.ncells, 0.1)
            solo, info = g.datainv(inp, mesh, S, ctx=solo_ctx,
                                   m_ref=_dev(m_ref) if m_ref is not None else None, **opts)
            out = torch.full((mesh.ncells,), float("nan"), dtype=torch.float64, device="cuda")
        jobs.append((kind, mesh, sv, S, inp, out, solo, opts, m_ref))
    torch.cuda.synchronize()
    ctx = g.Context(0)
    try:
        ctx.serve_config(3)
        ids = [ctx.submit(kind, mesh, S, inp, out, m_ref=_dev(m_ref) if m_ref is not None else None, **opts)
               for kind, mesh, sv, S, inp, out, solo, opts, m_ref in jobs]
        for jid in ids:
            assert ctx.wait(jid, 600.0) == g.GRAV_OK
        for jid, (kind, mesh, sv, S, inp, out, solo, opts, m_ref) in zip(ids, jobs):
            assert torch.equal(out, solo), (kind, opts["precision"])
            state, info = ctx.poll(jid)
            assert state == "done"
            if kind == "invert":
                assert info["converged"] and info["true_rel_res"] <= opts["tol"], info
            _oracle_check(kind, opts["precision"], mesh, sv, inp, out, opts.get("tol"), m_ref)
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
            inp = _dev(oracle.forward(mesh, sv, m))
            solo, info = g.datainv(inp, mesh, S, ctx=solo_ctx, **opts)
            assert info["converged"], info
            out = torch.full((mesh.ncells,), float("nan"), dtype=torch.float64, device="cuda")
        jobs.append((kind, mesh, sv, S, inp, out, solo, opts))
    torch.cuda.synchronize()
    ctx = g.Context(0)
    try:
        ctx.serve_config(3)
        ids = [ctx.submit(kind, mesh, S, inp, out, **opts) for kind, mesh, sv, S, inp, out, solo, opts in jobs]
        for jid in ids:
            assert ctx.wait(jid, 600.0) == g.GRAV_OK
        for jid, (kind, mesh, sv, S, inp, out, solo, opts) in zip(ids, jobs):
            state, info = ctx.poll(jid)
            assert state == "done"
            scale = float(solo.abs().max())
            assert float((out - solo).abs().max()) <= 1e-9 * scale, (kind, opts["precision"])
            _oracle_check(kind, opts["precision"], mesh, sv, inp, out, opts.get("tol"))
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


def test_backfill_and_resident_plans(g):
    """Admission by footprint with backfill, and resident plans.

    Two inversions L1, L2 on one mesh and survey (different data) and a small
    forward job S are submitted in the order L1, L2, S to a context whose HBM
    budget (2 f_L - 1, f the reserved footprints) holds L1 + S and L1's
    resident plan + L2, but not L1 + L2.  L2 must wait for L1's memory; S,
    behind it in the queue, starts at once and finishes before L2 starts
    (strict FIFO would hold it behind L2).  L2 then runs on the plan L1 left
    resident.  Every output equals the same job run through the one-shot
    calls, bitwise."""
    mesh, sv, m = _problem(60, 70, 60, 24, 4000, 25.0)
    S_big = g.Survey(sv.x, sv.y, sv.z)
    d1 = oracle.forward(mesh, sv, m)
    d2 = d1 * 0.5
    smesh, ssv, sm = _problem(62, 20, 18, 8, 300, 25.0)
    S_small = g.Survey(ssv.x, ssv.y, ssv.z)
    inv = dict(precision="mixed", tol=1e-5, max_iter=3000)
    solo_ctx = g.context()
    ref1, i1 = g.datainv(_dev(d1), mesh, S_big, ctx=solo_ctx, **inv)
    ref2, i2 = g.datainv(_dev(d2), mesh, S_big, ctx=solo_ctx, **inv)
    assert i1["converged"] and i2["converged"], (i1, i2)
    refs = g.forward(_dev(sm), smesh, S_small, ctx=solo_ctx, precision="mixed")
    # footprints, measured by the scheduler itself on a roomy context
    probe = g.Context(0)
    try:
        probe.plan_cache(0)
        o = torch.empty(mesh.ncells, dtype=torch.float64, device="cuda")
        a = probe.submit("invert", mesh, S_big, _dev(d1), o, **inv)
        os_ = torch.empty(ssv.n, dtype=torch.float64, device="cuda")
        b = probe.submit("forward", smesh, S_small, _dev(sm), os_, precision="mixed")
        assert probe.wait(a, 600.0) == g.GRAV_OK and probe.wait(b, 600.0) == g.GRAV_OK
        f_big, f_small = probe.job_plan(a)["footprint"], probe.job_plan(b)["footprint"]
    finally:
        probe.close()
    assert f_small < f_big // 4
    ctx = g.Context(0, hbm_budget=2 * f_big - 1)
    try:
        ctx.serve_config(3)
        out1 = torch.full((mesh.ncells,), float("nan"), dtype=torch.float64, device="cuda")
        out2 = torch.full((mesh.ncells,), float("nan"), dtype=torch.float64, device="cuda")
        outs = torch.full((ssv.n,), float("nan"), dtype=torch.float64, device="cuda")
        j1 = ctx.submit("invert", mesh, S_big, _dev(d1), out1, **inv)
        j2 = ctx.submit("invert", mesh, S_big, _dev(d2), out2, **inv)
        js = ctx.submit("forward", smesh, S_small, _dev(sm), outs, precision="mixed")
        for j in (j1, j2, js):
            assert ctx.wait(j, 600.0) == g.GRAV_OK
        t1, t2, ts = ctx.job_times(j1), ctx.job_times(j2), ctx.job_times(js)
        assert t2[1] >= t1[2], "L2 started before L1 released its memory"
        assert ts[1] < t2[1] and ts[2] <= t2[1], "the small job did not backfill ahead of L2"
        assert ctx.job_plan(j2)["plan_reused"] and not ctx.job_plan(j1)["plan_reused"]
        assert ctx.job_plan(j2)["setup_s"] == 0.0
        assert torch.equal(out1, ref1) and torch.equal(out2, ref2) and torch.equal(outs, refs)
    finally:
        ctx.close()


def test_resident_plan_stream_and_changed_survey(g):
    """An inversion stream on one survey through one slot builds one plan and
    reuses it; each result equals its one-shot run bitwise and the first one
    passes the oracle check.  Changing the survey's values in place (same
    device arrays) makes the next job build a fresh plan, whose result is the
    one-shot result for the new stations."""
    mesh, sv, m = _problem(70, 30, 26, 10, 700, 30.0)
    S = g.Survey(sv.x, sv.y, sv.z)
    d = oracle.forward(mesh, sv, m)
    opts = dict(precision="fp64", tol=1e-8, max_iter=3000)
    solo_ctx = g.context()
    ctx = g.Context(0)
    try:
        ctx.serve_config(1)
        datas = [d] + [d + synth.random_vector(sv.n, 71 + k, 0.005) for k in range(3)]
        ids, outs = [], []
        for dk in datas:
            out = torch.full((mesh.ncells,), float("nan"), dtype=torch.float64, device="cuda")
            ids.append(ctx.submit("invert", mesh, S, _dev(dk), out, **opts))
            outs.append(out)
        for j in ids:
            assert ctx.wait(j, 600.0) == g.GRAV_OK
        st = ctx.serve_stats()
        assert st["plans_built"] == 1 and st["plans_reused"] == 3 and st["plans_resident"] == 1
        assert [ctx.job_plan(j)["plan_reused"] for j in ids] == [False, True, True, True]
        for dk, out in zip(datas, outs):
            ref, _ = g.datainv(_dev(dk), mesh, S, ctx=solo_ctx, **opts)
            assert torch.equal(out, ref)
        _oracle_check("invert", "fp64", mesh, sv, _dev(datas[0]), outs[0], opts["tol"])
        # same arrays, new values: no reuse, and the result follows the new survey
        S.z.sub_(1.5)
        sv2 = synth.Survey(sv.x, sv.y, sv.z - 1.5)
        out = torch.full((mesh.ncells,), float("nan"), dtype=torch.float64, device="cuda")
        j = ctx.submit("invert", mesh, S, _dev(d), out, **opts)
        assert ctx.wait(j, 600.0) == g.GRAV_OK
        assert not ctx.job_plan(j)["plan_reused"]
        ref, _ = g.datainv(_dev(d), mesh, S, ctx=solo_ctx, **opts)
        assert torch.equal(out, ref)
        assert ctx.serve_stats()["plans_built"] == 2
        _oracle_check("invert", "fp64", mesh, sv2, _dev(d), out, opts["tol"])
    finally:
        ctx.close()


def test_resident_nystrom_preconditioner(g):
    """Nystrom-preconditioned inversions of three data vectors on one survey
    through one slot: the first job builds the plan and the preconditioner,
    the next two run on both (same lambda from the resident trace, same rank
    and coarsening) with no set-up, and every result equals its one-shot run
    within 1e-9 of max |m| and passes the oracle check."""
    mesh, sv, m = _problem(80, 40, 36, 12, 900, 50.0)
    S = g.Survey(sv.x, sv.y, sv.z)
    d = oracle.forward(mesh, sv, m)
    datas = [d, 0.7 * d, d + synth.random_vector(sv.n, 81, 0.002)]
    opts = dict(precision="mixed", tol=1e-5, max_iter=3000, precond="nystrom")
    solo_ctx = g.context()
    ctx = g.Context(0)
    try:
        ctx.serve_config(1)
        outs, ids = [], []
        for dk in datas:
            out = torch.full((mesh.ncells,), float("nan"), dtype=torch.float64, device="cuda")
            ids.append(ctx.submit("invert", mesh, S, _dev(dk), out, **opts))
            outs.append(out)
        for j in ids:
            assert ctx.wait(j, 600.0) == g.GRAV_OK
        infos = [ctx.poll(j)[1] for j in ids]
        assert [ctx.job_plan(j)["plan_reused"] for j in ids] == [False, True, True]
        assert infos[0]["nys_setup_s"] > 0
        assert all(i["nys_setup_s"] < 0.05 * infos[0]["nys_setup_s"] for i in infos[1:]), infos
        st = ctx.serve_stats()
        assert st["plans_built"] == 1 and st["bytes_resident"] > 0
        for dk, out in zip(datas, outs):
            ref, info = g.datainv(_dev(dk), mesh, S, ctx=solo_ctx, **opts)
            assert info["converged"]
            assert float((out - ref).abs().max()) <= 1e-9 * float(ref.abs().max())
            _oracle_check("invert", "mixed", mesh, sv, _dev(dk), out, opts["tol"])
    finally:
        ctx.close()
