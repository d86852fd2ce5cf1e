"""GPU tests of the differentiable forward operator: torch.autograd through
GravForward, whose backward is the hand-written adjoint kernel.

* torch.autograd.gradcheck (finite differences of the FP64 forward against the
  backward) on a tiny mesh;
* backward against the oracle's explicit G^T (FP64, 1e-10 of max);
* at paper scale (210 x 210 x 75 cells, 178,797 stations, mixed precision):
  the central finite difference of f(m) = <w, G m> along a random direction v
  equals <G^T w, v> from backward (f is linear, so the difference quotient is
  exact up to rounding; FP32 far-field rounding sets the 1e-6 tolerance).
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


def test_gradcheck_tiny_fp64(g):
    mesh, sv, m = synth.small_random_problem(3, 4, 2, 7, seed=91, irregular=True)
    plan = g.Plan(mesh, g.Survey(sv.x, sv.y, sv.z))
    mt = torch.tensor(m, dtype=torch.float64, device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(lambda x: g.gravity(x, plan), (mt,), eps=1e-3, atol=1e-12, rtol=1e-7)
    plan.close()


def test_backward_equals_oracle_transpose(g):
    mesh, sv, m = synth.small_random_problem(9, 8, 6, 120, seed=92)
    plan = g.Plan(mesh, g.Survey(sv.x, sv.y, sv.z))
    w = synth.random_vector(sv.n, 93)
    mt = torch.tensor(m, dtype=torch.float64, device="cuda", requires_grad=True)
    (g.gravity(mt, plan) * torch.tensor(w, device="cuda")).sum().backward()
    ref = oracle.G_explicit(mesh, sv).T @ w
    got = mt.grad.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()
    plan.close()


def test_directional_fd_paper_scale_mixed(g):
    wl = synth.make_workload("paper_210x210x75")
    plan = g.Plan(wl.mesh, g.Survey(wl.survey.x, wl.survey.y, wl.survey.z), precision="mixed")
    m = torch.tensor(wl.m, dtype=torch.float64, device="cuda", requires_grad=True)
    w = torch.tensor(synth.random_vector(wl.survey.n, 94), device="cuda")
    (g.gravity(m, plan) * w).sum().backward()
    v = torch.tensor(synth.random_vector(wl.mesh.ncells, 95, 10.0), device="cuda")
    h = 1.0
    with torch.no_grad():
        fp = torch.dot(w, plan.forward(m + h * v))
        fm = torch.dot(w, plan.forward(m - h * v))
        fd = float((fp - fm) / (2 * h))
        ad = float(torch.dot(m.grad, v))
        scale = float(torch.linalg.norm(plan.forward(v)) * torch.linalg.norm(w))
    assert abs(fd - ad) <= 1e-6 * scale, (fd, ad, scale)
    plan.close()
