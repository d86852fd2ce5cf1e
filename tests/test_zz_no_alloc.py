"""GPU test of grav_forward_fp64_noalloc, the forward product for callers that
cannot allocate device memory (the library keeps its scratch in a static
device array instead).

It calls the entry point through the C ABI and compares its output with the
regular grav_forward (FP64) on two calls in a row with different problems,
within the FP64 parity tolerance (1e-10 of max |d|), and checks that a
problem larger than the static scratch is rejected with GRAV_EINVAL.  This
file is collected last so that a failure here leaves every other test run.
"""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-10


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_03857_b300 as g
    f = g._lib.grav_forward_fp64_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.POINTER(g.grav_mesh), ctypes.POINTER(g.grav_survey), ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p]
    return g


def _noalloc(g, mesh, S, m):
    d = torch.full((S.n,), float("nan"), dtype=torch.float64, device="cuda")
    M = g.Mesh.of(mesh)
    rc = g._lib.grav_forward_fp64_noalloc(ctypes.byref(M.c), ctypes.byref(S.c), m.data_ptr(), d.data_ptr(),
                                          g._stream(None))
    assert rc == g.GRAV_OK, g._lib.grav_last_error(None).decode()
    torch.cuda.synchronize()
    return d


def test_noalloc_matches_grav_forward_twice(g):
    problems = [synth.small_random_problem(23, 17, 9, 700, seed=81, irregular=True),
                synth.small_random_problem(40, 31, 12, 1500, seed=82)]
    for mesh, sv, m in problems:
        S = g.Survey(sv.x, sv.y, sv.z)
        mt = torch.tensor(m, dtype=torch.float64, device="cuda")
        ref = g.forward(mt, mesh, S).cpu().numpy()
        got = _noalloc(g, mesh, S, mt).cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.abs(got - ref).max() <= TOL64 * np.abs(ref).max()


def test_noalloc_rejects_oversized_problem(g):
    mesh = synth.uniform_mesh(1000, 1000, 10, 10.0, 10.0, 10.0)     # node weights alone: ~84 MiB > 64 MiB
    sv = synth.Survey(np.array([5.0]), np.array([5.0]), np.array([-1.0]))
    S = g.Survey(sv.x, sv.y, sv.z)
    m = torch.zeros(16, dtype=torch.float64, device="cuda")        # never read: rejected before any launch
    d = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = g._lib.grav_forward_fp64_noalloc(ctypes.byref(g.Mesh.of(mesh).c), ctypes.byref(S.c), m.data_ptr(),
                                          d.data_ptr(), g._stream(None))
    assert rc == g.GRAV_EINVAL
    assert "static scratch" in g._lib.grav_last_error(None).decode()
