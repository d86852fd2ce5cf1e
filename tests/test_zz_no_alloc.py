"""GPU tests of grav_forward_fp64_noalloc, the forward product for callers that
cannot allocate device memory while they run (a framework whose allocator owns
all device memory, a fixed pre-reserved budget, code that cannot take the
synchronisation an allocation may cause).  The library keeps that entry
point's scratch in a static device array instead.

Every call goes through the C ABI.  Two calls in a row on different problems
are compared with the CPU oracle (every station) and with the regular
grav_forward in FP64, within the FP64 parity tolerance (1e-10 of max |d|).
A third problem is sized so that the static array cannot hold the partial
sums of as many chunks as the kernel would use to fill the GPU, so the
capped chunk count is the one that runs; it is checked against the oracle
on sampled stations and against grav_forward on every station.  Problems
beyond the array, the cell and node caps and the shared-memory row limit are
rejected before anything is enqueued.  This file is collected last so that
a failure here leaves every other test run.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-10
SCRATCH_DOUBLES = (64 << 20) // 8      # the documented 64 MiB static array
STATIONS_PER_CTA = 256                 # k_fwd64: 128 threads x 2 stations


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


def _call(g, mesh, S, m, d):
    return g._lib.grav_forward_fp64_noalloc(ctypes.byref(g.Mesh.of(mesh).c), ctypes.byref(S.c), m.data_ptr(),
                                            d.data_ptr(), g._stream(None))


def _noalloc(g, mesh, S, m):
    d = torch.full((S.n,), float("nan"), dtype=torch.float64, device="cuda")
    rc = _call(g, mesh, S, m, d)
    assert rc == g.GRAV_OK, g._lib.grav_last_error(None).decode()
    torch.cuda.synchronize()
    return d.cpu().numpy()


def test_noalloc_matches_oracle_twice(g):
    problems = [synth.small_random_problem(23, 17, 9, 700, seed=81, irregular=True),
                synth.small_random_problem(40, 31, 12, 1500, seed=82)]
    for mesh, sv, m in problems:
        S = g.Survey(sv.x, sv.y, sv.z)
        mt = torch.tensor(m, dtype=torch.float64, device="cuda")
        got = _noalloc(g, mesh, S, mt)
        ref = oracle.forward(mesh, sv, m)
        assert np.all(np.isfinite(got))
        assert np.abs(got - ref).max() <= TOL64 * np.abs(ref).max()
        lib = g.forward(mt, mesh, S).cpu().numpy()
        assert np.abs(got - lib).max() <= TOL64 * np.abs(ref).max()


def test_noalloc_scratch_capped_chunks(g):
    """200 x 200 x 180 cells: the node weights take 56 MiB of the 64 MiB array,
    leaving room for ~519 chunk rows of 2,000 partials while 740 chunks would
    fill the GPU; the call runs with the capped count."""
    nx, ny, nz, n = 200, 200, 180, 2000
    ldw = (nx + 2) // 2 * 2
    w_doubles = (ny + 1) * (nz + 1) * ldw
    tiles = -(-n // STATIONS_PER_CTA)
    wanted = -(-(148 * 40) // tiles)
    room = (SCRATCH_DOUBLES - w_doubles) // n
    assert room < wanted and room >= 1            # the cap binds (on a 148-SM B300)
    mesh = synth.uniform_mesh(nx, ny, nz, 25.0, 25.0, 25.0)
    rng = np.random.Generator(np.random.PCG64(83))
    sv = synth.Survey(rng.uniform(-200, 5200, n), rng.uniform(-200, 5200, n), -rng.uniform(1, 40, n))
    # a body in a noisy background, as in the paper's synthetics: a zero-mean
    # white-noise model over 7.2M cells cancels to max |d| ~ 0.04 mGal, below
    # which both FP64 evaluations (per prism and per node) carry ~2e-11 mGal
    # of rounding from their far-field terms
    m = rng.normal(0.0, 20.0, (nz, ny, nx))
    m[10:50, 80:120, 80:120] += 400.0
    m = m.ravel()
    S = g.Survey(sv.x, sv.y, sv.z)
    mt = torch.tensor(m, dtype=torch.float64, device="cuda")
    got = _noalloc(g, mesh, S, mt)
    assert np.all(np.isfinite(got))
    lib = g.forward(mt, mesh, S).cpu().numpy()
    scale = np.abs(lib).max()
    assert np.abs(got - lib).max() <= TOL64 * scale
    pick = np.linspace(0, n - 1, 6).astype(int)
    sub = synth.Survey(sv.x[pick].copy(), sv.y[pick].copy(), sv.z[pick].copy())
    ref = oracle.forward(mesh, sub, m)
    assert np.abs(got[pick] - ref).max() <= TOL64 * np.abs(ref).max()


def _rejected(g, mesh, what):
    sv = synth.Survey(np.array([5.0]), np.array([5.0]), np.array([-1.0]))
    S = g.Survey(sv.x, sv.y, sv.z)
    m = torch.zeros(16, dtype=torch.float64, device="cuda")        # never read: rejected before any launch
    d = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert _call(g, mesh, S, m, d) == g.GRAV_EINVAL
    assert what in g._lib.grav_last_error(None).decode()


def test_noalloc_rejects_oversized_problems(g):
    _rejected(g, synth.uniform_mesh(1000, 1000, 10, 10.0, 10.0, 10.0), "static scratch")   # ~84 MiB of weights
    # (ny+1)(nz+1) overflows a 32-bit int: must be caught by the node cap, not wrap
    _rejected(g, synth.uniform_mesh(1, 1 << 20, 4096, 10.0, 10.0, 10.0), "2^30 nodes")
    # one row of node weights beyond the kernel's shared-memory stage
    _rejected(g, synth.uniform_mesh(9000, 1, 1, 10.0, 10.0, 10.0), "nx+1 must be <=")
