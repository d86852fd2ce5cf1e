"""GPU test of the device-side failure path, without a GPU fault: a kernel's
bounded mbarrier wait that nothing completes gives up after its limit,
records the timeout in the context's status word and returns; the host reads
GRAV_EDEVICE, clears the word, and the context keeps working."""
import time

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


def test_bounded_wait_expires_and_context_survives(g):
    ctx = g.Context(0)
    try:
        stream = g._stream(None)
        for limit_ms in (20.0, 5.0):
            t0 = time.perf_counter()
            rc = g._lib.grav_selftest_wait(ctx.h, limit_ms, stream)
            dt = time.perf_counter() - t0
            assert rc == g.GRAV_EDEVICE
            assert "bounded device wait expired" in g._lib.grav_last_error(ctx.h).decode()
            assert limit_ms * 1e-3 <= dt < 5.0
        assert g._lib.grav_selftest_wait(ctx.h, 0.0, stream) == g.GRAV_EINVAL
        # the status word was cleared: ordinary work on the same context succeeds
        mesh, sv, m = synth.small_random_problem(6, 5, 4, 40, seed=200)
        d = g.forward(torch.tensor(m, device="cuda"), mesh, g.Survey(sv.x, sv.y, sv.z), ctx=ctx).cpu().numpy()
        ref = oracle.forward(mesh, sv, m)
        assert np.abs(d - ref).max() <= 1e-10 * np.abs(ref).max()
    finally:
        ctx.close()
