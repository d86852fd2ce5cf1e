"""GPU checks of the table-driven FP64 logarithm and arctangent that Eq. 2-3
uses (Tang's table method for log; a one-division table reduction for
atan(a/b)), against long-double references computed on the host (x86 80-bit
logl / atanl through numpy.longdouble).  log: at most one unit in the last
place (CUDA documents 1 ulp for its log).  atan(a/b), where the ratio's own
roundings count too: at most 1.5 ulp and no worse than CUDA's atan applied to
the rounded quotient a/b on the same inputs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_03857_b300 as g
    return g


def _ulp_err(got, ref_ld):
    ref64 = ref_ld.astype(np.float64)
    sp = np.spacing(np.abs(ref64))
    return np.abs(got.astype(np.longdouble) - ref_ld) / sp.astype(np.longdouble)


def _dev(x):
    return torch.as_tensor(np.asarray(x, dtype=np.float64), device="cuda")


def test_longdouble_is_extended():
    assert np.finfo(np.longdouble).nmant >= 63, "needs x86 80-bit long double for the reference"


def test_log64_within_one_ulp(g):
    rng = np.random.Generator(np.random.PCG64(7001))
    x = np.concatenate([
        np.exp(rng.uniform(-690, 690, 400_000)),                          # wide range
        1.0 + rng.uniform(-1e-3, 1e-3, 200_000),                          # near 1 (k = 0, j = 0 or 256)
        1.0 + np.ldexp(rng.uniform(-1, 1, 50_000), -40),
        rng.uniform(0.5, 4.0, 200_000),                                   # k in {-1, 0, 1}
        (1.0 + (np.arange(256) + 0.5) / 256)[None, :].repeat(8, 0).ravel() * np.ldexp(1.0, rng.integers(-20, 20, 2048)),
        np.ldexp(1.0, np.arange(-1021, 1023)),                            # powers of two
        rng.uniform(1.0, 60_000.0, 200_000),                              # the range of R + y in metres
    ])
    got = g.eval_fn64("log", _dev(x)).cpu().numpy()
    ref = np.log(x.astype(np.longdouble))
    err = _ulp_err(got, ref)
    cuda = g.eval_fn64("cuda_log", _dev(x)).cpu().numpy()
    err_cuda = _ulp_err(cuda, ref)
    print(f"log64: max {float(err.max()):.3f} ulp, mean {float(err.mean()):.3f}; CUDA log: max {float(err_cuda.max()):.3f}")
    assert float(err.max()) <= 1.0


def test_log64_special_values_match_cuda(g):
    x = np.array([0.0, -0.0, -1.0, np.inf, np.nan, 5e-324, 1e-310, 2.2250738585072014e-308, 1.0, 2.0])
    got = g.eval_fn64("log", _dev(x)).cpu().numpy()
    cuda = g.eval_fn64("cuda_log", _dev(x)).cpu().numpy()
    assert np.array_equal(got, cuda, equal_nan=True)
    assert got[8] == 0.0


def test_atan_ratio64_within_one_ulp(g):
    rng = np.random.Generator(np.random.PCG64(7002))
    n = 300_000
    b = np.exp(rng.uniform(-20, 20, n))
    a = np.concatenate([
        b[: n // 3] * rng.uniform(-1, 1, n // 3),                          # |a| <= b
        b[n // 3: 2 * n // 3] * np.exp(rng.uniform(0, 30, n // 3)) * rng.choice([-1, 1], n // 3),   # |a| > b
        b[2 * n // 3:] * np.exp(rng.uniform(-30, 30, n - 2 * (n // 3))),   # both regimes, tiny and huge ratios
    ])
    c = (np.arange(65) + 0.5) / 64                                         # reduction boundaries
    a2 = np.concatenate([a, c, -c, 1 / c, np.ones(4), [0.0, 1e-300]])
    b2 = np.concatenate([b, np.ones(65), np.ones(65), np.ones(65), [1.0, 2.0, 3.0, 1e-3], [1.0, 1.0]])
    a2[-6:-2] = b2[-6:-2]                                                  # |a| = b exactly
    got = g.eval_fn64("atan", _dev(a2), _dev(b2)).cpu().numpy()
    ref = np.arctan(a2.astype(np.longdouble) / b2.astype(np.longdouble))
    nz = ref != 0
    err = _ulp_err(got[nz], ref[nz])
    cuda = g.eval_fn64("cuda_atan", _dev(a2), _dev(b2)).cpu().numpy()
    err_cuda = _ulp_err(cuda[nz], ref[nz])
    print(f"atan_ratio64: max {float(err.max()):.3f} ulp, mean {float(err.mean()):.3f}; "
          f"CUDA atan(a/b): max {float(err_cuda.max()):.3f}")
    assert float(err.max()) <= 1.5 and float(err.max()) <= max(1.0, float(err_cuda.max()))
    assert np.all(got[~nz] == 0.0)


def _df_round(x):
    """x rounded to a double-float pair (the inputs the device sees)."""
    h = x.astype(np.float32).astype(np.float64)
    return h + (x - h).astype(np.float32).astype(np.float64)


def test_double_float_log_and_atan(g):
    """The double-float log and atan(a/b) of the near-field set-up (FP32
    pairs on the FP32 pipe) against the long-double reference, over the ranges
    the corner function meets: log within 2^-44 of |result| + 1, atan within
    2^-42 of max(|result|, 2^-9) (the FP32 cubic term of its series)."""
    rng = np.random.Generator(np.random.PCG64(7011))
    x = _df_round(np.exp(rng.uniform(-10, 12, 200_000)))
    got = g.eval_fn64("df_log", _dev(x)).cpu().numpy()
    ref = np.log(x.astype(np.longdouble))
    err = np.abs(got.astype(np.longdouble) - ref) / (np.abs(ref) + 1)
    assert float(err.max()) <= 2.0 ** -44
    a = _df_round(rng.normal(0, 1, 200_000) * np.exp(rng.uniform(-8, 8, 200_000)))
    b = _df_round(np.exp(rng.uniform(-8, 8, 200_000)))
    got = g.eval_fn64("df_atan", _dev(a), _dev(b)).cpu().numpy()
    ref = np.arctan(a.astype(np.longdouble) / b.astype(np.longdouble))
    err = np.abs(got.astype(np.longdouble) - ref) / np.maximum(np.abs(ref), 2.0 ** -9)
    assert float(err.max()) <= 2.0 ** -42


def test_double_float_corner_function_against_oracle(g):
    """Psi of Eq. 2-3 in double-float against the FP64 oracle at vertex
    offsets from 0.1 m to 30 km (x, y of either sign and exactly 0, z > 0):
    within 2^-42 of R (|ln R| + 1), the scale of the cancellation the
    near-field table's 8-corner differences face (they need ~2^-39)."""
    import oracle
    rng = np.random.Generator(np.random.PCG64(7012))
    n = 20_000
    s = 10.0 ** rng.uniform(-1, 4.5, n)
    x = s * rng.uniform(-1, 1, n)
    y = s * rng.uniform(-1, 1, n)
    z = s * rng.uniform(0.001, 1, n)
    x[::17] = 0.0
    y[::19] = 0.0
    x, y, z = _df_round(x), _df_round(y), _df_round(z)
    got = g.eval_fn64("df_psi", _dev(np.concatenate([x, z])), _dev(y)).cpu().numpy()
    ref = np.array([oracle.psi(float(a), float(b), float(c)) for a, b, c in zip(x, y, z)])
    R = np.sqrt(x * x + y * y + z * z)
    err = np.abs(got - ref) / (R * (np.abs(np.log(R)) + 1))
    assert err.max() <= 2.0 ** -42, err.max()
