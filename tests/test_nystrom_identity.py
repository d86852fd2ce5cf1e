"""CPU checks of the algebra behind the randomized Nystrom preconditioner
(precond = 2; Frangella, Tropp and Udell, SIAM J. Matrix Anal. Appl. 2023).

The library sketches K = B B^T (B the explicit, depth-weighted coarse
operator) with a Gaussian Omega: Z = B^T Omega, Y = B Z = K Omega, and takes
the Nystrom approximation in its Gram form
    K_hat = Y (M + nu I)^-1 Y^T,   M = Z^T Z  (= Omega^T K Omega),
applying (K_hat + lambda I)^-1 through the Woodbury identity as
    (r - Y T^-1 Y^T r) / lambda,   T = lambda (M + nu I) + Y^T Y,
with one Cholesky factor of T.  These tests check, with plain dense linear
algebra, that the Gram form is the published Nystrom approximation, that the
Woodbury expression is the inverse of K_hat + lambda I, that K_hat is exact
when K has rank <= ell, that T stays positive definite with FP32 sketch
products even when ell is a large share of N (where the published
Omega^T Y form loses definiteness), and that the preconditioned matrix of a
smooth-kernel system is far better conditioned than the system itself.
"""
import numpy as np


def _woodbury_apply(Y, M, lam, nu, r):
    T = lam * (M + nu * np.eye(M.shape[0])) + Y.T @ Y
    T = 0.5 * (T + T.T)
    L = np.linalg.cholesky(T)
    t = np.linalg.solve(L.T, np.linalg.solve(L, Y.T @ r))
    return (r - Y @ t) / lam


def _smooth_B(n, m, rng):
    """Point-mass kernel dz / R^3 of m buried cells at n surface stations,
    depth-weighted: a smooth operator with fast spectral decay."""
    cx, cy = rng.uniform(0, 1000, m), rng.uniform(0, 1000, m)
    cz = rng.uniform(50, 400, m)
    sx, sy = rng.uniform(0, 1000, n), rng.uniform(0, 1000, n)
    dx, dy, dz = cx[None] - sx[:, None], cy[None] - sy[:, None], cz[None] + 0.0 * sx[:, None]
    return dz / (dx * dx + dy * dy + dz * dz) ** 1.5 * 1e6 * (cz + 50.0)[None]


def _spd(n, rank, decay, rng):
    U, _ = np.linalg.qr(rng.normal(size=(n, rank)))
    return (U * decay ** np.arange(rank)) @ U.T


def test_gram_form_is_published_nystrom():
    rng = np.random.default_rng(2)
    n, m, ell = 250, 180, 30
    B = _smooth_B(n, m, rng)
    K = B @ B.T
    Om = rng.normal(size=(n, ell)) / np.sqrt(n)
    Z = B.T @ Om
    Y = B @ Z
    published = (K @ Om) @ np.linalg.solve(Om.T @ K @ Om, (K @ Om).T)
    gram = Y @ np.linalg.solve(Z.T @ Z, Y.T)
    assert np.linalg.norm(gram - published) <= 1e-8 * np.linalg.norm(published)
    # and it never exceeds K (K - K_hat = B (I - P_Z) B^T is PSD)
    assert np.linalg.eigvalsh(K - gram).min() >= -1e-9 * np.linalg.norm(K, 2)


def test_woodbury_form_inverts_nystrom_plus_shift():
    rng = np.random.default_rng(3)
    n, m, ell, lam, nu = 300, 200, 40, 1e-3, 1e-6
    B = _smooth_B(n, m, rng)
    B /= np.linalg.norm(B, 2)
    Om = rng.normal(size=(n, ell)) / np.sqrt(n)
    Z = B.T @ Om
    Y = B @ Z
    M = Z.T @ Z
    K_hat = Y @ np.linalg.solve(M + nu * np.eye(ell), Y.T)
    r = rng.normal(size=n)
    direct = np.linalg.solve(K_hat + lam * np.eye(n), r)
    got = _woodbury_apply(Y, M, lam, nu, r)
    assert np.linalg.norm(got - direct) <= 1e-8 * np.linalg.norm(direct)


def test_nystrom_exact_for_low_rank():
    rng = np.random.default_rng(4)
    n, rank, ell = 200, 15, 20
    K = _spd(n, rank, 0.8, rng)
    Om = rng.normal(size=(n, ell)) / np.sqrt(n)
    Y = K @ Om
    K_hat = Y @ np.linalg.pinv(Om.T @ Y) @ Y.T
    assert np.linalg.norm(K_hat - K) <= 1e-8 * np.linalg.norm(K)


def test_gram_form_stays_definite_with_fp32_products():
    """ell close to N: the sketch reaches eigenvalues far below the FP32
    rounding of the products.  T from the Gram form with nu = 1e-3 lambda
    factors; the published form's Omega^T Y (rounded products, Frangella's
    shift nu = sqrt(N) eps ||Y||_F) does not."""
    rng = np.random.default_rng(6)
    n, m, ell = 400, 600, 300
    B = _smooth_B(n, m, rng)
    K = B @ B.T
    lam = 1e-2 * np.trace(K) / n
    Om32 = (rng.normal(size=(n, ell)) / np.sqrt(n)).astype(np.float32)
    B32 = B.astype(np.float32)
    Z32 = B32.T @ Om32
    Y = (B32 @ Z32).astype(np.float64)
    M = Z32.astype(np.float64).T @ Z32.astype(np.float64)
    T = lam * (M + 1e-3 * lam * np.eye(ell)) + Y.T @ Y
    np.linalg.cholesky(0.5 * (T + T.T))          # raises if not positive definite
    Om = Om32.astype(np.float64)
    nu = np.sqrt(n) * np.finfo(float).eps * np.linalg.norm(Y)
    Yn = Y + nu * Om
    assert np.linalg.eigvalsh(0.5 * (Om.T @ Yn + Yn.T @ Om)).min() < 0.0


def test_preconditioned_condition_number():
    rng = np.random.default_rng(5)
    n, m, ell = 400, 500, 120
    B = _smooth_B(n, m, rng)
    K = B @ B.T
    lam = 1e-2 * np.trace(K) / n
    A = K + lam * np.eye(n)
    Om = rng.normal(size=(n, ell)) / np.sqrt(n)
    Z = B.T @ Om
    Y = B @ Z
    M = Z.T @ Z
    Pinv = np.column_stack([_woodbury_apply(Y, M, lam, 1e-3 * lam, e) for e in np.eye(n)])
    ev_A = np.linalg.eigvalsh(A)
    ev_P = np.sort(np.real(np.linalg.eigvals(Pinv @ A)))
    assert ev_P[0] > 0.0
    assert ev_P[-1] / ev_P[0] < 0.01 * ev_A[-1] / ev_A[0]
