"""CPU checks of the algebra behind the randomized Nystrom preconditioner
(precond = 2; Frangella, Tropp and Udell, SIAM J. Matrix Anal. Appl. 2023).

The library forms K_hat = Y (Omega^T Y)^-1 Y^T from Y = K Omega + nu Omega and
applies (K_hat + mu I)^-1 through the Woodbury identity as
    (r - Y T^-1 Y^T r) / mu,   T = mu Omega^T Y + Y^T Y,
with one Cholesky factor of T.  These tests check, with plain dense linear
algebra, that this expression is the inverse of K_hat + mu I, that K_hat is
exact when K has rank <= ell, and that the preconditioned matrix of a
smooth-kernel system is far better conditioned than the system itself.
"""
import numpy as np


def _woodbury_apply(Y, Om, mu, r):
    T = mu * (Om.T @ Y) + Y.T @ Y
    T = 0.5 * (T + T.T)
    L = np.linalg.cholesky(T)
    t = np.linalg.solve(L.T, np.linalg.solve(L, Y.T @ r))
    return (r - Y @ t) / mu


def _spd(n, rank, decay, rng):
    U, _ = np.linalg.qr(rng.normal(size=(n, rank)))
    return (U * decay ** np.arange(rank)) @ U.T


def test_woodbury_form_inverts_nystrom_plus_shift():
    rng = np.random.default_rng(3)
    n, ell, mu = 300, 40, 1e-3
    K = _spd(n, n, 0.97, rng)
    Om = rng.normal(size=(n, ell)) / np.sqrt(n)
    nu = 1e-9
    Y = K @ Om + nu * Om
    K_hat = Y @ np.linalg.solve(Om.T @ Y, Y.T)
    r = rng.normal(size=n)
    direct = np.linalg.solve(K_hat + mu * np.eye(n), r)
    got = _woodbury_apply(Y, Om, mu, r)
    assert np.linalg.norm(got - direct) <= 1e-8 * np.linalg.norm(direct)


def test_nystrom_exact_for_low_rank():
    rng = np.random.default_rng(4)
    n, rank, ell = 200, 15, 20
    K = _spd(n, rank, 0.8, rng)
    Om = rng.normal(size=(n, ell)) / np.sqrt(n)
    Y = K @ Om
    K_hat = Y @ np.linalg.pinv(Om.T @ Y) @ Y.T
    assert np.linalg.norm(K_hat - K) <= 1e-8 * np.linalg.norm(K)


def test_preconditioned_condition_number():
    rng = np.random.default_rng(5)
    n, ell = 400, 120
    K = _spd(n, n, 0.95, rng)            # eigenvalues decaying like a smooth kernel's
    lam = 1e-2 * np.trace(K) / n
    A = K + lam * np.eye(n)
    Om = rng.normal(size=(n, ell)) / np.sqrt(n)
    nu = np.sqrt(n) * np.finfo(float).eps * np.linalg.norm(K @ Om)
    Y = K @ Om + nu * Om
    mu = lam - nu
    Pinv = np.column_stack([_woodbury_apply(Y, Om, mu, e) for e in np.eye(n)])
    ev_A = np.linalg.eigvalsh(A)
    ev_P = np.sort(np.real(np.linalg.eigvals(Pinv @ A)))
    assert ev_P[0] > 0.0
    assert ev_P[-1] / ev_P[0] < 0.01 * ev_A[-1] / ev_A[0]
