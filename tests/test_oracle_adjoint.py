"""Pin of the oracle's coefficient gradient: central differences of the loss
through dense direct solves, on a grid small enough to perturb every
coefficient."""
import numpy as np
import scipy.sparse as sp

import amgdd_inputs as I
from oracle import kappa_gradient


def _solve(kappa, b):
    rp, ci, v = I.diffusion3d(kappa)
    A = sp.csr_matrix((v, ci, rp)).toarray()
    return np.linalg.solve(A, b), A


def test_gradient_matches_central_differences_everywhere():
    rng = np.random.default_rng(3)
    kappa = np.exp(rng.standard_normal((3, 4, 5)))
    n = kappa.size
    b = rng.uniform(-1, 1, n)
    xt = rng.uniform(-1, 1, n)
    x, A = _solve(kappa, b)
    lam = np.linalg.solve(A, x - xt)            # A symmetric
    g = kappa_gradient(kappa, x, lam)
    h = 1e-6
    fd = np.zeros(n)
    for m in range(n):
        kp = kappa.copy().reshape(-1)
        km = kappa.copy().reshape(-1)
        kp[m] += h
        km[m] -= h
        xp, _ = _solve(kp.reshape(kappa.shape), b)
        xm, _ = _solve(km.reshape(kappa.shape), b)
        fd[m] = (0.5 * np.sum((xp - xt) ** 2) - 0.5 * np.sum((xm - xt) ** 2)) / (2 * h)
    assert np.allclose(g, fd, rtol=1e-6, atol=1e-9 * abs(fd).max())


def test_gradient_is_minus_lambda_dA_x():
    """Against the definition: -lam^T (dA/dk_m) x with dA/dk_m by differencing
    the assembled matrix (exact up to rounding for this linear-fractional
    coefficient at small steps)."""
    rng = np.random.default_rng(4)
    kappa = np.exp(rng.standard_normal((2, 3, 3)))
    n = kappa.size
    x = rng.standard_normal(n)
    lam = rng.standard_normal(n)
    g = kappa_gradient(kappa, x, lam)
    for m in range(n):
        h = 1e-5 * kappa.reshape(-1)[m]
        kp = kappa.copy().reshape(-1)
        km = kappa.copy().reshape(-1)
        kp[m] += h
        km[m] -= h
        Ap = sp.csr_matrix((lambda r: (r[2], r[1], r[0]))(I.diffusion3d(kp.reshape(kappa.shape))))
        Am = sp.csr_matrix((lambda r: (r[2], r[1], r[0]))(I.diffusion3d(km.reshape(kappa.shape))))
        dA = (Ap - Am) / (2 * h)
        assert np.isclose(g[m], -(lam @ (dA @ x)), rtol=1e-7, atol=1e-12)
