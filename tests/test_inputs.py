"""Pins of the synthetic problem generators (shared by oracle and library)."""
import numpy as np
import scipy.sparse as sp

import amgdd_inputs as I


def _mat(rp, ci, v):
    return sp.csr_matrix((v, ci, rp))


def test_poisson_sizes_and_exact_symmetry():
    rp, ci, v = I.poisson2d(64, 64)
    assert len(rp) - 1 == 4096 and len(ci) == 20224
    rp, ci, v = I.poisson3d(12, 10, 8)
    A = _mat(rp, ci, v)
    assert (A - A.T).count_nonzero() == 0
    for i in range(A.shape[0]):  # ascending unique columns
        row = ci[rp[i]:rp[i + 1]]
        assert np.all(np.diff(row) > 0)


def test_dirichlet_laplacian_eigenpairs_2d():
    # lambda_ij = 4 - 2cos(i pi/(n+1)) - 2cos(j pi/(m+1)), v = sin (x) sin
    nx, ny = 9, 7
    A = _mat(*I.poisson2d(nx, ny))
    for (a, b) in [(1, 1), (2, 3), (9, 7), (5, 1)]:
        x = np.sin(a * np.pi * np.arange(1, nx + 1) / (nx + 1))
        y = np.sin(b * np.pi * np.arange(1, ny + 1) / (ny + 1))
        vec = np.outer(y, x).reshape(-1)  # idx = i + nx*j
        lam = 4 - 2 * np.cos(a * np.pi / (nx + 1)) - 2 * np.cos(b * np.pi / (ny + 1))
        assert np.allclose(A @ vec, lam * vec, rtol=0, atol=1e-13)


def test_dirichlet_laplacian_eigenpairs_3d():
    nx, ny, nz = 6, 5, 4
    A = _mat(*I.poisson3d(nx, ny, nz))
    for (a, b, c) in [(1, 1, 1), (2, 5, 3), (6, 1, 4)]:
        x = np.sin(a * np.pi * np.arange(1, nx + 1) / (nx + 1))
        y = np.sin(b * np.pi * np.arange(1, ny + 1) / (ny + 1))
        z = np.sin(c * np.pi * np.arange(1, nz + 1) / (nz + 1))
        vec = np.einsum("k,j,i->kji", z, y, x).reshape(-1)
        lam = (6 - 2 * np.cos(a * np.pi / (nx + 1)) - 2 * np.cos(b * np.pi / (ny + 1))
               - 2 * np.cos(c * np.pi / (nz + 1)))
        assert np.allclose(A @ vec, lam * vec, rtol=0, atol=1e-13)


def test_variable_coefficient_reduces_and_harmonic_mean():
    k = np.full((3, 4, 5), 2.5)
    A = _mat(*I.diffusion3d(k))
    B = _mat(*I.poisson3d(5, 4, 3))
    assert abs(A - 2.5 * B).max() < 1e-14
    k = np.ones((1, 1, 2))
    k[0, 0, 1] = 3.0
    A = _mat(*I.diffusion3d(k)).toarray()
    h = 2 * 1 * 3 / 4.0
    assert np.isclose(A[0, 1], -h) and np.isclose(A[1, 0], -h)
    assert np.isclose(A[0, 0], 5 * 1.0 + h) and np.isclose(A[1, 1], 5 * 3.0 + h)


def test_box_partition_and_rhs_seed():
    part, nsub = I.box_partition((64, 64), (16, 16))
    assert nsub == 16 and np.all(np.bincount(part) == 256)
    assert part[0] == 0 and part[16] == 1 and part[64 * 16] == 4
    part3, ns3 = I.box_partition((32, 32, 32), (16, 16, 16))
    assert ns3 == 8 and part3[32 * 32 * 16] == 4
    b0 = I.uniform_rhs(1000, 0)
    assert np.array_equal(b0, np.random.default_rng(0).uniform(-1, 1, 1000))
    assert b0.min() >= -1 and b0.max() <= 1


def test_batched_poisson_is_block_diagonal():
    """The batch is the direct sum of the single-system Poisson matrices, each
    partitioned into its own boxes (uneven at the far ends), in draw order."""
    rp, ci, v, part, nsub, B, picks, offs = I.batched_poisson(5, edges=(8, 12, 20), box=8, nrhs=4, seed=11)
    assert len(picks) == 5 and set(picks) <= {8, 12, 20}
    assert B.shape == (offs[-1], 4) and np.all(np.abs(B) <= 1.0)
    sub0 = 0
    for k, e in enumerate(picks):
        a, b = offs[k], offs[k + 1]
        assert b - a == e ** 3
        r1, c1, v1 = I.poisson3d(e, e, e)
        blk = rp[a:b + 1] - rp[a]
        assert np.array_equal(blk, r1)
        assert np.array_equal(ci[rp[a]:rp[b]] - a, c1) and np.array_equal(v[rp[a]:rp[b]], v1)
        p1, n1 = I.box_partition((e, e, e), (8, 8, 8))
        assert np.array_equal(part[a:b] - sub0, p1)
        sub0 += n1
    assert nsub == sub0 == part.max() + 1
    again = I.batched_poisson(5, edges=(8, 12, 20), box=8, nrhs=4, seed=11)
    assert np.array_equal(again[5], B) and again[6] == picks


def test_rotated_anisotropic_stencil():
    """9-point stencil of -div(K grad u), K = Q diag(1, eps) Q^T: symmetric,
    positive definite, interior rows sum to zero; theta = 0, eps = 1 is the
    5-point Laplacian (the mixed-derivative entries vanish); the stencil of an
    interior node carries the rotated tensor's entries."""
    import scipy.sparse as sp
    th, eps = 3 * np.pi / 16, 1e-3
    rp, ci, v = I.rotated_anisotropic2d(11, 9, th, eps)
    A = sp.csr_matrix((v, ci, rp)).toarray()
    assert np.array_equal(A, A.T) and np.linalg.eigvalsh(A).min() > 0
    c, s = np.cos(th), np.sin(th)
    K = np.array([[c, -s], [s, c]]) @ np.diag([1.0, eps]) @ np.array([[c, s], [-s, c]])
    i = 4 * 11 + 5                        # interior node (x = 5, y = 4)
    row = {j - i: A[i, j] for j in np.nonzero(A[i])[0]}
    assert np.isclose(row[0], 2 * K[0, 0] + 2 * K[1, 1]) and abs(sum(row.values())) < 1e-14
    assert np.isclose(row[1], -K[0, 0]) and np.isclose(row[-1], -K[0, 0])
    assert np.isclose(row[11], -K[1, 1]) and np.isclose(row[-11], -K[1, 1])
    assert np.isclose(row[12], -K[0, 1] / 2) and np.isclose(row[-12], -K[0, 1] / 2)
    assert np.isclose(row[10], K[0, 1] / 2) and np.isclose(row[-10], K[0, 1] / 2)
    rp0, ci0, v0 = I.rotated_anisotropic2d(7, 5, 0.0, 1.0)
    A0 = sp.csr_matrix((v0, ci0, rp0)).toarray()
    r5, c5, v5 = I.poisson2d(7, 5)
    assert np.array_equal(A0, sp.csr_matrix((v5, c5, r5)).toarray())
