"""Differentiable AMG-DD solve of -div(kappa grad x) = b: the GPU gradient
kernel against the oracle's formula, the whole backward pass against the
oracle's gradient (same AMG-DD solves, so the same x and lam), and central
differences of the loss (h = 1e-6) on random coefficients."""
import numpy as np
import pytest

import amgdd_inputs as I
from oracle import Oracle, kappa_gradient

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1906_10575_gb300 import capi  # noqa: E402
from paper_1906_10575_gb300.adjoint import diffusion_solve  # noqa: E402


def test_kernel_matches_oracle_formula():
    rng = np.random.default_rng(0)
    kappa = I.lognormal_kappa(17, seed=2)[:, :13, :11].copy()
    nz, ny, nx = kappa.shape
    n = kappa.size
    x = rng.standard_normal(n)
    lam = rng.standard_normal(n)
    g = torch.empty(n, dtype=torch.float64, device="cuda")
    capi.amgdd_kappa_grad_3d((nx, ny, nz), torch.from_numpy(kappa).cuda(), torch.from_numpy(x).cuda(),
                             torch.from_numpy(lam).cuda(), g)
    ref = kappa_gradient(kappa, x, lam)
    assert np.allclose(g.cpu().numpy(), ref, rtol=1e-13, atol=1e-15 * abs(ref).max())


def _loss_and_grad(kappa_np, b_np, xt_np, box, tol):
    kappa = torch.from_numpy(kappa_np).cuda().requires_grad_(True)
    b = torch.from_numpy(b_np).cuda().requires_grad_(True)
    xt = torch.from_numpy(xt_np).cuda()
    x = diffusion_solve(kappa, b, box=box, padding=2, tol=tol)
    loss = 0.5 * torch.sum((x - xt) ** 2)
    loss.backward()
    return float(loss.detach()), kappa.grad.cpu().numpy().reshape(-1), b.grad.cpu().numpy(), x.detach().cpu().numpy()


def _loss(kappa_np, b_np, xt_np, box, tol):
    with torch.no_grad():
        kappa = torch.from_numpy(kappa_np).cuda()
        b = torch.from_numpy(b_np).cuda()
        x = diffusion_solve(kappa, b, box=box, padding=2, tol=tol)
        return 0.5 * float(torch.sum((x - torch.from_numpy(xt_np).cuda()) ** 2))


def test_backward_matches_oracle_gradient_32():
    n = 32
    kappa = I.lognormal_kappa(n, seed=5)
    b = I.uniform_rhs(n ** 3, 6)
    xt = I.uniform_rhs(n ** 3, 7)
    _, gk, gb, x = _loss_and_grad(kappa, b, xt, (16, 16, 16), 1e-11)
    rp, ci, v = I.diffusion3d(kappa)
    part, nsub = I.box_partition((n, n, n), (16, 16, 16))
    o = Oracle(rp, ci, v, part, nsub, 2)
    xo, _ = o.amgdd_solve(b, 2, tol=1e-11)
    lo, _ = o.amgdd_solve(xo - xt, 2, tol=1e-11)
    assert np.array_equal(x, xo)
    assert np.array_equal(gb, lo)
    ref = kappa_gradient(kappa, xo, lo)
    assert np.allclose(gk, ref, rtol=1e-12, atol=1e-14 * abs(ref).max())


def test_gradient_matches_central_differences_32_coefficients():
    n = 32
    kappa = I.lognormal_kappa(n, seed=8)
    b = I.uniform_rhs(n ** 3, 9)
    xt = I.uniform_rhs(n ** 3, 10)
    _, gk, gb, _ = _loss_and_grad(kappa, b, xt, (16, 16, 16), 1e-13)
    rng = np.random.default_rng(11)
    idx = rng.choice(n ** 3, size=32, replace=False)
    h = 1e-6
    for m in idx:
        kp = kappa.copy().reshape(-1)
        km = kappa.copy().reshape(-1)
        kp[m] += h
        km[m] -= h
        fd = (_loss(kp.reshape(kappa.shape), b, xt, (16, 16, 16), 1e-13)
              - _loss(km.reshape(kappa.shape), b, xt, (16, 16, 16), 1e-13)) / (2 * h)
        assert abs(fd - gk[m]) <= 1e-5 * abs(gk[m]) + 1e-7 * abs(gk).max(), (m, fd, gk[m])
    # dL/db = lam: one directional difference
    d = np.random.default_rng(12).standard_normal(n ** 3)
    eps = 1e-6
    fdb = (_loss(kappa, b + eps * d, xt, (16, 16, 16), 1e-13)
           - _loss(kappa, b - eps * d, xt, (16, 16, 16), 1e-13)) / (2 * eps)
    assert np.isclose(fdb, gb @ d, rtol=1e-6)


def _refined_loss(s, rp_d, ci_d, v_np, b_d, xt_d, tol):
    """Loss of the solve of a perturbed matrix (same sparsity, values v_np):
    x += AMG-DD correction of b - A' x with the unperturbed handle s (its
    restriction and FAC launch), the residual with A' from the handle-free
    residual entry point, until ||b - A' x|| <= tol ||b||."""
    n = b_d.numel()
    v_d = torch.from_numpy(v_np).cuda()
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    r_all = torch.zeros(int(s.offsets[-1]), dtype=torch.float64, device="cuda")
    nrm = torch.zeros(1, dtype=torch.float64, device="cuda")
    bn = float(torch.linalg.vector_norm(b_d))
    for _ in range(300):
        capi.amgdd_residual_csr_noalloc(n, rp_d, ci_d, v_d, b_d, x, r_all[:n], nrm)
        if float(nrm[0]) ** 0.5 <= tol * bn:
            return 0.5 * float(torch.sum((x - xt_d) ** 2))
        capi.amgdd_restrict(s.h, r_all)
        capi.amgdd_fac(s.h, r_all, x)
    raise AssertionError("refinement did not converge")


def test_lognormal_96_gradient_32_coefficients():
    """96^3 diffusion with kappa = exp(g), g a Gaussian random field (length
    0.1, variance 1), loss 1/2 ||x - x_t||^2, 216 subdomains of 16^3, padding
    2: the GPU gradient equals the oracle's (same solves) on every node, and
    central differences (h = 1e-6) agree on 32 random coefficients. Each
    perturbed loss solves A(kappa +- h e_m) x = b to 1e-13 by refinement
    with the unperturbed AMG-DD hierarchy."""
    from paper_1906_10575_gb300 import Solver
    n = 96
    kappa = I.lognormal_kappa(n, seed=0)
    b = I.uniform_rhs(n ** 3, 1)
    xt = I.uniform_rhs(n ** 3, 2)
    _, gk, gb, x = _loss_and_grad(kappa, b, xt, (16, 16, 16), 1e-12)
    rp, ci, v = I.diffusion3d(kappa)
    part, nsub = I.box_partition((n, n, n), (16, 16, 16))
    o = Oracle(rp, ci, v, part, nsub, 2)
    xo, _ = o.amgdd_solve(b, 2, tol=1e-12)
    lo, _ = o.amgdd_solve(xo - xt, 2, tol=1e-12)
    assert np.array_equal(x, xo) and np.array_equal(gb, lo)
    ref = kappa_gradient(kappa, xo, lo)
    assert np.allclose(gk, ref, rtol=1e-12, atol=1e-14 * abs(ref).max())
    del o
    s = Solver(rp, ci, v, part, nsub, 2, n_fac=2)
    rp_d, ci_d = torch.from_numpy(rp).cuda(), torch.from_numpy(ci).cuda()
    b_d, xt_d = torch.from_numpy(b).cuda(), torch.from_numpy(xt).cuda()
    rng = np.random.default_rng(3)
    for m in rng.choice(n ** 3, size=32, replace=False):
        kp = kappa.copy().reshape(-1)
        km = kappa.copy().reshape(-1)
        kp[m] += 1e-6
        km[m] -= 1e-6
        vp = I.diffusion3d(kp.reshape(kappa.shape))[2]
        vm = I.diffusion3d(km.reshape(kappa.shape))[2]
        fd = (_refined_loss(s, rp_d, ci_d, vp, b_d, xt_d, 1e-13)
              - _refined_loss(s, rp_d, ci_d, vm, b_d, xt_d, 1e-13)) / 2e-6
        assert abs(fd - gk[m]) <= 1e-5 * abs(gk[m]) + 1e-7 * abs(gk).max(), (m, fd, gk[m])
    s.close()
