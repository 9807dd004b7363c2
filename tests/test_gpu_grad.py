"""Differentiation through x = A^{-1} b on the GPU: the autograd Function,
the adjoint solve and the link-force / dkappa kernels, against the oracle's
gradient and central finite differences (h = 1e-6).  Bar: 1e-6 relative.

A finite difference of two independent solves would carry the solvers'
error divided by h (1e-13 * cond / 1e-6 ~ 1e-5 here), so the perturbed
solutions are computed as corrections: x_+- = x + A_+-^{-1} (b - A_+- x),
whose right-hand side is O(h); the difference quotient is then accurate to
the correction solve's relative tolerance."""
import numpy as np
import pytest

from inputs import lattice as L
from oracle import dirac, grad, krylov

from .gpu_util import cuda, host, kappa_c_table

pytestmark = pytest.mark.gpu

TOL = 1e-13


@pytest.fixture(scope="module")
def wdl():
    import paper_0710_1988_gb300 as wdl
    wdl.lib()
    return wdl


def _oracle_grads(U, dims, kappa, b, eta, mu=0.0):
    v = U.shape[0]
    A = lambda x: dirac.apply_A(U, x.reshape(v, 4, 3), dims, kappa, mu).ravel()
    Ad = lambda x: dirac.apply_A_dagger(U, x.reshape(v, 4, 3), dims, kappa, mu).ravel()
    solve = lambda r: krylov.bicgstab(A, r, tol=1e-14, max_iter=20000)[0]
    solve_d = lambda r: krylov.bicgstab(Ad, r, tol=1e-14, max_iter=20000)[0]
    return grad.gradients(U, dims, kappa, b, eta, solve, solve_d, mu)


@pytest.mark.parametrize("mu", [0.0, 0.05])
def test_gradients_match_oracle(wdl, mu):
    import torch
    dims = (4, 4, 4, 8)
    U = L.gauge_field(dims, 0.5, 5000)
    kappa = 0.13
    b = L.gaussian_spinor(dims, 5001).ravel()
    eta = L.gaussian_spinor(dims, 5002).ravel()
    Lo, lam_o, dk_o, f_o = _oracle_grads(U, dims, kappa, b, eta, mu)
    op = wdl.WilsonOperator(dims, cuda(U), kappa, mu)
    x = torch.zeros(b.size, dtype=torch.complex128, device="cuda:0")
    op.dbicgstab(cuda(b), x, None, tol=TOL)
    lam = torch.zeros_like(x)
    op.adjoint_solve(cuda(eta), lam, None, tol=TOL)
    f = torch.empty((L.volume(dims), 4, 8), dtype=torch.float64, device="cuda:0")
    dk = op.gradients(lam, x, force=f)
    lam_h = host(lam)
    assert np.linalg.norm(lam_h - lam_o) <= 1e-9 * np.linalg.norm(lam_o)
    assert abs(dk - dk_o) <= 1e-8 * abs(dk_o)
    fh = host(f)
    assert np.linalg.norm(fh - f_o) <= 1e-8 * np.linalg.norm(f_o)
    op.close()


def test_autograd_against_finite_differences(wdl):
    import torch
    from paper_0710_1988_gb300.autograd import wilson_solve
    cfg = L.CONFIGS["grad_8x8x8x16"]
    dims = cfg.dims
    kappa = cfg.kappa_factor * kappa_c_table()[cfg.name]["kappa_c"]
    U = L.gauge_field(dims, cfg.eps, L.link_seed(cfg))
    v = L.volume(dims)
    b_h = L.gaussian_spinor(dims, 5101).ravel()
    eta = cuda(L.gaussian_spinor(dims, 5102).ravel())
    op = wdl.WilsonOperator(dims, cuda(U), kappa)

    b = cuda(b_h).requires_grad_(True)
    kap = torch.tensor(kappa, dtype=torch.float64, requires_grad=True)
    om = torch.zeros((v, 4, 8), dtype=torch.float64, device="cuda:0", requires_grad=True)
    x = wilson_solve(b, kap, om, op, None, TOL, 100000)
    loss = torch.real(torch.vdot(eta, x))
    loss.backward()

    xb = x.detach()
    tmp = torch.empty_like(xb)

    def correction(op_):
        # L at the perturbed operator: x + A_^{-1} (b - A_ x)
        op_.apply(xb, tmp)
        r = b.detach() - tmp
        d = torch.zeros_like(r)
        rc, st = op_.dbicgstab(r, d, None, tol=1e-10)
        assert rc == 0
        return torch.real(torch.vdot(eta, d)).item()

    h = 1e-6
    rng = np.random.Generator(np.random.PCG64(5103))
    # b: L is linear in b, so the difference quotient is Re eta^dagger A^{-1} d
    d = cuda(L.gaussian_spinor(dims, 5104).ravel())
    z = torch.zeros_like(d)
    op.dbicgstab(d, z, None, tol=TOL)
    fd = torch.real(torch.vdot(eta, z)).item()
    an = torch.real(torch.vdot(b.grad, d)).item()
    assert abs(fd - an) <= 1e-6 * abs(fd)
    # kappa
    op.set_params(kappa + h)
    lp = correction(op)
    op.set_params(kappa - h)
    lm = correction(op)
    op.set_params(kappa)
    fd = (lp - lm) / (2 * h)
    assert abs(fd - kap.grad.item()) <= 1e-6 * abs(fd)
    # link Lie-algebra parameters along a random direction
    omega = rng.standard_normal((v, 4, 8))
    opp = wdl.WilsonOperator(dims, cuda(L.move_links(U, omega, h)), kappa)
    opm = wdl.WilsonOperator(dims, cuda(L.move_links(U, omega, -h)), kappa)
    fd = (correction(opp) - correction(opm)) / (2 * h)
    an = float(np.sum(host(om.grad) * omega))
    assert abs(fd - an) <= 1e-6 * abs(fd)
    for o in (op, opp, opm):
        o.close()


def test_adjoint_solve_uses_the_deflation_space(wdl):
    import torch
    cfg = L.CONFIGS["wilson_4x4x4x4"]
    kappa = cfg.kappa_factor * kappa_c_table()[cfg.name]["kappa_c"]
    U = L.gauge_field(cfg.dims, cfg.eps, L.link_seed(cfg))
    op = wdl.WilsonOperator(cfg.dims, cuda(U), kappa)
    n = 12 * L.volume(cfg.dims)
    V = torch.zeros(cfg.k * n, dtype=torch.complex128, device="cuda:0")
    b0 = cuda(L.source(cfg, 0))
    op.gmresdr(b0, torch.zeros_like(b0), cfg.m, cfg.k, 1e-12, 100000, V_out=V)
    defl = op.deflation(V, cfg.k)
    g = cuda(L.gaussian_spinor(cfg.dims, 5200).ravel())
    lam = torch.zeros_like(g)
    rc, st = op.adjoint_solve(g, lam, defl, tol=1e-10)
    assert rc == 0 and st[0]["converged"]
    # A^dagger lam = g, checked with the oracle's adjoint operator
    r = host(g) - dirac.apply_A_dagger(U, host(lam).reshape(-1, 4, 3), cfg.dims, kappa).ravel()
    assert np.linalg.norm(r) <= 1.05e-10 * np.linalg.norm(host(g))
    defl.close()
    op.close()


@pytest.mark.parametrize("mu", [0.0, 0.05])
def test_mixed_autograd_matches_oracle(wdl, mu):
    """The autograd Function with mixed = True (FP32 iteration, restarted
    refinement, FP64 true residual 1e-12 for both solves): dL/db, dL/dkappa
    and the link force against the oracle's gradient (bars as the FP64 path
    at its 1e-13 solves, relaxed 10x for the 1e-12 ones)."""
    import torch
    from paper_0710_1988_gb300.autograd import wilson_solve
    dims = (4, 4, 4, 8)
    U = L.gauge_field(dims, 0.5, 5000)
    kappa = 0.13
    b_h = L.gaussian_spinor(dims, 5001).ravel()
    eta_h = L.gaussian_spinor(dims, 5002).ravel()
    Lo, lam_o, dk_o, f_o = _oracle_grads(U, dims, kappa, b_h, eta_h, mu)
    op = wdl.WilsonOperator(dims, cuda(U), kappa, mu)
    op.set_mixed_restart(1e-3)
    b = cuda(b_h).requires_grad_(True)
    kap = torch.tensor(kappa, dtype=torch.float64, requires_grad=True)
    om = torch.zeros((L.volume(dims), 4, 8), dtype=torch.float64, device="cuda:0",
                     requires_grad=True)
    x = wilson_solve(b, kap, om, op, None, 1e-12, 100000, mixed=True)
    loss = torch.real(torch.vdot(cuda(eta_h), x))
    loss.backward()
    assert abs(loss.item() - Lo) <= 1e-9 * abs(Lo)
    lam_h = host(b.grad)
    assert np.linalg.norm(lam_h - lam_o) <= 1e-8 * np.linalg.norm(lam_o)
    assert abs(kap.grad.item() - dk_o) <= 1e-7 * abs(dk_o)
    fh = host(om.grad)
    assert np.linalg.norm(fh - f_o) <= 1e-7 * np.linalg.norm(f_o)
    op.close()
