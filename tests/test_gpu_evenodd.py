"""Even-odd preconditioning on the GPU (wd_set_operator, wd_eo_prepare,
wd_eo_reconstruct, and the solvers on the Schur operator) against the
oracle's evenodd module.  Bars: 1e-12 relative per FP64 Schur application;
solutions through the Schur system satisfy the full system to the
tolerance (the odd residual is zero by construction, so ||b - A x|| equals
the Schur residual)."""
import numpy as np
import pytest

from inputs import lattice as L
from oracle import dirac, evenodd, krylov

from .gpu_util import cuda, host, kappa_c_table, rel_residual

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wdl():
    import paper_0710_1988_gb300 as wdl
    wdl.lib()
    return wdl


@pytest.mark.parametrize("dims,nrhs", [((4, 4, 4, 4), 1), ((6, 4, 2, 8), 3), ((8, 8, 8, 16), 2)])
@pytest.mark.parametrize("mu", [0.0, 0.05])
@pytest.mark.parametrize("dagger", [False, True])
def test_schur_apply_parity(wdl, dims, nrhs, mu, dagger):
    import torch
    U = L.gauge_field(dims, 0.5, 800)
    op = wdl.WilsonOperator(dims, cuda(U), 0.131, mu)
    op.set_operator(True)
    nh = 12 * L.volume(dims) // 2
    xe = L.gaussian_spinor(dims, 801, nrhs=nrhs)[:, : L.volume(dims) // 2].reshape(nrhs, nh)
    out = torch.empty(nrhs * nh, dtype=torch.complex128, device="cuda:0")
    op.apply(cuda(xe), out, dagger=dagger)
    got = host(out).reshape(nrhs, nh)
    g5 = lambda z: dirac.gamma5(z.reshape(-1, 4, 3)).ravel()
    for r in range(nrhs):
        if dagger:   # A_hat^dagger = gamma5 A_hat(-mu) gamma5
            ref = g5(evenodd.schur_apply(U, dims, 0.131, -mu, g5(xe[r])).ravel())
        else:
            ref = evenodd.schur_apply(U, dims, 0.131, mu, xe[r]).ravel()
        assert np.abs(got[r] - ref).max() <= 1e-12 * np.abs(ref).max()
    op.close()


@pytest.mark.parametrize("mu", [0.0, 0.08])
def test_prepare_and_reconstruct_parity(wdl, mu):
    import torch
    dims = (4, 4, 2, 6)
    U = L.gauge_field(dims, 0.5, 810)
    op = wdl.WilsonOperator(dims, cuda(U), 0.12, mu)
    op.set_operator(True)
    B = L.gaussian_spinor(dims, 811, nrhs=2)
    xe = L.gaussian_spinor(dims, 812, nrhs=2)[:, : L.volume(dims) // 2]
    nh = 12 * L.volume(dims) // 2
    Bh = torch.empty(2 * nh, dtype=torch.complex128, device="cuda:0")
    op.eo_prepare(cuda(B), Bh)
    X = torch.empty(B.size, dtype=torch.complex128, device="cuda:0")
    op.eo_reconstruct(cuda(B), cuda(xe), X)
    for r in range(2):
        ref = evenodd.prepare(U, dims, 0.12, mu, B[r]).ravel()
        assert np.abs(host(Bh).reshape(2, nh)[r] - ref).max() <= 1e-12 * np.abs(ref).max()
        refx = evenodd.reconstruct(U, dims, 0.12, mu, B[r], xe[r]).ravel()
        assert np.abs(host(X).reshape(2, -1)[r] - refx).max() <= 1e-12 * np.abs(refx).max()
    op.close()


def test_eo_gmresdr_dbicgstab_pipeline(wdl):
    """GMRES-DR(20,6) and D-BiCGStab(6) on the Schur system of the 4^4 preset;
    reconstructed solutions solve the full system, with fewer products."""
    import torch
    cfg = L.CONFIGS["wilson_4x4x4x4"]
    kappa = cfg.kappa_factor * kappa_c_table()[cfg.name]["kappa_c"]
    U = L.gauge_field(cfg.dims, cfg.eps, L.link_seed(cfg))
    op = wdl.WilsonOperator(cfg.dims, cuda(U), kappa)
    n = 12 * L.volume(cfg.dims)
    B = np.stack([L.source(cfg, j).ravel() for j in range(cfg.n_rhs + 1)])
    # full-operator reference counts
    Xf = cuda(np.zeros_like(B[1:]))
    _, sfull = op.dbicgstab(cuda(B[1:]), Xf, None, tol=cfg.tol)
    op.set_operator(True)
    Bh = torch.empty((cfg.n_rhs + 1) * n // 2, dtype=torch.complex128, device="cuda:0")
    op.eo_prepare(cuda(B), Bh)
    Bh = Bh.view(cfg.n_rhs + 1, n // 2)
    V = torch.zeros(cfg.k * n // 2, dtype=torch.complex128, device="cuda:0")
    xe0 = torch.zeros(n // 2, dtype=torch.complex128, device="cuda:0")
    rc, st, _, _ = op.gmresdr(Bh[0].contiguous(), xe0, cfg.m, cfg.k, cfg.tol, 100000, V_out=V)
    assert rc == 0
    defl = op.deflation(V, cfg.k)
    Xe = torch.zeros(cfg.n_rhs * n // 2, dtype=torch.complex128, device="cuda:0")
    rc, sts = op.dbicgstab(Bh[1:].contiguous(), Xe, defl, tol=cfg.tol)
    assert rc == 0 and all(s["converged"] for s in sts)
    X = torch.empty(cfg.n_rhs * n, dtype=torch.complex128, device="cuda:0")
    op.eo_reconstruct(cuda(B[1:]), Xe, X)
    Xh = host(X).reshape(cfg.n_rhs, n)
    Bhh = host(Bh)
    for j in range(cfg.n_rhs):
        scale = np.linalg.norm(Bhh[j + 1]) / np.linalg.norm(B[j + 1])
        assert rel_residual(U, cfg.dims, kappa, Xh[j], B[j + 1]) <= 1.05 * cfg.tol * scale
        assert sts[j]["mvp"] < sfull[j]["mvp"]
    defl.close()
    op.close()


@pytest.mark.parametrize("dims,nrhs", [((4, 4, 4, 4), 1), ((6, 4, 2, 8), 3), ((8, 8, 8, 16), 2)])
@pytest.mark.parametrize("mu", [0.0, 0.05])
@pytest.mark.parametrize("dagger", [False, True])
def test_f32_schur_apply_parity(wdl, dims, nrhs, mu, dagger):
    """The FP32 Schur operator (wd_apply_f32 in even-odd mode) against the
    oracle's FP64 Schur operator: 2e-6 of the largest entry (inputs rounded
    to FP32, ~200 FP32 terms per output over the two half hops)."""
    import torch
    U = L.gauge_field(dims, 0.5, 820)
    op = wdl.WilsonOperator(dims, cuda(U), 0.131, mu)
    op.set_operator(True)
    nh = 12 * L.volume(dims) // 2
    xe = L.gaussian_spinor(dims, 821, nrhs=nrhs)[:, : L.volume(dims) // 2].reshape(nrhs, nh)
    out = torch.empty(nrhs * nh, dtype=torch.complex128, device="cuda:0")
    op.apply_f32(cuda(xe), out, dagger=dagger)
    got = host(out).reshape(nrhs, nh)
    g5 = lambda z: dirac.gamma5(z.reshape(-1, 4, 3)).ravel()
    for r in range(nrhs):
        if dagger:
            ref = g5(evenodd.schur_apply(U, dims, 0.131, -mu, g5(xe[r])).ravel())
        else:
            ref = evenodd.schur_apply(U, dims, 0.131, mu, xe[r]).ravel()
        assert np.abs(got[r] - ref).max() <= 2e-6 * np.abs(ref).max()
    op.close()


@pytest.mark.parametrize("delta", [0.0, 1e-3])
def test_mixed_solver_on_the_schur_system(wdl, delta):
    """dbicgstab_mixed in even-odd mode (FP32 Schur iteration, FP64 Schur
    reliable updates), with and without the Schur deflation space: the
    reconstructed solutions satisfy the full system to tol * ||b_hat|| / ||b||
    under the oracle's operator."""
    import torch
    cfg = L.CONFIGS["wilson_4x4x4x4"]
    kappa = cfg.kappa_factor * kappa_c_table()[cfg.name]["kappa_c"]
    U = L.gauge_field(cfg.dims, cfg.eps, L.link_seed(cfg))
    n = 12 * L.volume(cfg.dims)
    B = np.stack([L.source(cfg, j).ravel() for j in range(cfg.n_rhs + 1)])
    op = wdl.WilsonOperator(cfg.dims, cuda(U), kappa)
    op.set_operator(True)
    op.set_mixed_restart(delta)
    Bh = torch.empty((cfg.n_rhs + 1) * n // 2, dtype=torch.complex128, device="cuda:0")
    op.eo_prepare(cuda(B), Bh)
    Bh = Bh.view(cfg.n_rhs + 1, n // 2)
    V = torch.zeros(cfg.k * n // 2, dtype=torch.complex128, device="cuda:0")
    xe0 = torch.zeros(n // 2, dtype=torch.complex128, device="cuda:0")
    rc, st, _, _ = op.gmresdr(Bh[0].contiguous(), xe0, cfg.m, cfg.k, cfg.tol, 100000, V_out=V)
    assert rc == 0
    defl = op.deflation(V, cfg.k)
    Bhh = host(Bh)
    for d in (None, defl):
        Xe = torch.zeros(cfg.n_rhs * n // 2, dtype=torch.complex128, device="cuda:0")
        rc, sts = op.dbicgstab_mixed(Bh[1:].contiguous(), Xe, d, tol=cfg.tol)
        assert rc == 0 and all(s["converged"] and s["true_rel_res"] <= cfg.tol for s in sts)
        X = torch.empty(cfg.n_rhs * n, dtype=torch.complex128, device="cuda:0")
        op.eo_reconstruct(cuda(B[1:]), Xe, X)
        Xh = host(X).reshape(cfg.n_rhs, n)
        for j in range(cfg.n_rhs):
            scale = np.linalg.norm(Bhh[j + 1]) / np.linalg.norm(B[j + 1])
            assert rel_residual(U, cfg.dims, kappa, Xh[j], B[j + 1]) <= 1.05 * cfg.tol * scale
    defl.close()
    op.close()


def test_mixed_schur_full_size_16x16x16x16(wdl):
    import torch
    cfg = L.CONFIGS["wilson_16x16x16x16"]
    table = kappa_c_table()
    if cfg.name not in table:
        pytest.skip("kappa_c of the 16^4 preset not recorded")
    kappa = cfg.kappa_factor * table[cfg.name]["kappa_c"]
    U = L.gauge_field(cfg.dims, cfg.eps, L.link_seed(cfg))
    n = 12 * L.volume(cfg.dims)
    B = np.stack([L.source(cfg, j).ravel() for j in (1, 2)])
    op = wdl.WilsonOperator(cfg.dims, cuda(U), kappa)
    op.set_operator(True)
    op.set_mixed_restart(1e-3)
    Bh = torch.empty(2 * n // 2, dtype=torch.complex128, device="cuda:0")
    op.eo_prepare(cuda(B), Bh)
    Xe = torch.zeros_like(Bh)
    rc, sts = op.dbicgstab_mixed(Bh, Xe, None, tol=cfg.tol)
    assert rc == 0 and all(s["converged"] for s in sts)
    X = torch.empty(2 * n, dtype=torch.complex128, device="cuda:0")
    op.eo_reconstruct(cuda(B), Xe, X)
    Xh = host(X).reshape(2, n)
    Bhh = host(Bh).reshape(2, n // 2)
    for j in range(2):
        scale = np.linalg.norm(Bhh[j]) / np.linalg.norm(B[j])
        assert rel_residual(U, cfg.dims, kappa, Xh[j], B[j]) <= 1.05 * cfg.tol * scale
    op.close()
