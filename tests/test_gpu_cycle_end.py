"""GMRES-DR's restart (Sec. 1) with the harmonic Ritz pairs from FP32
estimates refined in FP64 (the default) and from the FP64 QR iteration
alone (wd_set_eigen_estimates(h, 0), also the path taken when the refined
pairs fail their checks): the two must agree with each other and with the
oracle, so both stay covered."""
import numpy as np
import pytest

from .gpu_util import cuda, host, kappa_c_table, rel_residual

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wdl():
    import paper_0710_1988_gb300 as wdl
    wdl.lib()
    return wdl


def _solve(wdl, cfg, U, kappa, b0, B, fp32, m, k):
    import torch
    op = wdl.WilsonOperator(cfg.dims, cuda(U), kappa)
    op.set_eigen_estimates(fp32)
    V = torch.zeros(k * b0.size, dtype=torch.complex128, device="cuda:0")
    x0 = cuda(np.zeros_like(b0))
    rc, st, _, theta = op.gmresdr(cuda(b0), x0, m, k, 1e-12, 10000, V_out=V)
    assert rc == 0
    hist = op.gmresdr_history()
    defl = op.deflation(V, k)
    X = cuda(np.zeros_like(B))
    rc2, sts = op.dbicgstab(cuda(B), X, defl, tol=1e-12)
    assert rc2 == 0
    out = (st, np.asarray(theta), host(x0), [q["mvp"] for q in sts], host(X), hist)
    defl.close()
    op.close()
    return out


@pytest.mark.parametrize("m,k", [(20, 6), (40, 12), (80, 40)])
def test_fp32_estimates_and_fp64_iteration_agree(wdl, m, k):
    from inputs import lattice as L
    from oracle import krylov
    from .gpu_util import oracle_ops
    cfg = L.CONFIGS["wilson_4x4x4x4"]
    kappa = cfg.kappa_factor * kappa_c_table()[cfg.name]["kappa_c"]
    U = L.gauge_field(cfg.dims, cfg.eps, L.link_seed(cfg))
    b0 = L.source(cfg, 0).ravel()
    B = L.gaussian_spinor(cfg.dims, 3200, nrhs=6).reshape(6, -1)
    (s1, t1, x1, m1, X1, h1) = _solve(wdl, cfg, U, kappa, b0, B, True, m, k)
    (s2, t2, x2, m2, X2, h2) = _solve(wdl, cfg, U, kappa, b0, B, False, m, k)
    assert s1["mvp"] == s2["mvp"] and s1["cycles"] == s2["cycles"]
    np.testing.assert_allclose(h1, h2, rtol=1e-6, atol=0)
    scale = np.abs(t2).max()
    assert np.abs(np.sort(np.abs(t1)) - np.sort(np.abs(t2))).max() <= 1e-10 * scale
    assert np.linalg.norm(x1 - x2) <= 1e-9 * np.linalg.norm(x2)
    assert all(abs(a - b) <= 4 for a, b in zip(m1, m2))
    assert np.linalg.norm(X1 - X2) <= 1e-9 * np.linalg.norm(X2)
    # and the kept values are the oracle's
    A, _ = oracle_ops(U, cfg.dims, kappa)
    ref = krylov.gmresdr(A, b0, m, k, tol=1e-12)
    assert s1["mvp"] == ref.stats.mvp
    th_ref = np.sort(np.abs(ref.theta))
    for t in (t1, t2):
        assert np.abs(np.sort(np.abs(t)) - th_ref).max() <= 1e-8 * th_ref.max()
    assert rel_residual(U, cfg.dims, kappa, x1, b0) <= 1.05e-12
