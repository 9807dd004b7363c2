"""Sec. 4: serial twisted-mass shifts with the minimal-residual projection
over previous solutions, GPU (C ABI tm_multishift_solve) against the oracle.

Bars: every solution's true residual, recomputed with the oracle's
operator, <= 1.05e-10; solutions within 1e-8 relative of the oracle's
(sigma_min(A(mu)) >= mu bounds the conditioning by ||A|| / mu).  At kappa_c
and small mu BiCGStab's residual can sit just above the tolerance for tens
of iterations, so iteration counts depend on rounding and are not compared.
"""
import numpy as np
import pytest

from inputs import lattice as L
from oracle import krylov

from .gpu_util import cuda, host, kappa_c_table, oracle_ops, rel_residual

pytestmark = pytest.mark.gpu

MUS = (0.08, 0.04, 0.02)


@pytest.fixture(scope="module")
def wdl():
    import paper_0710_1988_gb300 as wdl
    wdl.lib()
    return wdl


@pytest.fixture(scope="module")
def tm():
    cfg = L.CONFIGS["wilson_4x4x4x4"]
    kc = kappa_c_table()[cfg.name]["kappa_c"]
    U = L.gauge_field(cfg.dims, cfg.eps, L.link_seed(cfg))
    B = np.stack([L.gaussian_spinor(cfg.dims, 3000 + j).ravel() for j in range(2)])
    oracle = []
    for j in range(2):
        xs, sts = krylov.serial_shifts(lambda mu: oracle_ops(U, cfg.dims, kc, mu)[0], B[j], MUS,
                                       tol=1e-10, project=True)
        oracle.append((xs, sts))
    return dict(cfg=cfg, kc=kc, U=U, B=B, oracle=oracle)


@pytest.mark.parametrize("mixed", [False, True])
def test_multishift_matches_oracle(wdl, tm, mixed):
    import torch
    cfg = tm["cfg"]
    op = wdl.WilsonOperator(cfg.dims, cuda(tm["U"]), tm["kc"])
    B = cuda(tm["B"])
    X = torch.zeros(len(MUS) * B.numel(), dtype=torch.complex128, device="cuda:0")
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        rc, sts = op.multishift(B, X, MUS, tol=1e-10, project=True, mixed=mixed, stream=st)
    st.synchronize()
    assert rc == 0
    Xh = host(X).reshape(len(MUS), 2, -1)
    for i, mu in enumerate(MUS):
        for j in range(2):
            s = sts[i][j]
            assert s["converged"] == 1
            assert rel_residual(tm["U"], cfg.dims, tm["kc"], Xh[i, j], tm["B"][j], mu) <= 1.05e-10
            xo = tm["oracle"][j][0][i]
            assert np.linalg.norm(Xh[i, j] - xo) / np.linalg.norm(xo) <= 1e-8
            if i > 0:
                assert s["mvp_extra"] >= i   # the projection's products
    op.close()


def test_projection_cuts_total_work(wdl, tm):
    import torch
    cfg = tm["cfg"]
    op = wdl.WilsonOperator(cfg.dims, cuda(tm["U"]), tm["kc"])
    B = cuda(tm["B"])
    tot = {}
    for project in (False, True):
        X = torch.zeros(len(MUS) * B.numel(), dtype=torch.complex128, device="cuda:0")
        rc, sts = op.multishift(B, X, MUS, tol=1e-10, project=project)
        assert rc == 0
        tot[project] = sum(s["mvp"] for row in sts for s in row)
    assert tot[True] < tot[False]
    op.close()


@pytest.mark.parametrize("mixed", [False, True])
def test_shifts_through_the_schur_system(wdl, mixed):
    """tm_multishift_solve in even-odd mode: full-lattice sources and
    solutions, each shift prepared with its own mu, solved on the Schur
    system (projected over the earlier shifts' even solutions) and
    reconstructed.  Every solution satisfies its full twisted system to
    tol * ||b_hat(mu)|| / ||b|| under the oracle's operator."""
    from oracle import evenodd
    dims = (4, 4, 4, 8)
    U = L.gauge_field(dims, 0.5, 760)
    kappa = 0.13
    B = L.gaussian_spinor(dims, 761, nrhs=2).reshape(2, -1)
    mus = [0.064, 0.016, 0.004]
    op = wdl.WilsonOperator(dims, cuda(U), kappa)
    op.set_operator(True)
    op.set_mixed_restart(1e-3)
    X = cuda(np.zeros((len(mus) * 2, B.shape[1]), dtype=np.complex128))
    rc, sts = op.multishift(cuda(B), X, mus, tol=1e-10, project=True, mixed=mixed)
    assert rc == 0
    Xh = host(X).reshape(len(mus), 2, -1)
    v = L.volume(dims)
    for i, mu in enumerate(mus):
        for j in range(2):
            assert sts[i][j]["converged"]
            bh = evenodd.prepare(U, dims, kappa, mu, B[j].reshape(v, 4, 3)).ravel()
            scale = np.linalg.norm(bh) / np.linalg.norm(B[j])
            assert rel_residual(U, dims, kappa, Xh[i, j], B[j], mu=mu) <= 1.05e-10 * scale
    op.close()
