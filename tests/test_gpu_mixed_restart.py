"""Restarted refinement in the mixed solver (wd_set_mixed_restart): the
low-precision BiCGStab runs until its recursive residual falls by delta, then
restarts from the FP64 residual.  Bars as for the mixed solver: FP64 true
residual <= 1e-10 under the oracle's operator, solution error <= cond * tol
on the 4^4 preset (2e-9, cond(A) = 41.6)."""
import numpy as np
import pytest

from inputs import lattice as L
from oracle import krylov

from .gpu_util import cuda, host, kappa_c_table, oracle_ops, rel_residual

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wdl():
    import paper_0710_1988_gb300 as wdl
    wdl.lib()
    return wdl


@pytest.mark.parametrize("bits", [32, 16])
@pytest.mark.parametrize("delta", [1e-3, 1e-5])
def test_restarted_refinement_4x4x4x4(wdl, bits, delta):
    cfg = L.CONFIGS["wilson_4x4x4x4"]
    kappa = cfg.kappa_factor * kappa_c_table()[cfg.name]["kappa_c"]
    U = L.gauge_field(cfg.dims, cfg.eps, L.link_seed(cfg))
    A, _ = oracle_ops(U, cfg.dims, kappa)
    B = np.stack([L.source(cfg, j).ravel() for j in range(1, cfg.n_rhs + 1)])
    op = wdl.WilsonOperator(cfg.dims, cuda(U), kappa)
    op.set_mixed_storage(bits)
    op.set_mixed_restart(delta, 500)
    X = cuda(np.zeros_like(B))
    rc, sts = op.dbicgstab_mixed(cuda(B), X, None, tol=1e-10)
    assert rc == 0
    Xh = host(X)
    for j in range(B.shape[0]):
        assert sts[j]["converged"] and sts[j]["restarts"] >= 1
        assert rel_residual(U, cfg.dims, kappa, Xh[j], B[j]) <= 1.05e-10
        xt, _ = krylov.bicgstab(A, B[j], tol=1e-14)
        assert np.linalg.norm(Xh[j] - xt) / np.linalg.norm(xt) <= 2e-9
    op.close()


def test_restarted_refinement_rejects_bad_delta(wdl):
    cfg = L.CONFIGS["wilson_4x4x4x4"]
    U = L.gauge_field(cfg.dims, cfg.eps, L.link_seed(cfg))
    op = wdl.WilsonOperator(cfg.dims, cuda(U), 0.12)
    for bad in ((1.0, 100), (-0.1, 100), (1e-3, 0)):
        with pytest.raises(Exception):
            op.set_mixed_restart(*bad)
    op.set_mixed_restart(0.0, 0)   # back to reliable updates
    op.close()


def test_twisted_at_kappa_c_converges_with_restarts(wdl):
    """16^4 twisted mass at kappa_c, mu = 0.002: the FP32 recurrence with
    reliable updates stalls near 1e-5 (20000 iterations); restarted
    refinement reaches 1e-10, checked by the oracle's operator."""
    cfg = L.CONFIGS["wilson_16x16x16x16"]
    table = kappa_c_table()
    if cfg.name not in table:
        pytest.skip("kappa_c of the 16^4 field not recorded")
    kappa = table[cfg.name]["kappa_c"]
    U = L.gauge_field(cfg.dims, cfg.eps, L.link_seed(cfg))
    B = L.gaussian_spinor(cfg.dims, 77).reshape(1, -1)
    op = wdl.WilsonOperator(cfg.dims, cuda(U), kappa)
    op.set_mixed_restart(1e-3, 4000)
    X = cuda(np.zeros_like(B))
    rc, sts = op.multishift(cuda(B), X, [0.002], tol=1e-10, max_iter=20000, project=False, mixed=True)
    assert rc == 0 and sts[0][0]["converged"]
    assert rel_residual(U, cfg.dims, kappa, host(X)[0], B[0], mu=0.002) <= 1.05e-10
    op.close()
