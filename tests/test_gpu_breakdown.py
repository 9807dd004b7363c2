"""WD_BREAKDOWN through the C ABI, reached by an input rather than a fault.

tests/gpu_util.breakdown_system builds a source b with <b, A b> = 0 exactly
(unit links, kappa = 3/16, constant + staggered modes), so with x0 = 0 the
first BiCGStab step has <r_hat, v> = 0 and alpha is undefined: the solver
must report a breakdown (the paper's "F", Sec. 3) for that system, write its
solution (x = 0, no step taken) and stats, and still solve the other systems
of the batch.  The oracle stops the same way (tests/test_oracle_pins.py).
"""
import numpy as np
import pytest

from inputs import lattice as L
from oracle import krylov

from .gpu_util import breakdown_system, cuda, host, oracle_ops, rel_residual

pytestmark = pytest.mark.gpu

DIMS = (4, 4, 2, 2)


@pytest.fixture(scope="module")
def wdl():
    import paper_0710_1988_gb300 as wdl
    wdl.lib()
    return wdl


@pytest.mark.parametrize("mixed", [False, True])
def test_breakdown_is_reported_per_system(wdl, mixed):
    from paper_0710_1988_gb300 import _lib
    U, kap, b = breakdown_system(DIMS)
    g = L.gaussian_spinor(DIMS, 4321).ravel()
    B = np.stack([b, g])
    op = wdl.WilsonOperator(DIMS, cuda(U), kap)
    X = cuda(np.full_like(B, np.nan + 0j))
    X.zero_()
    if mixed:
        # kappa = 3/16 lies beyond the free field's kappa_c = 1/8: the spectrum
        # surrounds the origin and FP64 BiCGStab converges only by its near
        # finite termination on the few distinct eigenvalues, which FP32
        # rounding destroys; restarting every pass from the FP64 residual
        # recovers it
        op.set_mixed_restart(1e-3, 40)
        rc, sts = op.dbicgstab_mixed(cuda(B), X, None, tol=1e-10, max_iter=4000)
    else:
        rc, sts = op.dbicgstab(cuda(B), X, None, tol=1e-10, max_iter=2000)
    assert rc == _lib.WD_BREAKDOWN
    xo, so = krylov.bicgstab(oracle_ops(U, DIMS, kap)[0], b, tol=1e-10)
    assert so.breakdown
    s0, s1 = sts
    assert s0["breakdown"] == 1 and s0["converged"] == 0
    assert s0["iters"] == so.iters == 0
    if not mixed:
        assert s0["mvp"] == so.mvp == 1
    Xh = host(X).reshape(2, -1)
    assert np.all(Xh[0] == 0)                  # no step was taken
    assert s0["true_rel_res"] == pytest.approx(1.0, rel=1e-12)
    # the other system of the batch is unaffected
    assert s1["breakdown"] == 0 and s1["converged"] == 1
    assert rel_residual(U, DIMS, kap, Xh[1], g) <= 1.05e-10
    op.close()
