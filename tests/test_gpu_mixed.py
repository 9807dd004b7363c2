"""Mixed precision (FP32 iteration, FP64 reliable updates): parity with the
CPU oracle.

Bars: the FP32 Wilson kernel agrees with the FP64 oracle to 2e-6 relative
(max-norm; inputs rounded to FP32, ~100 FP32 terms per output); a mixed
solve reaches the same FP64 true residual 1e-10 as the FP64 solver, checked
by the oracle's operator.  Its solution error against an oracle solve to
1e-14 is bounded by cond(A) * 1e-10; on the 4^4 preset cond(A) = 41.6
(sigma_max 1.968, sigma_min 0.0473 from an SVD of the oracle's dense
matrix), so the bar is 2e-9 where the FP64 solver's is 1e-9.
"""
import numpy as np
import pytest

from inputs import lattice as L
from oracle import dirac, krylov

from .gpu_util import cuda, host, kappa_c_table, oracle_ops, rel_residual

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wdl():
    import paper_0710_1988_gb300 as wdl
    wdl.lib()
    return wdl


@pytest.mark.parametrize("dims,nrhs", [((4, 4, 4, 4), 1), ((2, 3, 4, 5), 3), ((6, 4, 2, 8), 5),
                                       ((8, 8, 8, 16), 4), ((1, 4, 3, 2), 2), ((16, 16, 16, 16), 1)])
@pytest.mark.parametrize("dagger", [False, True])
def test_f32_wilson_parity(wdl, dims, nrhs, dagger):
    import torch
    U = L.gauge_field(dims, 0.5, 700)
    psi = L.gaussian_spinor(dims, 701, nrhs=nrhs)
    op = wdl.WilsonOperator(dims, cuda(U), 0.1337, 0.04)
    out = torch.empty(psi.size, dtype=torch.complex128, device="cuda:0")
    op.apply_f32(cuda(psi), out, dagger=dagger)
    got = host(out).reshape(psi.shape)
    f = dirac.apply_A_dagger if dagger else dirac.apply_A
    for r in range(nrhs):
        ref = f(U, psi[r], dims, 0.1337, 0.04)
        err = np.abs(got[r] - ref).max() / np.abs(ref).max()
        assert err <= 2e-6, (dims, r, err)
    op.close()


@pytest.fixture(scope="module")
def cfg0():
    cfg = L.CONFIGS["wilson_4x4x4x4"]
    kappa = cfg.kappa_factor * kappa_c_table()[cfg.name]["kappa_c"]
    U = L.gauge_field(cfg.dims, cfg.eps, L.link_seed(cfg))
    A, g5 = oracle_ops(U, cfg.dims, kappa)
    B = np.stack([L.source(cfg, j).ravel() for j in range(1, cfg.n_rhs + 1)])
    gd = krylov.gmresdr(A, L.source(cfg, 0).ravel(), cfg.m, cfg.k, tol=cfg.tol)
    return dict(cfg=cfg, kappa=kappa, U=U, A=A, g5=g5, B=B, gd=gd)


@pytest.mark.parametrize("every", [50, 7])
def test_mixed_bicgstab_reaches_fp64_residual(wdl, cfg0, every):
    c = cfg0
    op = wdl.WilsonOperator(c["cfg"].dims, cuda(c["U"]), c["kappa"])
    X = cuda(np.zeros_like(c["B"]))
    rc, sts = op.dbicgstab_mixed(cuda(c["B"]), X, None, tol=1e-10, reliable_every=every)
    Xh = host(X)
    assert rc == 0
    for j in range(c["B"].shape[0]):
        assert sts[j]["converged"] == 1 and sts[j]["true_rel_res"] <= 1e-10
        assert rel_residual(c["U"], c["cfg"].dims, c["kappa"], Xh[j], c["B"][j]) <= 1.05e-10
        xt, st = krylov.bicgstab(c["A"], c["B"][j], tol=1e-14)
        assert np.linalg.norm(Xh[j] - xt) / np.linalg.norm(xt) <= 2e-9
        # FP32 iterations cost at most ~40% more than the FP64 solver's
        _, s64 = krylov.bicgstab(c["A"], c["B"][j], tol=1e-10)
        assert sts[j]["iters"] <= 1.4 * s64.iters + 10
    op.close()


def test_mixed_dbicgstab_with_deflation(wdl, cfg0):
    c = cfg0
    cfg = c["cfg"]
    op = wdl.WilsonOperator(cfg.dims, cuda(c["U"]), c["kappa"])
    defl = op.deflation(cuda(c["gd"].V), cfg.k)
    X = cuda(np.zeros_like(c["B"]))
    rc, sts = op.dbicgstab_mixed(cuda(c["B"]), X, defl, tol=1e-10)
    assert rc == 0 and all(s["converged"] for s in sts)
    Xh = host(X)
    for j in range(c["B"].shape[0]):
        assert rel_residual(c["U"], cfg.dims, c["kappa"], Xh[j], c["B"][j]) <= 1.05e-10
    defl.close()
    op.close()


def test_mixed_streams_and_determinism(wdl, cfg0):
    import torch
    c = cfg0
    op = wdl.WilsonOperator(c["cfg"].dims, cuda(c["U"]), c["kappa"])
    B = cuda(c["B"])
    X1 = cuda(np.zeros_like(c["B"]))
    X2 = cuda(np.zeros_like(c["B"]))
    op.dbicgstab_mixed(B, X1, None, tol=1e-10)            # default stream: side stream + graph
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        op.dbicgstab_mixed(B, X2, None, tol=1e-10, stream=st)
    st.synchronize()
    assert torch.equal(X1, X2)
    op.close()


def test_mixed_batch_with_zero_and_host_buffers(wdl, cfg0):
    c = cfg0
    op = wdl.WilsonOperator(c["cfg"].dims, cuda(c["U"]), c["kappa"])
    B = np.stack([np.zeros_like(c["B"][0]), c["B"][0]])
    X = np.zeros_like(B)
    rc, sts = op.dbicgstab_mixed(B, X, None, tol=1e-10)
    assert rc == 0 and sts[0]["converged"] and sts[0]["iters"] == 0 and np.all(X[0] == 0)
    assert rel_residual(c["U"], c["cfg"].dims, c["kappa"], X[1], B[1]) <= 1.05e-10
    op.close()


def test_mixed_not_converged(wdl, cfg0):
    c = cfg0
    op = wdl.WilsonOperator(c["cfg"].dims, cuda(c["U"]), c["kappa"])
    X = cuda(np.zeros_like(c["B"][:1]))
    rc, sts = op.dbicgstab_mixed(cuda(c["B"][:1]), X, None, tol=1e-12, max_iter=5)
    assert rc == 2 and sts[0]["converged"] == 0 and sts[0]["iters"] <= 10
    assert 0 < sts[0]["true_rel_res"] < 1
    op.close()


def test_mixed_full_size_16x16x16x16(wdl):
    cfg = L.CONFIGS["wilson_16x16x16x16"]
    table = kappa_c_table()
    if cfg.name not in table:
        pytest.skip("kappa_c of the 16^4 preset not recorded")
    kappa = cfg.kappa_factor * table[cfg.name]["kappa_c"]
    U = L.gauge_field(cfg.dims, cfg.eps, L.link_seed(cfg))
    op = wdl.WilsonOperator(cfg.dims, cuda(U), kappa)
    Bh = np.stack([L.source(cfg, j) for j in range(1, 5)]).reshape(4, -1)
    X = cuda(np.zeros_like(Bh))
    rc, sts = op.dbicgstab_mixed(cuda(Bh), X, None, tol=1e-10)
    assert rc == 0 and all(s["converged"] and s["true_rel_res"] <= 1e-10 for s in sts)
    assert rel_residual(U, cfg.dims, kappa, host(X)[0], Bh[0]) <= 1.05e-10
    op.close()


@pytest.mark.parametrize("R", [1, 2, 4])
@pytest.mark.parametrize("threads", [64, 128, 256])
def test_every_f32_launch_shape(wdl, R, threads):
    import torch
    dims, nrhs = (6, 4, 2, 8), 5
    U = L.gauge_field(dims, 0.5, 710)
    psi = L.gaussian_spinor(dims, 711, nrhs=nrhs)
    op = wdl.WilsonOperator(dims, cuda(U), 0.13, 0.02)
    op.set_f32_shape(nrhs, R, threads)
    out = torch.empty(psi.size, dtype=torch.complex128, device="cuda:0")
    op.apply_f32(cuda(psi), out)
    got = host(out).reshape(psi.shape)
    for r in range(nrhs):
        ref = dirac.apply_A(U, psi[r], dims, 0.13, 0.02)
        assert np.abs(got[r] - ref).max() <= 2e-6 * np.abs(ref).max()
    op.close()


def test_autotuner_picks_a_shape_and_solves(wdl, cfg0):
    c = cfg0
    op = wdl.WilsonOperator(c["cfg"].dims, cuda(c["U"]), c["kappa"])
    R, T, ms = op.autotune_f32(3)
    assert R in (1, 2) and T in (64, 128, 256) and ms > 0
    X = cuda(np.zeros_like(c["B"]))
    rc, sts = op.dbicgstab_mixed(cuda(c["B"]), X, None, tol=1e-10)
    assert rc == 0 and all(s["converged"] for s in sts)
    op.close()
