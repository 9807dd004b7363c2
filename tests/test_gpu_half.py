"""FP16 storage of the mixed solver: parity with the CPU oracle.

Storage format under test: each site's 12 complex numbers are scaled by the
site's largest |re| or |im| and rounded to IEEE half (11-bit significand), so
every stored component carries an absolute error <= 2^-12 times its site's
scale; links keep rows 0 and 1 in half and rebuild row 2 as conj(row0 x row1).
Arithmetic is FP32.

Bars:
 * exact-input pin: with unit links and a Z4 source every input is exact in
   the half format, so the only error is the rounding of the output: each
   component within 2^-12 of its site's scale (plus FP32 arithmetic, 1e-6);
 * random inputs: ~100 products of half-rounded factors per output, each
   with relative rounding <= 2^-12, give a norm-wise relative error of a few
   1e-4; the bar is 2e-3 norm-wise (4e-3 in max-norm);
 * solves: the FP64 reliable updates and the FP64 true-residual test make
   the tolerance mean what it means for the FP64 solver, so the bars are
   those of the FP32-storage solver (true residual 1e-10; solution error
   against an oracle solve to 1e-14 within cond(A) * 1e-10 = 2e-9 on the
   4^4 preset, cond(A) = 41.6).
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


def _apply16(wdl, dims, U, psi, kappa, mu, dagger=False):
    import torch
    op = wdl.WilsonOperator(dims, cuda(U), kappa, mu)
    out = torch.empty(psi.size, dtype=torch.complex128, device="cuda:0")
    op.apply_f16(cuda(psi), out, dagger=dagger)
    op.close()
    return host(out).reshape(psi.shape)


def test_f16_exact_inputs_only_output_rounding(wdl):
    dims = (4, 4, 4, 8)
    U = L.unit_gauge_field(dims)
    psi = L.z4_spinor(dims, 720, nrhs=2)
    kappa = 0.125  # a power of two: kappa * (small integers) is exact in FP32
    got = _apply16(wdl, dims, U, psi, kappa, 0.0)
    for r in range(2):
        ref = dirac.apply_A(U, psi[r], dims, kappa, 0.0)
        scale = np.maximum(np.abs(ref.real), np.abs(ref.imag)).reshape(ref.shape[0], -1).max(axis=1)
        err = np.abs(got[r] - ref).reshape(ref.shape[0], -1).max(axis=1)
        assert np.all(err <= 2.0 ** -12 * scale * 1.0001 * np.sqrt(2) + 1e-6), err.max()


@pytest.mark.parametrize("dims,nrhs", [((4, 4, 4, 4), 1), ((2, 3, 4, 5), 3), ((6, 4, 2, 8), 5),
                                       ((8, 8, 8, 16), 4), ((1, 4, 3, 2), 2)])
@pytest.mark.parametrize("dagger", [False, True])
def test_f16_wilson_parity(wdl, dims, nrhs, dagger):
    U = L.gauge_field(dims, 0.5, 730)
    psi = L.gaussian_spinor(dims, 731, nrhs=nrhs)
    got = _apply16(wdl, dims, U, psi, 0.1337, 0.04, dagger)
    f = dirac.apply_A_dagger if dagger else dirac.apply_A
    for r in range(nrhs):
        ref = f(U, psi[r], dims, 0.1337, 0.04)
        assert np.linalg.norm(got[r] - ref) <= 2e-3 * np.linalg.norm(ref)
        assert np.abs(got[r] - ref).max() <= 4e-3 * np.abs(ref).max()


@pytest.fixture(scope="module")
def cfg0():
    cfg = L.CONFIGS["wilson_4x4x4x4"]
    kappa = cfg.kappa_factor * kappa_c_table()[cfg.name]["kappa_c"]
    U = L.gauge_field(cfg.dims, cfg.eps, L.link_seed(cfg))
    A, _ = oracle_ops(U, cfg.dims, kappa)
    B = np.stack([L.source(cfg, j).ravel() for j in range(1, cfg.n_rhs + 1)])
    gd = krylov.gmresdr(A, L.source(cfg, 0).ravel(), cfg.m, cfg.k, tol=cfg.tol)
    return dict(cfg=cfg, kappa=kappa, U=U, A=A, B=B, gd=gd)


@pytest.mark.parametrize("every", [50, 7])
def test_half_storage_solve_reaches_fp64_residual(wdl, cfg0, every):
    c = cfg0
    op = wdl.WilsonOperator(c["cfg"].dims, cuda(c["U"]), c["kappa"])
    op.set_mixed_storage(16)
    X = cuda(np.zeros_like(c["B"]))
    rc, sts = op.dbicgstab_mixed(cuda(c["B"]), X, None, tol=1e-10, reliable_every=every)
    Xh = host(X)
    assert rc == 0
    for j in range(c["B"].shape[0]):
        assert sts[j]["converged"] == 1 and sts[j]["true_rel_res"] <= 1e-10
        assert rel_residual(c["U"], c["cfg"].dims, c["kappa"], Xh[j], c["B"][j]) <= 1.05e-10
        xt, _ = krylov.bicgstab(c["A"], c["B"][j], tol=1e-14)
        assert np.linalg.norm(Xh[j] - xt) / np.linalg.norm(xt) <= 2e-9
    op.close()


def test_half_storage_with_deflation_and_determinism(wdl, cfg0):
    c = cfg0
    cfg = c["cfg"]
    op = wdl.WilsonOperator(cfg.dims, cuda(c["U"]), c["kappa"])
    op.set_mixed_storage(16)
    defl = op.deflation(cuda(c["gd"].V), cfg.k)
    X1 = cuda(np.zeros_like(c["B"]))
    X2 = cuda(np.zeros_like(c["B"]))
    rc, sts = op.dbicgstab_mixed(cuda(c["B"]), X1, defl, tol=1e-10)
    assert rc == 0 and all(s["converged"] for s in sts)
    op.dbicgstab_mixed(cuda(c["B"]), X2, defl, tol=1e-10)
    import torch
    assert torch.equal(X1, X2)
    Xh = host(X1)
    for j in range(c["B"].shape[0]):
        assert rel_residual(c["U"], cfg.dims, c["kappa"], Xh[j], c["B"][j]) <= 1.05e-10
    defl.close()
    op.close()


def test_half_storage_rejects_other_widths(wdl, cfg0):
    c = cfg0
    op = wdl.WilsonOperator(c["cfg"].dims, cuda(c["U"]), c["kappa"])
    with pytest.raises(Exception):
        op.set_mixed_storage(8)
    op.close()


def test_half_storage_twisted_shifts(wdl):
    dims = (4, 4, 4, 8)
    U = L.gauge_field(dims, 0.5, 740)
    kappa = 0.13
    B = L.gaussian_spinor(dims, 741, nrhs=2).reshape(2, -1)
    mus = [0.064, 0.016]
    op = wdl.WilsonOperator(dims, cuda(U), kappa)
    op.set_mixed_storage(16)
    X = cuda(np.zeros((len(mus) * 2, B.shape[1]), dtype=np.complex128))
    rc, sts = op.multishift(cuda(B), X, mus, tol=1e-10, mixed=True)
    assert rc == 0
    Xh = host(X).reshape(len(mus), 2, -1)
    for i, mu in enumerate(mus):
        for j in range(2):
            assert sts[i][j]["converged"]
            assert rel_residual(U, dims, kappa, Xh[i, j], B[j], mu=mu) <= 1.05e-10
    op.close()


def test_half_storage_full_size_16x16x16x16(wdl):
    cfg = L.CONFIGS["wilson_16x16x16x16"]
    table = kappa_c_table()
    if cfg.name not in table:
        pytest.skip("kappa_c of the 16^4 preset not recorded")
    kappa = cfg.kappa_factor * table[cfg.name]["kappa_c"]
    U = L.gauge_field(cfg.dims, cfg.eps, L.link_seed(cfg))
    op = wdl.WilsonOperator(cfg.dims, cuda(U), kappa)
    op.set_mixed_storage(16)
    Bh = np.stack([L.source(cfg, j) for j in range(1, 5)]).reshape(4, -1)
    X = cuda(np.zeros_like(Bh))
    rc, sts = op.dbicgstab_mixed(cuda(Bh), X, None, tol=1e-10)
    assert rc == 0 and all(s["converged"] and s["true_rel_res"] <= 1e-10 for s in sts)
    assert rel_residual(U, cfg.dims, kappa, host(X)[0], Bh[0]) <= 1.05e-10
    op.close()


@pytest.mark.parametrize("R", [1, 2, 4])
@pytest.mark.parametrize("threads", [64, 128, 256])
def test_every_f16_launch_shape(wdl, R, threads):
    import torch
    dims, nrhs = (6, 4, 2, 8), 5
    U = L.gauge_field(dims, 0.5, 750)
    psi = L.gaussian_spinor(dims, 751, nrhs=nrhs)
    op = wdl.WilsonOperator(dims, cuda(U), 0.13, 0.02)
    op.set_f16_shape(nrhs, R, threads)
    out = torch.empty(psi.size, dtype=torch.complex128, device="cuda:0")
    op.apply_f16(cuda(psi), out)
    got = host(out).reshape(psi.shape)
    for r in range(nrhs):
        ref = dirac.apply_A(U, psi[r], dims, 0.13, 0.02)
        assert np.linalg.norm(got[r] - ref) <= 2e-3 * np.linalg.norm(ref)
    op.close()


def test_f16_autotuner_picks_a_shape_and_solves(wdl, cfg0):
    c = cfg0
    op = wdl.WilsonOperator(c["cfg"].dims, cuda(c["U"]), c["kappa"])
    R, T, ms = op.autotune_f16(3)
    assert R in (1, 2) and T in (64, 128, 256) and ms > 0
    op.set_mixed_storage(16)
    X = cuda(np.zeros_like(c["B"]))
    rc, sts = op.dbicgstab_mixed(cuda(c["B"]), X, None, tol=1e-10)
    assert rc == 0 and all(s["converged"] for s in sts)
    op.close()
