"""Parity of the CUDA Wilson-Dirac apply (C ABI wd_apply) with the CPU oracle.

Bar: relative error <= 1e-12 per FP64 application (max-norm, relative to
the largest output component), on lattices that span several 128-site
blocks plus a ragged tail, odd extents, L = 1 and L = 2 directions, both
A and A^dagger, Wilson and twisted mass, batched right-hand sides.
"""
import numpy as np
import pytest

from inputs import lattice as L
from oracle import dirac

from .gpu_util import cuda, host

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def wdl():
    import paper_0710_1988_gb300 as wdl
    wdl.lib()
    return wdl


def _check(wdl, dims, kappa, mu, dagger, nrhs, seed):
    import torch
    U = L.gauge_field(dims, 0.5, seed)
    psi = L.gaussian_spinor(dims, seed + 1, nrhs=nrhs)
    op = wdl.WilsonOperator(dims, cuda(U), kappa, mu)
    out = torch.empty(psi.size, dtype=torch.complex128, device="cuda:0")
    op.apply(cuda(psi), out, dagger=dagger)
    got = host(out).reshape(psi.shape)
    f = dirac.apply_A_dagger if dagger else dirac.apply_A
    for r in range(nrhs):
        ref = f(U, psi[r], dims, kappa, mu)
        err = np.abs(got[r] - ref).max() / np.abs(ref).max()
        assert err <= TOL, (dims, kappa, mu, dagger, r, err)
    op.close()


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4), (2, 3, 4, 5), (6, 4, 2, 8),
                                  (1, 4, 3, 2), (5, 1, 1, 7), (8, 8, 8, 16)])
@pytest.mark.parametrize("dagger", [False, True])
def test_wilson_parity_small(wdl, dims, dagger):
    _check(wdl, dims, 0.1337, 0.0, dagger, 1, 100)


@pytest.mark.parametrize("mu", [0.05, -0.3])
@pytest.mark.parametrize("dagger", [False, True])
def test_twisted_mass_parity(wdl, mu, dagger):
    _check(wdl, (4, 2, 6, 4), 0.15, mu, dagger, 2, 200)


def test_batched_rhs_parity(wdl):
    _check(wdl, (4, 4, 4, 6), 0.12, 0.0, False, 5, 300)


def test_full_size_16x16x16x16(wdl):
    # the cfg of the benchmark: every site compared
    _check(wdl, (16, 16, 16, 16), 0.1366, 0.0, False, 1, 1001)


def test_large_lattice_sampled_sites(wdl):
    # 24^3 x 48: compare a few hundred sites against the per-site oracle
    import torch
    dims = (24, 24, 24, 48)
    v = L.volume(dims)
    rng = np.random.Generator(np.random.PCG64(5))
    U = L.gauge_field(dims, 0.5, 1004)
    psi = L.gaussian_spinor(dims, 1005)
    op = wdl.WilsonOperator(dims, cuda(U), 0.136)
    out = torch.empty(psi.size, dtype=torch.complex128, device="cuda:0")
    op.apply(cuda(psi), out)
    got = host(out).reshape(v, 4, 3)
    sites = np.concatenate([[0, v - 1, 23, 24 * 24 - 1, 24 * 24 * 24 - 1],
                            rng.integers(0, v, 300)])
    ref = dirac.apply_A_at_sites(U, psi, dims, 0.136, sites)
    err = np.abs(got[sites] - ref).max() / np.abs(ref).max()
    assert err <= TOL
    op.close()


def test_gamma5_hermiticity_on_gpu(wdl):
    import torch
    dims = (8, 4, 4, 8)
    U = L.gauge_field(dims, 0.5, 400)
    phi = L.gaussian_spinor(dims, 401)
    psi = L.gaussian_spinor(dims, 402)
    op = wdl.WilsonOperator(dims, cuda(U), 0.13)
    a = torch.empty(psi.size, dtype=torch.complex128, device="cuda:0")
    b = torch.empty_like(a)
    op.apply(cuda(psi), a)
    op.apply(cuda(phi), b, dagger=True)
    lhs = np.vdot(phi.ravel(), host(a))
    rhs = np.vdot(host(b), psi.ravel())
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)
    op.close()


def test_apply_is_deterministic(wdl):
    import torch
    dims = (8, 8, 8, 8)
    U = L.gauge_field(dims, 0.5, 500)
    psi = cuda(L.gaussian_spinor(dims, 501))
    op = wdl.WilsonOperator(dims, cuda(U), 0.13)
    a = torch.empty(psi.numel(), dtype=torch.complex128, device="cuda:0")
    b = torch.empty_like(a)
    op.apply(psi, a)
    op.apply(psi, b)
    assert torch.equal(a, b)
    op.close()


def test_apply_rejects_aliasing_and_host_pointers(wdl):
    dims = (2, 2, 2, 2)
    U = L.gauge_field(dims, 0.5, 600)
    op = wdl.WilsonOperator(dims, U, 0.1)     # host links: staged by wd_create
    x = cuda(L.gaussian_spinor(dims, 601))
    with pytest.raises(wdl.WdError) as e:
        op.apply(x, x)
    assert e.value.status == 1
    with pytest.raises(wdl.WdError):
        op.apply(L.gaussian_spinor(dims, 602), x)
    op.close()
