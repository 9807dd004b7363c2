"""Full-size parity of the growth rows, at the sizes `bench.py --config` times.

The oracle cannot solve these lattices in a test's time, so the checks are
properties that hold at any size, evaluated by the oracle:
 * every returned solution has true relative residual <= 1.05 tol under the
   oracle's own operator (whole lattice, or site by site where the lattice is
   too large for a whole-lattice numpy apply);
 * kernel outputs at sampled sites equal the oracle's per-site formulas
   (`dirac.apply_A_at_sites`, `grad.link_force_at`).
Bars: FP32 apply 2e-6 of the largest sampled entry (as in test_gpu_mixed);
FP64 link force 1e-12 of the largest sampled entry.
"""
import numpy as np
import pytest

from inputs import lattice as L
from oracle import dirac, grad

from .gpu_util import cuda, host, kappa_c_table, rel_residual

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wdl():
    import paper_0710_1988_gb300 as wdl
    wdl.lib()
    return wdl


def _kappa(cfg):
    table = kappa_c_table()
    if cfg.name not in table:
        pytest.skip(f"kappa_c of {cfg.name} not recorded")
    return cfg.kappa_factor * table[cfg.name]["kappa_c"]


@pytest.mark.parametrize("bits", [32, 16])
def test_mixed_20x20x20x32(wdl, bits):
    import torch
    cfg = L.CONFIGS["wilson_20x20x20x32_mixed"]
    kappa = _kappa(cfg)
    U = L.gauge_field(cfg.dims, cfg.eps, L.link_seed(cfg))
    op = wdl.WilsonOperator(cfg.dims, cuda(U), kappa)
    op.set_mixed_storage(bits)
    Bh = np.stack([L.source(cfg, j) for j in (1, 2)]).reshape(2, -1)
    X = cuda(np.zeros_like(Bh))
    rc, sts = op.dbicgstab_mixed(cuda(Bh), X, None, tol=cfg.tol, reliable_every=50)
    assert rc == 0 and all(s["converged"] and s["true_rel_res"] <= cfg.tol for s in sts)
    Xh = host(X)
    for j in range(2):
        assert rel_residual(U, cfg.dims, kappa, Xh[j], Bh[j]) <= 1.05 * cfg.tol
    # the FP32 kernel at sampled sites against the oracle's per-site walker
    if bits == 32:
        v = L.volume(cfg.dims)
        psi = L.gaussian_spinor(cfg.dims, 2300)
        out = torch.empty(psi.size, dtype=torch.complex128, device="cuda:0")
        op.apply_f32(cuda(psi), out)
        got = host(out).reshape(v, 4, 3)
        sites = np.random.Generator(np.random.PCG64(5)).choice(v, 24, replace=False)
        ref = dirac.apply_A_at_sites(U, psi, cfg.dims, kappa, sites)
        assert np.abs(got[sites] - ref).max() <= 2e-6 * np.abs(ref).max()
    op.close()


def test_twisted_shifts_24x24x24x48(wdl):
    cfg = L.CONFIGS["twisted_24x24x24x48"]
    kappa = _kappa(cfg)
    U = L.gauge_field(cfg.dims, cfg.eps, L.link_seed(cfg))
    op = wdl.WilsonOperator(cfg.dims, cuda(U), kappa)
    B = L.source(cfg, 0).reshape(1, -1)
    mus = [0.064, 0.032]
    X = cuda(np.zeros((len(mus), B.shape[1]), dtype=np.complex128))
    rc, sts = op.multishift(cuda(B), X, mus, tol=cfg.tol, project=True, mixed=True)
    assert rc == 0
    Xh = host(X)
    for i, mu in enumerate(mus):
        assert sts[i][0]["converged"] and sts[i][0]["true_rel_res"] <= cfg.tol
        assert rel_residual(U, cfg.dims, kappa, Xh[i], B[0], mu=mu) <= 1.05 * cfg.tol
    op.close()


def test_gradients_32x32x32x64(wdl):
    import torch
    cfg = L.CONFIGS["grad_32x32x32x64"]
    kappa = _kappa(cfg)
    U = L.gauge_field(cfg.dims, cfg.eps, L.link_seed(cfg))
    v = L.volume(cfg.dims)
    op = wdl.WilsonOperator(cfg.dims, cuda(U), kappa)
    b = L.gaussian_spinor(cfg.dims, L.rhs_seed(cfg, 0))
    eta = L.gaussian_spinor(cfg.dims, L.rhs_seed(cfg, 1))
    x = cuda(np.zeros(b.size, dtype=np.complex128))
    lam = cuda(np.zeros(b.size, dtype=np.complex128))
    rc, st = op.dbicgstab(cuda(b.reshape(1, -1)), x, None, tol=cfg.tol)
    assert rc == 0 and st[0]["converged"]
    rc, st = op.adjoint_solve(cuda(eta.reshape(1, -1)), lam, None, tol=cfg.tol)
    assert rc == 0 and st[0]["converged"]
    force = torch.empty((v, 4, 8), dtype=torch.float64, device="cuda:0")
    op.gradients(lam, x, force=force, want_dkappa=False)
    xh = host(x).reshape(v, 4, 3)
    lh = host(lam).reshape(v, 4, 3)
    fh = host(force)
    rng = np.random.Generator(np.random.PCG64(6))
    sites = rng.choice(v, 12, replace=False)
    # x solves A x = b and lam solves A^dagger lam = eta, site by site:
    # every site's residual is bounded by the global one
    r = dirac.apply_A_at_sites(U, xh, cfg.dims, kappa, sites) - b[sites]
    assert np.sqrt((np.abs(r) ** 2).sum(axis=(1, 2))).max() <= 1.05 * cfg.tol * np.linalg.norm(b)
    g5l = dirac.gamma5(lh)            # A^dagger = gamma5 A gamma5 (mu = 0)
    r = dirac.gamma5(dirac.apply_A_at_sites(U, g5l, cfg.dims, kappa, sites)) - eta[sites]
    assert np.sqrt((np.abs(r) ** 2).sum(axis=(1, 2))).max() <= 1.05 * cfg.tol * np.linalg.norm(eta)
    # the force kernel at sampled links against the oracle's per-link formula
    pairs = [(int(s), int(m)) for s, m in zip(rng.choice(v, 16, replace=False), rng.integers(0, 4, 16))]
    ref = grad.link_force_at(U, cfg.dims, kappa, lh, xh, pairs)
    got = np.stack([fh[s, m] for s, m in pairs])
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    op.close()
