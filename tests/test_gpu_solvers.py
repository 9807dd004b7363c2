"""Parity of the CUDA solvers (C ABI gmresdr_solve, dbicgstab_solve*) with
the CPU oracle, plus the properties that hold at any size.

Bars (FP64): iterate-by-iterate agreement with the oracle to <= 1e-10
relative for the first BiCGStab iterations (same arithmetic, different
rounding order); converged solutions within 1e-9 relative of an oracle
solve to 1e-14; every converged system's true residual, recomputed by the
oracle's operator, <= tol (with 5% slack for the recomputation itself).
"""
import math

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


@pytest.fixture(scope="module")
def cfg0():
    """4^4, eps = 0.3, kappa = 0.95 kappa_c, GMRES-DR(20,6), 3 Gaussian RHS."""
    cfg = L.CONFIGS["wilson_4x4x4x4"]
    kc = kappa_c_table()[cfg.name]["kappa_c"]
    kappa = cfg.kappa_factor * kc
    U = L.gauge_field(cfg.dims, cfg.eps, L.link_seed(cfg))
    A, g5 = oracle_ops(U, cfg.dims, kappa)
    b0 = L.source(cfg, 0).ravel()
    B = np.stack([L.source(cfg, j).ravel() for j in range(1, cfg.n_rhs + 1)])
    gd = krylov.gmresdr(A, b0, cfg.m, cfg.k, tol=cfg.tol)
    return dict(cfg=cfg, dims=cfg.dims, U=U, kappa=kappa, A=A, g5=g5, b0=b0, B=B, gd=gd)


def _op(wdl, c):
    return wdl.WilsonOperator(c["dims"], cuda(c["U"]), c["kappa"])


def _rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


# ------------------------------------------------------------------ BiCGStab

@pytest.mark.parametrize("iters", [1, 2, 5, 10, 20])
def test_bicgstab_iterates_match_oracle(wdl, cfg0, iters):
    op = _op(wdl, cfg0)
    b = cfg0["B"][0]
    X = cuda(np.zeros_like(b))
    rc, sts = op.dbicgstab(cuda(b), X, None, tol=1e-14, max_iter=iters)
    xo, so = krylov.bicgstab(cfg0["A"], b, tol=1e-14, max_iter=iters)
    assert sts[0]["iters"] == so.iters == iters
    assert sts[0]["mvp"] == so.mvp == 2 * iters
    assert _rel(host(X), xo) <= 1e-10
    assert abs(sts[0]["rel_res"] - so.history[-1]) <= 1e-8 * so.history[-1]
    op.close()


def test_bicgstab_converges_like_oracle(wdl, cfg0):
    op = _op(wdl, cfg0)
    b = cfg0["B"][1]
    X = cuda(np.zeros_like(b))
    rc, sts = op.dbicgstab(cuda(b), X, None, tol=1e-10)
    xo, so = krylov.bicgstab(cfg0["A"], b, tol=1e-10)
    xt, _ = krylov.bicgstab(cfg0["A"], b, tol=1e-14)
    s = sts[0]
    assert rc == 0 and s["converged"] == 1 and so.converged
    assert abs(s["iters"] - so.iters) <= 2
    assert s["true_rel_res"] <= 1e-10
    assert rel_residual(cfg0["U"], cfg0["dims"], cfg0["kappa"], host(X), b) <= 1.05e-10
    assert _rel(host(X), xt) <= 1e-9
    op.close()


# ------------------------------------------------------------------ GMRES-DR

def test_gmresdr_matches_oracle(wdl, cfg0):
    import torch
    c = cfg0
    cfg = c["cfg"]
    op = _op(wdl, c)
    n = c["b0"].size
    x = cuda(np.zeros_like(c["b0"]))
    V = torch.zeros(cfg.k * n, dtype=torch.complex128, device="cuda:0")
    rc, st, Hbar, theta = op.gmresdr(cuda(c["b0"]), x, cfg.m, cfg.k, cfg.tol, 100000, V_out=V)
    gd = c["gd"]
    assert rc == 0 and st["converged"] == 1
    assert st["mvp"] == gd.stats.mvp and st["cycles"] == gd.stats.cycles
    assert st["mvp"] == cfg.m + (cfg.m - cfg.k) * (st["cycles"] - 1)
    assert abs(st["rel_res"] - gd.stats.rel_res) <= 1e-4 * gd.stats.rel_res
    assert st["true_rel_res"] <= cfg.tol * 1.05
    assert _rel(host(x), gd.x) <= 1e-9
    # harmonic Ritz values: same set, same order
    assert np.abs(theta - gd.theta).max() <= 1e-8 * np.abs(gd.theta).max()
    # same deflation space (basis-independent): projector distance
    Vg = host(V).reshape(cfg.k, n)
    assert np.abs(Vg.conj() @ Vg.T - np.eye(cfg.k)).max() < 1e-12
    Vo = gd.V
    dist = np.linalg.norm(Vg.T - Vo.T @ (Vo.conj() @ Vg.T), 2)
    assert dist < 1e-7
    # Arnoldi relation through the returned Hbar: V^dagger A V = Hbar[:k]
    AV = np.stack([c["A"](v) for v in Vg])
    assert np.abs(Vg.conj() @ AV.T - Hbar[: cfg.k]).max() < 1e-11
    op.close()


def test_gmresdr_k0_is_restarted_gmres(wdl, cfg0):
    c = cfg0
    op = _op(wdl, c)
    x = cuda(np.zeros_like(c["b0"]))
    rc, st, _, _ = op.gmresdr(cuda(c["b0"]), x, 15, 0, 1e-9, 100000)
    r = krylov.gmresdr(c["A"], c["b0"], 15, 0, tol=1e-9)
    assert st["cycles"] == r.stats.cycles and st["mvp"] == r.stats.mvp == 15 * st["cycles"]
    assert _rel(host(x), r.x) <= 1e-8
    op.close()


def test_gmresdr_nonzero_guess(wdl, cfg0):
    c = cfg0
    op = _op(wdl, c)
    x0 = L.gaussian_spinor(c["dims"], 77).ravel() * 0.1
    x = cuda(x0)
    rc, st, _, _ = op.gmresdr(cuda(c["b0"]), x, 20, 6, 1e-10, 100000)
    r = krylov.gmresdr(c["A"], c["b0"], 20, 6, tol=1e-10, x0=x0)
    assert rc == 0 and st["mvp"] == r.stats.mvp and st["mvp_extra"] == 2
    assert _rel(host(x), r.x) <= 1e-9
    op.close()


def test_gmresdr_lucky_breakdown_gives_exact_solution(wdl):
    # n = 24: the Krylov space is exhausted before m = 24 steps
    dims = (1, 1, 1, 2)
    U = L.gauge_field(dims, 0.5, 88)
    A, _ = oracle_ops(U, dims, 0.1)
    from oracle import dirac
    Ad = dirac.dense_A(U, dims, 0.1)
    b = L.gaussian_spinor(dims, 89).ravel()
    op = wdl.WilsonOperator(dims, cuda(U), 0.1)
    x = cuda(np.zeros_like(b))
    rc, st, _, _ = op.gmresdr(cuda(b), x, 24, 4, 1e-12, 1000)
    assert rc == 0 and st["converged"] == 1 and st["cycles"] == 1
    assert _rel(host(x), np.linalg.solve(Ad, b)) < 1e-10
    op.close()


def test_gmresdr_budget_exhausted(wdl, cfg0):
    c = cfg0
    op = _op(wdl, c)
    x = cuda(np.zeros_like(c["b0"]))
    rc, st, _, _ = op.gmresdr(cuda(c["b0"]), x, 20, 6, 1e-13, 40)
    assert rc == 2 and st["converged"] == 0 and st["mvp"] <= 40
    op.close()


# ------------------------------------------------------------------ D-BiCGStab (Sec. 2)

@pytest.mark.parametrize("iters", [1, 4, 12])
def test_projection_and_iterates_match_oracle(wdl, cfg0, iters):
    # same V on both sides: the projection and the first iterations agree
    c = cfg0
    cfg = c["cfg"]
    op = _op(wdl, c)
    V = cuda(c["gd"].V)
    defl = op.deflation(V, cfg.k)
    B = c["B"]
    X = cuda(np.zeros_like(B))
    rc, sts = op.dbicgstab(cuda(B), X, defl, tol=1e-14, max_iter=iters)
    for j in range(B.shape[0]):
        xo, so = krylov.dbicgstab(c["A"], B[j], c["gd"].V, tol=1e-14, max_iter=iters,
                                  gamma5=c["g5"])
        assert sts[j]["iters"] == so.iters
        assert _rel(host(X)[j], xo) <= 1e-10
    defl.close()
    op.close()


def test_dbicgstab_pipeline_on_gpu(wdl, cfg0):
    """GMRES-DR on the GPU, then D-BiCGStab(6) on 3 more RHS, all batched."""
    import torch
    c = cfg0
    cfg = c["cfg"]
    op = _op(wdl, c)
    n = c["b0"].size
    V = torch.zeros(cfg.k * n, dtype=torch.complex128, device="cuda:0")
    op.gmresdr(cuda(c["b0"]), cuda(np.zeros_like(c["b0"])), cfg.m, cfg.k, cfg.tol, 100000,
               V_out=V)
    defl = op.deflation(V, cfg.k)
    B = c["B"]
    X = cuda(np.zeros_like(B))
    rc, sts = op.dbicgstab(cuda(B), X, defl, tol=cfg.tol)
    assert rc == 0
    Xh = host(X)
    for j in range(B.shape[0]):
        assert sts[j]["converged"] == 1 and sts[j]["mvp"] % 2 == 0
        assert rel_residual(c["U"], c["dims"], c["kappa"], Xh[j], B[j]) <= 1.05 * cfg.tol
        xt, _ = krylov.bicgstab(c["A"], B[j], tol=1e-14)
        assert _rel(Xh[j], xt) <= 1e-9
        xo, so = krylov.dbicgstab(c["A"], B[j], c["gd"].V, tol=cfg.tol, gamma5=c["g5"])
        assert abs(sts[j]["iters"] - so.iters) <= 3
    defl.close()
    op.close()


def test_host_pointer_path_matches_device_path(wdl, cfg0):
    c = cfg0
    op = _op(wdl, c)
    B = c["B"][:2].copy()
    Xh = np.zeros_like(B)
    rc1, s1 = op.dbicgstab(B, Xh, None, tol=1e-10)
    Xd = cuda(np.zeros_like(B))
    rc2, s2 = op.dbicgstab(cuda(B), Xd, None, tol=1e-10)
    assert np.array_equal(Xh, host(Xd))
    assert [s["iters"] for s in s1] == [s["iters"] for s in s2]
    op.close()


def test_solver_is_deterministic(wdl, cfg0):
    c = cfg0
    op = _op(wdl, c)
    B = cuda(c["B"])
    X1 = cuda(np.zeros_like(c["B"]))
    X2 = cuda(np.zeros_like(c["B"]))
    op.dbicgstab(B, X1, None, tol=1e-10)
    op.dbicgstab(B, X2, None, tol=1e-10)
    import torch
    assert torch.equal(X1, X2)
    op.close()


def test_mixed_systems_in_one_batch(wdl, cfg0):
    # a zero right-hand side, one inside the deflation space, and a generic one
    c = cfg0
    cfg = c["cfg"]
    op = _op(wdl, c)
    Vo = c["gd"].V
    defl = op.deflation(cuda(Vo), cfg.k)
    inside = np.stack([c["A"](v) for v in Vo]).T @ np.arange(1, cfg.k + 1)  # A V y
    B = np.stack([np.zeros_like(c["b0"]), inside, c["B"][2]])
    X = cuda(np.zeros_like(B))
    rc, sts = op.dbicgstab(cuda(B), X, defl, tol=1e-10)
    assert rc == 0 and all(s["converged"] for s in sts)
    assert np.all(host(X)[0] == 0) and sts[0]["iters"] == 0
    assert sts[1]["iters"] == 0          # solved by the projection alone
    assert sts[2]["iters"] > 5
    defl.close()
    op.close()


def test_not_converged_reports_and_writes_x(wdl, cfg0):
    c = cfg0
    op = _op(wdl, c)
    b = c["B"][0]
    X = cuda(np.zeros_like(b))
    rc, sts = op.dbicgstab(cuda(b), X, None, tol=1e-12, max_iter=3)
    assert rc == 2 and sts[0]["converged"] == 0 and sts[0]["iters"] == 3
    assert np.linalg.norm(host(X)) > 0
    assert math.isfinite(sts[0]["true_rel_res"]) and sts[0]["true_rel_res"] < 1
    op.close()


def test_singular_projection_is_reported(wdl, cfg0):
    c = cfg0
    op = _op(wdl, c)
    v = c["gd"].V[0]
    V = cuda(np.stack([v, v]))
    with pytest.raises(wdl.WdError) as e:
        op.deflation(V, 2)
    assert e.value.status == 4
    op.close()


def test_explicit_left_basis_equals_gamma5_default(wdl, cfg0):
    c = cfg0
    cfg = c["cfg"]
    op = _op(wdl, c)
    Vo = c["gd"].V
    Uo = np.stack([c["g5"](v) for v in Vo])
    B = cuda(c["B"][:1])
    X1 = cuda(np.zeros_like(c["B"][:1]))
    X2 = cuda(np.zeros_like(c["B"][:1]))
    op.dbicgstab_oneshot(B, X1, V=cuda(Vo), k=cfg.k, tol=1e-10)
    op.dbicgstab_oneshot(B, X2, V=cuda(Vo), U=cuda(Uo), k=cfg.k, tol=1e-10)
    assert _rel(host(X1), host(X2)) <= 1e-12
    op.close()


# ------------------------------------------------------------------ full size

def test_full_size_16x16x16x16_pipeline(wdl):
    """The benchmark workload: GMRES-DR(80,40) on a Z4 source to 1e-10, then
    D-BiCGStab(40) on 10 Z4 sources, every true residual checked; two of them
    recomputed by the oracle's operator.

    On this synthetic gauge field (eps = 0.5, 0.99 kappa_c) the 40 smallest
    harmonic Ritz values are not isolated from the rest of the spectrum, and
    deflating them changes the BiCGStab product count by about 1% (the
    oracle gives the same counts); the Sec. 3 trend is therefore checked as
    "deflation, and more accurate eigenvectors, never cost products"."""
    import torch
    cfg = L.CONFIGS["wilson_16x16x16x16"]
    kc = kappa_c_table()[cfg.name]["kappa_c"]
    kappa = cfg.kappa_factor * kc
    U = L.gauge_field(cfg.dims, cfg.eps, L.link_seed(cfg))
    op = wdl.WilsonOperator(cfg.dims, cuda(U), kappa)
    n = 12 * L.volume(cfg.dims)
    b0 = cuda(L.source(cfg, 0))
    V = torch.zeros(cfg.k * n, dtype=torch.complex128, device="cuda:0")
    rc, st, _, theta = op.gmresdr(b0, torch.zeros_like(b0), cfg.m, cfg.k, cfg.tol, 200000,
                                  V_out=V)
    assert rc == 0 and st["true_rel_res"] <= 1.05 * cfg.tol
    defl = op.deflation(V, cfg.k)
    Bh = np.stack([L.source(cfg, j) for j in range(1, cfg.n_rhs + 1)])
    X = cuda(np.zeros_like(Bh))
    rc, sts = op.dbicgstab(cuda(Bh), X, defl, tol=cfg.tol)
    assert rc == 0 and all(s["converged"] and s["true_rel_res"] <= cfg.tol for s in sts)
    Xh = host(X)
    for j in (0, cfg.n_rhs - 1):
        assert rel_residual(U, cfg.dims, kappa, Xh[j], Bh[j]) <= 1.05 * cfg.tol
    X0 = cuda(np.zeros_like(Bh[:1]))
    rc, s0 = op.dbicgstab(cuda(Bh[:1]), X0, None, tol=cfg.tol)
    assert sts[0]["mvp"] <= s0[0]["mvp"] * 1.05
    V3 = torch.zeros_like(V)
    op.gmresdr(b0, torch.zeros_like(b0), cfg.m, cfg.k, 1e-14, 400000, V_out=V3)
    defl3 = op.deflation(V3, cfg.k)
    X3 = cuda(np.zeros_like(Bh[:1]))
    rc, s3 = op.dbicgstab(cuda(Bh[:1]), X3, defl3, tol=cfg.tol)
    assert rc == 0 and s3[0]["mvp"] <= s0[0]["mvp"] * 1.02
    assert s3[0]["mvp"] <= sts[0]["mvp"] * 1.02
    defl3.close()
    defl.close()
    op.close()
