"""The tensor-core form of the tall-skinny product V Y (GMRES-DR's restart
V_{m+1} P_{k+1}, Sec. 1; the projection's x0 += V y, r0 -= (A V) y, Sec. 2)
against its definition.

The reference is the plain sum in extended precision (numpy longdouble, at
least 64 significand bits) on the host.  The bar follows from the method:
each FP64 value is held to 2^-55 of its row's (column's) largest magnitude
and the digit pairs left out weigh below 2^-56 of (row maximum) x (column
maximum), so every element is within 8 K 2^-53 x row max x column max of
the exact sum (K = 2 kv real terms) -- the same order as an FP64 dot
product's rounding.  Sizes span several 128-row tiles with a ragged tail,
one to three 24-column tiles, kv from 1 to the maximum 88.
"""
import numpy as np
import pytest

from .gpu_util import cuda, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wdl():
    import paper_0710_1988_gb300 as wdl
    wdl.lib()
    return wdl


def _rand(rng, shape, spread=0.0):
    z = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    if spread:
        z *= 10.0 ** rng.uniform(-spread, spread, size=shape)
    return z


def _reference(V, Y, IN, sign):
    ref = (Y.T.astype(np.clongdouble) @ V.astype(np.clongdouble)) * sign
    if IN is not None:
        ref = ref + IN.astype(np.clongdouble)
    return ref


def _bound(V, Y, kv):
    rowmax = np.maximum(np.abs(V.real), np.abs(V.imag)).max(axis=0)      # per element i
    colmax = np.maximum(np.abs(Y.real), np.abs(Y.imag)).max(axis=0)      # per column c
    return 8 * (2 * kv) * 2.0 ** -53 * colmax[:, None] * rowmax[None, :]


def _run(wdl, V, Y, IN, sign, tc):
    kv, n = V.shape
    ncol = Y.shape[1]
    out = cuda(np.full((ncol, n), np.nan + 0j)) if IN is None else cuda(IN.copy())
    wdl.tsgemm(cuda(V), kv, cuda(Y), ncol, out, IN=out if IN is not None else None,
               sign=sign, tensor_cores=tc)
    return host(out)


@pytest.mark.parametrize("kv,ncol,n,beta,sign,spread", [
    (81, 41, 1157, False, 1.0, 0.0),      # GMRES-DR(80,40) restart shape
    (61, 61, 700, False, 1.0, 0.0),       # (80,60): three column tiles
    (40, 10, 1300, True, 1.0, 0.0),       # x0 += V y for 10 right-hand sides
    (40, 10, 1300, True, -1.0, 0.0),      # r0 -= W y
    (88, 8, 257, True, -1.0, 3.0),        # largest kv, magnitudes over 6 decades
    (1, 24, 129, False, 1.0, 0.0),        # one row of V
    (17, 30, 128, True, 1.0, 8.0),        # exactly one row tile, 16 decades
])
def test_tensor_core_product_matches_definition(wdl, kv, ncol, n, beta, sign, spread):
    rng = np.random.Generator(np.random.PCG64(1000 * kv + ncol))
    V = _rand(rng, (kv, n), spread)
    Y = _rand(rng, (kv, ncol), spread)
    IN = _rand(rng, (ncol, n)) if beta else None
    got = _run(wdl, V, Y, IN, sign, True)
    ref = _reference(V, Y, IN, sign)
    err = np.abs(got - ref).astype(np.float64)
    bound = _bound(V, Y, kv)
    assert np.all(np.isfinite(got))
    assert np.all(err <= bound), float((err / bound).max())
    # deterministic: the same call gives the same bits
    assert np.array_equal(_run(wdl, V, Y, IN, sign, True), got)
    # and it is as accurate as the FP64 form overall
    fp = _run(wdl, V, Y, IN, sign, False)
    e_tc = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    e_fp = np.linalg.norm(fp - ref) / np.linalg.norm(ref)
    assert e_tc <= max(4 * e_fp, 1e-15), (e_tc, e_fp)


def test_zero_rows_columns_and_tiny_entries(wdl):
    rng = np.random.Generator(np.random.PCG64(77))
    kv, ncol, n = 33, 12, 300
    V = _rand(rng, (kv, n))
    V[:, 5] = 0                        # an all-zero row of the product
    V[3, 7] = 1e-300                   # a tiny entry beside normal ones
    V[:, 9] *= 1e-280                  # a row of tiny magnitude
    Y = _rand(rng, (kv, ncol))
    Y[:, 4] = 0                        # an all-zero column
    Y[2, 6] = 1e250                    # one huge entry in a column
    got = _run(wdl, V, Y, None, 1.0, True)
    ref = _reference(V, Y, None, 1.0)
    err = np.abs(got - ref).astype(np.float64)
    assert np.all(got[:, 5] == 0) and np.all(got[4, :] == 0)
    assert np.all(err <= _bound(V, Y, kv))


def test_solvers_agree_in_both_forms(wdl):
    """GMRES-DR(20,6) and D-BiCGStab(6) on 10 sources at 4^4 with the
    products on the tensor cores and in FP64: the same MVP counts, harmonic
    Ritz values and solutions to the solver tolerance."""
    from inputs import lattice as L
    from .gpu_util import kappa_c_table
    cfg = L.CONFIGS["wilson_4x4x4x4"]
    kappa = cfg.kappa_factor * kappa_c_table()[cfg.name]["kappa_c"]
    U = L.gauge_field(cfg.dims, cfg.eps, L.link_seed(cfg))
    b0 = L.source(cfg, 0).ravel()
    B = L.gaussian_spinor(cfg.dims, 3100, nrhs=10).reshape(10, -1)
    res = {}
    for tc in (True, False):
        op = wdl.WilsonOperator(cfg.dims, cuda(U), kappa)
        op.set_contraction(tc)
        import torch
        V = torch.zeros(cfg.k * b0.size, dtype=torch.complex128, device="cuda:0")
        x0 = cuda(np.zeros_like(b0))
        rc, st, _, theta = op.gmresdr(cuda(b0), x0, cfg.m, cfg.k, 1e-12, 10000, V_out=V)
        assert rc == 0
        defl = op.deflation(V, cfg.k)
        X = cuda(np.zeros_like(B))
        rc2, sts = op.dbicgstab(cuda(B), X, defl, tol=1e-12)
        assert rc2 == 0
        res[tc] = (st, theta, host(x0), [q["mvp"] for q in sts], host(X))
        defl.close()
        op.close()
    (s1, t1, x1, m1, X1), (s2, t2, x2, m2, X2) = res[True], res[False]
    assert s1["mvp"] == s2["mvp"] and s1["cycles"] == s2["cycles"]
    assert np.abs(np.sort(np.abs(t1)) - np.sort(np.abs(t2))).max() <= 1e-10 * np.abs(t2).max()
    assert np.linalg.norm(x1 - x2) <= 1e-9 * np.linalg.norm(x2)
    assert all(abs(a - b) <= 4 for a, b in zip(m1, m2))
    assert np.linalg.norm(X1 - X2) <= 1e-9 * np.linalg.norm(X2)
