"""Pins for the oracle's gradients of L = Re(eta^dagger A^{-1} b): central
finite differences (h = 1e-6) on a 2x2x2x4 lattice with dense LU solves."""
import numpy as np
import pytest

from inputs import lattice as L
from oracle import dirac, grad

DIMS = (2, 2, 2, 4)


@pytest.fixture(scope="module")
def prob():
    U = L.gauge_field(DIMS, 0.5, 4100)
    kap = 0.12
    b = L.gaussian_spinor(DIMS, 4101).ravel()
    eta = L.gaussian_spinor(DIMS, 4102).ravel()
    return U, kap, b, eta


def _loss(U, kap, b, eta, mu=0.0):
    A = dirac.dense_A(U, DIMS, kap, mu)
    return float(np.vdot(eta, np.linalg.solve(A, b)).real)


def _grads(U, kap, b, eta, mu=0.0):
    A = dirac.dense_A(U, DIMS, kap, mu)
    v = U.shape[0]

    def solve_dagger(r):   # A^{-dagger} = gamma5 A(-mu)^{-1} gamma5
        g5 = lambda z: dirac.gamma5(z.reshape(v, 4, 3)).ravel()
        Am = dirac.dense_A(U, DIMS, kap, -mu)
        return g5(np.linalg.solve(Am, g5(r)))
    return grad.gradients(U, DIMS, kap, b, eta, lambda r: np.linalg.solve(A, r), solve_dagger, mu)


def test_adjoint_solve_is_dagger_solve(prob):
    U, kap, b, eta = prob
    A = dirac.dense_A(U, DIMS, kap)
    _, lam, _, _ = _grads(U, kap, b, eta)
    assert np.abs(lam - np.linalg.solve(A.conj().T, eta)).max() < 1e-12 * np.abs(lam).max()


def test_grad_b_finite_difference(prob):
    U, kap, b, eta = prob
    _, lam, _, _ = _grads(U, kap, b, eta)
    d = L.gaussian_spinor(DIMS, 4103).ravel()
    h = 1e-6
    fd = (_loss(U, kap, b + h * d, eta) - _loss(U, kap, b - h * d, eta)) / (2 * h)
    assert abs(fd - np.vdot(lam, d).real) <= 1e-6 * abs(fd)


def test_grad_kappa_finite_difference(prob):
    U, kap, b, eta = prob
    _, _, dk, _ = _grads(U, kap, b, eta)
    h = 1e-6
    fd = (_loss(U, kap + h, b, eta) - _loss(U, kap - h, b, eta)) / (2 * h)
    assert abs(fd - dk) <= 1e-6 * abs(fd)


@pytest.mark.parametrize("mu", [0.0, 0.07])
def test_link_force_finite_difference(prob, mu):
    U, kap, b, eta = prob
    _, _, _, f = _grads(U, kap, b, eta, mu)
    rng = np.random.Generator(np.random.PCG64(4104))
    om = rng.standard_normal(f.shape)
    h = 1e-6
    lp = _loss(grad.move_links(U, om, h), kap, b, eta, mu)
    lm = _loss(grad.move_links(U, om, -h), kap, b, eta, mu)
    fd = (lp - lm) / (2 * h)
    assert abs(fd - np.sum(f * om)) <= 1e-6 * abs(fd)
    # one single component as well
    e = np.zeros_like(om)
    e[3, 2, 5] = 1.0
    fd1 = (_loss(grad.move_links(U, e, h), kap, b, eta, mu)
           - _loss(grad.move_links(U, e, -h), kap, b, eta, mu)) / (2 * h)
    assert abs(fd1 - f[3, 2, 5]) <= 1e-6 * max(abs(fd1), 1e-3)


def test_link_force_at_matches_the_array_form():
    """The per-link walker used for full-size checks equals the rolled-array
    form on a lattice with unequal extents (every (s, mu) of it)."""
    dims = (2, 3, 4, 2)
    v = L.volume(dims)
    U = L.gauge_field(dims, 0.7, 91)
    x = L.gaussian_spinor(dims, 92)
    lam = L.gaussian_spinor(dims, 93)
    full = grad.link_force(U, dims, 0.13, lam, x)
    pairs = [(s, mu) for s in range(v) for mu in range(4)]
    at = grad.link_force_at(U, dims, 0.13, lam, x, pairs)
    assert np.abs(at - full.reshape(-1, 8)).max() <= 1e-13 * np.abs(full).max()
