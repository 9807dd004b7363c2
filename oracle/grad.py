"""Gradients of L = Re(eta^dagger x), x = A^{-1} b (oracle, FP64).

Not in the paper: this is the differentiation growth line of the workload.
With dL = Re(g^dagger dx) and dx = A^{-1} (db - dA x), the adjoint vector
lambda = A^{-dagger} g gives

  dL/db     = lambda                       (dL = Re(lambda^dagger db))
  dL/dkappa = Re(lambda^dagger D x)        (A = 1 - kappa D + i mu gamma5)
  dL/domega_{s,mu,a} = kappa Re(lambda^dagger (dD/domega) x)

for links moved as U_mu(s) -> exp(i omega_a T_a) U_mu(s), T_a = lambda_a / 2
(Gell-Mann).  U_mu(s) enters D in the forward hop of site s and, as its
adjoint, in the backward hop of site s+mu, so

  dL/domega_{s,mu,a} = -kappa Im tr[T_a (W1 - W2)],
  W1 = U_mu(s) sum_spin phi lambda(s)^dagger,      phi = (1 - gamma_mu) x(s+mu),
  W2 = sum_spin psi lambda(s+mu)^dagger U_mu(s)^dagger,  psi = (1 + gamma_mu) x(s).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
from __future__ import annotations

import numpy as np

from . import dirac

T = None


def _generators():
    l = np.zeros((8, 3, 3), dtype=np.complex128)
    l[0][0, 1] = l[0][1, 0] = 1
    l[1][0, 1], l[1][1, 0] = -1j, 1j
    l[2][0, 0], l[2][1, 1] = 1, -1
    l[3][0, 2] = l[3][2, 0] = 1
    l[4][0, 2], l[4][2, 0] = -1j, 1j
    l[5][1, 2] = l[5][2, 1] = 1
    l[6][1, 2], l[6][2, 1] = -1j, 1j
    l[7][0, 0] = l[7][1, 1] = 1 / np.sqrt(3)
    l[7][2, 2] = -2 / np.sqrt(3)
    return l / 2.0


T = _generators()        # T_a = lambda_a / 2


def link_force(links, dims, kappa, lam, x):
    """dL/domega, shape (V, 4, 8), for adjoint lam and solution x (V, 4, 3)."""
    v = links.shape[0]
    shape = dirac._shape(dims)
    u = links.reshape(shape + (4, 3, 3))
    lf = lam.reshape(shape + (4, 3))
    xf = x.reshape(shape + (4, 3))
    out = np.zeros(shape + (4, 8))
    for mu in range(4):
        ax = dirac.AXIS[mu]
        umu = u[..., mu, :, :]
        phi = (dirac.ONE4 - dirac.GAMMA[mu]) @ np.roll(xf, -1, axis=ax)   # from x(s+mu)
        psi = (dirac.ONE4 + dirac.GAMMA[mu]) @ xf                         # from x(s)
        lam_up = np.roll(lf, -1, axis=ax)                                 # lambda(s+mu)
        # sum over spin of colour outer products  phi_c conj(lambda_d)
        o1 = np.einsum("...sc,...sd->...cd", phi, np.conj(lf))
        o2 = np.einsum("...sc,...sd->...cd", psi, np.conj(lam_up))
        w1 = umu @ o1
        w2 = o2 @ np.conj(np.swapaxes(umu, -1, -2))
        m = w1 - w2
        tr = np.einsum("aij,...ji->...a", T, m)
        out[..., mu, :] = -kappa * tr.imag
    return out.reshape(v, 4, 8)


def link_force_at(links, dims, kappa, lam, x, pairs):
    """dL/domega_{s,mu,a} for a few (s, mu) pairs, shape (len(pairs), 8): the
    same formula as `link_force`, walked site by site through explicit
    coordinates, so that a full-size result can be checked one link at a time."""
    out = np.zeros((len(pairs), 8))
    for i, (s, mu) in enumerate(pairs):
        c = list(dirac.site_coords(dims, int(s)))
        c[mu] += 1
        sp = dirac.site_index(dims, *c)
        u = links[s, mu]
        phi = (dirac.ONE4 - dirac.GAMMA[mu]) @ x[sp]          # spin x colour
        psi = (dirac.ONE4 + dirac.GAMMA[mu]) @ x[s]
        o1 = phi.T @ np.conj(lam[s])                          # sum over spin
        o2 = psi.T @ np.conj(lam[sp])
        m = u @ o1 - o2 @ np.conj(u.T)
        out[i] = -kappa * np.array([np.trace(T[a] @ m).imag for a in range(8)])
    return out


def gradients(links, dims, kappa, b, eta, solve, solve_dagger, mu: float = 0.0):
    """(L, dL/db, dL/dkappa, dL/domega) for L = Re(eta^dagger A^{-1} b).

    ``solve(rhs)`` returns A^{-1} rhs and ``solve_dagger(rhs)`` A^{-dagger} rhs
    (flat complex vectors)."""
    v = links.shape[0]
    x = solve(b.ravel())
    L = float(np.vdot(eta.ravel(), x).real)
    lam = solve_dagger(eta.ravel())
    dx = dirac.hopping(links, x.reshape(v, 4, 3), dims).ravel()
    dkappa = float(np.vdot(lam, dx).real)
    f = link_force(links, dims, kappa, lam.reshape(v, 4, 3), x.reshape(v, 4, 3))
    return L, lam, dkappa, f


def move_links(links, omega, h):
    """U_mu(s) -> exp(i h omega_a T_a) U_mu(s) for omega of shape (V, 4, 8)."""
    herm = np.einsum("sma,aij->smij", omega, T) * h
    w, q = np.linalg.eigh(herm)
    ex = np.einsum("...ij,...j,...kj->...ik", q, np.exp(1j * w), np.conj(q))
    return ex @ links
