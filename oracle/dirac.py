"""Wilson-Dirac operator on a periodic 4-D lattice (oracle, FP64).

The paper names the Wilson matrix A_W and uses only its gamma5-hermiticity
gamma5 A_W gamma5 = A_W^dagger (Sec. 1); it never writes the stencil out.
This file takes the standard hopping-parameter form

  (D psi)(x) = sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu)
                      + (1 + gamma_mu) U_mu(x-mu)^dagger psi(x-mu) ]
  A = 1 - kappa*D + i*mu*gamma5            (mu = 0: plain Wilson)

with periodic boundaries in all four directions and the chiral gamma basis

  gamma_k = [[0, -i sigma_k], [i sigma_k, 0]]  (k = 1, 2, 3 for x, y, z)
  gamma_4 = [[0, 1], [1, 0]]                   (t)
  gamma5  = gamma_1 gamma_2 gamma_3 gamma_4 = diag(1, 1, -1, -1).

The twisted term i*mu*gamma5 is the Sec. 4 twisted-mass operator with the
twist written as the workload defines it (no 2*kappa factor).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Arrays: links U[s, mu, a, b], spinors psi[s, sigma, a], complex128, with the
site index s = x + Lx*(y + Ly*(z + Lz*t)).  Internally reshaped to
(Lt, Lz, Ly, Lx, ...) so that direction mu rolls numpy axis AXIS[mu].
"""
from __future__ import annotations

import numpy as np

# -------------------------------------------------------------- gammas

SIGMA = np.array([[[0, 1], [1, 0]],
                  [[0, -1j], [1j, 0]],
                  [[1, 0], [0, -1]]], dtype=np.complex128)
_I2 = np.eye(2, dtype=np.complex128)
_Z2 = np.zeros((2, 2), dtype=np.complex128)


def _block(a, b, c, d):
    return np.block([[a, b], [c, d]])


GAMMA = np.stack(
    [_block(_Z2, -1j * SIGMA[k], 1j * SIGMA[k], _Z2) for k in range(3)]
    + [_block(_Z2, _I2, _I2, _Z2)])          # GAMMA[mu], mu = x, y, z, t
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
ONE4 = np.eye(4, dtype=np.complex128)

AXIS = (3, 2, 1, 0)      # numpy axis of (Lt, Lz, Ly, Lx) rolled by mu


def _shape(dims):
    lx, ly, lz, lt = dims
    return (lt, lz, ly, lx)


def _as_field(a, dims, tail):
    return a.reshape(_shape(dims) + tail)


# -------------------------------------------------------------- operator

def hopping(links: np.ndarray, psi: np.ndarray, dims) -> np.ndarray:
    """D psi, the 8-neighbour hopping term (no diagonal)."""
    u = _as_field(links, dims, (4, 3, 3))
    f = _as_field(psi, dims, (4, 3))
    out = np.zeros_like(f)
    for mu in range(4):
        ax = AXIS[mu]
        umu = u[..., mu, :, :]
        # forward: (1 - gamma_mu) U_mu(x) psi(x + mu)
        fwd = np.roll(f, -1, axis=ax)                     # psi(x + mu)
        col = fwd @ np.swapaxes(umu, -1, -2)              # U psi, per spin
        out += (ONE4 - GAMMA[mu]) @ col
        # backward: (1 + gamma_mu) U_mu(x - mu)^dagger psi(x - mu)
        y = f @ np.conj(umu)                              # U^dagger psi at x
        out += (ONE4 + GAMMA[mu]) @ np.roll(y, 1, axis=ax)
    return out.reshape(psi.shape)


def gamma5(psi: np.ndarray) -> np.ndarray:
    """gamma5 psi for psi[..., 4, 3]."""
    return np.einsum("st,...ta->...sa", GAMMA5, psi)


def apply_A(links, psi, dims, kappa: float, mu: float = 0.0) -> np.ndarray:
    """A psi = psi - kappa * D psi + i*mu*gamma5 psi."""
    out = psi - kappa * hopping(links, psi, dims)
    if mu != 0.0:
        out = out + 1j * mu * gamma5(psi)
    return out


def apply_A_dagger(links, psi, dims, kappa: float, mu: float = 0.0):
    """A^dagger psi = gamma5 A(-mu) gamma5 psi (gamma5-hermiticity, Sec. 1)."""
    return gamma5(apply_A(links, gamma5(psi), dims, kappa, -mu))


def site_index(dims, x, y, z, t) -> int:
    lx, ly, lz, lt = dims
    return (x % lx) + lx * ((y % ly) + ly * ((z % lz) + lz * (t % lt)))


def site_coords(dims, s: int):
    lx, ly, lz, lt = dims
    return (s % lx, (s // lx) % ly, (s // (lx * ly)) % lz, s // (lx * ly * lz))


def apply_A_at_sites(links, psi, dims, kappa, sites, mu: float = 0.0):
    """(A psi)(s) for a few sites s, straight from the definition.

    Used to check a full-size result one site at a time; walks the
    neighbours through explicit coordinates instead of array rolls.
    """
    out = np.zeros((len(sites), 4, 3), dtype=np.complex128)
    for i, s in enumerate(sites):
        c = list(site_coords(dims, int(s)))
        acc = np.zeros((4, 3), dtype=np.complex128)
        for m in range(4):
            up = list(c)
            up[m] += 1
            dn = list(c)
            dn[m] -= 1
            sp = site_index(dims, *up)
            sm = site_index(dims, *dn)
            acc += (ONE4 - GAMMA[m]) @ (psi[sp] @ links[s, m].T)
            acc += (ONE4 + GAMMA[m]) @ (psi[sm] @ np.conj(links[sm, m]))
        out[i] = psi[s] - kappa * acc + 1j * mu * (GAMMA5 @ psi[s])
    return out


def dense_A(links, dims, kappa, mu: float = 0.0) -> np.ndarray:
    """The n x n matrix of A (n = 12 V), column by column; small lattices only."""
    v = links.shape[0]
    n = 12 * v
    a = np.zeros((n, n), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for j in range(n):
        e[:] = 0
        e[j] = 1
        a[:, j] = apply_A(links, e.reshape(v, 4, 3), dims, kappa, mu).ravel()
    return a


def dense_D(links, dims) -> np.ndarray:
    """The n x n hopping matrix D (A = 1 - kappa*D at mu = 0)."""
    n = 12 * links.shape[0]
    return (np.eye(n) - dense_A(links, dims, 1.0)).astype(np.complex128)
