"""Even-odd (Schur complement) preconditioned operator (oracle, FP64).

Sec. 3 solves "the even-odd preconditioned system" (and Sec. 4 its twisted
mass form); the paper does not write it out.  With sites split by parity
(x + y + z + t) mod 2, the hopping term only connects opposite parities:

  A = [[A_ee, -kappa D_eo], [-kappa D_oe, A_oo]],   A_ee = A_oo = 1 + i mu gamma5,

and A x = b is equivalent to the Schur system on the even sites

  A_hat x_e = b_hat,   A_hat = A_ee - kappa^2 D_eo A_oo^{-1} D_oe,
  b_hat = b_e + kappa D_eo A_oo^{-1} b_o,
  x_o = A_oo^{-1} (b_o + kappa D_oe x_e),

with A_oo^{-1} = (1 - i mu gamma5) / (1 + mu^2).

Half-lattice vectors hold the sites of one parity in increasing site order;
for even Lx that is compact index s // 2 (the two sites of every x-pair have
opposite parities).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
from __future__ import annotations

import numpy as np

from . import dirac


def parity(dims) -> np.ndarray:
    lx, ly, lz, lt = dims
    s = np.arange(lx * ly * lz * lt)
    x = s % lx
    y = (s // lx) % ly
    z = (s // (lx * ly)) % lz
    t = s // (lx * ly * lz)
    return (x + y + z + t) % 2


def sites(dims, p: int) -> np.ndarray:
    """Full site indices of parity p, increasing."""
    return np.nonzero(parity(dims) == p)[0]


def embed(v_half, dims, p: int) -> np.ndarray:
    """Half-lattice spinor of parity p -> full spinor with zeros elsewhere."""
    vol = int(np.prod(dims))
    out = np.zeros((vol, 4, 3), dtype=np.complex128)
    out[sites(dims, p)] = v_half.reshape(-1, 4, 3)
    return out


def restrict(v_full, dims, p: int) -> np.ndarray:
    return v_full.reshape(-1, 4, 3)[sites(dims, p)]


def hop(links, dims, v_half, p_in: int) -> np.ndarray:
    """D restricted to parity p_in -> 1 - p_in (D_{1-p, p} v)."""
    full = dirac.hopping(links, embed(v_half, dims, p_in), dims)
    return restrict(full, dims, 1 - p_in)


def aoo_inv(v, mu: float) -> np.ndarray:
    return (v - 1j * mu * dirac.gamma5(v.reshape(-1, 4, 3))) / (1.0 + mu * mu)


def schur_apply(links, dims, kappa: float, mu: float, xe) -> np.ndarray:
    """A_hat x_e = (1 + i mu gamma5) x_e - kappa^2 D_eo A_oo^{-1} D_oe x_e."""
    xe = xe.reshape(-1, 4, 3)
    t = aoo_inv(hop(links, dims, xe, 0), mu)
    return xe + 1j * mu * dirac.gamma5(xe) - kappa * kappa * hop(links, dims, t, 1)


def prepare(links, dims, kappa: float, mu: float, b) -> np.ndarray:
    """b_hat = b_e + kappa D_eo A_oo^{-1} b_o."""
    be = restrict(b, dims, 0)
    bo = restrict(b, dims, 1)
    return be + kappa * hop(links, dims, aoo_inv(bo, mu), 1)


def reconstruct(links, dims, kappa: float, mu: float, b, xe) -> np.ndarray:
    """Full solution from x_e: x_o = A_oo^{-1} (b_o + kappa D_oe x_e)."""
    bo = restrict(b, dims, 1)
    xo = aoo_inv(bo + kappa * hop(links, dims, xe.reshape(-1, 4, 3), 0), mu)
    x = embed(xe, dims, 0)
    x[sites(dims, 1)] = xo
    return x
