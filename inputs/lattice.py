"""Seeded synthetic gauge fields and right-hand sides.

The paper measures on quenched Wilson-plaquette ensembles at beta = 6.0
(Sec. 3), which are not available here.  They are replaced by random SU(3)
links U = exp(i*eps*H), H a Gaussian Hermitian traceless 3x3 matrix, and by
Gaussian or Z4 noise sources.  Nothing in this module implements the solver;
it only draws and shapes random numbers.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional, Tuple

import numpy as np

# ---------------------------------------------------------------- presets


@dataclass(frozen=True)
class LatticeConfig:
    """One named workload: lattice extents, link recipe and solver sizes."""
    name: str
    dims: Tuple[int, int, int, int]          # (Lx, Ly, Lz, Lt)
    eps: float                               # link spread in exp(i*eps*H)
    kappa_factor: float                      # kappa = kappa_factor * kappa_c
    m: int = 0                               # GMRES-DR subspace size
    k: int = 0                               # deflation vectors
    rhs_kind: str = "gaussian"               # "gaussian" or "z4"
    n_rhs: int = 1                           # right-hand sides after the first
    tol: float = 1e-10
    mus: Tuple[float, ...] = field(default_factory=tuple)
    index: int = 0


CONFIGS = {
    "wilson_4x4x4x4": LatticeConfig(
        "wilson_4x4x4x4", (4, 4, 4, 4), 0.3, 0.95, m=20, k=6,
        rhs_kind="gaussian", n_rhs=3, index=0),
    "wilson_16x16x16x16": LatticeConfig(
        "wilson_16x16x16x16", (16, 16, 16, 16), 0.5, 0.99, m=80, k=40,
        rhs_kind="z4", n_rhs=10, index=1),
    "wilson_20x20x20x32_mixed": LatticeConfig(
        "wilson_20x20x20x32_mixed", (20, 20, 20, 32), 0.5, 0.995, m=80, k=60,
        rhs_kind="z4", n_rhs=12, index=2),
    "twisted_24x24x24x48": LatticeConfig(
        "twisted_24x24x24x48", (24, 24, 24, 48), 0.5, 1.0,
        rhs_kind="gaussian", n_rhs=16,
        mus=(0.064, 0.032, 0.016, 0.008, 0.004, 0.002), index=3),
    "grad_8x8x8x16": LatticeConfig(
        "grad_8x8x8x16", (8, 8, 8, 16), 0.5, 0.99,
        rhs_kind="gaussian", n_rhs=1, index=4),
    "grad_32x32x32x64": LatticeConfig(
        "grad_32x32x32x64", (32, 32, 32, 64), 0.5, 0.99,
        rhs_kind="gaussian", n_rhs=1, index=4),
}


def link_seed(cfg: LatticeConfig) -> int:
    return 1000 + cfg.index


def rhs_seed(cfg: LatticeConfig, j: int) -> int:
    return 2000 + 100 * cfg.index + j


def volume(dims) -> int:
    lx, ly, lz, lt = dims
    return lx * ly * lz * lt


# ---------------------------------------------------------------- SU(3)

def _gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices lambda_a (shape (8, 3, 3))."""
    l = np.zeros((8, 3, 3), dtype=np.complex128)
    l[0][0, 1] = l[0][1, 0] = 1
    l[1][0, 1] = -1j
    l[1][1, 0] = 1j
    l[2][0, 0] = 1
    l[2][1, 1] = -1
    l[3][0, 2] = l[3][2, 0] = 1
    l[4][0, 2] = -1j
    l[4][2, 0] = 1j
    l[5][1, 2] = l[5][2, 1] = 1
    l[6][1, 2] = -1j
    l[6][2, 1] = 1j
    l[7][0, 0] = l[7][1, 1] = 1 / np.sqrt(3)
    l[7][2, 2] = -2 / np.sqrt(3)
    return l


GELL_MANN = _gell_mann()


def _reunitarise(u: np.ndarray) -> np.ndarray:
    """Gram-Schmidt on rows 0 and 1, row 2 = conj(row0 x row1): det = 1."""
    r0 = u[..., 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=-1, keepdims=True)
    r1 = u[..., 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=-2)


def _exp_i_hermitian(h: np.ndarray, eps: float) -> np.ndarray:
    """exp(i*eps*H) for a batch of Hermitian H, by eigendecomposition."""
    w, q = np.linalg.eigh(h)
    ph = np.exp(1j * eps * w)
    return np.einsum("...ij,...j,...kj->...ik", q, ph, np.conj(q))


def random_su3(rng: np.random.Generator, shape, eps: float) -> np.ndarray:
    """SU(3) matrices exp(i*eps*sum_a h_a lambda_a/2), h_a ~ N(0,1)."""
    h = rng.standard_normal(tuple(shape) + (8,))
    herm = np.einsum("...a,aij->...ij", h, GELL_MANN) * 0.5
    return _reunitarise(_exp_i_hermitian(herm, eps))


def gauge_field(dims, eps: float, seed: int) -> np.ndarray:
    """Random links, shape (V, 4, 3, 3), complex128."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.ascontiguousarray(random_su3(rng, (volume(dims), 4), eps))


def unit_gauge_field(dims) -> np.ndarray:
    """Free field: every link the identity."""
    v = volume(dims)
    u = np.zeros((v, 4, 3, 3), dtype=np.complex128)
    u[:, :, 0, 0] = u[:, :, 1, 1] = u[:, :, 2, 2] = 1
    return u


def gauge_transform_field(dims, seed: int, eps: float = 1.5) -> np.ndarray:
    """One random SU(3) matrix per site, shape (V, 3, 3)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.ascontiguousarray(random_su3(rng, (volume(dims),), eps))


def move_links(links: np.ndarray, omega: np.ndarray, h: float) -> np.ndarray:
    """Links displaced along Lie-algebra directions: exp(i h omega_a lambda_a/2) U.

    omega has shape (V, 4, 8); used to build finite-difference inputs."""
    herm = np.einsum("sma,aij->smij", omega, GELL_MANN) * (0.5 * h)
    w, q = np.linalg.eigh(herm)
    ex = np.einsum("...ij,...j,...kj->...ik", q, np.exp(1j * w), np.conj(q))
    return np.ascontiguousarray(ex @ links)


# ---------------------------------------------------------------- sources

def gaussian_spinor(dims, seed: int, nrhs: Optional[int] = None) -> np.ndarray:
    """Re and Im i.i.d. N(0,1) per component: shape (V, 4, 3) or (nrhs, V, 4, 3)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = (volume(dims), 4, 3) if nrhs is None else (nrhs, volume(dims), 4, 3)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def z4_spinor(dims, seed: int, nrhs: Optional[int] = None) -> np.ndarray:
    """Each component uniform on {1, i, -1, -i}."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = (volume(dims), 4, 3) if nrhs is None else (nrhs, volume(dims), 4, 3)
    k = rng.integers(0, 4, size=shape)
    return (np.array([1, 1j, -1, -1j], dtype=np.complex128))[k]


def source(cfg: LatticeConfig, j: int) -> np.ndarray:
    """The j-th right-hand side of a preset (j = 0 is the GMRES-DR one)."""
    if cfg.rhs_kind == "z4":
        return z4_spinor(cfg.dims, rhs_seed(cfg, j))
    return gaussian_spinor(cfg.dims, rhs_seed(cfg, j))
