"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package draws random numbers and lays them out; it holds none of the
solver's arithmetic (no Wilson operator, no Krylov method, no projection).
Both the CPU oracle and the CUDA path consume exactly the arrays produced
here, so the two sides see bit-identical inputs.

Canonical host layout (complex128, C order):
  site index  s = x + Lx*(y + Ly*(z + Lz*t)),  dims = (Lx, Ly, Lz, Lt)
  gauge field U[s, mu, a, b]   mu = 0..3 for x, y, z, t;  a, b colour
  spinor     psi[s, sigma, a]  sigma = 0..3 spin, a = 0..2 colour
"""
from .lattice import (
    LatticeConfig,
    CONFIGS,
    volume,
    gauge_field,
    unit_gauge_field,
    gaussian_spinor,
    z4_spinor,
    random_su3,
    gauge_transform_field,
    link_seed,
    rhs_seed,
    source,
    move_links,
)

__all__ = [
    "LatticeConfig", "CONFIGS", "volume", "gauge_field", "unit_gauge_field",
    "gaussian_spinor", "z4_spinor", "random_su3", "gauge_transform_field",
    "link_seed", "rhs_seed", "source", "move_links",
]
