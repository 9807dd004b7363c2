"""Helpers shared by the GPU tests: tensors on cuda:0 and the oracle operator."""
import json
import os

import numpy as np

from inputs import lattice as L

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def host(t):
    return t.detach().cpu().numpy()


def kappa_c_table():
    path = os.path.join(GOLDEN, "kappa_c.json")
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        return json.load(f)


def oracle_ops(links, dims, kappa, mu=0.0):
    from oracle import dirac
    v = L.volume(dims)
    A = lambda x: dirac.apply_A(links, x.reshape(v, 4, 3), dims, kappa, mu).ravel()
    g5 = lambda x: dirac.gamma5(x.reshape(v, 4, 3)).ravel()
    return A, g5


def rel_residual(links, dims, kappa, x, b, mu=0.0):
    """||b - A x|| / ||b|| with the oracle's operator (a property check)."""
    A, _ = oracle_ops(links, dims, kappa, mu)
    x = np.asarray(x).ravel()
    b = np.asarray(b).ravel()
    return np.linalg.norm(b - A(x)) / np.linalg.norm(b)


def breakdown_system(dims):
    """A Wilson system on which BiCGStab breaks down at its first step, exactly.

    Unit links, kappa = 3/16, and b = b1 + b2 with b1 = 1 on (spin 0, colour 0)
    at every site (momentum 0: A b1 = (1 - 8 kappa) b1 = -b1/2) and b2 =
    (-1)^x on (spin 0, colours 1, 2) (momentum (pi,0,0,0): A b2 = (1 - 4 kappa)
    b2 = b2/4).  With x0 = 0 the shadow vector is r_hat = b, and
    <r_hat, A b> = V (-1/2 + 2/4) = 0 with every term and partial sum a
    dyadic rational, so the zero is exact in FP64 and FP32 while A b != 0.
    dims[0] must be even.  Returns (links, kappa, b flat)."""
    assert dims[0] % 2 == 0
    v = L.volume(dims)
    x = np.arange(v) % dims[0]           # site = x + Lx (y + Ly (z + Lz t))
    b = np.zeros((v, 4, 3), dtype=np.complex128)
    b[:, 0, 0] = 1.0
    b[:, 0, 1] = (-1.0) ** x
    b[:, 0, 2] = (-1.0) ** x
    return L.unit_gauge_field(dims), 0.1875, b.ravel()
