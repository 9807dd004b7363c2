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
