"""Critical hopping parameter kappa_c (oracle).

Sec. 3 defines kappa_c per gauge configuration: the kappa at which the
leftmost eigenvalue of A reaches the imaginary axis.  Every eigenvalue of
A = 1 - kappa*D is 1 - kappa*lambda with lambda an eigenvalue of D, so for
kappa > 0 the smallest real part is 1 - kappa*max Re lambda(D) and

  kappa_c = 1 / max Re lambda(D).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as sla

from . import dirac


def kappa_c_dense(links, dims) -> float:
    """kappa_c from the full spectrum of D (small lattices)."""
    lam = np.linalg.eigvals(dirac.dense_D(links, dims))
    return float(1.0 / np.max(lam.real))


def kappa_c_bisect(links, dims, lo: float, hi: float, iters: int = 60) -> float:
    """The workload's own definition: bisect kappa until min Re lambda(A) = 0.

    Uses the dense matrix of A at every trial kappa, so it is for tiny
    lattices only; it serves as an independent check of kappa_c_dense.
    """
    def min_re(kappa):
        return np.min(np.linalg.eigvals(dirac.dense_A(links, dims, kappa)).real)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if min_re(mid) > 0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def kappa_c_arnoldi(links, dims, tol: float = 1e-12, ncv: int = 40, nev: int = 4) -> float:
    """kappa_c from the rightmost eigenvalue of D by implicitly restarted Arnoldi.

    The rightmost eigenvalues of D come in a tight cluster (the low modes of
    A), so large lattices take thousands of products; ``tol`` is ARPACK's
    relative accuracy on the Ritz values.
    """
    n = 12 * links.shape[0]
    v = links.shape[0]

    def mv(x):
        return dirac.hopping(links, x.reshape(v, 4, 3), dims).ravel()

    op = sla.LinearOperator((n, n), matvec=mv, dtype=np.complex128)
    rng = np.random.Generator(np.random.PCG64(7))
    v0 = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    lam = sla.eigs(op, k=nev, which="LR", tol=tol, ncv=ncv, v0=v0,
                   return_eigenvectors=False)
    return float(1.0 / np.max(lam.real))


def kappa_c_krylov(links, dims, steps: int = 300, seed: int = 7) -> float:
    """kappa_c from the rightmost Ritz value of a `steps`-step Arnoldi
    factorisation of D (classical Gram-Schmidt applied twice, no restart).

    Exterior eigenvalues are the first Ritz values to converge; on 8^4 the
    rightmost one agrees with implicitly restarted Arnoldi to 3e-6 after 200
    steps and to 1e-11 after 400.  Used where restarted Arnoldi stalls on
    the cluster of near-critical eigenvalues."""
    v = links.shape[0]
    n = 12 * v
    steps = min(steps, n)
    rng = np.random.Generator(np.random.PCG64(seed))
    q = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    Q = np.zeros((steps + 1, n), dtype=np.complex128)
    H = np.zeros((steps + 1, steps), dtype=np.complex128)
    Q[0] = q / np.linalg.norm(q)
    for j in range(steps):
        w = dirac.hopping(links, Q[j].reshape(v, 4, 3), dims).ravel()
        for _ in range(2):
            h = (Q[: j + 1] @ w.conj()).conj()  # Q^dagger w without a conjugated copy of Q
            w = w - Q[: j + 1].T @ h
            H[: j + 1, j] += h
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j].real <= 1e-14:
            steps = j + 1
            break
        Q[j + 1] = w / H[j + 1, j]
    ritz = np.linalg.eigvals(H[:steps, :steps])
    return float(1.0 / np.max(ritz.real))


def kappa_c(links, dims) -> float:
    """Dense spectrum up to n = 3072; implicitly restarted Arnoldi up to
    n = 1e5; a 300-step Arnoldi factorisation up to n = 4e6 and a 200-step
    one beyond (the basis of (steps + 1) n complex numbers must fit in host
    memory: 26 GB at 24^3 x 48)."""
    n = 12 * links.shape[0]
    if n <= 3072:
        return kappa_c_dense(links, dims)
    if n <= 100_000:
        return kappa_c_arnoldi(links, dims, tol=1e-10, ncv=100, nev=6)
    if n <= 4_000_000:
        return kappa_c_krylov(links, dims, steps=300)
    return kappa_c_krylov(links, dims, steps=200)
