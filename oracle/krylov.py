"""Krylov solvers and projections (oracle, FP64, one right-hand side at a time).

  bicgstab      BiCGStab (van der Vorst 1992), the method Sec. 2 deflates.
  gmresdr       GMRES with deflated restarting, GMRES-DR(m,k) (Morgan 2002,
                cited in Sec. 1), which solves the first right-hand side and
                returns approximate right eigenvectors.
  lr_projection the k x k left-right projection of Sec. 2:
                (U^dagger A V) y = U^dagger r0,  x0_new = x0 + V y.
  dbicgstab     D-BiCGStab(k) of Sec. 2: lr_projection once, then BiCGStab.
  minres_previous  the minimal-residual projection over previous solutions
                of Sec. 4: Q^dagger A^dagger A Q d = Q^dagger A^dagger r0.

Vectors are flat complex128 arrays of length n = 12 V; a basis is stored as
rows (shape (k, n)).  ``apply`` is any callable x -> A x.

Readings where the paper is silent:
  * Inner products are <a, b> = a^dagger b (np.vdot).
  * Residuals are relative to ||b||; with x0 = 0 that is the paper's "norm
    of the initial residual" (Sec. 3).
  * BiCGStab tests convergence on the recursive residual after each full
    iteration (two MVPs, so every count is even, as in Tables 1-2), then
    checks the true residual b - A x and restarts from it (shadow vector
    r_hat = r) at most three times if that is above tol.
  * GMRES-DR tests convergence only at the end of a cycle; the first cycle
    costs m MVPs and every later one m - k (the counts of Tables 1-3 all
    have that form).
  * Harmonic Ritz values are ordered by (|theta|, Re theta, Im theta) and
    the k smallest kept.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np

Apply = Callable[[np.ndarray], np.ndarray]


@dataclass
class SolveStats:
    mvp: int = 0              # MVPs the paper counts (inside the iteration)
    mvp_extra: int = 0        # initial / true residuals and setup products
    iters: int = 0
    cycles: int = 0
    restarts: int = 0
    converged: bool = False
    breakdown: bool = False
    rel_res: float = np.inf   # recursive (or least-squares) residual / ||b||
    true_rel_res: float = np.inf
    history: List[float] = field(default_factory=list)
    x0: Optional[np.ndarray] = None   # starting guess after a projection (Sec. 2, 4)


def _norm(x):
    return float(np.sqrt(np.vdot(x, x).real))


# ------------------------------------------------------------------ BiCGStab

def bicgstab(apply: Apply, b: np.ndarray, x0: Optional[np.ndarray] = None,
             tol: float = 1e-10, max_iter: int = 10000, max_restarts: int = 3,
             r0: Optional[np.ndarray] = None, bnorm: Optional[float] = None):
    """BiCGStab for A x = b.  Returns (x, SolveStats).

    One iteration, with <.,.> the complex inner product:
      rho   = <r_hat, r>;  beta = (rho / rho_old) (alpha / omega)
      p     = r + beta (p - omega v);   v = A p;   alpha = rho / <r_hat, v>
      s     = r - alpha v;              t = A s;   omega = <t, s> / <t, t>
      x    += alpha p + omega s;        r = s - omega t
    """
    st = SolveStats()
    x = np.zeros_like(b) if x0 is None else x0.copy()
    if bnorm is None:
        bnorm = _norm(b)
    if bnorm == 0.0:
        st.converged, st.rel_res, st.true_rel_res = True, 0.0, 0.0
        return np.zeros_like(b), st
    if r0 is not None:
        r = r0.copy()
    elif x0 is None:
        r = b.copy()
    else:
        r = b - apply(x)
        st.mvp_extra += 1
    rn = _norm(r)
    for restart in range(max_restarts + 1):
        st.restarts = restart
        if rn / bnorm <= tol:
            st.converged = True
            break
        r_hat = r.copy()
        rho_old = alpha = omega = 1.0 + 0j
        p = np.zeros_like(b)
        v = np.zeros_like(b)
        while st.iters < max_iter:
            rho = np.vdot(r_hat, r)
            if abs(rho) <= 1e-30 * _norm(r_hat) * rn:
                st.breakdown = True
                break
            beta = (rho / rho_old) * (alpha / omega)
            p = r + beta * (p - omega * v)
            v = apply(p)
            st.mvp += 1
            rv = np.vdot(r_hat, v)
            if abs(rv) <= 1e-30 * _norm(r_hat) * _norm(v):
                st.breakdown = True
                break
            alpha = rho / rv
            s = r - alpha * v
            st.iters += 1
            if _norm(s) == 0.0:            # exact solution in this step
                x = x + alpha * p
                r = s
                rn = 0.0
                st.history.append(0.0)
                break
            t = apply(s)
            st.mvp += 1
            omega = np.vdot(t, s) / np.vdot(t, t)
            x = x + alpha * p + omega * s
            r = s - omega * t
            rho_old = rho
            rn = _norm(r)
            st.history.append(rn / bnorm)
            if rn / bnorm <= tol:
                break
        st.rel_res = rn / bnorm
        if st.breakdown or st.iters >= max_iter and rn / bnorm > tol:
            break
        r = b - apply(x)                   # true residual
        st.mvp_extra += 1
        rn = _norm(r)
        st.true_rel_res = rn / bnorm
        if rn / bnorm <= tol:
            st.converged = True
            break
    if st.true_rel_res == np.inf:
        st.true_rel_res = _norm(b - apply(x)) / bnorm
        st.mvp_extra += 1
    return x, st


# ------------------------------------------------------------------ GMRES-DR

@dataclass
class GmresDrResult:
    x: np.ndarray
    V: np.ndarray            # (k, n): orthonormal basis of the harmonic Ritz vectors
    Vk1: np.ndarray          # (k+1, n): V and one more column
    Hbar: np.ndarray         # (k+1, k): A V = Vk1 Hbar
    theta: np.ndarray        # (k,) harmonic Ritz values kept
    stats: SolveStats


def _harmonic_ritz(H: np.ndarray, m: int, k: int):
    """Harmonic Ritz pairs of the (m+1) x m Hessenberg-like H, k smallest |theta|.

    With H_m the top m x m block and f = H_m^{-dagger} e_m, the harmonic Ritz
    pairs are the eigenpairs of H_m + |h_{m+1,m}|^2 f e_m^T.
    """
    hm = H[:m, :m]
    em = np.zeros(m, dtype=np.complex128)
    em[-1] = 1.0
    f = np.linalg.solve(hm.conj().T, em)
    hh = hm + abs(H[m, m - 1]) ** 2 * np.outer(f, em)
    theta, g = np.linalg.eig(hh)
    order = sorted(range(m), key=lambda i: (abs(theta[i]), theta[i].real,
                                            theta[i].imag))[:k]
    return theta[order], g[:, order]


def gmresdr(apply: Apply, b: np.ndarray, m: int, k: int, tol: float = 1e-10,
            max_mv: int = 100000, x0: Optional[np.ndarray] = None,
            lucky_tol: float = 1e-14) -> GmresDrResult:
    """GMRES-DR(m,k) for A x = b (Morgan 2002, as used in Sec. 1 and Sec. 3).

    Cycle: Arnoldi (classical Gram-Schmidt applied twice) extends
    A V_j = V_{j+1} Hbar_j up to j = m; d = argmin ||c - Hbar_m d||,
    x += V_m d, rho = c - Hbar_m d.  Converged if ||rho|| / ||r0|| <= tol.
    Restart: harmonic Ritz vectors g_1..g_k (k smallest |theta|); P_k = QR
    of [g; 0]; p_{k+1} = rho orthonormalised against P_k;
    Hbar_k = P_{k+1}^dagger Hbar_m P_k, V_{k+1} = V_{m+1} P_{k+1},
    c = P_{k+1}^dagger rho; continue Arnoldi from column k+1.
    The basis returned is the first k columns of V_{k+1} after the restart
    step that follows the converged cycle.
    """
    n = b.size
    st = SolveStats()
    x = np.zeros_like(b) if x0 is None else x0.copy()
    if x0 is None:
        r = b.copy()
    else:
        r = b - apply(x)
        st.mvp_extra += 1
    beta = _norm(r)
    bnorm = beta
    V = np.zeros((m + 1, n), dtype=np.complex128)
    H = np.zeros((m + 1, m), dtype=np.complex128)
    c = np.zeros(m + 1, dtype=np.complex128)
    V[0] = r / beta
    c[0] = beta
    j0 = 0
    theta = np.zeros(k, dtype=np.complex128)
    Hk = np.zeros((k + 1, k), dtype=np.complex128)
    Vk1 = np.zeros((k + 1, n), dtype=np.complex128)
    while True:
        # ---- Arnoldi from column j0 to m-1
        m_eff = m
        for j in range(j0, m):
            w = apply(V[j])
            st.mvp += 1
            w0 = _norm(w)
            h = V[: j + 1].conj() @ w
            w = w - V[: j + 1].T @ h
            h2 = V[: j + 1].conj() @ w
            w = w - V[: j + 1].T @ h2
            H[: j + 1, j] = h + h2
            hn = _norm(w)
            H[j + 1, j] = hn
            if hn <= lucky_tol * w0:           # invariant subspace: exact
                m_eff = j + 1
                break
            V[j + 1] = w / hn
        st.cycles += 1
        # ---- least squares min || c - Hbar d ||
        Hs = H[: m_eff + 1, :m_eff]
        d = np.linalg.lstsq(Hs, c[: m_eff + 1], rcond=None)[0]
        x = x + V[:m_eff].T @ d
        rho = c[: m_eff + 1] - Hs @ d
        res = _norm(rho)
        st.history.append(res / bnorm)
        st.rel_res = res / bnorm
        if m_eff < m:                           # lucky breakdown
            st.converged = True
            break
        done = res / bnorm <= tol
        # ---- deflated restart (also after the final cycle, to emit V)
        if k > 0:
            theta, g = _harmonic_ritz(H, m, k)
            gpad = np.vstack([g, np.zeros((1, k), dtype=np.complex128)])
            pk, _ = np.linalg.qr(gpad)
            p = rho.copy()
            for _ in range(2):
                p = p - pk @ (pk.conj().T @ p)
            p = p / _norm(p)
            P = np.hstack([pk, p[:, None]])                    # (m+1, k+1)
            Hk = P.conj().T @ H @ pk[:m]                       # (k+1, k)
            Vk1 = P.T @ V                                      # (k+1, n)
            ck = P.conj().T @ rho
        if done:
            st.converged = True
            break
        if st.mvp + (m - k) > max_mv:
            break
        Vfull = V.copy() if k == 0 else None
        V[:] = 0
        H[:] = 0
        c[:] = 0
        if k > 0:
            V[: k + 1] = Vk1
            H[: k + 1, :k] = Hk
            c[: k + 1] = ck
            # re-orthogonalise v_{k+1} against v_1..v_k
            vk = V[k] - V[:k].T @ (V[:k].conj() @ V[k])
            V[k] = vk / _norm(vk)
        else:                                   # plain GMRES(m) restart
            r = Vfull.T @ rho                   # residual = V_{m+1} rho
            V[0] = r / res
            c[0] = res
        j0 = k
    rt = b - apply(x)
    st.mvp_extra += 1
    st.true_rel_res = _norm(rt) / bnorm
    V_out = Vk1[:k].copy() if k > 0 else np.zeros((0, n), dtype=np.complex128)
    return GmresDrResult(x=x, V=V_out, Vk1=Vk1, Hbar=Hk, theta=theta, stats=st)


# ------------------------------------------------------------------ Sec. 2 projection

def lr_projection(apply: Apply, V: np.ndarray, U: np.ndarray, r0: np.ndarray):
    """Solve (U^dagger A V) y = U^dagger r0 (Sec. 2).  Returns (y, G, AV)."""
    AV = np.stack([apply(v) for v in V])           # k MVPs
    G = U.conj() @ AV.T                            # G[i, j] = u_i^dagger A v_j
    y = np.linalg.solve(G, U.conj() @ r0)
    return y, G, AV


def dbicgstab(apply: Apply, b: np.ndarray, V: np.ndarray,
              U: Optional[np.ndarray] = None, tol: float = 1e-10,
              max_iter: int = 10000, x0: Optional[np.ndarray] = None,
              gamma5: Optional[Callable] = None):
    """D-BiCGStab(k), Sec. 2: x0_new = x0 + V y, then BiCGStab from x0_new.

    U defaults to gamma5 V (left eigenvectors from right ones, Sec. 1);
    ``gamma5`` maps a flat vector to gamma5 times it.
    """
    x = np.zeros_like(b) if x0 is None else x0.copy()
    extra = 0
    if x0 is None:
        r0 = b.copy()
    else:
        r0 = b - apply(x)
        extra += 1
    if V.shape[0] > 0:
        if U is None:
            U = np.stack([gamma5(v) for v in V])
        y, _, _ = lr_projection(apply, V, U, r0)
        extra += V.shape[0]
        x = x + V.T @ y
        r0 = b - apply(x)
        extra += 1
    x0_proj = x.copy()
    x, st = bicgstab(apply, b, x0=x, tol=tol, max_iter=max_iter, r0=r0,
                     bnorm=_norm(b))
    st.mvp_extra += extra
    st.x0 = x0_proj
    return x, st


# ------------------------------------------------------------------ Sec. 4 projection

def minres_previous(apply: Apply, Q: np.ndarray, r0: np.ndarray):
    """Solve Q^dagger A^dagger A Q d = Q^dagger A^dagger r0 (Sec. 4); returns d."""
    AQ = np.stack([apply(q) for q in Q]).T          # (n, k), k MVPs
    M = AQ.conj().T @ AQ
    return np.linalg.solve(M, AQ.conj().T @ r0)


def serial_shifts(apply_mu: Callable[[float], Apply], b: np.ndarray, mus,
                  tol: float = 1e-10, max_iter: int = 10000,
                  project: bool = True):
    """Sec. 4: solve A(mu_i) x_i = b one shift after another; before each
    solve, project over the solutions already found.  Returns (xs, stats)."""
    xs, stats = [], []
    for mu in mus:
        apply = apply_mu(mu)
        x0 = np.zeros_like(b)
        r0 = b.copy()
        extra = 0
        if project and xs:
            Q = np.stack(xs)
            d = minres_previous(apply, Q, r0)
            extra += len(xs)
            x0 = Q.T @ d
            r0 = b - apply(x0)
            extra += 1
        x, st = bicgstab(apply, b, x0=x0, tol=tol, max_iter=max_iter, r0=r0,
                         bnorm=_norm(b))
        st.mvp_extra += extra
        st.x0 = x0
        xs.append(x)
        stats.append(st)
    return xs, stats
