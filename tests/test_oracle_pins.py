"""Pins for the CPU oracle: facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: the
Clifford algebra, the free-field momentum-space spectrum, gauge covariance,
an independently assembled dense matrix and its LU solve, library routines
that special cases reduce to, and the structure of the paper's MVP counts.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.sparse.linalg as sla

from inputs import lattice as L
from oracle import dirac, kappa, krylov

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _vec(dims, seed):
    return L.gaussian_spinor(dims, seed)


def _ops(U, dims, kap, mu=0.0):
    v = U.shape[0]
    A = lambda x: dirac.apply_A(U, x.reshape(v, 4, 3), dims, kap, mu).ravel()
    g5 = lambda x: dirac.gamma5(x.reshape(v, 4, 3)).ravel()
    return A, g5


# ------------------------------------------------------------------ gammas

def test_gamma_clifford_algebra():
    g = dirac.GAMMA
    for a in range(4):
        assert np.allclose(g[a], g[a].conj().T, atol=0)
        for b in range(4):
            ac = g[a] @ g[b] + g[b] @ g[a]
            assert np.allclose(ac, 2.0 * (a == b) * np.eye(4), atol=1e-15)
    assert np.array_equal(dirac.GAMMA5, np.diag([1, 1, -1, -1]).astype(complex))
    for a in range(4):   # gamma5 anticommutes with every gamma_mu
        assert np.allclose(dirac.GAMMA5 @ g[a] + g[a] @ dirac.GAMMA5, 0)


def test_gamma_chiral_block_form():
    # chiral basis: every gamma_mu is block off-diagonal, gamma_4 has unit blocks
    for a in range(4):
        assert np.all(dirac.GAMMA[a][:2, :2] == 0)
        assert np.all(dirac.GAMMA[a][2:, 2:] == 0)
    assert np.array_equal(dirac.GAMMA[3][:2, 2:], np.eye(2))


# ------------------------------------------------------------------ inputs

def test_links_are_su3():
    U = L.gauge_field((2, 2, 2, 4), 0.5, 11)
    uu = np.einsum("...ab,...cb->...ac", U, U.conj())
    assert np.abs(uu - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-14


# ------------------------------------------------------------------ operator

def _dense_by_blocks(U, dims, kap):
    """Independent assembly of A = 1 - kappa D from 12x12 Kronecker blocks."""
    v = U.shape[0]
    n = 12 * v
    A = np.eye(n, dtype=complex)
    g = dirac.GAMMA
    lx, ly, lz, lt = dims
    for t in range(lt):
        for z in range(lz):
            for y in range(ly):
                for x in range(lx):
                    s = x + lx * (y + ly * (z + lz * t))
                    c = [x, y, z, t]
                    for mu in range(4):
                        up = list(c)
                        up[mu] = (up[mu] + 1) % dims[mu]
                        dn = list(c)
                        dn[mu] = (dn[mu] - 1) % dims[mu]
                        sp = up[0] + lx * (up[1] + ly * (up[2] + lz * up[3]))
                        sm = dn[0] + lx * (dn[1] + ly * (dn[2] + lz * dn[3]))
                        A[12 * s:12 * s + 12, 12 * sp:12 * sp + 12] -= kap * np.kron(
                            np.eye(4) - g[mu], U[s, mu])
                        A[12 * s:12 * s + 12, 12 * sm:12 * sm + 12] -= kap * np.kron(
                            np.eye(4) + g[mu], U[sm, mu].conj().T)
    return A


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 3, 2, 4)])
def test_dense_matrix_matches_block_assembly(dims):
    U = L.gauge_field(dims, 0.5, 21)
    kap = 0.13
    Ad = dirac.dense_A(U, dims, kap)
    Ab = _dense_by_blocks(U, dims, kap)
    assert np.abs(Ad - Ab).max() < 1e-15


def test_gamma5_hermiticity_dense():
    dims = (2, 2, 2, 2)
    U = L.gauge_field(dims, 0.5, 22)
    A = _dense_by_blocks(U, dims, 0.14)
    g5 = np.kron(np.eye(16), np.kron(dirac.GAMMA5, np.eye(3)))
    assert np.abs(g5 @ A @ g5 - A.conj().T).max() < 1e-15
    H = g5 @ A
    assert np.abs(H - H.conj().T).max() < 1e-15
    lam = np.linalg.eigvals(A)
    # spectrum closed under complex conjugation
    d = np.abs(lam[:, None] - lam.conj()[None, :]).min(axis=1)
    assert d.max() < 1e-10


def test_gamma5_hermiticity_inner_product():
    dims = (4, 4, 4, 4)
    U = L.gauge_field(dims, 0.5, 23)
    A, g5 = _ops(U, dims, 0.125)
    phi = _vec(dims, 24).ravel()
    psi = _vec(dims, 25).ravel()
    lhs = np.vdot(phi, A(psi))
    rhs = np.vdot(g5(A(g5(phi))), psi)
    assert abs(lhs - rhs) <= 1e-14 * abs(lhs)


def test_free_field_spectrum_2x2x2x2():
    # unit links, L = 2: p_mu in {0, pi}, lambda = 1 - 2 kappa (4 - 2j),
    # multiplicity 12 * C(4, j)
    dims = (2, 2, 2, 2)
    kap = 0.1
    A = dirac.dense_A(L.unit_gauge_field(dims), dims, kap)
    lam = np.sort(np.linalg.eigvals(A).real)
    expect = np.sort(np.concatenate(
        [np.full(12 * math.comb(4, j), 1 - 2 * kap * (4 - 2 * j)) for j in range(5)]))
    assert np.abs(lam - expect).max() < 1e-12
    assert np.abs(np.linalg.eigvals(A).imag).max() < 1e-12


def _plane_wave(dims, p, chi):
    lx, ly, lz, lt = dims
    v = L.volume(dims)
    s = np.arange(v)
    x = np.stack([s % lx, (s // lx) % ly, (s // (lx * ly)) % lz, s // (lx * ly * lz)])
    phase = np.exp(1j * (p[:, None] * x).sum(0))
    return phase[:, None, None] * chi[None]


@pytest.mark.parametrize("dims,nmom", [((4, 4, 4, 4), 12), ((16, 16, 16, 16), 2)])
def test_free_field_plane_waves(dims, nmom):
    # A e^{ipx} chi = e^{ipx} [(1 - 2k sum cos p) + 2ik sum gamma_mu sin p_mu] chi
    kap = 0.11
    U = L.unit_gauge_field(dims)
    rng = _rng(31)
    for _ in range(nmom):
        n = np.array([rng.integers(0, d) for d in dims])
        p = 2 * np.pi * n / np.array(dims)
        chi = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        psi = _plane_wave(dims, p, chi)
        out = dirac.apply_A(U, psi, dims, kap)
        M = (1 - 2 * kap * np.cos(p).sum()) * np.eye(4) + 2j * kap * sum(
            dirac.GAMMA[m] * np.sin(p[m]) for m in range(4))
        expect = _plane_wave(dims, p, M @ chi)
        assert np.abs(out - expect).max() < 1e-13
        # eigenvalues 1 - 2k sum cos p +- 2ik sqrt(sum sin^2 p)
        ev = np.linalg.eigvals(M)
        r = 1 - 2 * kap * np.cos(p).sum()
        im = 2 * kap * math.sqrt((np.sin(p) ** 2).sum())
        assert np.sum(np.abs(ev - (r + 1j * im)) < 1e-12) >= 2
        assert np.sum(np.abs(ev - (r - 1j * im)) < 1e-12) >= 2


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 3, 4, 2)])
def test_gauge_covariance(dims):
    U = L.gauge_field(dims, 0.5, 41)
    om = L.gauge_transform_field(dims, 42)
    psi = _vec(dims, 43)
    v = L.volume(dims)
    Up = np.empty_like(U)
    for mu in range(4):
        fwd = np.array([dirac.site_index(dims, *[c + (i == mu) for i, c in
                                                  enumerate(dirac.site_coords(dims, s))])
                        for s in range(v)])
        Up[:, mu] = om @ U[:, mu] @ np.conj(np.swapaxes(om[fwd], -1, -2))
    psip = np.einsum("sab,sib->sia", om, psi)
    lhs = dirac.apply_A(Up, psip, dims, 0.13)
    rhs = np.einsum("sab,sib->sia", om, dirac.apply_A(U, psi, dims, 0.13))
    assert np.abs(lhs - rhs).max() < 1e-13


def test_apply_at_sites_matches_field_apply():
    dims = (4, 2, 4, 6)
    U = L.gauge_field(dims, 0.5, 51)
    psi = _vec(dims, 52)
    full = dirac.apply_A(U, psi, dims, 0.12, 0.03)
    sites = [0, 5, 17, 63, L.volume(dims) - 1]
    part = dirac.apply_A_at_sites(U, psi, dims, 0.12, sites, 0.03)
    assert np.abs(full[sites] - part).max() < 1e-14


# ------------------------------------------------------------------ even-odd

def test_eo_compact_index():
    from oracle import evenodd
    for dims in [(4, 2, 2, 4), (6, 4, 2, 2)]:
        v = L.volume(dims)
        for p in (0, 1):
            assert np.array_equal(evenodd.sites(dims, p) // 2, np.arange(v // 2))


def _dense_schur(U, dims, kap, mu):
    from oracle import evenodd
    nh = 12 * L.volume(dims) // 2
    M = np.zeros((nh, nh), dtype=complex)
    e = np.zeros(nh, dtype=complex)
    for j in range(nh):
        e[:] = 0
        e[j] = 1
        M[:, j] = evenodd.schur_apply(U, dims, kap, mu, e).ravel()
    return M


@pytest.mark.parametrize("mu", [0.0, 0.1])
def test_eo_schur_solve_equals_full_solve(mu):
    from oracle import evenodd
    dims = (4, 2, 2, 4)
    U = L.gauge_field(dims, 0.5, 4300)
    kap = 0.12
    b = L.gaussian_spinor(dims, 4301)
    A = dirac.dense_A(U, dims, kap, mu)
    x_full = np.linalg.solve(A, b.ravel())
    Ah = _dense_schur(U, dims, kap, mu)
    xe = np.linalg.solve(Ah, evenodd.prepare(U, dims, kap, mu, b).ravel())
    x = evenodd.reconstruct(U, dims, kap, mu, b, xe)
    assert np.abs(x.ravel() - x_full).max() <= 1e-12 * np.abs(x_full).max()


def test_eo_schur_gamma5_hermiticity():
    dims = (4, 2, 2, 4)
    U = L.gauge_field(dims, 0.5, 4302)
    nh = 12 * L.volume(dims) // 2
    g5 = np.kron(np.eye(nh // 12), np.kron(dirac.GAMMA5, np.eye(3)))
    for mu in (0.0, 0.07):
        Ap = _dense_schur(U, dims, 0.13, mu)
        Am = _dense_schur(U, dims, 0.13, -mu)
        assert np.abs(g5 @ Ap @ g5 - Am.conj().T).max() < 1e-14


# ------------------------------------------------------------------ twisted mass

def test_twisted_mass_identities():
    dims = (4, 4, 4, 4)
    U = L.gauge_field(dims, 0.5, 61)
    psi = _vec(dims, 62)
    phi = _vec(dims, 63)
    kap, mu = 0.13, 0.05
    # gamma5 A(mu) gamma5 = A(-mu)^dagger
    lhs = np.vdot(phi, dirac.gamma5(dirac.apply_A(U, dirac.gamma5(psi), dims, kap, mu)))
    rhs = np.vdot(dirac.apply_A(U, phi, dims, kap, -mu), psi)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)
    # ||A(mu) psi||^2 = ||A_W psi||^2 + mu^2 ||psi||^2 (gamma5 A_W Hermitian)
    a = dirac.apply_A(U, psi, dims, kap, mu)
    aw = dirac.apply_A(U, psi, dims, kap, 0.0)
    n2 = np.vdot(psi, psi).real
    assert abs(np.vdot(a, a).real - np.vdot(aw, aw).real - mu * mu * n2) <= 1e-12 * n2


# ------------------------------------------------------------------ kappa_c

def test_kappa_c_free_field():
    dims = (2, 2, 2, 2)
    assert abs(kappa.kappa_c_dense(L.unit_gauge_field(dims), dims) - 0.125) < 1e-14
    dims = (4, 4, 4, 4)
    assert abs(kappa.kappa_c_arnoldi(L.unit_gauge_field(dims), dims) - 0.125) < 1e-10


def test_kappa_c_krylov_full_space_is_exact():
    # with as many steps as the dimension the Ritz values are the eigenvalues
    dims = (2, 2, 2, 2)
    U = L.gauge_field(dims, 0.3, 72)
    assert abs(kappa.kappa_c_krylov(U, dims, steps=192) - kappa.kappa_c_dense(U, dims)) < 1e-10


def test_kappa_c_three_ways_agree():
    dims = (2, 2, 2, 2)
    U = L.gauge_field(dims, 0.3, 71)
    kd = kappa.kappa_c_dense(U, dims)
    kb = kappa.kappa_c_bisect(U, dims, 0.1, 0.3)
    ka = kappa.kappa_c_arnoldi(U, dims, ncv=60)
    assert abs(kd - kb) < 1e-12
    assert abs(kd - ka) < 1e-10
    assert 0.125 < kd < 0.2


# ------------------------------------------------------------------ solvers

@pytest.fixture(scope="module")
def small_system():
    dims = (2, 2, 2, 2)
    U = L.gauge_field(dims, 0.3, 81)
    kc = kappa.kappa_c_dense(U, dims)
    kap = 0.95 * kc
    Ad = _dense_by_blocks(U, dims, kap)
    A, g5 = _ops(U, dims, kap)
    b = _vec(dims, 82).ravel()
    return dict(dims=dims, U=U, kap=kap, Ad=Ad, A=A, g5=g5, b=b,
                x=np.linalg.solve(Ad, b), cond=np.linalg.cond(Ad))


def test_bicgstab_matches_lu(small_system):
    s = small_system
    x, st = krylov.bicgstab(s["A"], s["b"], tol=1e-12)
    assert st.converged and st.mvp % 2 == 0
    assert st.true_rel_res <= 1e-12
    err = np.linalg.norm(x - s["x"]) / np.linalg.norm(s["x"])
    assert err <= s["cond"] * 1e-12 * 2


def test_dbicgstab_with_k0_is_bicgstab(small_system):
    s = small_system
    b2 = _vec(s["dims"], 83).ravel()
    x1, st1 = krylov.bicgstab(s["A"], b2, tol=1e-10)
    x2, st2 = krylov.dbicgstab(s["A"], b2, np.zeros((0, b2.size), complex), tol=1e-10,
                               gamma5=s["g5"])
    assert st1.history == st2.history and np.array_equal(x1, x2)


def test_gmresdr_full_space_is_exact(small_system):
    # m >= dimension of the Krylov space: GMRES terminates with the exact solution
    s = small_system
    r = krylov.gmresdr(s["A"], s["b"], m=200, k=5, tol=1e-12)
    assert r.stats.converged and r.stats.cycles == 1
    err = np.linalg.norm(r.x - s["x"]) / np.linalg.norm(s["x"])
    assert err < 1e-10


def test_gmresdr_k0_is_restarted_gmres(small_system):
    # k = 0 reduces to GMRES(m); compare with SciPy's restarted GMRES
    s = small_system
    m = 15
    r = krylov.gmresdr(s["A"], s["b"], m=m, k=0, tol=1e-9)
    n = s["b"].size
    op = sla.LinearOperator((n, n), matvec=s["A"], dtype=complex)
    hist = []
    xs, info = sla.gmres(op, s["b"], restart=m, rtol=1e-9, atol=0, maxiter=1000,
                         callback=lambda pr: hist.append(pr), callback_type="pr_norm")
    assert info == 0
    # the number of MVPs SciPy needed (inner iterations) bounds ours from below
    assert r.stats.converged
    assert r.stats.mvp == m * r.stats.cycles
    assert len(hist) <= r.stats.mvp
    # same GMRES(m) residual after the first full cycle (both minimise over K_m)
    assert abs(r.stats.history[0] - hist[m - 1]) <= 1e-6 * r.stats.history[0]
    assert np.linalg.norm(r.x - xs) / np.linalg.norm(xs) < 1e-7


def test_gmresdr_invariants(small_system):
    s = small_system
    m, k = 20, 6
    r = krylov.gmresdr(s["A"], s["b"], m=m, k=k, tol=1e-12)
    st = r.stats
    assert st.converged
    # MVP count: m for the first cycle, m - k for every later cycle
    assert st.mvp == m + (m - k) * (st.cycles - 1)
    # minimal residual: non-increasing across cycles
    assert all(b <= a * (1 + 1e-12) for a, b in zip(st.history, st.history[1:]))
    # orthonormal basis and the Arnoldi relation A V_k = V_{k+1} Hbar_k
    assert np.abs(r.Vk1.conj() @ r.Vk1.T - np.eye(k + 1)).max() < 1e-13
    AV = np.stack([s["A"](v) for v in r.V])
    normA = np.linalg.norm(s["Ad"], 2)
    assert np.linalg.norm(AV.T - r.Vk1.T @ r.Hbar, 2) <= 1e-12 * normA
    assert np.linalg.norm(r.x - s["x"]) / np.linalg.norm(s["x"]) <= s["cond"] * 2e-12


def test_harmonic_ritz_is_petrov_galerkin(small_system):
    # theta solves (A V g - theta V g) orthogonal to A V, i.e. the generalised
    # problem Hbar^H Hbar g = theta H_m^H g, solved here by SciPy directly
    s = small_system
    m, k = 12, 4
    n = s["b"].size
    H = np.zeros((m + 1, m), complex)
    V = np.zeros((m + 1, n), complex)
    V[0] = s["b"] / np.linalg.norm(s["b"])
    for j in range(m):
        w = s["A"](V[j])
        for i in range(j + 1):
            H[i, j] = np.vdot(V[i], w)
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        V[j + 1] = w / H[j + 1, j]
    theta, _ = krylov._harmonic_ritz(H, m, k)
    gen = scipy.linalg.eigvals(H.conj().T @ H, H[:m].conj().T)
    gen = np.array(sorted(gen, key=lambda z: (abs(z), z.real, z.imag))[:k])
    assert np.abs(theta - gen).max() < 1e-9 * np.abs(gen).max()


def test_harmonic_ritz_values_approach_small_eigenvalues(small_system):
    s = small_system
    k = 4
    # keep cycling past the solution: deflated restarting keeps refining the
    # eigen-part even when the linear system is already solved
    r = krylov.gmresdr(s["A"], s["b"], m=30, k=k, tol=1e-30, max_mv=600)
    lam = np.linalg.eigvals(s["Ad"])
    small = np.array(sorted(lam, key=abs)[:k])
    # each kept harmonic Ritz value sits on one of the k smallest eigenvalues
    for t in r.theta:
        assert np.min(np.abs(small - t)) < 1e-5 * abs(t)
    # and the eigen-residuals of the harmonic Ritz pairs are small
    Vm = r.V
    G = Vm.conj() @ np.stack([s["A"](v) for v in Vm]).T
    ev = np.linalg.eigvals(G)
    assert np.abs(ev[:, None] - small[None, :]).min(axis=1).max() < 1e-5


# ------------------------------------------------------------------ projection

def test_lr_projection_properties(small_system):
    s = small_system
    r = krylov.gmresdr(s["A"], s["b"], m=20, k=6, tol=1e-12)
    V = r.V
    U = np.stack([s["g5"](v) for v in V])
    b2 = _vec(s["dims"], 84).ravel()
    y, G, AV = krylov.lr_projection(s["A"], V, U, b2)
    x0 = V.T @ y
    rn = b2 - s["A"](x0)
    # Petrov-Galerkin: U^dagger r_new = 0
    assert np.abs(U.conj() @ rn).max() <= 1e-12 * np.linalg.norm(b2)
    # G = (gamma5 V)^dagger A V is Hermitian
    assert np.abs(G - G.conj().T).max() <= 1e-12 * np.abs(G).max()
    # basis invariance: V -> V R (R unitary) leaves x0_new unchanged
    R, _ = np.linalg.qr(_rng(85).standard_normal((6, 6)) + 1j * _rng(86).standard_normal((6, 6)))
    VR = R.T @ V
    UR = np.stack([s["g5"](v) for v in VR])
    y2, _, _ = krylov.lr_projection(s["A"], VR, UR, b2)
    assert np.linalg.norm(VR.T @ y2 - x0) <= 1e-11 * np.linalg.norm(x0)


def test_lr_projection_removes_exact_eigencomponents(small_system):
    s = small_system
    lam, W = np.linalg.eig(s["Ad"])
    idx = np.argsort(np.abs(lam))[:4]
    V, _ = np.linalg.qr(W[:, idx])
    V = V.T
    U = np.stack([s["g5"](v) for v in V])
    b2 = _vec(s["dims"], 87).ravel()
    y, _, _ = krylov.lr_projection(s["A"], V, U, b2)
    rn = b2 - s["A"](V.T @ y)
    # left eigenvectors of the same eigenvalues see no residual
    lamL, WL = np.linalg.eig(s["Ad"].conj().T)
    for i in idx:
        j = np.argmin(np.abs(lamL - np.conj(lam[i])))
        assert abs(np.vdot(WL[:, j], rn)) <= 1e-10 * np.linalg.norm(b2)


def test_minres_previous_is_least_squares():
    dims = (2, 2, 2, 4)
    U = L.gauge_field(dims, 0.5, 91)
    A, _ = _ops(U, dims, 0.12, mu=0.01)
    b = _vec(dims, 92).ravel()
    Q = np.stack([_vec(dims, 93 + j).ravel() for j in range(3)])
    d = krylov.minres_previous(A, Q, b)
    AQ = np.stack([A(q) for q in Q]).T
    dl = np.linalg.lstsq(AQ, b, rcond=None)[0]
    assert np.abs(d - dl).max() <= 1e-10 * np.abs(dl).max()
    assert np.linalg.norm(b - AQ @ d) <= np.linalg.norm(b)


def test_serial_shift_projection_cuts_work():
    dims = (4, 4, 4, 4)
    U = L.gauge_field(dims, 0.5, 95)
    kc = 0.1425
    b = _vec(dims, 96).ravel()
    mus = [0.08, 0.06, 0.04, 0.03]
    apply_mu = lambda mu: _ops(U, dims, kc, mu)[0]
    _, st0 = krylov.serial_shifts(apply_mu, b, mus, tol=1e-9, project=False)
    xs, st1 = krylov.serial_shifts(apply_mu, b, mus, tol=1e-9, project=True)
    assert all(s.converged for s in st1)
    assert sum(s.mvp for s in st1) < sum(s.mvp for s in st0)


def _dense_gamma5(v):
    """gamma5 = diag(1, 1, -1, -1) on spin, identity on site and colour, built
    as a dense n x n matrix (independent of dirac.gamma5)."""
    return np.kron(np.eye(v), np.kron(np.diag([1.0, 1.0, -1.0, -1.0]), np.eye(3))).astype(complex)


def _exact_right_eigvecs(Ad, k):
    lam, W = np.linalg.eig(Ad)
    idx = np.argsort(np.abs(lam))[:k]
    Q, _ = np.linalg.qr(W[:, idx])
    return Q.T, lam[idx]


@pytest.mark.parametrize("basis", ["gmresdr", "exact"])
def test_dbicgstab_starts_from_the_left_right_projection(small_system, basis):
    """Sec. 2: before BiCGStab, x0 = V y with (U^H A V) y = U^H b and U =
    gamma5 V.  With max_iter = 0 the oracle returns that x0; it must equal
    the projection computed here from the dense matrix and an explicitly
    built gamma5, and satisfy the Petrov-Galerkin condition for gamma5 V
    (a default U = V, or a projection on the wrong residual, fails both)."""
    s = small_system
    k = 6
    if basis == "gmresdr":
        V = krylov.gmresdr(s["A"], s["b"], m=20, k=k, tol=1e-12).V
    else:
        V, _ = _exact_right_eigvecs(s["Ad"], k)
    n = s["b"].size
    G5 = _dense_gamma5(n // 12)
    Vc = V.T                                     # n x k, columns
    U = G5 @ Vc
    b2 = _vec(s["dims"], 88).ravel()
    G = U.conj().T @ s["Ad"] @ Vc
    y = np.linalg.solve(G, U.conj().T @ b2)
    x_ref = Vc @ y
    x, st = krylov.dbicgstab(s["A"], b2, V, tol=1e-12, max_iter=0, gamma5=s["g5"])
    assert st.iters == 0 and st.mvp == 0
    # G = (gamma5 V)^H A V is Hermitian indefinite and can be ill-conditioned:
    # two LU solves agree to a few ulps times cond(G)
    assert np.linalg.norm(x - x_ref) <= 64 * np.linalg.cond(G) * 2.2e-16 * np.linalg.norm(x_ref)
    assert np.array_equal(st.x0, x)
    assert np.abs(U.conj().T @ (b2 - s["Ad"] @ x)).max() <= 1e-12 * np.linalg.norm(b2)


def test_dbicgstab_iterates_on_the_projected_residual(small_system):
    """After one BiCGStab iteration from the projected x0 the recursive
    residual equals the true residual b - A x (exact in arithmetic), and, with
    exact right eigenvectors, that residual stays orthogonal to the k left
    eigenvectors of the same eigenvalues (A maps their orthogonal complement
    into itself).  A stale residual handed to BiCGStab breaks both."""
    s = small_system
    k = 4
    V, lam = _exact_right_eigvecs(s["Ad"], k)
    b2 = _vec(s["dims"], 89).ravel()
    x1, st = krylov.dbicgstab(s["A"], b2, V, tol=1e-14, max_iter=1, gamma5=s["g5"])
    assert st.iters == 1 and st.mvp == 2 and len(st.history) == 1
    r_true = np.linalg.norm(b2 - s["Ad"] @ x1) / np.linalg.norm(b2)
    assert abs(st.history[0] - r_true) <= 1e-10 * r_true
    lamL, WL = np.linalg.eig(s["Ad"].conj().T)
    r1 = b2 - s["Ad"] @ x1
    for l in lam:
        j = np.argmin(np.abs(lamL - np.conj(l)))
        assert abs(np.vdot(WL[:, j], r1)) <= 1e-10 * np.linalg.norm(b2)


def test_dbicgstab_solution_matches_lu(small_system):
    s = small_system
    V = krylov.gmresdr(s["A"], s["b"], m=20, k=6, tol=1e-12).V
    b2 = _vec(s["dims"], 90).ravel()
    x, st = krylov.dbicgstab(s["A"], b2, V, tol=1e-12, gamma5=s["g5"])
    assert st.converged and st.mvp % 2 == 0 and st.true_rel_res <= 1e-12
    xs = np.linalg.solve(s["Ad"], b2)
    assert np.linalg.norm(x - xs) <= 2 * s["cond"] * 1e-12 * np.linalg.norm(xs)


def test_serial_shifts_start_from_least_squares_over_previous_solutions():
    """Sec. 4: shift i starts from x0 = Q d with d = argmin ||b - A(mu_i) Q d||
    over the solutions Q of the shifts already solved.  Checked against
    lstsq on the dense A(mu_i) = A_W + i mu_i gamma5 assembled here (the
    operator of the previous shift, or no projection, fails)."""
    dims = (2, 2, 2, 4)
    U = L.gauge_field(dims, 0.5, 97)
    kap = 0.13
    v = U.shape[0]
    Aw = _dense_by_blocks(U, dims, kap)
    G5 = _dense_gamma5(v)
    b = _vec(dims, 98).ravel()
    mus = [0.2, 0.1, 0.05, 0.02]
    apply_mu = lambda mu: _ops(U, dims, kap, mu)[0]
    xs, sts = krylov.serial_shifts(apply_mu, b, mus, tol=1e-12, project=True)
    assert all(st.converged for st in sts)
    assert np.array_equal(sts[0].x0, np.zeros_like(b))
    for i in range(1, len(mus)):
        Ai = Aw + 1j * mus[i] * G5
        Q = np.stack(xs[:i]).T                   # n x i
        d = np.linalg.lstsq(Ai @ Q, b, rcond=None)[0]
        x0 = Q @ d
        assert np.linalg.norm(sts[i].x0 - x0) <= 1e-10 * np.linalg.norm(x0), i
        # and the projected start never has a larger residual than x0 = 0
        assert np.linalg.norm(b - Ai @ sts[i].x0) <= np.linalg.norm(b)
        # the solution itself is the dense solve of the shift's system
        xd = np.linalg.solve(Ai, b)
        cond = np.linalg.cond(Ai)
        assert np.linalg.norm(xs[i] - xd) <= 2 * cond * 1e-12 * np.linalg.norm(xd)


def test_bicgstab_reports_breakdown_when_r_hat_is_orthogonal_to_A_r0():
    """<r_hat, A r0> = 0 exactly (constant + staggered free-field modes at
    kappa = 3/16, see tests/gpu_util.breakdown_system): alpha is undefined, so
    BiCGStab stops at its first step with the breakdown flag (the paper's "F"
    of Sec. 3), having spent one MVP and left x = 0."""
    from .gpu_util import breakdown_system
    dims = (4, 2, 2, 2)
    U, kap, b = breakdown_system(dims)
    A, _ = _ops(U, dims, kap)
    assert np.vdot(b, A(b)) == 0 and np.linalg.norm(A(b)) > 0
    x, st = krylov.bicgstab(A, b, tol=1e-10)
    assert st.breakdown and not st.converged
    assert st.iters == 0 and st.mvp == 1
    assert not np.any(x) and st.true_rel_res == 1.0


# ------------------------------------------------------------------ paper's counts

def test_paper_counts_have_cycle_structure():
    """Every GMRES-DR count in Tables 1-3 is m + (m - k) c and every BiCGStab
    count is even: convergence is tested at cycle ends and per full iteration,
    the convention the oracle follows."""
    with open(os.path.join(GOLDEN, "paper_mvp_counts.json")) as f:
        g = json.load(f)
    for tab in ("table1_16x16x16x16", "table2_20x20x20x32"):
        for m, k, counts in g[tab]["gmresdr_first_rhs"]:
            assert m - k == 20
            for c in counts:
                if c is not None:
                    assert c >= m and (c - m) % (m - k) == 0, (tab, m, k, c)
        for key in ("dbicgstab_L1", "dbicgstab_L2", "dbicgstab_L3"):
            for _, counts in g[tab][key]:
                assert all(c % 2 == 0 for c in counts)
        assert all(c % 2 == 0 for c in g[tab]["bicgstab"])
    t3 = g["table3_twisted_mass"]
    m, k = t3["m"], t3["k"]
    cols = ("x0_zero", "projection_high_to_low", "projection_low_to_high")
    for key, total in zip(cols, t3["totals"]):
        assert sum(t3[key]) == total
        assert all(c >= m and (c - m) % (m - k) == 0 for c in t3[key])
