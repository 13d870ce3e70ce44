"""Pins of the CPU oracle against facts that the paper and the mathematics fix (no GPU).

Each test checks one oracle function against something other than itself: closed-form values,
algebraic identities, brute force on tiny inputs, or an independent exact solver.
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import ib, krylov, mac, multigrid, peskin, smoothers, system, transfer
from paper_1612_02208_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Peskin kernel (Appendix)
def test_phi_closed_form_values():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "phi_closed_form.txt")) if l.strip() and l[0] != "#"]
    r = np.array([float(x[0]) for x in rows])
    v = np.array([float(x[2]) for x in rows])
    np.testing.assert_allclose(peskin.phi(r), v, rtol=0, atol=1e-15)


def test_phi_moment_identities():
    rng = np.random.default_rng(11)
    r = rng.uniform(-3, 3, 10000)
    js = np.arange(-5, 6)
    w = peskin.phi(r[:, None] - js[None, :])
    np.testing.assert_allclose(w.sum(1), 1.0, atol=1e-14)                               # partition of unity
    np.testing.assert_allclose((w * (r[:, None] - js[None, :])).sum(1), 0.0, atol=1e-14)  # first moment
    np.testing.assert_allclose((w * w).sum(1), 3.0 / 8.0, atol=1e-14)                    # sum of squares
    # even/odd split: sum over even j equals sum over odd j (= 1/2)
    even = (js % 2) == 0
    np.testing.assert_allclose(w[:, even].sum(1), 0.5, atol=1e-14)


def test_phi_c1_and_derivative():
    eps = 1e-7
    for r0 in (0.0, 1.0, 2.0, -1.0):
        assert abs(peskin.phi(r0 - 1e-12) - peskin.phi(r0 + 1e-12)) < 1e-11
        assert abs(peskin.dphi(r0 - 1e-9) - peskin.dphi(r0 + 1e-9)) < 1e-6
    r = np.linspace(-2.4, 2.4, 997)
    fd = (peskin.phi(r + eps) - peskin.phi(r - eps)) / (2 * eps)
    np.testing.assert_allclose(peskin.dphi(r), fd, atol=1e-7)


# ---------------------------------------------------------------- MAC operators
def test_divergence_is_minus_gradient_transpose():
    for N in (4, 8, 12):
        assert abs(mac.divergence(N) + mac.gradient(N).T).max() < 1e-12


def test_mac_fourier_symbols():
    N = 16
    h = 1.0 / N
    j, i = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    for k1, k2 in ((1, 0), (3, 5), (8, 8), (0, 7)):
        t1, t2 = 2 * np.pi * k1 / N, 2 * np.pi * k2 / N
        e = np.exp(1j * (t1 * i + t2 * j)).ravel()
        lap = mac.laplacian(N)
        sym = -(4 * np.sin(t1 / 2) ** 2 + 4 * np.sin(t2 / 2) ** 2) / h ** 2
        np.testing.assert_allclose(lap @ e, sym * e, atol=1e-8 * abs(sym) + 1e-9)
        G = mac.gradient(N)
        gp = G @ e
        np.testing.assert_allclose(gp[:N * N], (1 - np.exp(-1j * t1)) / h * e, atol=1e-9)
        np.testing.assert_allclose(gp[N * N:], (1 - np.exp(-1j * t2)) / h * e, atol=1e-9)
        D = mac.divergence(N)
        np.testing.assert_allclose(D @ np.concatenate([e, 0 * e]), (np.exp(1j * t1) - 1) / h * e, atol=1e-9)


# ---------------------------------------------------------------- interpolation / spreading / springs
def _random_markers(M, seed, near_seam=True):
    rng = np.random.default_rng(seed)
    X = rng.uniform(0, 1, (M, 2))
    if near_seam:
        X[0] = [1e-3, 0.5]
        X[1] = [0.9999, 0.9999]
        X[2] = [0.5, 0.0]
    return X


@pytest.mark.parametrize("N", [8, 16])
def test_interp_local_equals_bruteforce(N):
    X = _random_markers(9, N)
    for c in (0, 1):
        np.testing.assert_allclose(ib.interp_matrix(N, X, c).toarray(), ib.interp_matrix_bruteforce(N, X, c),
                                   atol=1e-15)


def test_interp_partition_of_unity_and_adjointness():
    N = 32
    h = 1.0 / N
    X = _random_markers(40, 3)
    rng = np.random.default_rng(4)
    for c in (0, 1):
        J = ib.interp_matrix(N, X, c)
        np.testing.assert_allclose(np.asarray(J.sum(1)).ravel(), 1.0, atol=1e-14)
        S = ib.spread_matrix(N, X, c)
        F = rng.standard_normal(X.shape[0])
        u = rng.standard_normal(N * N)
        lhs = h * h * (S @ F) @ u
        rhs = F @ (J @ u)
        assert abs(lhs - rhs) < 1e-12 * (abs(rhs) + 1)
        # a single marker spreads a total force F: sum_f (S F)_f h^2 = F
        one = np.zeros(X.shape[0]); one[5] = 2.5
        assert abs((S @ one).sum() * h * h - 2.5) < 1e-13


def test_spring_operator():
    # hand-computed three-marker ring: F_a = sum kappa (X_b - X_a)
    X = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    E = np.array([[0, 1], [1, 2], [2, 0]], dtype=np.int32)
    k = np.array([1.0, 2.0, 3.0])
    expect = np.array([[1.0, 3.0], [-3.0, 2.0], [2.0, -5.0]])
    np.testing.assert_allclose(ib.spring_force(X, E, k), expect)
    K = ib.stiffness(3, E, k)
    np.testing.assert_allclose(K @ X, expect)
    s = I.elastic_disk(32, kappa=7.0)
    K = ib.stiffness(s.M, s.edges, s.kappa)
    np.testing.assert_allclose(K @ np.ones(s.M), 0.0, atol=1e-12)   # translation
    assert abs(K - K.T).max() == 0
    small = I.elastic_disk(8, kappa=1.0)
    ev = np.linalg.eigvalsh(ib.stiffness(small.M, small.edges, small.kappa).toarray())
    assert ev.max() < 1e-12                                    # negative semidefinite
    np.testing.assert_allclose(ib.stiffness(s.M, s.edges, s.kappa) @ s.X,
                               ib.spring_force(s.X, s.edges, s.kappa), atol=1e-9)


def test_zero_force_at_rest():
    # all markers collapsed to one point: any rigid translation of that configuration is at rest
    s = I.thin_interface(32)
    Xc = np.tile([[0.37, 0.61]], (s.M, 1))
    K = ib.stiffness(s.M, s.edges, s.kappa)
    assert np.abs(K @ Xc).max() == 0.0
    prob = I.Problem(32, 0.0, 1.0, 1e-2, I.Structure(Xc, s.edges, s.kappa), np.zeros(3 * 32 * 32))
    b = system.rhs(prob)
    assert np.abs(b).max() == 0.0
    w, _ = system.solve_direct(system.operator_of(prob), b, 32, 0.0)
    assert np.abs(w).max() < 1e-14


# ---------------------------------------------------------------- the Stokes-IB system
def test_operator_symmetric_and_kernel():
    prob = I.thin_ellipse_stokes(16, kappa=1e3)
    L = system.operator_of(prob)
    assert abs(L - L.T).max() < 1e-9 * abs(L).max()
    Z = system.null_basis(16, 0.0)
    assert np.abs(L @ Z).max() < 1e-9
    # nothing else in the kernel: the smallest singular values beyond the gauge are O(1)
    s = np.linalg.svd(L.toarray(), compute_uv=False)
    assert s[-3] < 1e-8 and s[-4] > 1e-3


def test_fluid_only_matches_fourier_solve():
    for rho, mu, dt in ((0.0, 1.0, 1e-2), (1.0, 1e-2, 1e-3)):
        prob = I.no_structure(16, rho=rho, mu=mu, dt=dt, seed=5)
        L = system.operator_of(prob)
        b = system.rhs(prob)
        w, _ = system.solve_direct(L, b, 16, rho)
        wf = system.fft_stokes(16, rho, mu, dt, b)
        np.testing.assert_allclose(system.project(w, 16, rho), system.project(wf, 16, rho), atol=1e-12)


@pytest.mark.parametrize("maker,N", [(I.thin_ellipse_stokes, 16), (I.disk_stokes, 16), (I.thin_ellipse_re, 16)])
def test_three_exact_solves_agree(maker, N):
    prob = maker(N)
    L = system.operator_of(prob)
    b = system.rhs(prob)
    w, lam = system.solve_direct(L, b, N, prob.rho)
    assert np.abs(lam).max() < 1e-10 * np.abs(b).max()        # consistent right-hand side
    w = system.project(w, N, prob.rho)
    w3, X3 = system.solve_full_system(prob)
    wl, Xl = system.solve_lagrangian(prob)
    scale = np.abs(w).max()
    assert np.abs(system.project(w3, N, prob.rho) - w).max() < 1e-10 * scale
    assert np.abs(system.project(wl, N, prob.rho) - w).max() < 1e-10 * scale
    assert np.abs(X3 - Xl).max() < 1e-12
    # discrete incompressibility of the exact solution
    n = N * N
    D = mac.divergence(N)
    assert np.linalg.norm(D @ w[:2 * n]) < 1e-12 * np.linalg.norm(w[:2 * n]) * N
    # the structure moves with the interpolated velocity: X^{n+1} = X^n + dt J u
    U = ib.interp_velocity(N, prob.structure.X, w)
    np.testing.assert_allclose(X3, prob.structure.X + prob.dt * U, atol=1e-12)


def test_homogeneous_form_matches_full_system():
    prob = I.thin_ellipse_stokes(16, kappa=50.0)
    L = system.operator_of(prob)
    b = system.rhs(prob, add_SKXn=False)
    w, _ = system.solve_direct(L, b, 16, 0.0)
    w3, _ = system.solve_full_system(prob, add_SKXn=False)
    np.testing.assert_allclose(system.project(w, 16, 0.0), system.project(w3, 16, 0.0), atol=1e-11)


def test_rhs_spring_force_has_zero_mean():
    prob = I.disk_stokes(32, kappa=3.0)
    s = prob.structure
    F = ib.stiffness(s.M, s.edges, s.kappa) @ s.X
    f = ib.spread_force(32, s.X, F)
    assert abs(f[:1024].sum()) < 1e-9 and abs(f[1024:].sum()) < 1e-9


# ---------------------------------------------------------------- transfers (Sec. 3.2)
def test_transfer_identities():
    for Nc in (4, 8):
        Nf = 2 * Nc
        Pu, Pv = transfer.prolong_u(Nc), transfer.prolong_v(Nc)
        Ru = transfer.restrict_velocity(Nc)
        np.testing.assert_allclose(Ru @ np.ones(2 * Nf * Nf), 1.0, atol=1e-15)
        Pvel = transfer.prolong_velocity(Nc)
        # RT0 keeps divergence: D_f P_u = Inj D_c, Inj = piecewise-constant injection = 4 R_p^T
        Inj = 4.0 * transfer.restrict_p(Nc).T
        lhs = (mac.divergence(Nf) @ Pvel).toarray()
        rhs = (Inj @ mac.divergence(Nc)).toarray()
        np.testing.assert_allclose(lhs, rhs, atol=1e-12)
        # and its adjoint: R_u G_f = G_c R_p
        np.testing.assert_allclose((Ru @ mac.gradient(Nf)).toarray(),
                                   (mac.gradient(Nc) @ transfer.restrict_p(Nc)).toarray(), atol=1e-12)
        Pp = transfer.prolong_p(Nc)
        np.testing.assert_allclose(Pp @ np.ones(Nc * Nc), 1.0)
        np.testing.assert_allclose(transfer.restrict_p(Nc) @ np.ones(Nf * Nf), 1.0)
    # bilinear reproduction of a linear field away from the seam
    Nc = 8
    Nf = 16
    jc, ic = np.meshgrid(np.arange(Nc), np.arange(Nc), indexing="ij")
    pc = (2.0 * (ic + 0.5) / Nc + 3.0 * (jc + 0.5) / Nc).ravel()
    jf, if_ = np.meshgrid(np.arange(Nf), np.arange(Nf), indexing="ij")
    pf = (2.0 * (if_ + 0.5) / Nf + 3.0 * (jf + 0.5) / Nf).ravel()
    interior = ((if_ > 0) & (if_ < Nf - 1) & (jf > 0) & (jf < Nf - 1)).ravel()
    np.testing.assert_allclose((transfer.prolong_p(Nc) @ pc)[interior], pf[interior], atol=1e-13)
    # RT0: a field linear in x and constant in y on x-faces is reproduced away from the seam
    uc = (1.0 + 5.0 * ic / Nc).ravel()
    uf = (1.0 + 5.0 * if_ / Nf).ravel()
    inner = (if_ < Nf - 1).ravel()
    np.testing.assert_allclose((transfer.prolong_u(Nc) @ uc)[inner], uf[inner], atol=1e-13)


def test_galerkin_coarse_ib_operator():
    prob = I.thin_ellipse_stokes(32, kappa=1e3)
    H = multigrid.Hierarchy(prob)
    s = prob.structure
    K = ib.stiffness(s.M, s.edges, s.kappa)
    Pchain = None
    for l in range(H.lmax - 1, -1, -1):
        B = H.levels[l].B
        assert abs(B - B.T).max() < 1e-9 * abs(B).max()
        Nc = H.levels[l].N
        Pv = transfer.prolong_velocity(Nc)
        Pchain = Pv if Pchain is None else (Pchain @ Pv)
        hc = 1.0 / Nc
        for c in (0, 1):
            n_f = H.levels[-1].n
            n_c = Nc * Nc
            Jl = ib.interp_matrix(32, s.X, c) @ Pchain[c * n_f:(c + 1) * n_f, c * n_c:(c + 1) * n_c]
            ref = (Jl.T @ K @ Jl) / hc ** 2
            blk = B[c * n_c:(c + 1) * n_c, c * n_c:(c + 1) * n_c]
            assert abs(blk - ref).max() < 1e-9 * abs(ref).max()


def test_coarse_pseudo_inverse():
    prob = I.thin_ellipse_stokes(16, kappa=1e2)
    H = multigrid.Hierarchy(prob)
    L0 = H.levels[0].L.toarray()
    Z = system.null_basis(8, 0.0)
    b = system.project(np.random.default_rng(0).standard_normal(192), 8, 0.0)
    x = H.coarse_pinv @ b
    np.testing.assert_allclose(L0 @ x, b, atol=1e-10)
    assert np.abs(Z.T @ x).max() < 1e-12
    np.testing.assert_allclose(H.coarse_pinv, np.linalg.pinv(L0, rcond=1e-10), atol=1e-9)


# ---------------------------------------------------------------- smoothers (Sec. 3.3)
def test_vanka_fixed_point_and_bruteforce():
    prob = I.thin_ellipse_stokes(8, kappa=1e2)
    H = multigrid.Hierarchy(prob, n_min=4)
    lev = H.fine
    L = lev.L
    N, n = 8, 64
    b = system.rhs(prob)
    w, _ = system.solve_direct(L, b, N, 0.0)
    x1 = smoothers.vanka_sweep(L, lev.dofs, lev.patches, w, b, 0.8)
    np.testing.assert_allclose(x1, w, atol=1e-11)
    # brute force: B = sum_c W_c R_c^T (R_c L R_c^T)^{-1} R_c with dofs found from face geometry
    Ld = L.toarray()
    Bm = np.zeros((3 * n, 3 * n))
    h = 1.0 / N
    for j in range(N):
        for i in range(N):
            cx, cy = (i + 0.5) * h, (j + 0.5) * h
            dofs = []
            for comp, (ox, oy) in ((0, (0.0, 0.5)), (1, (0.5, 0.0))):
                for jj in range(N):
                    for ii in range(N):
                        fx, fy = (ii + ox) * h, (jj + oy) * h
                        dx = (fx - cx) - np.round(fx - cx)
                        dy = (fy - cy) - np.round(fy - cy)
                        if abs(np.hypot(dx, dy) - 0.5 * h) < 1e-12:
                            dofs.append((comp * n + jj * N + ii, 0.5))
            dofs.append((2 * n + j * N + i, 1.0))
            idx = np.array([d for d, _ in dofs])
            wts = np.array([wt for _, wt in dofs])
            Lc = Ld[np.ix_(idx, idx)]
            Bm[np.ix_(idx, np.arange(3 * n))] += wts[:, None] * np.linalg.solve(Lc, np.eye(3 * n)[idx])
    rng = np.random.default_rng(1)
    x0 = rng.standard_normal(3 * n)
    bb = rng.standard_normal(3 * n)
    ref = x0 + 0.8 * Bm @ (bb - Ld @ x0)
    np.testing.assert_allclose(smoothers.vanka_sweep(L, lev.dofs, lev.patches, x0, bb, 0.8), ref, atol=1e-10)


def test_chebyshev_residual_polynomial():
    rng = np.random.default_rng(2)
    lam_max = 3.0
    ev = rng.uniform(0.1 * lam_max, lam_max, 50)
    b = rng.standard_normal(50)
    for k in (1, 2, 3, 5):
        x = smoothers.chebyshev(lambda z: ev * z, np.ones(50), b, lam_max, k, 0.1, 1.1)
        lmin, lmax = 0.1 * lam_max, 1.1 * lam_max
        theta, delta = (lmax + lmin) / 2, (lmax - lmin) / 2
        Tk = np.polynomial.chebyshev.Chebyshev.basis(k)
        p = Tk((theta - ev) / delta) / Tk(theta / delta)
        np.testing.assert_allclose(b - ev * x, p * b, atol=1e-12)
    # with a diagonal preconditioner: operator diag(d) * ev on the same interval
    d = rng.uniform(0.5, 2.0, 50)
    x = smoothers.chebyshev(lambda z: (ev / d) * z * d, 1.0 / d, b, lam_max, 2, 0.1, 1.1)
    lmin, lmax = 0.1 * lam_max, 1.1 * lam_max
    theta, delta = (lmax + lmin) / 2, (lmax - lmin) / 2
    p = np.polynomial.chebyshev.Chebyshev.basis(2)((theta - ev / d) / delta) / \
        np.polynomial.chebyshev.Chebyshev.basis(2)(theta / delta)
    np.testing.assert_allclose(b - ev * x, p * b, atol=1e-12)


def test_power_estimate_on_diagonal():
    ev = np.linspace(0.5, 4.0, 40)
    lam = smoothers.power_max(lambda z: ev * z, np.ones(40), 40, 400)
    assert abs(lam - 4.0) < 1e-3
    assert smoothers.hash_vector(3)[0] == (2654435761 % 2 ** 32) / 2 ** 32 - 0.5


def test_schur_factorisation_exact_inverse():
    prob = I.thin_ellipse_re(16, kappa=1e3)
    L = system.operator_of(prob)
    n = 256
    G, D = mac.gradient(16), mac.divergence(16)
    AIB = L[:2 * n, :2 * n].toarray()
    Ainv = np.linalg.inv(AIB)
    Mexact = D.toarray() @ Ainv @ G.toarray()
    Mp = np.linalg.pinv(Mexact, rcond=1e-10)
    r = system.project(np.random.default_rng(3).standard_normal(3 * n), 16, 1.0)
    x = smoothers.sc_apply(r, 2 * n, lambda q: Ainv @ q, lambda q: Mp @ q, G, D)
    ref, _ = system.solve_direct(L, r, 16, 1.0)
    np.testing.assert_allclose(system.project(x, 16, 1.0), system.project(ref, 16, 1.0), atol=1e-10)


# ---------------------------------------------------------------- multigrid (Alg. 1)
@pytest.mark.parametrize("smoother", ["vanka", "sc"])
def test_two_grid_equals_dense_operator(smoother):
    prob = I.thin_ellipse_stokes(16, kappa=1e2)
    H = multigrid.Hierarchy(prob, smoother=smoother)
    assert H.lmax == 1
    n3 = 3 * 256
    L = H.fine.L.toarray()
    # dense smoother iteration matrix S (b = 0) and its affine part
    Eye = np.eye(n3)
    S = np.stack([H.smooth(1, Eye[:, k], np.zeros(n3), 1) for k in range(n3)], axis=1)
    Bs = np.stack([H.smooth(1, np.zeros(n3), Eye[:, k], 1) for k in range(n3)], axis=1)
    P, R = H.P[1].toarray(), H.R[1].toarray()
    CG = P @ H.coarse_pinv @ R
    b = np.random.default_rng(7).standard_normal(n3)
    x = np.zeros(n3)
    for _ in range(H.nu1):
        x = S @ x + Bs @ b
    x = x + CG @ (b - L @ x)
    for _ in range(H.nu2):
        x = S @ x + Bs @ b
    np.testing.assert_allclose(H.vcycle(b), x, atol=1e-9 * np.abs(x).max())


def test_vcycle_iteration_contracts():
    prob = I.thin_ellipse_stokes(32, kappa=1e2)
    H = multigrid.Hierarchy(prob)
    L = H.fine.L
    b = system.rhs(prob)
    x = np.zeros_like(b)
    r0 = np.linalg.norm(b)
    for _ in range(8):
        x = x + H.vcycle(b - L @ x)
    assert np.linalg.norm(b - L @ x) < 1e-3 * r0


# ---------------------------------------------------------------- FGMRES
def test_fgmres_minimal_residual_identity_preconditioner():
    rng = np.random.default_rng(9)
    n = 30
    A = rng.standard_normal((n, n)) + 6 * np.eye(n)
    b = rng.standard_normal(n)
    for k in (1, 3, 7):
        x, its, hist, _ = krylov.fgmres(lambda z: A @ z, lambda z: z, b, rtol=1e-30, max_it=k)
        Kb = np.stack([np.linalg.matrix_power(A, i) @ b for i in range(k)], axis=1)
        Q, _ = np.linalg.qr(Kb)
        y = np.linalg.lstsq(A @ Q, b, rcond=None)[0]
        best = np.linalg.norm(b - A @ Q @ y)
        assert abs(np.linalg.norm(b - A @ x) - best) < 1e-10
        assert abs(hist[-1] - best) < 1e-10
    x, its, hist, conv = krylov.fgmres(lambda z: A @ z, lambda z: z, b, rtol=1e-13, max_it=n)
    assert conv and np.linalg.norm(A @ x - b) < 1e-11 * np.linalg.norm(b)


def test_fgmres_vcycle_converges_to_direct_solution():
    prob = I.thin_ellipse_stokes(32, kappa=1e2)
    L = system.operator_of(prob)
    b = system.rhs(prob)
    w, _ = system.solve_direct(L, b, 32, 0.0)
    w = system.project(w, 32, 0.0)
    for sm in ("vanka", "sc"):
        H = multigrid.Hierarchy(prob, smoother=sm)
        x, its, hist, conv = krylov.fgmres(lambda z: L @ z, H.vcycle, b, rtol=1e-13,
                                           project=lambda z: system.project(z, 32, 0.0))
        assert conv and its < 40
        assert np.abs(x - w).max() < 1e-10 * np.abs(w).max()
        assert np.linalg.norm(b - L @ x) < 2e-13 * np.linalg.norm(b)


def _iters(prob, smoother="vanka", rtol=1e-8):
    L = system.operator_of(prob)
    b = system.rhs(prob)
    H = multigrid.Hierarchy(prob, smoother=smoother)
    return krylov.fgmres(lambda z: L @ z, H.vcycle, b, rtol=rtol)[1]


def test_iteration_trends():
    """Paper Sec. 1 and 6: iterations grow with stiffness and Reynolds number, and are roughly
    mesh-independent for Stokes flow at moderate stiffness."""
    its_k = [_iters(I.thin_ellipse_stokes(32, kappa=k)) for k in (1e0, 1e2, 1e4, 1e5)]
    assert all(a <= b for a, b in zip(its_k, its_k[1:])), its_k
    assert its_k[-1] > its_k[0]
    i32 = _iters(I.thin_ellipse_stokes(32, kappa=1e2))
    i64 = _iters(I.thin_ellipse_stokes(64, kappa=1e2))
    assert abs(i64 - i32) <= 3, (i32, i64)
    # Reynolds number: rho = 1, dt = 1e-2, mu decreasing
    its_re = []
    for mu in (1.0, 1e-2, 1e-4):
        p = I.thin_ellipse_stokes(32, kappa=1e3)
        p.rho, p.mu = 1.0, mu
        its_re.append(_iters(p))
    assert all(a <= b for a, b in zip(its_re, its_re[1:])), its_re


def test_time_loop_matches_chained_full_system_solves():
    """Two semi-implicit steps (Eq. imp-X-new after each eliminated solve) give the same u, p and X
    as solving the full (u, p, X^{n+1}) system of Eq. system-impib twice, each time at the new X."""
    from oracle import timestep
    prob = I.disk_stokes(16, kappa=30.0)
    ws, Xs = timestep.run(prob, 2)
    p = prob
    for k in range(2):
        w3, X3 = system.solve_full_system(p)
        np.testing.assert_allclose(system.project(w3, 16, 0.0), ws[k], atol=1e-10 * np.abs(ws[k]).max())
        np.testing.assert_allclose(X3, Xs[k + 1], atol=1e-12)
        p = timestep.with_positions(p, X3)
    assert np.abs(Xs[2] - Xs[0]).max() > 1e-6      # the structure moved


def test_fgmres_smooth_is_gmres_with_identity_preconditioner():
    """With B = identity the wrapped smoothing step is k steps of GMRES: x + argmin over the Krylov
    space K_k(L, r) of the residual, checked against a brute-force least-squares solve on the
    explicit Krylov basis."""
    rng = np.random.default_rng(7)
    n, k = 40, 3
    L = np.eye(n) * 3.0 + rng.standard_normal((n, n)) * 0.3
    x = rng.standard_normal(n)
    b = rng.standard_normal(n)
    out = smoothers.fgmres_smooth(L, lambda v: v.copy(), x, b, k)
    r = b - L @ x
    Kb = np.stack([np.linalg.matrix_power(L, i) @ r for i in range(k)], axis=1)
    c = np.linalg.lstsq(L @ Kb, r, rcond=None)[0]
    np.testing.assert_allclose(out, x + Kb @ c, rtol=1e-9, atol=1e-12)


def test_fgmres_smooth_with_exact_preconditioner_solves_in_one_step():
    rng = np.random.default_rng(8)
    n = 30
    L = np.eye(n) * 2.0 + rng.standard_normal((n, n)) * 0.2
    x = rng.standard_normal(n)
    b = rng.standard_normal(n)
    out = smoothers.fgmres_smooth(L, lambda v: np.linalg.solve(L, v), x, b, 1)
    assert np.linalg.norm(b - L @ out) < 1e-12 * np.linalg.norm(b)
    # a zero residual returns x unchanged
    I3 = np.eye(5)
    v = rng.standard_normal(5)
    np.testing.assert_array_equal(smoothers.fgmres_smooth(I3, lambda q: q, v, v.copy(), 2), v)


@pytest.mark.parametrize("smoother", ["vanka", "sc"])
def test_krylov_wrapped_vcycle_is_a_convergent_preconditioner(smoother):
    """The wrapped smoothers (FGMRES(nu) preconditioned by one undamped sweep) inside the V-cycle:
    FGMRES on the 32^2 thin ellipse converges to 1e-8, and no slower than with the damped sweeps
    by more than two iterations."""
    prob = I.thin_ellipse_stokes(32)
    L = system.operator_of(prob)
    b = system.rhs(prob)
    its = {}
    for wrap in (False, True):
        H = multigrid.Hierarchy(prob, smoother=smoother, krylov=wrap)
        x, it, hist, conv = krylov.fgmres(lambda z: L @ z, H.vcycle, b, rtol=1e-8, max_it=100, restart=100,
                                          project=lambda v: system.project(v, 32, prob.rho))
        assert conv, (smoother, wrap, it)
        its[wrap] = it
    assert its[True] <= its[False] + 2, its


# ------------------------------------------- multicolour Gauss-Seidel inside SC (Sec. 3.3, SC smoothing)
def _red_black_perm(colours):
    return np.concatenate([np.flatnonzero(colours == 0), np.flatnonzero(colours == 1)])


@pytest.mark.parametrize("which", ["A", "Mh"])
def test_multicolour_sgs_is_textbook_symmetric_gauss_seidel(which):
    """Without IB couplings the colour passes are Gauss-Seidel in red-black order: a forward sweep is
    the lower-triangular solve (D + L) z = r of the red-black permuted operator and the backward
    sweep adds (D + U)^{-1} (r - Op z).  Triangular solves from scipy, not the colour passes."""
    from scipy.sparse.linalg import spsolve_triangular
    N = 16
    A = mac.momentum(N, 1.0, 1e-2, 1e-3).tocsr()
    dA = A.diagonal()
    if which == "A":
        Op, d, col = A, dA, smoothers.rb_colours(N, 2)
    else:
        Op = (mac.divergence(N) @ sp.diags(1.0 / dA) @ mac.gradient(N)).tocsr()
        d, col = Op.diagonal(), smoothers.rb_colours(N, 1)
    r = np.random.default_rng(4).standard_normal(Op.shape[0])
    perm = _red_black_perm(col)
    Pm = Op[perm][:, perm].tocsr()
    lower = sp.tril(Pm, format="csr")
    upper = sp.triu(Pm, format="csr")
    rp = r[perm]
    z1 = spsolve_triangular(lower, rp, lower=True)
    z2 = z1 + spsolve_triangular(upper, rp - Pm @ z1, lower=False)
    ref = np.empty_like(r)
    ref[perm] = z2
    got = smoothers.sgs_multicolour(Op, d, col, r)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_multicolour_sgs_is_symmetric_positive_with_ib_couplings():
    """With the IB couplings (which link faces of one colour) the forward-backward colour order
    still gives a symmetric preconditioner, positive on this problem: r1.P r2 = r2.P r1, r.P r > 0."""
    prob = I.thin_ellipse_re(32, kappa=1e4, seed=2)
    H = multigrid.Hierarchy(prob, smoother="sc", sc_relax="sgs")
    lev = H.fine
    assert (lev.AIB - lev.A).nnz > 0
    P = lambda q: smoothers.sgs_multicolour(lev.AIB, lev.dA, smoothers.rb_colours(lev.N, 2), q)
    rng = np.random.default_rng(5)
    r1, r2 = rng.standard_normal((2, 2 * lev.n))
    a, b = r1 @ P(r2), r2 @ P(r1)
    assert abs(a - b) <= 1e-12 * max(abs(a), abs(b))
    assert r1 @ P(r1) > 0 and r2 @ P(r2) > 0


def test_chebyshev_with_exact_preconditioner_closed_form():
    """A callable preconditioner enters the Chebyshev iteration as P: with P = Op^{-1} every
    eigenvalue of P Op is 1, so with lam_max = 1 the iterate is (1 - T_k((theta - 1)/delta) /
    T_k(theta/delta)) Op^{-1} b."""
    rng = np.random.default_rng(6)
    n = 30
    Q = rng.standard_normal((n, n))
    Op = Q @ Q.T + n * np.eye(n)
    b = rng.standard_normal(n)
    exact = np.linalg.solve(Op, b)
    theta, delta = 0.6, 0.5
    for k in (1, 2, 4):
        x = smoothers.chebyshev(lambda z: Op @ z, lambda q: np.linalg.solve(Op, q), b, 1.0, k, 0.1, 1.1)
        Tk = np.polynomial.chebyshev.Chebyshev.basis(k)
        np.testing.assert_allclose(x, (1 - Tk((theta - 1) / delta) / Tk(theta / delta)) * exact, atol=1e-12)


def test_sc_with_multicolour_gs_is_a_convergent_preconditioner():
    """SC smoothing with symmetric red-black Gauss-Seidel inside both Chebyshev iterations: FGMRES
    with its V-cycle converges to 1e-8 on the 32^2 thin ellipse (Stokes and kappa = 1e4 with inertia)."""
    for prob in (I.thin_ellipse_stokes(32), I.thin_ellipse_re(32, kappa=1e4, seed=2)):
        L = system.operator_of(prob)
        b = system.rhs(prob)
        H = multigrid.Hierarchy(prob, smoother="sc", sc_relax="sgs")
        x, it, hist, conv = krylov.fgmres(lambda z: L @ z, H.vcycle, b, rtol=1e-8, max_it=100, restart=100,
                                          project=lambda v: system.project(v, 32, prob.rho))
        assert conv, it


# ------------------------------------------------------ box RAS smoother (Sec. 3.3, Alg. 2 with boxes)
def test_ras_one_cell_boxes_are_restricted_vanka():
    """b = 1, o = 0: each subdomain is the 5-dof cell patch, and each face takes the correction of the
    cell to its right (u) or above (v): the Vanka patch solve with weights (1, 0, 1, 0, 1)."""
    prob = I.thin_ellipse_re(16, kappa=1e3)
    L = system.operator_of(prob).tocsr()
    N = 16
    rng = np.random.default_rng(9)
    x, bb = rng.standard_normal((2, 3 * N * N))
    boxes = smoothers.ras_boxes(N, 1, 0)
    got = smoothers.ras_sweep(L, boxes, smoothers.ras_factors(L, boxes), x, bb, 0.9)
    dofs = smoothers.vanka_patch_dofs(N)
    P = smoothers.vanka_patches(L, dofs)
    r = bb - L @ x
    delta = np.linalg.solve(P, r[dofs][..., None])[..., 0]
    dx = np.zeros_like(x)
    np.add.at(dx, dofs.ravel(), (delta * np.array([1.0, 0.0, 1.0, 0.0, 1.0])).ravel())
    np.testing.assert_allclose(got, x + 0.9 * dx, rtol=0, atol=1e-10 * np.abs(x + 0.9 * dx).max())


@pytest.mark.parametrize("b,o", [(4, 1), (2, 2), (4, 0), (2, 1)])
def test_ras_subdomains_are_the_geometric_boxes(b, o):
    """Each subdomain's dofs are exactly the faces and cell centres inside its extended square (faces on
    its edges included), periodically; it owns those inside the core square (left and bottom edges
    included); the owned sets partition all dofs.  Checked from dof positions, not index loops."""
    N = 16
    h = 1.0 / N
    idx = np.arange(N * N)
    i, j = idx % N, idx // N
    pos = [(i * h, (j + 0.5) * h), ((i + 0.5) * h, j * h), ((i + 0.5) * h, (j + 0.5) * h)]
    owners = np.zeros(3 * N * N, dtype=int)
    for k, (d, own) in enumerate(smoothers.ras_boxes(N, b, o)):
        I0, J0 = (k % (N // b)) * b, (k // (N // b)) * b
        expect, expect_own = [], []
        for comp, (px, py) in enumerate(pos):
            rx = np.round(((px - (I0 - o) * h) % 1.0) / h * 2) / 2   # offsets in cells from the box corner
            ry = np.round(((py - (J0 - o) * h) % 1.0) / h * 2) / 2
            inside = (rx <= b + 2 * o) & (ry <= b + 2 * o)
            if comp == 0:
                inside &= ry > 0
            elif comp == 1:
                inside &= rx > 0
            else:
                inside &= (rx > 0) & (ry > 0)
            core = inside & (rx >= o) & (rx < o + b) & (ry >= o) & (ry < o + b)
            expect += list(comp * N * N + idx[inside])
            expect_own += list(comp * N * N + idx[core])
        assert sorted(d.tolist()) == sorted(expect)
        assert sorted(d[own].tolist()) == sorted(expect_own)
        owners[d[own]] += 1
    assert (owners == 1).all()


def test_ras_fixed_point_and_convergent_vcycle():
    """The exact solution is a fixed point of a RAS sweep; FGMRES with the RAS V-cycle (4 x 4 boxes,
    overlap 1) converges to 1e-8, including the 32^2 disk at kappa = 1e6."""
    prob = I.disk_stokes(32, kappa=1e6, seed=1)
    L = system.operator_of(prob)
    b = system.rhs(prob)
    H = multigrid.Hierarchy(prob, smoother="ras", box=4, overlap=1)
    xs, _ = system.solve_direct(L, b, 32, prob.rho)
    lev = H.fine
    y = smoothers.ras_sweep(lev.L, lev.boxes, lev.factors, xs, b, 1.0)
    assert np.abs(y - xs).max() <= 1e-9 * np.abs(xs).max()
    x, it, hist, conv = krylov.fgmres(lambda z: L @ z, H.vcycle, b, rtol=1e-8, max_it=100, restart=100,
                                      project=lambda v: system.project(v, 32, prob.rho))
    assert conv, it


def test_ras_16x16_boxes_and_the_exact_level_reading():
    """16 x 16 boxes with overlap 4 (Sec. 5.1.1, 5.2.1) on the 32^2 disk: level 2 (32^2) holds four
    boxes of 1,776 dofs whose subdomains are the geometric extended squares and whose owned sets
    partition the dofs; level 1 (16^2) is too small for them (`ras_wraps`), and its sweep is the exact
    level solve: from any x, the new residual lies in the operator's kernel (constant pressure, and
    constant velocities at rho = 0), and a second sweep leaves x unchanged up to that kernel.  The exact
    solution is a fixed point on both levels."""
    prob = I.disk_stokes(32, kappa=1e2, seed=1)
    H = multigrid.Hierarchy(prob, smoother="ras", box=16, overlap=4)
    lev2, lev1 = H.levels[2], H.levels[1]
    assert lev1.boxes is None and smoothers.ras_wraps(16, 16, 4) and not smoothers.ras_wraps(32, 16, 4)
    assert len(lev2.boxes) == 4 and all(len(d) == 3 * 24 * 24 + 2 * 24 for d, _ in lev2.boxes)
    owners = np.zeros(3 * 32 * 32, dtype=int)
    for d, own in lev2.boxes:
        owners[d[own]] += 1
    assert (owners == 1).all()
    rng = np.random.default_rng(16)
    x = rng.standard_normal(3 * lev1.n)
    b = rng.standard_normal(3 * lev1.n)
    y = H.smooth(1, x, b, 1)
    r = b - lev1.L @ y
    Z = system.null_basis(16, prob.rho)
    assert np.abs(r - Z @ (Z.T @ r)).max() <= 1e-10 * np.abs(b).max()
    y2 = H.smooth(1, y, b, 1)
    assert np.abs(y2 - y).max() <= 1e-10 * np.abs(y).max()
    L = system.operator_of(prob)
    bf = system.rhs(prob)
    xs, _ = system.solve_direct(L, bf, 32, prob.rho)
    assert np.abs(H.smooth(2, xs, bf, 1) - xs).max() <= 1e-9 * np.abs(xs).max()


# ------------------------------------------------ the paper's structures (Sec. 5.1, 5.2), periodic box
def test_paper_structures_geometry():
    """Thick annulus: M1 = 19N/8 by M2 = 3N/32 + 1 markers on circles of radius r + s2_m, fibres closed
    along s1 only; thin circle: M1 markers on radius r; marker spacing about 2h/3 (Sec. 5.1)."""
    N = 64
    a = I.thick_annulus(N, 50.0)
    M1, M2 = 19 * N // 8, 3 * N // 32 + 1
    assert a.M == M1 * M2 and a.E == M1 * M2
    rad = np.hypot(a.X[:, 0] - 0.5, a.X[:, 1] - 0.5).reshape(M2, M1)
    np.testing.assert_allclose(rad, (0.25 + np.arange(M2) / (M2 - 1) / 16)[:, None] * np.ones(M1), atol=1e-15)
    e = a.edges
    assert ((e[:, 0] // M1) == (e[:, 1] // M1)).all()                 # links stay on one fibre
    assert (((e[:, 1] - e[:, 0]) % M1) == 1).all()                    # s1 neighbours, closed
    c = I.thin_circle(N, 50.0)
    assert c.M == M1
    spacing = np.linalg.norm(c.X - np.roll(c.X, -1, axis=0), axis=1)
    np.testing.assert_allclose(spacing, 2 * 0.25 * np.sin(np.pi / M1), rtol=1e-13)   # chord of the step
    assert 0.6 < spacing.mean() * N < 0.7                             # about 2h/3


@pytest.mark.parametrize("kind", ["circle", "annulus"])
def test_paper_structures_force_continuum_limit(kind):
    """The spring force of the initial configuration is the discrete alpha d^2X/ds1^2 with the nodal
    quadrature weight: on a circle of radius R each marker's force points to the centre with magnitude
    alpha R ds1 wq (2 sin(ds1/2)/ds1)^2, so the total magnitude tends to 2 pi R alpha wq (wq = 1 for
    the thin circle; ds2 per fibre of the annulus).  Checked with the oracle's spring operator."""
    N, gamma = 64, 5.0
    st = I.thin_circle(N, gamma) if kind == "circle" else I.thick_annulus(N, gamma)
    F = ib.spring_force(st.X, st.edges, st.kappa)
    M1 = 19 * N // 8
    ds1 = 2 * np.pi / M1
    alpha = (7.0 if kind == "circle" else 1.0) * gamma * I.ALPHA_UNIT
    radial = st.X - 0.5
    rad = np.linalg.norm(radial, axis=1)
    cosang = -(F * radial).sum(1) / (np.linalg.norm(F, axis=1) * rad)
    np.testing.assert_allclose(cosang, 1.0, atol=1e-12)                # points to the centre
    if kind == "circle":
        wq, radii = np.ones(M1), np.full(M1, 0.25)
    else:
        M2 = 3 * N // 32 + 1
        wq = np.full(M1 * M2, (1.0 / 16) / (M2 - 1))
        radii = rad
    expect = alpha * radii * ds1 * wq * (2 * np.sin(ds1 / 2) / ds1) ** 2
    np.testing.assert_allclose(np.linalg.norm(F, axis=1), expect, rtol=1e-12)


def test_paper_workload_trends_on_the_oracle():
    """Iteration trends the paper states (Sec. 5.1, 5.2), at 32^2 with box RAS (4 x 4, overlap 1) to
    1e-12: more iterations for the thin circle than for the annulus at the same gamma, and no fewer
    as gamma grows (5 -> 500)."""
    its = {}
    for kind in ("annulus", "circle"):
        for gamma in (5.0, 500.0):
            prob = I.paper_problem(kind, 32, gamma)
            L = system.operator_of(prob)
            b = system.rhs(prob)
            H = multigrid.Hierarchy(prob, smoother="ras", box=4, overlap=1)
            _, it, _, conv = krylov.fgmres(lambda z: L @ z, H.vcycle, b, rtol=1e-12, max_it=100, restart=100,
                                           project=lambda v: system.project(v, 32, prob.rho))
            its[kind, gamma] = it
    assert its["annulus", 500.0] >= its["annulus", 5.0], its
    assert its["circle", 500.0] >= its["circle", 5.0], its
    assert its["circle", 500.0] >= its["annulus", 500.0], its


def test_ras_overlap_trend_on_the_thin_membrane():
    """The paper's finding for the thin membrane in Stokes flow at gamma = 500 (Sec. 5.2.1): solver
    performance depends strongly on the overlap width, and only larger subdomains with more overlap
    converge.  At 32^2 to 1e-12: 4 x 4 boxes with overlap 1 hit the 100-iteration cap, 8 x 8 boxes
    with overlap 2 converge, and more overlap on the 4 x 4 boxes helps."""
    prob = I.paper_problem("circle", 32, 500.0)
    L = system.operator_of(prob)
    b = system.rhs(prob)
    its = {}
    for bx, o in ((4, 1), (4, 2), (8, 2)):
        H = multigrid.Hierarchy(prob, smoother="ras", box=bx, overlap=o)
        _, it, _, conv = krylov.fgmres(lambda z: L @ z, H.vcycle, b, rtol=1e-12, max_it=100, restart=100,
                                       project=lambda v: system.project(v, 32, prob.rho))
        its[bx, o] = (it, conv)
    assert not its[4, 1][1], its
    assert its[4, 2][1] and its[8, 2][1], its
    assert its[8, 2][0] < its[4, 2][0] < 100, its
