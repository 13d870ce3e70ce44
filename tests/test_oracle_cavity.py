"""Pins of the lid-driven cavity oracle (Sec. 5: no-slip walls, regularised lid) against facts the
mathematics fixes: identities, agreement with the (separately pinned) periodic operator away from
the walls, second-order convergence to a manufactured Stokes solution, Cauchy convergence of the
lid-driven flow, and convergence of the multigrid-preconditioned solve."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import cavity, ib, krylov, mac, system
from paper_1612_02208_gb300 import inputs as I


def _annulus(N, gamma):
    return I.thick_annulus(N, gamma)


def test_cavity_operator_identities():
    N = 16
    G, D = cavity.gradient(N), cavity.divergence(N)
    assert abs(D + G.T).max() == 0
    A = cavity.momentum(N, 1.0, 1e-2, 1e-3)
    assert abs(A - A.T).max() == 0
    st = _annulus(32, 5.0)
    L = cavity.operator(32, 0.0, 1.0, 0.01, st.X, st.edges, st.kappa)
    assert abs(L - L.T).max() <= 1e-9 * abs(L).max()
    assert L.shape[0] == 3 * 32 * 32 - 2 * 32
    # the kernel is the constant pressure only
    Z = cavity.null_basis(32)
    assert np.abs(L @ Z[:, 0]).max() <= 1e-12 * abs(L).max()


def test_cavity_matches_periodic_operator_away_from_walls():
    """Rows of unknowns two or more cells from every wall equal the periodic operator's rows."""
    N = 16
    st = _annulus(32, 5.0)          # markers only matter through the shared restriction
    Lc = cavity.operator(N, 1.0, 1e-2, 1e-3, np.zeros((0, 2)), np.zeros((0, 2), np.int32), np.zeros(0))
    Lp = system.stokes_ib_operator(N, 1.0, 1e-2, 1e-3, np.zeros((0, 2)), np.zeros((0, 2), np.int32), np.zeros(0))
    idx = cavity.interior(N)
    n = N * N
    for r, g in enumerate(idx):
        comp, loc = g // n, g % n
        i, j = loc % N, loc // N
        if min(i, j, N - 1 - i, N - 1 - j) < 2:
            continue
        row_c = Lc.getrow(r).toarray().ravel()
        row_p = Lp.getrow(g).toarray().ravel()[idx]
        np.testing.assert_allclose(row_c, row_p, rtol=0, atol=1e-12 * np.abs(row_p).max())
    del st


def _manufactured():
    """Stokes (rho = 0, mu = 1) with the stream function psi = sin^2(pi x) sin^2(pi y): u = psi_y,
    v = -psi_x vanish on all walls and are divergence-free; p = cos(pi x) cos(pi y); the forcing
    f = -Lap u + grad p, derived symbolically."""
    import sympy as sy
    x, y = sy.symbols("x y")
    psi = sy.sin(sy.pi * x) ** 2 * sy.sin(sy.pi * y) ** 2
    u, v = sy.diff(psi, y), -sy.diff(psi, x)
    p = sy.cos(sy.pi * x) * sy.cos(sy.pi * y)
    fu = -(sy.diff(u, x, 2) + sy.diff(u, y, 2)) + sy.diff(p, x)
    fv = -(sy.diff(v, x, 2) + sy.diff(v, y, 2)) + sy.diff(p, y)
    f = lambda e: sy.lambdify((x, y), e, "numpy")
    return f(u), f(v), f(fu), f(fv)


def _faces(N):
    h = 1.0 / N
    j, i = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    i, j = i.ravel(), j.ravel()
    return (i * h, (j + 0.5) * h), ((i + 0.5) * h, j * h)


def test_cavity_manufactured_stokes_converges_at_second_order():
    ue, ve, fu, fv = _manufactured()
    errs = []
    for N in (16, 32, 64):
        (xu, yu), (xv, yv) = _faces(N)
        n = N * N
        full = np.concatenate([fu(xu, yu), fv(xv, yv), np.zeros(n)])
        idx = cavity.interior(N)
        b = full[idx]
        L = cavity.operator(N, 0.0, 1.0, 1.0, np.zeros((0, 2)), np.zeros((0, 2), np.int32), np.zeros(0))
        w = cavity.solve_direct(L, b, N)
        exact = np.concatenate([ue(xu, yu), ve(xv, yv), np.zeros(n)])[idx]
        nv = 2 * n - 2 * N
        errs.append(np.abs(w[:nv] - exact[:nv]).max())
        D = cavity.divergence(N)
        assert np.abs(D @ w[:nv]).max() <= 1e-9 * np.abs(w[:nv]).max()     # discretely divergence-free
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0, errs


def test_cavity_manufactured_lid_converges_at_second_order():
    """A manufactured Stokes flow (mu = 1) whose top-wall velocity is the regularised lid: stream
    function psi = u_lid(x) (y^3 - y^2), so u = psi_y equals u_lid on y = 1 and vanishes on the other
    walls, v = -psi_x vanishes on all walls (u_lid' = 0 at x = 0, 1), and the flow is divergence-free.
    With the lid's right-hand side term the solve converges at second order; a wrong factor, sign or
    face position of that term leaves an O(1) or O(h) error."""
    import sympy as sy
    x, y = sy.symbols("x y")
    lid = (1 - sy.cos(2 * sy.pi * x)) / 2
    psi = lid * (y ** 3 - y ** 2)
    u, v = sy.diff(psi, y), -sy.diff(psi, x)
    p = sy.cos(sy.pi * x) * sy.cos(sy.pi * y)
    fu = -(sy.diff(u, x, 2) + sy.diff(u, y, 2)) + sy.diff(p, x)
    fv = -(sy.diff(v, x, 2) + sy.diff(v, y, 2)) + sy.diff(p, y)
    F = lambda e: sy.lambdify((x, y), e, "numpy")
    ue, ve, fue, fve = F(u), F(v), F(fu), F(fv)
    xs = np.linspace(0.0, 1.0, 11)
    np.testing.assert_allclose(cavity.lid_velocity(xs), F(lid)(xs, 0.0), atol=1e-15)   # the oracle's lid
    errs = []
    for N in (16, 32, 64):
        (xu, yu), (xv, yv) = _faces(N)
        n = N * N
        idx = cavity.interior(N)
        b = np.concatenate([fue(xu, yu), fve(xv, yv), np.zeros(n)])[idx] + cavity.lid_rhs(N, 1.0)
        L = cavity.operator(N, 0.0, 1.0, 1.0, np.zeros((0, 2)), np.zeros((0, 2), np.int32), np.zeros(0))
        w = cavity.solve_direct(L, b, N)
        exact = np.concatenate([ue(xu, yu) * np.ones(n), ve(xv, yv) * np.ones(n), np.zeros(n)])[idx]
        nv = 2 * n - 2 * N
        errs.append(np.abs(w[:nv] - exact[:nv]).max())
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5, errs


def test_cavity_pressure_prolongation_is_local_and_reproduces_linears():
    """Bilinear prolongation reproduces linear fields on fine cells whose four coarse neighbours lie
    inside, and fields linear in one coordinate away from the walls across that coordinate; no fine
    cell takes a value from a coarse cell on the far side of a wall (the periodic wrap is gone), and
    every row sums to 1, so a zero or wrapped ghost fails."""
    Nc = 8
    Nf = 2 * Nc
    P = cavity.prolong_pressure(Nc)
    Xc = (np.arange(Nc) + 0.5) / Nc
    Xf = (np.arange(Nf) + 0.5) / Nf
    YYc, XXc = np.meshgrid(Xc, Xc, indexing="ij")
    YYf, XXf = np.meshgrid(Xf, Xf, indexing="ij")
    inner = (slice(1, Nf - 1), slice(1, Nf - 1))
    lin = (P @ (0.3 + 1.7 * XXc - 0.9 * YYc).ravel()).reshape(Nf, Nf)
    np.testing.assert_allclose(lin[inner], (0.3 + 1.7 * XXf - 0.9 * YYf)[inner], atol=1e-14)
    fy = (P @ (2.0 * YYc).ravel()).reshape(Nf, Nf)
    np.testing.assert_allclose(fy[1:Nf - 1, :], (2.0 * YYf)[1:Nf - 1, :], atol=1e-14)
    fx = (P @ (2.0 * XXc).ravel()).reshape(Nf, Nf)
    np.testing.assert_allclose(fx[:, 1:Nf - 1], (2.0 * XXf)[:, 1:Nf - 1], atol=1e-14)
    C = P.tocoo()
    fi, fj, ci, cj = C.row % Nf, C.row // Nf, C.col % Nc, C.col // Nc
    assert np.all(np.abs(Xf[fi] - Xc[ci]) < 1.0 / Nc) and np.all(np.abs(Xf[fj] - Xc[cj]) < 1.0 / Nc)
    np.testing.assert_allclose(np.asarray(P.sum(axis=1)).ravel(), 1.0, atol=1e-15)


def test_cavity_lid_driven_flow_cauchy_convergence():
    """Stokes flow driven by the regularised lid alone: u sampled on the coarse u faces (the mean of the
    two fine faces around each coarse face centre) converges at about second order."""
    def solve(N):
        L = cavity.operator(N, 0.0, 1.0, 1.0, np.zeros((0, 2)), np.zeros((0, 2), np.int32), np.zeros(0))
        return cavity.embed(N, cavity.solve_direct(L, cavity.lid_rhs(N, 1.0), N))

    def u_on(Nc, wf, Nf):
        uf = wf[: Nf * Nf].reshape(Nf, Nf)          # [j][i]
        r = Nf // Nc
        return 0.5 * (uf[r // 2 - 1::r, ::r] + uf[r // 2::r, ::r])   # rows around the coarse centres

    w16, w32, w64 = solve(16), solve(32), solve(64)
    u16 = w16[:256].reshape(16, 16)
    d1 = np.abs(u_on(16, w32, 32) - u16).max()
    d2 = np.abs(u_on(16, w64, 64) - u_on(16, w32, 32)).max()
    assert d1 / d2 > 3.0, (d1, d2)
    assert np.abs(w64[: 64 * 64]).max() > 0.1     # the lid drives a flow


def test_cavity_transfers():
    """RT0: D_f P_u = (injection) D_c on the cavity; the pressure prolongation keeps constants."""
    Nc, Nf = 8, 16
    rng = np.random.default_rng(3)
    wc = rng.standard_normal(2 * Nc * Nc - 2 * Nc)
    dc = cavity.divergence(Nc) @ wc
    df = cavity.divergence(Nf) @ (cavity.prolong_velocity(Nc) @ wc)
    inj = dc.reshape(Nc, Nc).repeat(2, axis=0).repeat(2, axis=1).ravel()
    np.testing.assert_allclose(df, inj, atol=1e-12 * np.abs(inj).max())
    np.testing.assert_allclose(cavity.prolong_pressure(Nc) @ np.ones(Nc * Nc), 1.0, atol=1e-15)


@pytest.mark.parametrize("smoother", ["vanka", "sc"])
def test_cavity_multigrid_preconditioned_solve(smoother):
    """The paper's annulus (gamma = 5) in the lid-driven cavity, Stokes, one step from the initial
    configuration: FGMRES with the cavity V-cycle reaches 1e-8 and the direct solution; the exact
    solution is a fixed point of a Vanka sweep."""
    N = 32
    st = _annulus(N, 5.0)
    rho, mu, dt = 0.0, 1.0, 0.32 / N
    L = cavity.operator(N, rho, mu, dt, st.X, st.edges, st.kappa)
    F = ib.spring_force(st.X, st.edges, st.kappa)
    skx = ib.spread_force(N, st.X, F)              # S K X^n on the periodic layout's faces
    b = cavity.lid_rhs(N, mu) + np.concatenate([skx, np.zeros(N * N)])[cavity.interior(N)]
    H = cavity.Hierarchy(N, rho, mu, dt, st.X, st.edges, st.kappa, smoother=smoother)
    x, it, hist, conv = krylov.fgmres(lambda z: L @ z, H.vcycle, b, rtol=1e-8, max_it=100, restart=100,
                                      project=lambda v: cavity.project(v, N))
    assert conv, it
    ref = cavity.solve_direct(L, b, N)
    assert np.abs(x - ref).max() <= 1e-6 * np.abs(ref).max()
    if smoother == "vanka":
        lev = H.levels[-1]
        y = cavity.vanka_sweep(lev.L, lev.patches, lev.factors, ref, b, 0.8)
        assert np.abs(y - ref).max() <= 1e-9 * np.abs(ref).max()
