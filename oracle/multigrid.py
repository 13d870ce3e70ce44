"""Level hierarchy and recursive V-cycle (Sec. 3.1, Alg. 1; Sec. 3.2).

Levels l = 0..lmax with N_l = n_min * 2^l (n_min = 8, the paper's 8 x 8 coarsest grid), h_l = 1/N_l.
On every level A^l, G^l, D^l are rediscretised; the IB part of the momentum operator is the
Galerkin projection [S K J]^l = R_u [S K J]^{l+1} P_u with R_u = P_u^T / 4 (formed here as the
literal sparse triple product), and L^l = [[A^l - dt [SKJ]^l, G^l], [-D^l, 0]].
The coarsest level is solved exactly with the pseudo-inverse of the dense L^0, written with the
orthonormal kernel basis Z as (L^0 + Z Z^T)^{-1} - Z Z^T (valid for symmetric L^0 whose kernel is
exactly span Z), which is the gauge-fixed exact coarse solve.

With the box RAS smoother, a level too small for the boxes (b does not divide N_l, or a subdomain's
e + 1 = b + 2o + 1 face columns would wrap onto themselves: 16 x 16 boxes with overlap 4 on 16^2) is
smoothed by the exact level solve with its gauge-fixed pseudo-inverse: the paper's cavity clips such a
box to the domain (Sec. 5), which makes the one box the whole level (smoothers.exact_level_sweep).

V-cycle (Alg. 1): on level l > 0 apply nu1 pre-smoothing sweeps, form r = b - L w, restrict,
recurse with a zero initial guess, prolong and add the correction, apply nu2 post-smoothing
sweeps; on level 0 solve exactly.

Pinned by: the Galerkin coarse operator is symmetric and equals (1/h_l^2) (J P)^T K (J P);
a two-level cycle equals the dense two-grid operator S^nu2 (I - P L0^+ R L) S^nu1 applied to b;
V-cycle iteration converges on Stokes-IB problems; iteration-count trends in stiffness and Re.
"""
import numpy as np
import scipy.sparse as sp

from . import ib, mac, smoothers, system, transfer


class Level:
    def __init__(self, N, rho, mu, dt, B):
        self.N = N
        self.n = N * N
        self.h = 1.0 / N
        self.A = mac.momentum(N, rho, mu, dt)
        self.G = mac.gradient(N)
        self.D = mac.divergence(N)
        self.B = B.tocsr()                          # [S K J]^l on the velocity faces
        self.AIB = (self.A - dt * self.B).tocsr()
        self.L = sp.bmat([[self.AIB, self.G], [-self.D, None]], format="csr")


class Hierarchy:
    def __init__(self, prob, n_min=8, smoother="vanka", omega=None, nu1=2, nu2=2,
                 cheb_iters=2, cheb_lo=0.1, cheb_hi=1.1, power_iters=10, lam_override=None, krylov=False,
                 sc_relax="jacobi", box=4, overlap=1):
        N = prob.N
        if N < n_min or (N // n_min) * n_min != N or (N // n_min) & (N // n_min - 1):
            raise ValueError("N must be n_min * 2^k")
        self.prob = prob
        self.rho, self.mu, self.dt = prob.rho, prob.mu, prob.dt
        self.smoother = smoother
        # krylov: each smoothing stage is FGMRES(nu) preconditioned by one undamped basic sweep
        # (Sec. 3.3); otherwise nu damped sweeps
        self.krylov = krylov
        # sc_relax: the point relaxation preconditioning the SC smoother's Chebyshev iterations,
        # "jacobi" or "sgs" (symmetric red-black Gauss-Seidel)
        self.sc_relax = sc_relax
        self.omega = 1.0 if krylov else ((0.8 if smoother == "vanka" else 1.0) if omega is None else omega)
        # smoother "ras": box subdomains of box x box cells with `overlap` cells on each side
        self.box, self.overlap = box, overlap
        self.nu1, self.nu2 = nu1, nu2
        self.cheb_iters, self.cheb_lo, self.cheb_hi = cheb_iters, cheb_lo, cheb_hi
        self.power_iters = power_iters
        lmax = int(round(np.log2(N // n_min)))
        s = prob.structure
        Bs = [None] * (lmax + 1)
        Bs[lmax] = ib.ib_operator(N, s.X, s.edges, s.kappa)
        self.P = [None] * (lmax + 1)     # P[l]: level l-1 -> l
        self.R = [None] * (lmax + 1)     # R[l]: level l -> l-1
        for l in range(lmax, 0, -1):
            Nc = n_min * 2 ** (l - 1)
            self.P[l] = transfer.prolong(Nc)
            self.R[l] = transfer.restrict(Nc)
            Pu = transfer.prolong_velocity(Nc)
            Ru = transfer.restrict_velocity(Nc)
            Bs[l - 1] = (Ru @ Bs[l] @ Pu).tocsr()
        self.levels = [Level(n_min * 2 ** l, self.rho, self.mu, self.dt, Bs[l]) for l in range(lmax + 1)]
        self.lmax = lmax
        L0 = self.levels[0].L.toarray()
        Z = system.null_basis(self.levels[0].N, self.rho)
        self.coarse_pinv = np.linalg.inv(L0 + Z @ Z.T) - Z @ Z.T
        for l, lev in enumerate(self.levels):
            if l == 0:
                continue
            if smoother == "vanka":
                lev.dofs = smoothers.vanka_patch_dofs(lev.N)
                lev.patches = smoothers.vanka_patches(lev.L, lev.dofs)
            elif smoother == "ras":
                if smoothers.ras_wraps(lev.N, box, overlap):   # exact level solve (smoothers.exact_level_sweep)
                    Z = system.null_basis(lev.N, self.rho)
                    lev.pinv = np.linalg.inv(lev.L.toarray() + Z @ Z.T) - Z @ Z.T
                    lev.boxes = None
                else:
                    lev.boxes = smoothers.ras_boxes(lev.N, box, overlap)
                    lev.factors = smoothers.ras_factors(lev.L, lev.boxes)
            else:
                lev.dA = lev.AIB.diagonal()
                PA, PM, lev.dM = smoothers.sc_preconditioners(lev.AIB, lev.G, lev.D, lev.dA, sc_relax)
                if lam_override is not None:
                    lev.lamA, lev.lamM = lam_override[l]
                else:
                    lev.lamA = smoothers.power_max(lambda z: lev.AIB @ z, PA, 2 * lev.n, power_iters)
                    Ainv = lambda q: smoothers.chebyshev(lambda z: lev.AIB @ z, PA, q, lev.lamA,
                                                         cheb_iters, cheb_lo, cheb_hi)
                    lev.lamM = smoothers.power_max(lambda q: lev.D @ Ainv(lev.G @ q), PM, lev.n,
                                                   power_iters)

    @property
    def fine(self):
        return self.levels[-1]

    def basic(self, l, x, b):
        """One sweep of the basic smoother with the hierarchy's damping."""
        lev = self.levels[l]
        if self.smoother == "vanka":
            return smoothers.vanka_sweep(lev.L, lev.dofs, lev.patches, x, b, self.omega)
        if self.smoother == "ras":
            return self._ras(lev, x, b)
        return smoothers.sc_sweep(lev.L, lev.G, lev.D, lev.AIB, lev.dA, lev.dM, lev.lamA, lev.lamM,
                                  x, b, self.omega, self.cheb_iters, self.cheb_lo, self.cheb_hi, self.sc_relax)

    def _ras(self, lev, x, b):
        if lev.boxes is None:
            return smoothers.exact_level_sweep(lev.L, lev.pinv, x, b, self.omega)
        return smoothers.ras_sweep(lev.L, lev.boxes, lev.factors, x, b, self.omega)

    def smooth(self, l, x, b, sweeps):
        lev = self.levels[l]
        if self.krylov:
            if sweeps == 0:
                return x
            return smoothers.fgmres_smooth(lev.L, lambda v: self.basic(l, np.zeros_like(v), v), x, b, sweeps)
        for _ in range(sweeps):
            if self.smoother == "vanka":
                x = smoothers.vanka_sweep(lev.L, lev.dofs, lev.patches, x, b, self.omega)
            elif self.smoother == "ras":
                x = self._ras(lev, x, b)
            else:
                x = smoothers.sc_sweep(lev.L, lev.G, lev.D, lev.AIB, lev.dA, lev.dM, lev.lamA, lev.lamM,
                                       x, b, self.omega, self.cheb_iters, self.cheb_lo, self.cheb_hi,
                                       self.sc_relax)
        return x

    def mg(self, l, w, b):
        """Alg. 1 on level l."""
        if l == 0:
            return self.coarse_pinv @ b
        lev = self.levels[l]
        w = self.smooth(l, w, b, self.nu1)
        r = b - lev.L @ w
        rc = self.R[l] @ r
        ec = self.mg(l - 1, np.zeros_like(rc), rc)
        w = w + self.P[l] @ ec
        w = self.smooth(l, w, b, self.nu2)
        return w

    def vcycle(self, b):
        """The preconditioner: one V-cycle from a zero initial guess on the finest level."""
        return self.mg(self.lmax, np.zeros_like(b), b)
