"""Seeded synthetic inputs for the Stokes-IB solve: grids, marker layouts, springs, stiffnesses, forcing.

This module only *generates* problem data.  It holds none of the solver's arithmetic (no kernel
weights, no operators, no projections); both the CUDA path and the CPU oracle consume what it
returns, so that the two sides see bit-identical inputs.

Problem statement (paper Sec. 2.2, Eq. (system-impib) and Eq. (matrix-impib)): a periodic unit
square discretised on an N x N staggered (MAC) grid, h = 1/N, with fluid parameters rho, mu, dt,
Lagrangian markers X^n (M x 2) joined by zero-rest-length linear springs (edge list with
per-spring stiffness kappa_e, Appendix "Lagrangian discretization"), and a right-hand side g on
the velocity faces (pressure right-hand side 0).

Layouts (shared with the C ABI):
  * Eulerian vectors are float64 arrays of length 3*N*N laid out [u | v | p], each block
    row-major [j][i];  u[j][i] lives on the x-face (i*h, (j+1/2)*h), v[j][i] on the y-face
    ((i+1/2)*h, j*h), p[j][i] at the cell centre ((i+1/2)*h, (j+1/2)*h).
  * X is float64 (M, 2) C-contiguous (x, y interleaved), edges int32 (E, 2), kappa float64 (E,).

Workload recipes (the shapes of the paper's thick and thin structures, Sec. 5.1 and 5.2, at the
marker spacing of one half grid cell):
  * thin interface: markers at uniform angles on a base circle of radius r0 with arc spacing
    h/2, M = round(2*pi*r0 / (h/2)), then displaced onto an ellipse with semi-axes (a, b);
    closed ring of E = M springs.
  * thick disk of radius R: K = round(R / (h/2)) concentric rings, ring k at radius k*R/K with
    n_k = max(6, round(2*pi*r_k / (h/2))) markers at angles 2*pi*m/n_k, plus one centre marker.
    Tangential springs close every ring; each ring-k marker is joined radially to the
    ring-(k-1) marker nearest in angle (index round-half-down of m*n_{k-1}/n_k, modulo
    n_{k-1}); ring-1 markers join the centre.  E = 2*(M-1).

The paper's own structures (Sec. 5.1 thick annulus, Sec. 5.2 thin circle), in the periodic box:
  * thick annulus, Eq. (annulus): X(s1, s2) = c + (r + s2)(cos s1, sin s1), (s1, s2) in
    [0, 2 pi) x [0, w], w = 1/16, r = 1/4, c = (1/2, 1/2); M1 = 19N/8 points in s1 (s1_k = 2 pi k/M1)
    and M2 = 3N/32 + 1 in s2 (s2_m = m w/(M2 - 1)); fibres along s1 only.  The force
    F = alpha d^2X/ds1^2 with alpha = gamma 3.93/0.005, taken with the nodal quadrature weight
    ds1 ds2 per marker, is the force of zero-rest-length springs between s1-neighbours of one fibre
    with kappa_e = alpha ds2/ds1 (ds1 = 2 pi/M1, ds2 = w/(M2 - 1)).
  * thin circle, Eq. (circle): X(s1) = c + r (cos s1, sin s1), M1 = 19N/8 points,
    alpha = 7 gamma 3.93/0.005, weight ds1 per marker: kappa_e = alpha/ds1.
  The paper's single linear solve: dt = 0.32 h, no external forcing (g = 0), so the right-hand side
  is the elastic force S K X^n of the initial configuration; Stokes (rho = 0, mu = 1) or rho = 1
  with mu in {1, 0.1, 0.01}; tolerance 1e-12, at most 100 iterations.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def _round_half_up(x: float) -> int:
    return int(np.floor(x + 0.5))


@dataclass
class Structure:
    X: np.ndarray          # (M, 2) float64
    edges: np.ndarray      # (E, 2) int32
    kappa: np.ndarray      # (E,) float64

    @property
    def M(self) -> int:
        return int(self.X.shape[0])

    @property
    def E(self) -> int:
        return int(self.edges.shape[0])


@dataclass
class Problem:
    N: int
    rho: float
    mu: float
    dt: float
    structure: Structure
    g: np.ndarray                      # (3*N*N,) float64, pressure block zero
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def h(self) -> float:
        return 1.0 / self.N


def thin_interface(N: int, center=(0.5, 0.5), axes=(0.30, 0.20), r0: float = 0.25,
                   kappa: float = 1e2) -> Structure:
    """Closed elliptical ring of markers at half-cell arc spacing on the base circle of radius r0."""
    h = 1.0 / N
    M = _round_half_up(2.0 * np.pi * r0 / (0.5 * h))
    theta = 2.0 * np.pi * np.arange(M) / M
    X = np.empty((M, 2), dtype=np.float64)
    X[:, 0] = center[0] + axes[0] * np.cos(theta)
    X[:, 1] = center[1] + axes[1] * np.sin(theta)
    a = np.arange(M, dtype=np.int32)
    edges = np.stack([a, (a + 1) % M], axis=1).astype(np.int32)
    return Structure(X, edges, np.full(M, float(kappa)))


def elastic_disk(N: int, center=(0.5, 0.5), R: float = 0.25, kappa: float = 1e2) -> Structure:
    """Concentric-ring disk with tangential and radial springs (recipe in the module docstring)."""
    h = 1.0 / N
    K = max(1, _round_half_up(R / (0.5 * h)))
    xs = [np.array([center[0]])]
    ys = [np.array([center[1]])]
    edges = []
    start_prev, n_prev = 0, 1
    start = 1
    for k in range(1, K + 1):
        rk = k * R / K
        nk = max(6, _round_half_up(2.0 * np.pi * rk / (0.5 * h)))
        m = np.arange(nk)
        th = 2.0 * np.pi * m / nk
        xs.append(center[0] + rk * np.cos(th))
        ys.append(center[1] + rk * np.sin(th))
        idx = start + m
        edges.append(np.stack([idx, start + (m + 1) % nk], axis=1))          # tangential
        if n_prev == 1:
            inner = np.zeros(nk, dtype=np.int64)
        else:
            # round-half-down of m * n_prev / nk, in exact integer arithmetic
            num = 2 * m * n_prev - nk
            inner = -((-num) // (2 * nk))                                     # ceil(num / (2 nk))
            inner = np.mod(inner, n_prev)
        edges.append(np.stack([idx, start_prev + inner], axis=1))             # radial
        start_prev, n_prev = start, nk
        start += nk
    X = np.stack([np.concatenate(xs), np.concatenate(ys)], axis=1).astype(np.float64)
    E = np.concatenate(edges, axis=0).astype(np.int32)
    return Structure(np.ascontiguousarray(X), np.ascontiguousarray(E), np.full(E.shape[0], float(kappa)))


ALPHA_UNIT = 3.93 / 0.005   # the explicit-stability stiffness that gamma is measured in (Sec. 5.1)


def thick_annulus(N: int, gamma: float, center=(0.5, 0.5), r: float = 0.25, w: float = 1.0 / 16) -> Structure:
    """The paper's thick annulus (Eq. annulus) with s1 fibres; recipe in the module docstring."""
    if N % 32:
        raise ValueError("N must be a multiple of 32 (M1 = 19N/8, M2 = 3N/32 + 1)")
    M1, M2 = 19 * N // 8, 3 * N // 32 + 1
    s1 = 2.0 * np.pi * np.arange(M1) / M1
    s2 = w * np.arange(M2) / (M2 - 1)
    rr = r + s2[:, None]                                        # (M2, M1)
    X = np.stack([(center[0] + rr * np.cos(s1)).ravel(), (center[1] + rr * np.sin(s1)).ravel()], axis=1)
    k = np.arange(M1)
    edges = np.concatenate([np.stack([m * M1 + k, m * M1 + (k + 1) % M1], axis=1) for m in range(M2)])
    alpha = gamma * ALPHA_UNIT
    kappa = alpha * (w / (M2 - 1)) / (2.0 * np.pi / M1)
    return Structure(np.ascontiguousarray(X, dtype=np.float64), edges.astype(np.int32),
                     np.full(edges.shape[0], kappa))


def thin_circle(N: int, gamma: float, center=(0.5, 0.5), r: float = 0.25) -> Structure:
    """The paper's thin circular membrane (Eq. circle); recipe in the module docstring."""
    if N % 8:
        raise ValueError("N must be a multiple of 8 (M1 = 19N/8)")
    M1 = 19 * N // 8
    s1 = 2.0 * np.pi * np.arange(M1) / M1
    X = np.stack([center[0] + r * np.cos(s1), center[1] + r * np.sin(s1)], axis=1)
    k = np.arange(M1)
    edges = np.stack([k, (k + 1) % M1], axis=1).astype(np.int32)
    kappa = 7.0 * gamma * ALPHA_UNIT / (2.0 * np.pi / M1)
    return Structure(np.ascontiguousarray(X, dtype=np.float64), edges, np.full(M1, kappa))


def paper_problem(kind: str, N: int, gamma: float, mu: float | None = None) -> Problem:
    """One linear solve of the paper's tests: structure `kind` ("annulus" or "circle"), dt = 0.32 h,
    g = 0 (the elastic force of the initial configuration drives the flow); mu None: Stokes
    (rho = 0, mu = 1), else rho = 1 with that mu."""
    s = thick_annulus(N, gamma) if kind == "annulus" else thin_circle(N, gamma)
    rho, mu_ = (0.0, 1.0) if mu is None else (1.0, float(mu))
    flow = "stokes" if mu is None else f"mu{mu:g}"
    return Problem(N, rho, mu_, 0.32 / N, s, np.zeros(3 * N * N), name=f"paper_{kind}_N{N}_gamma{gamma:g}_{flow}",
                   meta=dict(gamma=gamma, kind=kind))


def merge(*parts: Structure) -> Structure:
    Xs, Es, Ks = [], [], []
    off = 0
    for s in parts:
        Xs.append(s.X)
        Es.append(s.edges + off)
        Ks.append(s.kappa)
        off += s.M
    return Structure(np.ascontiguousarray(np.concatenate(Xs)),
                     np.ascontiguousarray(np.concatenate(Es).astype(np.int32)),
                     np.concatenate(Ks))


def empty_structure() -> Structure:
    return Structure(np.zeros((0, 2)), np.zeros((0, 2), dtype=np.int32), np.zeros(0))


def loguniform_kappa(E: int, lo: float, hi: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size=E))


def forcing(N: int, seed: int) -> np.ndarray:
    """Seeded N(0,1) forcing on every velocity face; pressure block 0."""
    rng = np.random.default_rng(seed)
    g = np.zeros(3 * N * N)
    g[: 2 * N * N] = rng.standard_normal(2 * N * N)
    return g


def random_vector(n: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(n)


# --------------------------------------------------------------------------------------------
# Workloads with the sizes of the build's configurations.
# --------------------------------------------------------------------------------------------

def thin_ellipse_stokes(N: int = 32, kappa: float = 1e2, seed: int = 0) -> Problem:
    """Stokes (rho=0, mu=1, dt=1e-2), thin ellipse 0.30/0.20 at the centre."""
    s = thin_interface(N, kappa=kappa)
    return Problem(N, 0.0, 1.0, 1e-2, s, forcing(N, seed), name=f"thin_ellipse_stokes_N{N}",
                   meta=dict(kappa=kappa, seed=seed))


def disk_stokes(N: int = 128, kappa: float = 1e2, seed: int = 1) -> Problem:
    """Stokes (rho=0, mu=1, dt=1e-2), thick disk of radius 0.25 at the centre."""
    s = elastic_disk(N, R=0.25, kappa=kappa)
    return Problem(N, 0.0, 1.0, 1e-2, s, forcing(N, seed), name=f"disk_stokes_N{N}",
                   meta=dict(kappa=kappa, seed=seed))


def thin_ellipse_re(N: int = 512, kappa: float = 1e2, seed: int = 2) -> Problem:
    """Nonzero Reynolds number (rho=1, mu=1e-2, dt=1e-3), thin ellipse 0.30/0.20."""
    s = thin_interface(N, kappa=kappa)
    return Problem(N, 1.0, 1e-2, 1e-3, s, forcing(N, seed), name=f"thin_ellipse_re_N{N}",
                   meta=dict(kappa=kappa, seed=seed))


def thin_ellipse_loguniform(N: int = 256, seed_kappa: int = 3, seed: int = 3) -> Problem:
    """Stokes, thin ellipse with per-spring kappa ~ LogUniform(1e2, 1e4)."""
    s = thin_interface(N)
    s.kappa = loguniform_kappa(s.E, 1e2, 1e4, seed_kappa)
    return Problem(N, 0.0, 1.0, 1e-2, s, forcing(N, seed), name=f"thin_ellipse_loguniform_N{N}",
                   meta=dict(seed_kappa=seed_kappa, seed=seed))


def disk_and_ellipse_re(N: int = 1024, kappa: float = 1e4, seed: int = 4) -> Problem:
    """rho=1, mu=1e-2, dt=1e-3: disk R=0.15 at (0.3,0.5) plus ellipse 0.15/0.10 at (0.7,0.5)."""
    d = elastic_disk(N, center=(0.3, 0.5), R=0.15, kappa=kappa)
    e = thin_interface(N, center=(0.7, 0.5), axes=(0.15, 0.10), r0=0.125, kappa=kappa)
    return Problem(N, 1.0, 1e-2, 1e-3, merge(d, e), forcing(N, seed),
                   name=f"disk_and_ellipse_re_N{N}", meta=dict(kappa=kappa, seed=seed))


def no_structure(N: int, rho: float = 0.0, mu: float = 1.0, dt: float = 1e-2, seed: int = 0) -> Problem:
    return Problem(N, rho, mu, dt, empty_structure(), forcing(N, seed), name=f"fluid_only_N{N}")
