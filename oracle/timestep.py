"""Time stepping of the semi-implicit scheme (Sec. 2.2, Eqs. imp-momentum to imp-F), for tests only.

Each step solves the eliminated system (Eq. matrix-impib) at the lagged configuration X^n and moves
the structure with the interpolated new velocity, X^{n+1} = X^n + dt J^n u^{n+1} (Eq. imp-X-new).
The momentum right-hand side g is the same at every step (steady forcing); with rho > 0 a caller
that wants the (rho/dt) u^n term puts it into g.  Test infrastructure only: nothing on the GPU
path imports it.
"""
import dataclasses

import numpy as np

from . import ib, system


def advance(prob, w):
    """X^{n+1} = X^n + dt J^n u^{n+1} (Eq. imp-X-new) for the solution w = [u | v | p] of the step."""
    X = prob.structure.X
    return X + prob.dt * ib.interp_velocity(prob.N, X, w)


def with_positions(prob, X):
    """The same problem with the markers at X."""
    return dataclasses.replace(prob, structure=dataclasses.replace(prob.structure, X=np.array(X, dtype=np.float64)))


def run(prob, steps, add_SKXn=True):
    """`steps` time steps from prob's configuration; returns the solutions and positions
    [w^1 .. w^steps], [X^0 .. X^steps] (solutions gauge-fixed)."""
    ws, Xs = [], [prob.structure.X.copy()]
    for _ in range(steps):
        L = system.operator_of(prob)
        b = system.rhs(prob, add_SKXn)
        w, _ = system.solve_direct(L, b, prob.N, prob.rho)
        w = system.project(w, prob.N, prob.rho)
        X = advance(prob, w)
        ws.append(w)
        Xs.append(X)
        prob = with_positions(prob, X)
    return ws, Xs
