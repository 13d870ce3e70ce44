"""Peskin's four-point regularised delta kernel (Appendix, "Lagrangian-Eulerian interaction").

The one-dimensional kernel phi(r) is piecewise in |r| with square roots on [0,1) and [1,2) and
vanishes for |r| >= 2; the two-dimensional regularised delta is
delta_h(x) = phi(x_1/h) phi(x_2/h) / h^2.

Pinned by: phi(0)=1/2, phi(1)=1/4, phi(2)=0; partition of unity, zero first moment and
sum of squares 3/8 for every shift; C^1 continuity; the derivative against central differences.
"""
import numpy as np


def phi(r):
    """phi(r) of the four-point kernel, elementwise, float64."""
    a = np.abs(np.asarray(r, dtype=np.float64))
    out = np.zeros_like(a)
    inner = a < 1.0
    outer = (a >= 1.0) & (a < 2.0)
    ai = a[inner]
    out[inner] = (3.0 - 2.0 * ai + np.sqrt(1.0 + 4.0 * ai - 4.0 * ai * ai)) / 8.0
    ao = a[outer]
    out[outer] = (5.0 - 2.0 * ao - np.sqrt(-7.0 + 12.0 * ao - 4.0 * ao * ao)) / 8.0
    return out


def dphi(r):
    """d phi / d r (signed r), elementwise, float64."""
    r = np.asarray(r, dtype=np.float64)
    a = np.abs(r)
    sgn = np.sign(r)
    out = np.zeros_like(a)
    inner = a < 1.0
    outer = (a >= 1.0) & (a < 2.0)
    ai = a[inner]
    out[inner] = (-2.0 + (4.0 - 8.0 * ai) / (2.0 * np.sqrt(1.0 + 4.0 * ai - 4.0 * ai * ai))) / 8.0
    ao = a[outer]
    out[outer] = (-2.0 - (12.0 - 8.0 * ao) / (2.0 * np.sqrt(-7.0 + 12.0 * ao - 4.0 * ao * ao))) / 8.0
    return out * sgn
