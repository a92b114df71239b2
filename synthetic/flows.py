"""Closed-form flow fields that the test problems prescribe as input data.

* Ethier-Steinman Beltrami flow with a = pi/4, d = pi/2, the exact Navier-Stokes solution with
  zero forcing given in Appendix A (Beltrami flow).  Used for initial histories, Dirichlet data
  and for the error norms of Eq. (errors), Section 4.1.
* Steady Poiseuille flow in a straight pipe of radius R along +z with peak velocity U: the
  parabolic inflow whose flow rate the unit-flow-rate profile of Section 2.2.1 scales.

These are data, not part of the discretisation; both the oracle's tests and the GPU tests use
them to build inputs and to score results.
"""
from __future__ import annotations

import math

import numpy as np


def _c(t, rho, mu):
    # c(t) = pi * exp(-pi^2 mu t / (4 rho))
    return math.pi * math.exp(-math.pi ** 2 * mu * t / (4.0 * rho))


def _f_and_grad(x, y, z, c):
    """f(x,y,z) = -c/4 [exp(pi x/4) sin(pi(y+2z)/4) + exp(pi z/4) cos(pi(x+2y)/4)] and its
    partial derivatives with respect to its three arguments.  The three velocity components are
    f(x,y,z), f(y,z,x), f(z,x,y) (the formula of Appendix A is cyclic in x->y->z)."""
    q = math.pi / 4.0
    ea, eb = np.exp(q * x), np.exp(q * z)
    sa, ca = np.sin(q * (y + 2 * z)), np.cos(q * (y + 2 * z))
    sb, cb = np.sin(q * (x + 2 * y)), np.cos(q * (x + 2 * y))
    k = -c / 4.0
    f = k * (ea * sa + eb * cb)
    f1 = k * (q * ea * sa - q * eb * sb)
    f2 = k * (q * ea * ca - 2 * q * eb * sb)
    f3 = k * (2 * q * ea * ca + q * eb * cb)
    return f, f1, f2, f3


def beltrami_u(X, t, rho=1.0, mu=1.0):
    """Velocity [n,3] at points X [n,3] and time t (Appendix A)."""
    X = np.asarray(X, dtype=np.float64)
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    c = _c(t, rho, mu)
    ux = _f_and_grad(x, y, z, c)[0]
    uy = _f_and_grad(y, z, x, c)[0]
    uz = _f_and_grad(z, x, y, c)[0]
    return np.stack([ux, uy, uz], axis=1)


def beltrami_grad_u(X, t, rho=1.0, mu=1.0):
    """Velocity gradient [n,3,3], entry [i,j] = d u_i / d x_j."""
    X = np.asarray(X, dtype=np.float64)
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    c = _c(t, rho, mu)
    G = np.empty((X.shape[0], 3, 3))
    _, f1, f2, f3 = _f_and_grad(x, y, z, c)       # u_x = f(x,y,z)
    G[:, 0, 0], G[:, 0, 1], G[:, 0, 2] = f1, f2, f3
    _, f1, f2, f3 = _f_and_grad(y, z, x, c)       # u_y = f(y,z,x)
    G[:, 1, 1], G[:, 1, 2], G[:, 1, 0] = f1, f2, f3
    _, f1, f2, f3 = _f_and_grad(z, x, y, c)       # u_z = f(z,x,y)
    G[:, 2, 2], G[:, 2, 0], G[:, 2, 1] = f1, f2, f3
    return G


def beltrami_p(X, t, rho=1.0, mu=1.0):
    """Pressure [n] at points X and time t (Appendix A)."""
    X = np.asarray(X, dtype=np.float64)
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    q = math.pi / 4.0
    s = (np.exp(2 * q * x) + np.exp(2 * q * y) + np.exp(2 * q * z)
         + 2 * np.exp(q * (x + y)) * np.cos(q * (y + 2 * z)) * np.sin(q * (2 * x + z))
         + 2 * np.exp(q * (x + z)) * np.cos(q * (x + 2 * y)) * np.sin(q * (y + 2 * z))
         + 2 * np.exp(q * (y + z)) * np.cos(q * (2 * x + z)) * np.sin(q * (x + 2 * y)))
    return -rho * math.pi ** 2 / 32.0 * math.exp(-math.pi ** 2 * t * mu / (2.0 * rho)) * s


def poiseuille_u(X, radius, peak):
    """Axial Poiseuille velocity along +z: u_z = U (1 - r^2/R^2)."""
    X = np.asarray(X, dtype=np.float64)
    r2 = X[:, 0] ** 2 + X[:, 1] ** 2
    u = np.zeros_like(X)
    u[:, 2] = peak * np.clip(1.0 - r2 / radius ** 2, 0.0, None)
    return u


def poiseuille_p(X, radius, length, peak, mu):
    """Poiseuille pressure with p = 0 at the outlet z = L: p = 4 mu U (L - z) / R^2."""
    X = np.asarray(X, dtype=np.float64)
    return 4.0 * mu * peak * (length - X[:, 2]) / radius ** 2


def zero_net_flux(nodes, bfaces, node_ids, values):
    """Make Dirichlet velocity data discretely compatible with incompressibility when the whole
    boundary is Dirichlet: subtract c * n_k from the value at each boundary node k, n_k being the
    node's share of the face area vectors (sum over its faces of A_f n_f / 3), with c chosen so
    that the net flux sum_k values_k . n_k of the piecewise-linear boundary data is zero.
    ``node_ids`` must cover every node of ``bfaces``.  Returns the corrected values."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = nodes[bfaces]
    an = 0.5 * np.cross(x[:, 1] - x[:, 0], x[:, 2] - x[:, 0]) / 3.0
    nk = np.zeros_like(nodes)
    for k in range(3):
        np.add.at(nk, bfaces[:, k], an)
    nk = nk[node_ids]
    v = np.asarray(values, dtype=np.float64)
    c = np.sum(v * nk) / np.sum(nk * nk)
    return v - c * nk
