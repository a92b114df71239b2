"""Pins of the oracle's per-quadrature-point stabilisation coefficients (Section 2.3): the LES
factor tau_M r_M(u^EXT, p^EXT) of the semi-implicit LES term and the resistive (RIIS) part of
tau_M.  Each is checked against a closed form computed here from the paper's definitions with
fields whose derivatives are known exactly, not against the oracle's own loops.

* Linear fields u^EXT = a + B x, p^EXT = p0 + c.x, u^BDF = b + D x on one tetrahedron: every
  derivative is exact for P1, so the strong residual
  r_M = rho((alpha u^EXT - u^BDF)/dt + (u*.grad) u^EXT) + grad p^EXT + sum_k (R_k/eps_k) delta_k u^EXT - f
  at each quadrature point is known in closed form (time part, advection, pressure gradient,
  body force and a resistive band all nonzero).
* A manufactured history with r_M = 0 exactly makes the LES factor vanish.
* The element matrix depends on u^BDF only through the LES factor, so the difference of two
  element matrices that differ only in u^BDF is the LES term -(Delta s (x) tau_M r~_M, rho grad v)
  alone, with (a (x) b, grad v) = sum_ij a_i b_j d_j v_i.
* tau_M with two resistive surfaces: (sigma^2 rho^2/dt^2 + rho^2 u*.G u* + C_r mu^2 G:G
  + sum_k (R_k delta_k/eps_k)^2)^(-1/2) on the reference element (G = I)."""
import math

import numpy as np
import pytest

import oracle as O
from synthetic import single_tet


def _bary_points(x):
    # 4-point degree-2 rule: barycentric (a, b, b, b) and its permutations,
    # a = (5 + 3 sqrt 5)/20, b = (5 - sqrt 5)/20.
    a = (5.0 + 3.0 * math.sqrt(5.0)) / 20.0
    b = (5.0 - math.sqrt(5.0)) / 20.0
    lam = np.full((4, 4), b)
    np.fill_diagonal(lam, a)
    return lam, lam @ x


def _delta(phi, eps):
    return np.where(np.abs(phi) <= eps, (1.0 + np.cos(np.pi * phi / eps)) / (2.0 * eps), 0.0)


def _linear_case(seed):
    rng = np.random.default_rng(seed)
    x = single_tet(seed, "random").nodes
    a, B = rng.standard_normal(3), rng.standard_normal((3, 3))       # u^EXT = a + B x
    b, D = rng.standard_normal(3), rng.standard_normal((3, 3))       # u^BDF = b + D x
    p0, c = rng.standard_normal(), rng.standard_normal(3)            # p^EXT = p0 + c.x
    f = rng.standard_normal(3)
    # two resistive surfaces: planes through the element's centroid (normal n_k), band half-width
    # wider than part of the element so that delta varies between the quadrature points
    cen = x.mean(axis=0)
    normals = [np.array([0.0, 0.0, 1.0]), rng.standard_normal(3)]
    normals = [n / np.linalg.norm(n) for n in normals]
    phi_lin = [(lambda X, n=n: (X - cen) @ n) for n in normals]
    eps = [0.7 * np.ptp(phi_lin[0](x)), 0.9 * np.ptp(phi_lin[1](x))]
    res = [3.0e3, 7.0e2]
    return x, (a, B), (b, D), (p0, c), f, phi_lin, eps, res


@pytest.mark.parametrize("seed,order", [(0, 1), (1, 2), (2, 3), (3, 2)])
def test_les_factor_is_tau_m_times_the_strong_residual_of_linear_fields(seed, order):
    x, (a, B), (b, D), (p0, c), f, phi_lin, eps, res = _linear_case(seed)
    rho, mu, dt, c_r = 1.06, 0.035, 1e-3, 30.0
    alpha = O.bdf_coefficients(order)[0]
    P = O.Params(rho=rho, mu=mu, dt=dt, bdf_order=order, c_r=c_r, f=tuple(f), stab=2)
    uext_n = a + x @ B.T
    ubdf_n = b + x @ D.T
    pext_n = p0 + x @ c
    phinod = np.stack([pl(x) for pl in phi_lin])
    riis = [O.RIIS(r, e, None) for r, e in zip(res, eps)]
    J = (x[1:] - x[0]).T
    Ji = np.linalg.inv(J)
    G = Ji.T @ Ji
    lam, xq = _bary_points(x)
    deltas_seen = []
    for q in range(4):
        d = O.qp_coefficients(P, x, ubdf_n, uext_n, pext_n, q, phinod, riis)
        u = a + B @ xq[q]
        ubdf = b + D @ xq[q]
        dl = np.array([_delta(pl(xq[q][None, :])[0], e) for pl, e in zip(phi_lin, eps)])
        deltas_seen.append(dl)
        sR = float(np.sum(np.array(res) / np.array(eps) * dl))
        rm = rho * ((alpha * u - ubdf) / dt + B @ u) + c + sR * u - f
        tm = (order ** 2 * rho ** 2 / dt ** 2 + rho ** 2 * u @ G @ u + c_r * mu ** 2 * np.sum(G * G)
              + np.sum((np.array(res) * dl / np.array(eps)) ** 2)) ** -0.5
        assert d["tau_m"] == pytest.approx(tm, rel=1e-12)
        assert np.allclose(d["us"], u, rtol=1e-12, atol=1e-12 * np.abs(u).max())
        assert d["sR"] == pytest.approx(sR, rel=1e-12, abs=1e-12 * sR + 1e-300)
        assert np.allclose(d["m"], rho * ubdf / dt + f, rtol=1e-12, atol=1e-12 * np.abs(rho * ubdf / dt).max())
        scale = tm * max(np.abs(rho * alpha * u / dt).max(), np.abs(rho * ubdf / dt).max())
        assert np.abs(d["s"] - tm * rm).max() <= 1e-11 * scale, (d["s"], tm * rm)
        # every part of r_M is large enough here that dropping it or flipping its sign shows
        for part in (rho * (alpha * u - ubdf) / dt, rho * B @ u, c, sR * u, f):
            assert np.abs(tm * part).max() > 1e-6 * scale
    deltas_seen = np.array(deltas_seen)
    assert (deltas_seen > 0).any() and np.ptp(deltas_seen) > 0     # the band is active and varies


def test_les_factor_vanishes_for_an_exact_discrete_solution():
    # u^EXT = (y, 1, 0), p^EXT = -rho x, u^BDF = alpha u^EXT, f = 0: (u.grad)u = (1, 0, 0) and
    # grad p = (-rho, 0, 0) cancel, the time part is zero, so r_M = 0 at every point.
    x = single_tet(4, "random").nodes
    for order in (1, 2, 3):
        rho = 1.06
        alpha = O.bdf_coefficients(order)[0]
        P = O.Params(rho=rho, mu=0.035, dt=1e-3, bdf_order=order, stab=2)
        uext = np.stack([x[:, 1], np.ones(4), np.zeros(4)], axis=1)
        pext = -rho * x[:, 0]
        ubdf = alpha * uext
        for q in range(4):
            d = O.qp_coefficients(P, x, ubdf, uext, pext, q)
            assert np.abs(d["s"]).max() <= 1e-13 * d["tau_m"] * rho * alpha / 1e-3 * np.abs(uext).max()
        # and the element matrix no longer depends on how the zero residual splits: adding the
        # same multiple of u^EXT to u^BDF and to alpha u^EXT's companion body force keeps r_M = 0
        P2 = O.Params(rho=rho, mu=0.035, dt=1e-3, bdf_order=order, stab=2, f=(0.0, rho * 0.5 / 1e-3, 0.0))
        ubdf2 = ubdf.copy()
        ubdf2[:, 1] -= 0.5                       # rho (alpha u - u^BDF)/dt gains rho*0.5/dt in y = f_y
        A1, _ = O.element(P, x, ubdf, uext, pext)
        A2, _ = O.element(P2, x, ubdf2, uext, pext)
        assert np.abs(A1 - A2).max() <= 1e-12 * np.abs(A1).max()


@pytest.mark.parametrize("seed", [5, 6])
def test_matrix_depends_on_the_history_only_through_the_les_term(seed):
    # A(u^BDF_1) - A(u^BDF_2) = -(Delta s (x) tau_M r~_M(trial), rho grad v): for the velocity
    # trial phi_b e_j, r~_M = c_b e_j with c_b = (rho alpha/dt + sR) phi_b + rho u*.grad phi_b;
    # for the pressure trial phi_b, r~_M = grad phi_b.  Pressure-test rows do not change.
    x, (a, B), (b, D), (p0, c), f, phi_lin, eps, res = _linear_case(seed)
    rho, dt, order = 1.06, 1e-3, 2
    alpha = O.bdf_coefficients(order)[0]
    P = O.Params(rho=rho, mu=0.035, dt=dt, bdf_order=order, f=tuple(f), stab=2)
    uext_n, pext_n = a + x @ B.T, p0 + x @ c
    phinod = np.stack([pl(x) for pl in phi_lin])
    riis = [O.RIIS(r, e, None) for r, e in zip(res, eps)]
    rng = np.random.default_rng(seed)
    ub1 = b + x @ D.T
    ub2 = ub1 + 5.0e3 * rng.standard_normal((4, 3))
    A1, _ = O.element(P, x, ub1, uext_n, pext_n, phinod, riis)
    A2, _ = O.element(P, x, ub2, uext_n, pext_n, phinod, riis)
    Ji = np.linalg.inv((x[1:] - x[0]).T)
    gphi = np.concatenate([-Ji.sum(axis=0, keepdims=True), Ji], axis=0)   # rows: grad phi_a
    lam, _ = _bary_points(x)
    dA = np.zeros((16, 16))
    for q in range(4):
        d1 = O.qp_coefficients(P, x, ub1, uext_n, pext_n, q, phinod, riis)
        d2 = O.qp_coefficients(P, x, ub2, uext_n, pext_n, q, phinod, riis)
        ds = d1["s"] - d2["s"]
        tm, w, us, sR = d1["tau_m"], d1["w"], d1["us"], d1["sR"]
        for aa in range(4):
            for bb in range(4):
                cb = (rho * alpha / dt + sR) * lam[q, bb] + rho * us @ gphi[bb]
                for i in range(3):
                    for j in range(3):
                        dA[4 * aa + i, 4 * bb + j] -= w * rho * ds[i] * tm * cb * gphi[aa, j]
                    dA[4 * aa + i, 4 * bb + 3] -= w * rho * ds[i] * tm * (gphi[bb] @ gphi[aa])
    assert np.abs(dA).max() > 1e-5 * np.abs(A1).max()                   # the LES term is visible
    assert np.abs((A1 - A2) - dA).max() <= 1e-10 * np.abs(A1).max()


def test_tau_m_with_two_resistive_surfaces_on_the_reference_element():
    rho, mu, dt = 1.06, 0.035, 5e-4
    P = O.Params(rho=rho, mu=mu, dt=dt, bdf_order=2, c_r=30.0)
    riis = [O.RIIS(1.0e4, 0.05, None), O.RIIS(3.0e3, 0.2, None)]
    deltas = (2.0, 15.0)
    us = np.array([0.5, -2.0, 1.5])
    tm, tc = O.tau(P, np.eye(3), np.ones(3), us, deltas, riis)
    ref = (4 * rho ** 2 / dt ** 2 + rho ** 2 * us @ us + 30.0 * mu ** 2 * 3
           + (1.0e4 * 2.0 / 0.05) ** 2 + (3.0e3 * 15.0 / 0.2) ** 2) ** -0.5
    assert tm == pytest.approx(ref, rel=1e-14)
    assert tc == pytest.approx(1.0 / (3.0 * ref), rel=1e-14)
    # the resistive part dominates here, so a dropped square or a missing surface shows
    tm1, _ = O.tau(P, np.eye(3), np.ones(3), us, deltas[:1], riis[:1])
    assert abs(tm1 - tm) > 1e-3 * tm
