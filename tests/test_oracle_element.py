"""Pins of the oracle's element routines against facts fixed by the paper and by mathematics
(not by re-typing the oracle's own formulas)."""
import math

import numpy as np
import pytest

import oracle as O
from synthetic import single_tet


def _x(seed, kind="random"):
    m = single_tet(seed, kind)
    return m.nodes[m.tets[0]]


def _fields(seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((4, 3)), rng.standard_normal((4, 3)), rng.standard_normal(4)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    O.load_library()


def test_reference_geometry():
    # On the unit right simplex J = I: G = I, g = (1,1,1), |K| = 1/6, sum of gradients = 0.
    x = _x(0, "reference")
    det, gp, G, g, vol = O.geometry(x)
    assert det == pytest.approx(1.0)
    assert np.allclose(G, np.eye(3), atol=0, rtol=0)
    assert np.allclose(g, [1, 1, 1])
    assert vol == pytest.approx(1.0 / 6.0)
    assert np.allclose(gp.sum(axis=0), 0.0)
    assert np.allclose(gp, [[-1, -1, -1], [1, 0, 0], [0, 1, 0], [0, 0, 1]])


@pytest.mark.parametrize("seed", range(4))
def test_gradients_reproduce_linear_fields(seed):
    # grad phi_a must reproduce the gradient of any linear field exactly (partition of unity +
    # linear completeness of P1).
    x = _x(seed)
    _, gp, G, g, vol = O.geometry(x)
    rng = np.random.default_rng(seed)
    c, a0 = rng.standard_normal(3), rng.standard_normal()
    vals = x @ c + a0
    assert np.allclose(vals @ gp, c, rtol=1e-12, atol=1e-12)
    J = (x[1:] - x[0]).T
    Ji = np.linalg.inv(J)
    assert np.allclose(G, Ji.T @ Ji, rtol=1e-12)
    assert np.allclose(g, Ji.T @ np.ones(3), rtol=1e-12)
    assert vol == pytest.approx(abs(np.linalg.det(J)) / 6.0, rel=1e-13)


def test_tau_closed_form_on_reference_element():
    # u* = 0, no RIIS: tau_M = (sigma^2 rho^2/dt^2 + C_r mu^2 G:G)^-1/2, G:G = 3 on the reference tet;
    # tau_C = 1/(tau_M g.g) with g.g = 3.
    P = O.Params(rho=1.06, mu=0.035, dt=1e-3, bdf_order=2, c_r=30.0)
    tm, tc = O.tau(P, np.eye(3), np.ones(3), np.zeros(3))
    ref = (4 * 1.06 ** 2 / 1e-6 + 30 * 0.035 ** 2 * 3) ** -0.5
    assert tm == pytest.approx(ref, rel=1e-14)
    assert tc == pytest.approx(1.0 / (ref * 3.0), rel=1e-14)
    # advective part: u* = (1,0,0) adds rho^2 G_00
    tm2, _ = O.tau(P, np.eye(3), np.ones(3), np.array([1.0, 0, 0]))
    assert tm2 == pytest.approx((4 * 1.06 ** 2 / 1e-6 + 1.06 ** 2 + 30 * 0.035 ** 2 * 3) ** -0.5, rel=1e-14)


def test_delta_function():
    lib = O.load_library()
    eps = 0.05
    assert lib.orc_delta(0.0, eps) == pytest.approx(1.0 / eps)
    assert lib.orc_delta(eps, eps) == pytest.approx(0.0, abs=1e-12)
    assert lib.orc_delta(1.01 * eps, eps) == 0.0
    s = np.linspace(-eps, eps, 20001)
    vals = np.array([lib.orc_delta(v, eps) for v in s])
    assert np.trapezoid(vals, s) == pytest.approx(1.0, rel=1e-6)    # unit mass


@pytest.mark.parametrize("order", [1, 2, 3])
def test_bdf_polynomial_exactness(order):
    # BDF of order s differentiates polynomials of degree s exactly at t^{n+1}; the extrapolation
    # reproduces degree s-1 polynomials.
    alpha, beta, gamma = O.bdf_coefficients(order)
    dt, tn = 0.1, 0.7
    for deg in range(order + 1):
        c = np.arange(1, deg + 2, dtype=float)
        f = lambda t: sum(ci * t ** k for k, ci in enumerate(c))
        df = lambda t: sum(k * ci * t ** (k - 1) for k, ci in enumerate(c) if k)
        hist = [f(tn - j * dt) for j in range(order)]
        approx = (alpha * f(tn + dt) - sum(b * h for b, h in zip(beta, hist))) / dt
        assert approx == pytest.approx(df(tn + dt), rel=1e-10, abs=1e-10)
        if deg < order:
            assert sum(g * h for g, h in zip(gamma, hist)) == pytest.approx(f(tn + dt), rel=1e-12)


CASES = [(s, k, d) for s in range(3) for k in ("random", "sliver") for d in (0, 1)]


@pytest.mark.parametrize("seed,kind,diff", [(i, k, d) for i, (s, k, d) in enumerate(CASES)])
def test_matrix_is_jacobian_of_residual(seed, kind, diff):
    # The element residual is written from the strong residual r_M, r_C at each quadrature point;
    # it is affine in the 16 unknowns with u* frozen, so central differences give its Jacobian up
    # to round-off.  Checks every term of the matrix (signs, indices, transposes).
    stab = CASES[seed][0]
    x = _x(seed, kind)
    ub, ue, pe = _fields(100 + seed)
    P = O.Params(rho=1.06, mu=0.035, dt=1e-3, bdf_order=2, stab=stab, diffusion=diff,
                 f=(0.3, -0.2, 0.1))
    A, b = O.element(P, x, ub, ue, pe)
    sol = np.random.default_rng(seed).standard_normal(16)
    J = np.zeros((16, 16))
    h = 1e-2
    for k in range(16):
        e = np.zeros(16)
        e[k] = h
        J[:, k] = (O.element_residual(P, x, ub, ue, pe, sol + e) - O.element_residual(P, x, ub, ue, pe, sol - e)) / (2 * h)
    assert np.abs(J - A).max() <= 1e-9 * np.abs(A).max()
    R0 = O.element_residual(P, x, ub, ue, pe, np.zeros(16))
    assert np.abs(R0 + b).max() <= 1e-12 * np.abs(b).max()


def test_riis_band_jacobian():
    # Element cut by a resistive surface (phi changes sign inside): same finite-difference pin.
    x = _x(7)
    ub, ue, pe = _fields(7)
    c = x.mean(axis=0)
    phi = np.stack([(x - c) @ np.array([0.0, 0.0, 1.0])])
    eps = 0.6 * np.ptp(phi)
    riis = [O.RIIS(1e4, eps, None)]
    P = O.Params(rho=1.06, mu=0.035, dt=1e-3, bdf_order=2, stab=2)
    A, b = O.element(P, x, ub, ue, pe, phi, riis)
    A0, _ = O.element(P, x, ub, ue, pe)
    assert np.abs(A - A0).max() > 1e-3 * np.abs(A).max()       # the term is active
    sol = np.random.default_rng(1).standard_normal(16)
    J = np.zeros((16, 16))
    for k in range(16):
        e = np.zeros(16)
        e[k] = 1e-2
        J[:, k] = (O.element_residual(P, x, ub, ue, pe, sol + e, phi, riis)
                   - O.element_residual(P, x, ub, ue, pe, sol - e, phi, riis)) / 2e-2
    assert np.abs(J - A).max() <= 1e-9 * np.abs(A).max()


def _mass(vol):
    return vol * (np.ones((4, 4)) + np.eye(4)) / 20.0


@pytest.mark.parametrize("seed", range(3))
def test_mass_block_closed_form(seed):
    # mu = 0, u* = 0, no stabilisation: the velocity block is rho alpha/dt * M_e (x) I_3 with the
    # exact P1 mass matrix |K|(1+delta_ab)/20 (the 4-point rule is exact for degree 2).
    x = _x(seed)
    vol = O.geometry(x)[4]
    z3, z = np.zeros((4, 3)), np.zeros(4)
    P = O.Params(rho=1.3, mu=0.0, dt=0.01, bdf_order=3, stab=0)
    A, b = O.element(P, x, z3, z3, z)
    alpha = 11.0 / 6.0
    M = _mass(vol)
    for i in range(3):
        assert np.allclose(A[i::4, i::4], 1.3 * alpha / 0.01 * M, rtol=1e-13)
        for j in range(3):
            if j != i:
                assert np.abs(A[i::4, j::4]).max() == 0.0
    assert np.abs(A[3::4, 3::4]).max() == 0.0


def test_resistive_block_closed_form():
    # Whole element on the surface (phi = 0 at all nodes): delta = 1/eps everywhere, so the
    # resistive term adds (R/eps^2) M_e to each velocity component (Eq. riis).
    x = _x(3)
    vol = O.geometry(x)[4]
    z3, z = np.zeros((4, 3)), np.zeros(4)
    P = O.Params(rho=1.0, mu=0.0, dt=0.01, bdf_order=1, stab=0)
    riis = [O.RIIS(200.0, 0.1, None)]
    A, _ = O.element(P, x, z3, z3, z, np.zeros((1, 4)), riis)
    A0, _ = O.element(P, x, z3, z3, z)
    for i in range(3):
        assert np.allclose(A[i::4, i::4] - A0[i::4, i::4], 200.0 / 0.1 ** 2 * _mass(vol), rtol=1e-12)


@pytest.mark.parametrize("diff", [0, 1, 2])
def test_diffusion_annihilates_translations(diff):
    # Diffusion (any of the three forms of Eq. diffusion-term) vanishes on constant velocity
    # fields; the symmetric forms also vanish on rigid rotations.
    x = _x(5)
    z3, z = np.zeros((4, 3)), np.zeros(4)
    base = O.Params(rho=1.0, mu=0.0, dt=1.0, bdf_order=1, stab=0)
    P = O.Params(rho=1.0, mu=2.5, dt=1.0, bdf_order=1, stab=0, diffusion=diff)
    K = O.element(P, x, z3, z3, z)[0] - O.element(base, x, z3, z3, z)[0]
    t = np.zeros(16)
    t[0::4], t[1::4], t[2::4] = 0.3, -1.2, 0.7
    assert np.abs(K @ t).max() <= 1e-12 * np.abs(K).max()
    if diff:
        w = np.array([0.4, -0.3, 0.9])
        rot = np.zeros(16)
        for a in range(4):
            rot[4 * a:4 * a + 3] = np.cross(w, x[a])
        assert np.abs(K @ rot).max() <= 1e-12 * np.abs(K).max() * np.abs(rot).max()


def test_divergence_rows_vanish_on_rigid_motions():
    # Galerkin continuity rows (div u, q) vanish on translations and rotations (divergence-free,
    # exactly represented by P1).
    x = _x(6)
    ub, ue, pe = _fields(6)
    P = O.Params(rho=1.0, mu=0.1, dt=0.1, bdf_order=1, stab=0)
    A, _ = O.element(P, x, ub, ue, pe)
    w = np.array([0.4, -0.3, 0.9])
    for v in (np.tile([1.0, 2.0, -1.0, 0.0], 4), None):
        if v is None:
            v = np.zeros(16)
            for a in range(4):
                v[4 * a:4 * a + 3] = np.cross(w, x[a])
        assert np.abs(A[3::4] @ v).max() <= 1e-13 * np.abs(A).max() * np.abs(v).max()


def test_pressure_gradient_rows_integrate_by_parts():
    # -(p, div v) with p constant equals -p * (surface flux of v) = 0 summed over a closed
    # element for v constant: the rows of the pressure column sum to zero over the nodes.
    x = _x(8)
    ub, ue, pe = _fields(8)
    P = O.Params(rho=1.0, mu=0.1, dt=0.1, bdf_order=1, stab=0)
    A, _ = O.element(P, x, ub, ue, pe)
    for i in range(3):
        assert abs(A[i::4, 3::4].sum()) <= 1e-13 * np.abs(A).max()
    # and -(p, div v) = (grad p, v) for linear p with v vanishing nowhere: check against the
    # exact integral  -int p div(phi_a e_i) = -d_i phi_a int p = -d_i phi_a |K| mean(p)
    _, gp, _, _, vol = O.geometry(x)
    p = np.array([0.3, -1.0, 2.0, 0.5])
    for a in range(4):
        for i in range(3):
            assert A[4 * a + i, 3::4] @ p == pytest.approx(-gp[a, i] * vol * p.mean(), rel=1e-12, abs=1e-14)
