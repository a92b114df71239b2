"""Oracle pins for the outlet conditions of Section 2.2: inertial backflow stabilisation on
Neumann faces and the resistance condition.

Backflow: with u* . n >= 0 on the faces the term vanishes; for a uniform inflow u* = -U n it is the
constant c = beta rho U / 2 times the face mass matrix, whose closed form is A (1 + delta_ab) / 12
per face; for any u* it is symmetric positive semi-definite.  Resistance: w . u is the exact flux
of a P1 velocity (checked on a linear field against the centroid rule per face); with C_R = 0 the
condition is Neumann data h = p_0; with C_R > 0 the solution is the Neumann one with the pressure
shifted by C_R Q (Q the flux, fixed by the inlet data)."""
import math

import numpy as np
import scipy.sparse as sp

import oracle as O
from synthetic import cylinder, poiseuille_p, poiseuille_u

R, L, U, MU, RHO = 1.0, 2.0, 20.0, 0.035, 1.06


def _mesh():
    return cylinder(R, L, n_tets=3000, seed=7)


def _outlet_faces(m):
    return m.bfaces[m.btags == 2].astype(np.int64)


def _problem(outlet):
    P = O.Params(rho=RHO, mu=MU, dt=1e-3, bdf_order=2, stab=2)
    Q = U * math.pi * R * R / 2.0
    return O.Problem(P, [O.BC(tag=0, kind="noslip"),
                         O.BC(tag=1, kind="dirichlet", time="constant", tparams={"value": Q},
                              space="parabolic", radius=R),
                         outlet])


def test_backflow_vanishes_for_outflow():
    m = _mesh()
    prob = _problem(O.BC(tag=2, kind="neumann", tparams={"value": 0.0}, beta=1.0))
    u = np.zeros((m.n_nodes, 3))
    u[:, 2] = 3.0                       # the outlet normal is +z: u . n > 0 everywhere
    assert abs(O.backflow_matrix(m, prob, u)).sum() == 0.0


def test_backflow_for_uniform_inflow_is_scaled_face_mass():
    m = _mesh()
    beta, Uin = 0.7, 2.5
    prob = _problem(O.BC(tag=2, kind="neumann", tparams={"value": 0.0}, beta=beta))
    u = np.zeros((m.n_nodes, 3))
    u[:, 2] = -Uin
    K = O.backflow_matrix(m, prob, u).toarray()
    # closed-form face mass, c = beta rho Uin / 2, on each velocity component
    f = _outlet_faces(m)
    x = m.nodes[f]
    area = 0.5 * np.linalg.norm(np.cross(x[:, 1] - x[:, 0], x[:, 2] - x[:, 0]), axis=1)
    Kref = np.zeros_like(K)
    c = beta * RHO * Uin / 2.0
    for fi in range(f.shape[0]):
        for a in range(3):
            for b in range(3):
                mab = area[fi] * (1.0 + (a == b)) / 12.0
                for comp in range(3):
                    Kref[4 * f[fi, a] + comp, 4 * f[fi, b] + comp] += c * mab
    assert np.allclose(K, Kref, rtol=1e-12, atol=1e-14 * np.abs(Kref).max())


def test_backflow_symmetric_positive_semidefinite():
    m = _mesh()
    prob = _problem(O.BC(tag=2, kind="neumann", tparams={"value": 0.0}, beta=1.0))
    u = np.random.default_rng(3).standard_normal((m.n_nodes, 3))
    K = O.backflow_matrix(m, prob, u)
    nz = np.unique(K.nonzero()[0])
    Kd = K[nz][:, nz].toarray()
    assert np.allclose(Kd, Kd.T, atol=1e-15 * np.abs(Kd).max())
    assert np.linalg.eigvalsh(Kd).min() >= -1e-12 * np.abs(Kd).max()


def test_resistance_vector_gives_exact_flux_of_p1_fields():
    m = _mesh()
    w = O.resistance_vectors(m, 2)
    f = _outlet_faces(m)
    x = m.nodes[f]
    an = 0.5 * np.cross(x[:, 1] - x[:, 0], x[:, 2] - x[:, 0])
    # u = (0, 0, a + b x + c y): the flux through each flat face is A_f n_z (u at the centroid)
    a, b, c = 1.3, -0.4, 0.9
    X = m.nodes
    u = np.zeros((m.n_nodes, 4))
    u[:, 2] = a + b * X[:, 0] + c * X[:, 1]
    cen = x.mean(axis=1)
    exact = np.sum(an[:, 2] * (a + b * cen[:, 0] + c * cen[:, 1]))
    assert abs(w @ u.ravel() - exact) <= 1e-12 * abs(exact)
    # a plain plug flow U e_z through the flat outlet: Q = U * (pi R^2 up to the polygonal rim)
    u[:, 2] = 2.0
    assert abs(w @ u.ravel() - 2.0 * an[:, 2].sum()) <= 1e-12 * 2.0 * an[:, 2].sum()


def _developed_step(outlet):
    m = _mesh()
    prob = _problem(outlet)
    X = m.nodes
    u0 = poiseuille_u(X, R, U)
    p0 = poiseuille_p(X, R, L, U, MU)
    st = O.step(m, prob, [u0, u0], [p0, p0], 1e-3)
    return m, st.x.reshape(-1, 4), st


def test_resistance_with_zero_coefficient_is_neumann_data():
    p_base = 3.0
    _, xr, _ = _developed_step(O.BC(tag=2, kind="resistance", tparams={"value": p_base}, resistance=0.0))
    _, xn, _ = _developed_step(O.BC(tag=2, kind="neumann", tparams={"value": p_base}))
    assert np.allclose(xr, xn, rtol=0, atol=1e-10 * np.abs(xn).max())


def test_resistance_shifts_the_pressure_by_cr_times_flux():
    """With the flux fixed by the inlet data, the resistance outlet's solution is the Neumann
    (h = p_0) one with the same velocity and the pressure raised by C_R Q everywhere: a constant
    pressure c changes the weak form only through -(c, div v) = -c int_Gamma_out v . n (v = 0 on
    the Dirichlet part), which the extra traction C_R Q n balances, and the stabilisation terms
    see only grad p."""
    p_base, CR = 5.0, 0.8
    m, xn, _ = _developed_step(O.BC(tag=2, kind="neumann", tparams={"value": p_base}))
    _, xr, _ = _developed_step(O.BC(tag=2, kind="resistance", tparams={"value": p_base}, resistance=CR))
    Q = O.resistance_vectors(m, 2) @ xn.ravel()
    assert Q > 0.0
    scale_u = np.abs(xn[:, :3]).max()
    assert np.allclose(xr[:, :3], xn[:, :3], rtol=0, atol=1e-9 * scale_u)
    shift = xr[:, 3] - xn[:, 3]
    assert np.allclose(shift, CR * Q, rtol=1e-9, atol=1e-9 * abs(CR * Q)), (shift.min(), shift.max(), CR * Q)
