"""Oracle pins for the moving-domain (ALE) parts of Section 2.1-2.3: the lifting problem
(Eq. lifting, harmonic extension), the BDF mesh velocity and the semi-implicit convective
velocity u* = u^EXT - u_ALE (Eq. u_star).

* Lifting: P1 reproduces linear fields, so linear Dirichlet data on the whole boundary give the
  linear field inside; on a cube, data varying only along z imposed on the faces z = 0, 1 give it
  too, because that field has zero normal flux through the side faces (the natural condition).
* Mesh velocity: the BDF derivative of order k is exact on polynomials of degree <= k.
* Element: with a mesh velocity the matrix is still the Jacobian of the residual.
* Step (Galilean invariance of the semi-implicit ALE form): on a domain translating at constant
  velocity v, with history v + w and Dirichlet data shifted by v, the step gives v + (the fixed-
  domain step for w) and the same pressure.  The BDF weights sum to alpha and the extrapolation
  weights to 1, so the v parts cancel in the time derivative and u* = w^EXT; every other term sees
  only gradients of v (zero).  A missing or mis-signed u_ALE, or a wrong mesh velocity, breaks it."""
import numpy as np
import pytest

import oracle as O
from synthetic import cube_kuhn, cylinder
from tests.test_oracle_element import _fields, _x


def _mesh():
    return cylinder(1.0, 3.0, n_tets=4000, seed=13)


def test_lifting_reproduces_linear_boundary_data():
    m = _mesh()
    rng = np.random.default_rng(1)
    A, c = rng.standard_normal((3, 3)), rng.standard_normal(3)
    bd = np.unique(m.bfaces.ravel())
    d = O.lifting(m, bd, m.nodes[bd] @ A.T + c)
    assert np.allclose(d, m.nodes @ A.T + c, rtol=0, atol=1e-10)


def test_lifting_natural_condition_on_the_wall():
    # the unit cube: the side faces are exactly parallel to z, so a field varying along z only has
    # zero normal flux there (a Delaunay cylinder's wall facets are not exactly axis-parallel)
    m = cube_kuhn(5)
    caps = np.nonzero((np.abs(m.nodes[:, 2]) < 1e-12) | (np.abs(m.nodes[:, 2] - 1.0) < 1e-12))[0]
    a, c = np.array([0.2, -0.1, 0.05]), np.array([0.01, 0.02, 0.03])
    vals = m.nodes[caps, 2:3] * a[None, :] + c[None, :]
    alpha = np.full(m.tets.shape[0], 2.5)   # a constant stiffening leaves the solution unchanged
    d = O.lifting(m, caps, vals, alpha=alpha)
    assert np.allclose(d, m.nodes[:, 2:3] * a[None, :] + c[None, :], rtol=0, atol=1e-10)


@pytest.mark.parametrize("order", [1, 2, 3])
def test_mesh_velocity_exact_on_polynomials(order):
    dt, t1 = 1e-2, 0.37
    rng = np.random.default_rng(order)
    coef = [rng.standard_normal((5, 3)) for _ in range(order + 1)]
    d = lambda t: sum(ck * t ** k for k, ck in enumerate(coef))
    v = lambda t: sum(k * ck * t ** (k - 1) for k, ck in enumerate(coef) if k)
    hist = [d(t1 - j * dt) for j in range(order + 1)]
    assert np.allclose(O.ale_velocity(order, hist, dt), v(t1), rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("seed", range(3))
def test_matrix_is_jacobian_of_residual_with_mesh_velocity(seed):
    x = _x(seed, "random")
    ub, ue, pe = _fields(200 + seed)
    ua = np.random.default_rng(300 + seed).standard_normal((4, 3))
    P = O.Params(rho=1.06, mu=0.035, dt=1e-3, bdf_order=2, stab=2, diffusion=0, f=(0.3, -0.2, 0.1))
    A, b = O.element(P, x, ub, ue, pe, uale=ua)
    A0, _ = O.element(P, x, ub, ue, pe)
    assert np.abs(A - A0).max() > 1e-6 * np.abs(A0).max()            # the mesh velocity matters
    sol = np.random.default_rng(seed).standard_normal(16)
    J = np.zeros((16, 16))
    h = 1e-2
    for k in range(16):
        e = np.zeros(16)
        e[k] = h
        J[:, k] = (O.element_residual(P, x, ub, ue, pe, sol + e, uale=ua)
                   - O.element_residual(P, x, ub, ue, pe, sol - e, uale=ua)) / (2 * h)
    assert np.abs(J - A).max() <= 1e-9 * np.abs(A).max()
    assert np.abs(O.element_residual(P, x, ub, ue, pe, np.zeros(16), uale=ua) + b).max() <= 1e-12 * np.abs(b).max()


@pytest.mark.parametrize("order", [1, 2])
def test_translating_domain_is_the_fixed_domain_step_plus_v(order):
    m = _mesh()
    V, dt, t1 = m.n_nodes, 1e-3, 0.05
    v = np.array([0.3, -0.2, 0.5])
    rng = np.random.default_rng(17)
    r2 = m.nodes[:, 0] ** 2 + m.nodes[:, 1] ** 2
    base = np.zeros((V, 3))
    base[:, 2] = 20.0 * np.clip(1.0 - r2, 0.0, None)
    wh = [base + rng.standard_normal((V, 3)) for _ in range(order)]
    ph = [rng.standard_normal(V) for _ in range(order)]
    inflow = np.zeros((V, 3))
    inflow[:, 2] = 20.0 * np.clip(1.0 - r2, 0.0, None)
    P = O.Params(rho=1.06, mu=0.035, dt=dt, bdf_order=order, stab=2)
    prob = O.Problem(P, [O.BC(tag=0, kind="nodal"), O.BC(tag=1, kind="nodal"),
                         O.BC(tag=2, kind="neumann", tparams={"value": 2.0})])
    fixed = O.step(m, prob, wh, ph, t1, nodal={0: np.zeros((V, 3)), 1: inflow})
    shift = np.broadcast_to(v, (V, 3))
    d_hist = [shift * (t1 - j * dt) for j in range(order + 1)]       # d^{n+1}, d^n, ...
    moving = O.step(m, prob, [w + shift for w in wh], ph, t1, nodal={0: shift.copy(), 1: inflow + shift},
                    d_hist=d_hist)
    xf, xm = fixed.x.reshape(-1, 4), moving.x.reshape(-1, 4)
    su, sp_ = np.abs(xf[:, :3]).max(), np.abs(xf[:, 3]).max()
    assert np.allclose(xm[:, :3] - v, xf[:, :3], rtol=0, atol=1e-9 * su)
    assert np.allclose(xm[:, 3], xf[:, 3], rtol=0, atol=1e-9 * sp_)
    # and without the mesh velocity the translated step differs
    plain = O.step(m, prob, [w + shift for w in wh], ph, t1, nodal={0: shift.copy(), 1: inflow + shift})
    assert np.abs(plain.x.reshape(-1, 4)[:, :3] - v - xf[:, :3]).max() > 1e-6 * su
