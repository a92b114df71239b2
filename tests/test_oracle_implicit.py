"""Oracle pins for the fully implicit formulation (Eq. u_star implicit, implicit LES term),
linearised by Newton's method (Section 2.4).

* Newton converges superlinearly from the semi-implicit solution (the second contraction factor is
  below the first to the power 1.4 and below a twentieth of it, which a fixed-factor contraction
  cannot meet): the element Jacobians (central differences of the implicit element residual) are
  consistent with the residual.  A Jacobian spoiled on purpose fails the same criterion.
* The converged solution U is the fixed point of the semi-implicit system assembled with the
  extrapolated fields replaced by U itself (u* = u, tau_M(u), r_M(u, p)): checked through the
  ordinary assembly, Dirichlet rows and direct solve, a path independent of the Newton routine.
* Galilean invariance on a domain translating at constant velocity v (ALE): the implicit step with
  history v + w and data shifted by v is v + the fixed-domain implicit step for w."""
import numpy as np
import pytest

import oracle as O
from synthetic import cylinder
from tests import cases as C


@pytest.mark.parametrize("order,riis", [(1, False), (2, True)])
def test_newton_converges_quadratically(order, riis):
    case = C.vessel_case(3000, seed=21, order=order, riis=riis)
    prob = C.oracle_problem(case)
    uh = [case.u_hist[j] for j in range(order)]
    ph = [case.p_hist[j] for j in range(order)]
    r = O.implicit_step(case.mesh, prob, uh, ph, case.t0 + case.dt)
    res = r.residuals
    assert res[-1] <= 1e-11 * r.scale and len(res) <= 5, res
    assert _superlinear(res), res
    # The criterion separates Newton from a method that contracts by a fixed factor.  A Jacobian
    # spoiled on purpose (central differences of step 3, far outside the residual's linear range)
    # still contracts by about 1e-4 per iteration, as often as Newton's first step, but linearly.
    bad = O.implicit_step(case.mesh, prob, uh, ph, case.t0 + case.dt, h=3.0, tol=1e-14, max_newton=3)
    assert not _superlinear(bad.residuals), bad.residuals


def _superlinear(res):
    """Newton's contraction factors shrink from one iteration to the next: c_2 <= c_1^1.4 and
    c_2 <= c_1/20 (c_k = ||F_k|| / ||F_{k-1}||).  A fixed-factor (linear) contraction fails
    both: c_2 = c_1."""
    c1, c2 = res[1] / res[0], res[2] / res[1]
    return c2 <= c1 ** 1.4 and c2 <= c1 / 20.0


def test_implicit_solution_is_the_picard_fixed_point():
    case = C.vessel_case(3000, seed=22, order=2, riis=True)
    prob = C.oracle_problem(case)
    uh = [case.u_hist[j] for j in range(2)]
    ph = [case.p_hist[j] for j in range(2)]
    t1 = case.t0 + case.dt
    r = O.implicit_step(case.mesh, prob, uh, ph, t1)
    U = r.x.reshape(-1, 4)
    prm = prob.params
    _, beta, _ = O.bdf_coefficients(2)
    ubdf = beta[0] * uh[0] + beta[1] * uh[1]
    A, b = O.assemble(prm, case.mesh.nodes, case.mesh.tets, ubdf, U[:, :3].copy(), U[:, 3].copy(), prob.riis)
    b = b + O.neumann_rhs(case.mesh, prob, t1)
    ids, vals = O.dirichlet_data(case.mesh, prob, t1)
    rows = (4 * ids[:, None] + np.arange(3)[None, :]).ravel()
    A, b = O.apply_dirichlet(A, b, rows, vals.ravel())
    x = O.solve_direct(A, b)
    assert np.linalg.norm(x - r.x) <= 1e-8 * np.linalg.norm(r.x)
    # and it is not the semi-implicit solution
    semi = O.step(case.mesh, prob, uh, ph, t1)
    assert np.linalg.norm(semi.x - r.x) > 1e-6 * np.linalg.norm(r.x)


def test_implicit_translating_domain_is_the_fixed_domain_step_plus_v():
    m = cylinder(1.0, 3.0, n_tets=3000, seed=13)
    V, dt, t1 = m.n_nodes, 1e-3, 0.05
    v = np.array([0.3, -0.2, 0.5])
    rng = np.random.default_rng(19)
    r2 = m.nodes[:, 0] ** 2 + m.nodes[:, 1] ** 2
    inflow = np.zeros((V, 3))
    inflow[:, 2] = 20.0 * np.clip(1.0 - r2, 0.0, None)
    wh = [inflow + rng.standard_normal((V, 3)) for _ in range(2)]
    ph = [rng.standard_normal(V) for _ in range(2)]
    P = O.Params(rho=1.06, mu=0.035, dt=dt, bdf_order=2, stab=2)
    prob = O.Problem(P, [O.BC(tag=0, kind="nodal"), O.BC(tag=1, kind="nodal"),
                         O.BC(tag=2, kind="neumann", tparams={"value": 2.0})])
    fixed = O.implicit_step(m, prob, wh, ph, t1, nodal={0: np.zeros((V, 3)), 1: inflow})
    shift = np.broadcast_to(v, (V, 3))
    moving = O.implicit_step(m, prob, [w + shift for w in wh], ph, t1, nodal={0: shift.copy(), 1: inflow + shift},
                             d_hist=[shift * (t1 - j * dt) for j in range(3)])
    xf, xm = fixed.x.reshape(-1, 4), moving.x.reshape(-1, 4)
    assert np.allclose(xm[:, :3] - v, xf[:, :3], rtol=0, atol=1e-8 * np.abs(xf[:, :3]).max())
    assert np.allclose(xm[:, 3], xf[:, 3], rtol=0, atol=1e-8 * np.abs(xf[:, 3]).max())
