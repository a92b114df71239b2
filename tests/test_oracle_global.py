"""Pins of the oracle's global routines: whole steps against closed-form flows, boundary data
against the paper's definitions, and the linear-algebra reference against exact inverses."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from synthetic import (beltrami_grad_u, beltrami_p, beltrami_u, cube_kuhn, cylinder,
                       poiseuille_p, poiseuille_u, zero_net_flux)


def beltrami_run(n, steps=10, dt=1e-3, order=1, stab=2):
    """Beltrami set-up: unit cube, rho = mu = 1, exact Dirichlet data on all faces (made
    discretely flux-free), pressure pinned at node 0 to the exact value."""
    m = cube_kuhn(n)
    P = O.Params(rho=1.0, mu=1.0, dt=dt, bdf_order=order, stab=stab)
    prob = O.Problem(P, [O.BC(tag=t, kind="nodal") for t in range(1, 7)], pin_node=0)
    X = m.nodes
    bd = np.unique(m.bfaces.ravel())
    uh = [beltrami_u(X, -k * dt) for k in range(order)]
    ph = [beltrami_p(X, -k * dt) for k in range(order)]
    t1 = 0.0
    for s in range(steps):
        t1 = (s + 1) * dt
        ue = beltrami_u(X, t1)
        ue[bd] = zero_net_flux(X, m.bfaces, bd, ue[bd])
        st = O.step(m, prob, uh, ph, t1, nodal={tg: ue for tg in range(1, 7)},
                    pin_value=float(beltrami_p(X[:1], t1)[0]))
        x = st.x.reshape(-1, 4)
        uh = [x[:, :3].copy()] + uh[:order - 1]
        ph = [x[:, 3].copy()] + ph[:order - 1]
    return O.relative_errors(X, m.tets, uh[0], ph[0], lambda q: beltrami_u(q, t1),
                             lambda q: beltrami_grad_u(q, t1), lambda q: beltrami_p(q, t1),
                             p_mean_free=True)


def test_beltrami_convergence_rates():
    # Section 4.1: e_L2^u ~ h^2, e_H1^u ~ h, pressure at least ~h for P1-P1 with stabilisation.
    e4 = beltrami_run(4)
    e8 = beltrami_run(8)
    rates = [math.log2(a / b) for a, b in zip(e4, e8)]
    assert rates[0] > 1.7, rates
    assert rates[1] > 0.9, rates
    assert rates[2] > 1.2, rates
    assert e8[0] < 0.01 and e8[1] < 0.16


def _iterative(A, b):
    return O.fgmres(A, b, M=O.ASimple(A).apply, restart=60, tol=1e-12)[0]


def _poiseuille(n_tets, steps=6):
    R, L, U, mu, rho = 1.0, 2.0, 20.0, 0.035, 1.06
    m = cylinder(R, L, n_tets=n_tets, seed=2)
    P = O.Params(rho=rho, mu=mu, dt=1e-3, bdf_order=2, stab=2)
    Q = U * math.pi * R * R / 2.0
    prob = O.Problem(P, [O.BC(tag=0, kind="noslip"),
                         O.BC(tag=1, kind="dirichlet", time="constant", tparams={"value": Q},
                              space="parabolic", radius=R),
                         O.BC(tag=2, kind="neumann", tparams={"value": 0.0})])
    X = m.nodes
    u0, p0 = poiseuille_u(X, R, U), poiseuille_p(X, R, L, U, mu)
    uh, ph = [u0, u0], [p0, p0]
    for s in range(steps):
        st = O.step(m, prob, uh, ph, (s + 1) * 1e-3, solver=_iterative)
        x = st.x.reshape(-1, 4)
        uh = [x[:, :3].copy(), uh[0]]
        ph = [x[:, 3].copy(), ph[0]]
    eu = np.linalg.norm(uh[0] - u0) / np.linalg.norm(u0)
    dp = ph[0][m.tag_nodes(1)].mean()
    return eu, dp, 4 * mu * U * L / R ** 2


def test_poiseuille_near_fixed_point():
    # Exact Poiseuille (grad-grad form) is a steady solution with zero traction at the outlet;
    # started from it, the discrete steps stay close to it, and the inlet pressure (= pressure
    # drop, p = 0 at the outlet) converges to 4 mu U L / R^2 under refinement.
    eu1, dp1, ex = _poiseuille(6000)
    eu2, dp2, _ = _poiseuille(24000)
    assert eu1 < 0.03 and eu2 < 0.012, (eu1, eu2)
    assert abs(dp2 - ex) < 0.2 * ex, (dp2, ex)
    assert abs(dp2 - ex) * 2.5 < abs(dp1 - ex), (dp1, dp2, ex)


def test_time_laws():
    assert O.time_law("constant", 3.0, {"value": 2.5}) == 2.5
    tp = {"gmin": 1.0, "gmax": 5.0, "period": 0.8}
    assert O.time_law("pulsatile", 0.0, tp) == pytest.approx(1.0)
    assert O.time_law("pulsatile", 0.4, tp) == pytest.approx(5.0)
    assert O.time_law("pulsatile", 0.8, tp) == pytest.approx(1.0)
    rp = {"g0": 1.0, "g1": 3.0, "t0": 0.5, "tL": 0.2}
    assert O.time_law("ramp", 0.1, rp) == 1.0
    assert O.time_law("ramp", 0.6, rp) == pytest.approx(2.0)
    assert O.time_law("ramp", 0.8, rp) == 3.0
    fp = {"period": 1.0, "a": [1.0, 0.5], "b": [0.0, 0.25]}
    assert O.time_law("fourier", 0.25, fp) == pytest.approx(1.0 + 0.25)


def test_parabolic_profile_has_unit_flow_rate():
    # Section 2.2.1 remark: the parabolic profile has unit flow rate; with Q = U pi R^2 / 2 its
    # peak is U.
    R = 1.0
    m = cylinder(R, 3.0, n_tets=20000, seed=5)
    prob = O.Problem(O.Params(), [O.BC(tag=1, kind="dirichlet", time="constant",
                                       tparams={"value": 1.0}, space="parabolic", radius=R)])
    ids, vals = O.dirichlet_data(m, prob, 0.0)
    f = m.bfaces[m.btags == 1]
    x = m.nodes[f]
    area_n = 0.5 * np.cross(x[:, 1] - x[:, 0], x[:, 2] - x[:, 0])
    full = np.zeros((m.n_nodes, 3))
    full[ids] = vals
    flux = -np.sum(np.einsum("fkj,fj->fk", full[f], area_n).mean(axis=1))
    assert flux == pytest.approx(1.0, rel=0.02)
    assert vals[:, 2].max() == pytest.approx(2.0 / math.pi, rel=0.05)
    assert np.allclose(vals[:, :2], 0.0, atol=1e-12)


def test_neumann_total_force():
    # -(h n, v) summed over all test functions = -h * (area vector of the tagged boundary).
    m = cylinder(1.0, 3.0, n_tets=8000, seed=6)
    prob = O.Problem(O.Params(), [O.BC(tag=2, kind="neumann", tparams={"value": 7.0})])
    r = O.neumann_rhs(m, prob, 0.0).reshape(-1, 4)
    _, n, area = O.boundary_geometry(m.nodes, m.bfaces, m.btags, 2)
    assert np.allclose(r[:, :3].sum(axis=0), -7.0 * area * n, rtol=1e-12, atol=1e-12)
    assert np.allclose(r[:, 3], 0.0)


def test_apply_dirichlet_rows():
    rng = np.random.default_rng(0)
    A = sp.random(40, 40, density=0.2, random_state=1, format="csr") + sp.eye(40) * 3.0
    b = rng.standard_normal(40)
    rows, vals = np.array([3, 7, 11]), np.array([1.0, -2.0, 0.5])
    A2, b2 = O.apply_dirichlet(A, b, rows, vals)
    x = np.linalg.solve(A2.toarray(), b2)
    assert np.allclose(x[rows], vals)
    for r in rows:
        row = A2[r].toarray().ravel()
        assert np.count_nonzero(row) == 1 and row[r] == pytest.approx(abs(A[r, r]))
    keep = np.setdiff1d(np.arange(40), rows)
    assert np.allclose(A2[keep].toarray(), A[keep].toarray())


# ---------------------------- linear algebra reference ----------------------------------
def test_jacobi_exact_on_diagonal():
    d = np.linspace(1.0, 5.0, 30)
    M = sp.diags(d).tocsr()
    b = np.random.default_rng(1).standard_normal(30)
    assert np.allclose(O.jacobi(M, 1.0 / d, b, 1.0, 1), b / d)


def test_chebyshev_error_bound():
    # For SPD D^-1 M with spectrum in [lmin, lmax], k Chebyshev steps reduce the error by at
    # least 2 q^k / (1 + q^2k), q = (sqrt(kappa)-1)/(sqrt(kappa)+1) (Saad, Sec. 12.3).
    n = 200
    lam = np.linspace(0.1, 2.0, n)
    Q, _ = np.linalg.qr(np.random.default_rng(2).standard_normal((n, n)))
    M = sp.csr_matrix(Q @ np.diag(lam) @ Q.T)
    dinv = np.ones(n)
    x_true = np.random.default_rng(3).standard_normal(n)
    b = M @ x_true
    kappa = 20.0
    q = (math.sqrt(kappa) - 1) / (math.sqrt(kappa) + 1)
    for k in (1, 3, 8, 15):
        x = O.chebyshev(M, dinv, b, 0.1, 2.0, k)
        bound = 2 * q ** k / (1 + q ** (2 * k))
        assert np.linalg.norm(x - x_true) <= bound * np.linalg.norm(x_true) * (1 + 1e-9)


def test_asimple_exact_when_F_diagonal():
    # With a diagonal velocity block and converged Schur smoothing, the SIMPLE factorisation is
    # an exact inverse: z = A^-1 r.  Pins the block formula (order and signs of D, G, S).
    rng = np.random.default_rng(4)
    V = 30
    N = 4 * V
    vel = (4 * np.arange(V)[:, None] + np.arange(3)[None, :]).ravel()
    pre = 4 * np.arange(V) + 3
    A = np.zeros((N, N))
    A[vel, vel] = rng.uniform(2.0, 4.0, vel.size)
    G = rng.standard_normal((vel.size, V)) * (rng.random((vel.size, V)) < 0.2)
    A[np.ix_(vel, pre)] = G
    A[np.ix_(pre, vel)] = -G.T
    A[np.ix_(pre, pre)] = np.diag(rng.uniform(1.0, 2.0, V))
    A = sp.csr_matrix(A)
    opts = O.ASimpleOpts(f=O.SmootherOpts("jacobi", 1, 1.0), s=O.SmootherOpts("jacobi", 400, 0.6))
    pc = O.ASimple(A, opts)
    r = rng.standard_normal(N)
    z = pc.apply(r)
    assert np.allclose(z, np.linalg.solve(A.toarray(), r), rtol=1e-9, atol=1e-9)


def test_fgmres_matches_direct_solve():
    rng = np.random.default_rng(5)
    n = 300
    A = sp.random(n, n, density=0.03, random_state=6, format="csr") + sp.eye(n) * 4.0
    b = rng.standard_normal(n)
    x, its, hist = O.fgmres(A, b, restart=20, tol=1e-12)
    assert np.linalg.norm(A @ x - b) <= 1e-11 * np.linalg.norm(b)
    assert np.allclose(x, np.linalg.solve(A.toarray(), b), rtol=1e-9)


def test_asimple_gmres_solves_navier_stokes_system():
    # The preconditioned solve reaches the direct solution of an assembled cube system.
    m = cube_kuhn(4)
    P = O.Params(rho=1.0, mu=1.0, dt=1e-3, bdf_order=1, stab=2)
    u0, p0 = beltrami_u(m.nodes, 0.0), beltrami_p(m.nodes, 0.0)
    A, b = O.assemble(P, m.nodes, m.tets, u0, u0, p0)
    bd = np.unique(m.bfaces.ravel())
    rows = np.r_[(4 * bd[:, None] + np.arange(3)).ravel(), 3]
    vals = np.r_[beltrami_u(m.nodes[bd], 1e-3).ravel(), 0.0]
    A, b = O.apply_dirichlet(A, b, rows, vals)
    xd = O.solve_direct(A, b)
    x, its, _ = O.fgmres(A, b, M=O.ASimple(A).apply, restart=40, tol=1e-13)
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)


# ---------------------------- Womersley inlet profile (Section 2.2.1) ----------------------
def test_womersley_unit_flux_and_wall_value():
    from scipy.integrate import quad

    R, nu = 1.0, 0.035 / 1.06
    for omega in (2 * math.pi, 10 * math.pi):
        re = quad(lambda r: np.real(O.womersley_profile(r, R, omega, nu)) * 2 * math.pi * r, 0, R, limit=200)[0]
        im = quad(lambda r: np.imag(O.womersley_profile(r, R, omega, nu)) * 2 * math.pi * r, 0, R, limit=200)[0]
        assert re == pytest.approx(1.0, abs=1e-9) and abs(im) < 1e-9
        assert abs(O.womersley_profile(R, R, omega, nu)) < 1e-12


def test_womersley_small_frequency_is_poiseuille():
    R, nu = 0.8, 1.0
    r = np.linspace(0, R, 9)
    W = O.womersley_profile(r, R, 1e-6, nu)
    assert np.allclose(W.real, 2 * (R * R - r * r) / (math.pi * R ** 4), rtol=1e-6, atol=1e-9)
    assert np.abs(W.imag).max() < 1e-5


def test_womersley_solves_the_oscillatory_pipe_equation():
    # For u = W(r) e^{i w t}: i w W = -dp/dz + nu (W'' + W'/r) with a uniform pressure gradient,
    # so W'' + W'/r - (i w / nu) W is the same constant at every radius.
    R, nu, omega = 1.0, 0.05, 4.0
    h = 1e-4
    vals = []
    for r in (0.2, 0.45, 0.7, 0.9):
        Wm, W0, Wp = O.womersley_profile(np.array([r - h, r, r + h]), R, omega, nu)
        lap = (Wp - 2 * W0 + Wm) / h ** 2 + (Wp - Wm) / (2 * h * r)
        vals.append(lap - 1j * omega / nu * W0)
    vals = np.array(vals)
    assert np.abs(vals - vals[0]).max() <= 1e-5 * np.abs(vals[0])
