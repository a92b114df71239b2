"""The seeded synthetic inputs that stand in for the paper's meshes: the recipes hold what the
design notes state (host only, no GPU).

* Seeded: the same seed gives the same mesh bit for bit; another seed gives another mesh.
* Shuffled: node order carries no spatial order.  The library's space-filling-curve renumbering
  is exercised, not bypassed.
* Valid: every tetrahedron is positively oriented; the tagged faces are exactly the boundary faces.
* Tagged as in Test II: the wall is tag 0, the inlet (z = 0) tag 1, the outlet (z = L) tag 2.  The
  wall nodes lie on the cylinder, or on the stenosed radius r_s(z) = R (1 - s (1 + cos(pi
  (z - z_c) / h))) within |z - z_c| <= h.
* Shaped like the tetrahedral meshes of Table tab:mesh (Section 4; `golden/table_mesh_tetrahedral.txt`).
  At 100k tets, the tetrahedra per vertex and the mean edge ratio lie within the range of the
  table's two tetrahedral meshes, and the largest edge ratio stays below the table's largest.
  The count is within 5 % of the requested one.
* Batched unions keep every member's nodes, and offset member i's tags by 10 i.
* The Beltrami flow of Appendix A, which gives the Beltrami histories, boundary data and error
  norms, is an exact Navier-Stokes solution for any rho and mu (checked by finite differences);
  so is the steady Poiseuille pipe flow, with the flow rate its peak velocity implies.
"""
import os

import numpy as np
import pytest

import synthetic as S
from synthetic.meshes import _signed_volumes, boundary_faces

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _table_mesh():
    rows = {}
    with open(os.path.join(GOLDEN, "table_mesh_tetrahedral.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, *v = line.split()
                rows[name] = dict(zip(("elements", "vertices", "h_min", "h_avg", "h_max", "q_min", "q_avg", "q_max"),
                                      map(float, v)))
    return rows


def _same(a, b):
    return all(np.array_equal(getattr(a, k), getattr(b, k)) for k in ("nodes", "tets", "bfaces", "btags"))


def _face_keys(f):
    return set(map(tuple, np.sort(f, axis=1)))


def test_seeded_and_shuffled():
    a = S.cylinder(1.0, 10.0, n_tets=20000, seed=2)
    assert _same(a, S.cylinder(1.0, 10.0, n_tets=20000, seed=2))
    assert not _same(a, S.cylinder(1.0, 10.0, n_tets=20000, seed=5))
    assert abs(np.corrcoef(np.arange(a.n_nodes), a.nodes[:, 2])[0, 1]) < 0.1


@pytest.mark.parametrize("make", [lambda: S.cylinder(1.0, 10.0, n_tets=20000, seed=2),
                                  lambda: S.stenosis(1.0, 10.0, n_tets=20000, seed=3),
                                  lambda: S.bifurcation(n_tets=20000, seed=1001)])
def test_valid_oriented_and_tagged(make):
    m = make()
    assert np.all(_signed_volumes(m.nodes, m.tets) > 0.0)
    assert _face_keys(m.bfaces) == _face_keys(boundary_faces(m.nodes, m.tets))
    assert len(_face_keys(m.bfaces)) == len(m.bfaces)
    tags = set(np.unique(m.btags).tolist())
    assert {0, 1, 2} <= tags


def test_cylinder_tags_and_table_statistics():
    m = S.cylinder(1.0, 10.0, n_tets=100_000, seed=2)
    z = m.nodes[m.bfaces][:, :, 2]
    assert np.all(z[m.btags == 1] == 0.0) and np.all(z[m.btags == 2] == 10.0)
    wall = np.unique(m.bfaces[m.btags == 0])
    assert np.abs(np.hypot(m.nodes[wall, 0], m.nodes[wall, 1]) - 1.0).max() < 1e-12
    st = S.mesh_stats(m)
    table = _table_mesh()
    ratio = [r["elements"] / r["vertices"] for r in table.values()]
    assert min(ratio) <= st["tets_per_vertex"] <= max(ratio)                 # 5.37 .. 6.26
    assert min(r["q_avg"] for r in table.values()) <= st["q_avg"] <= max(r["q_avg"] for r in table.values())
    assert st["q_max"] <= max(r["q_max"] for r in table.values())
    assert abs(m.n_tets - 100_000) <= 5_000


def test_stenosis_wall_follows_the_radial_map():
    m = S.stenosis(1.0, 10.0, n_tets=50_000, seed=3, z_center=3.0, half_length=1.0, severity=0.25)
    wall = np.unique(m.bfaces[m.btags == 0])
    x = m.nodes[wall]
    r, z = np.hypot(x[:, 0], x[:, 1]), x[:, 2]
    rs = np.where(np.abs(z - 3.0) <= 1.0, 1.0 - 0.25 * (1.0 + np.cos(np.pi * (z - 3.0))), 1.0)
    assert np.abs(r - rs).max() < 1e-12
    assert r.min() == pytest.approx(0.5, abs=0.02)        # the throat keeps half the radius: 75 % of the area gone


def test_bifurcation_has_an_inlet_and_two_outlets():
    m = S.bifurcation(n_tets=30_000, seed=1001)
    assert set(np.unique(m.btags).tolist()) == {0, 1, 2, 3}
    for tag in (1, 2, 3):
        assert np.count_nonzero(m.btags == tag) > 10


def test_batch_union_offsets_members():
    a = S.cylinder(1.0, 10.0, n_tets=20000, seed=2)
    b = S.bifurcation(n_tets=20_000, seed=1001)
    u = S.batch([a, b])
    assert u.n_nodes == a.n_nodes + b.n_nodes and u.n_tets == a.n_tets + b.n_tets
    assert np.array_equal(u.nodes[:a.n_nodes], a.nodes) and np.array_equal(u.tets[a.n_tets:], b.tets + a.n_nodes)
    assert set(np.unique(u.btags).tolist()) == set(np.unique(a.btags).tolist()) | {10 + t for t in np.unique(b.btags)}


@pytest.mark.parametrize("rho,mu", [(1.0, 1.0), (1.06, 0.035)])
def test_beltrami_flow_solves_navier_stokes(rho, mu):
    """The closed form of Appendix A used for the Beltrami data and errors: by central differences
    at random points, u is divergence-free, beltrami_grad_u is its gradient, and
    rho (du/dt + (u . grad) u) - mu lap u + grad p = 0 with no forcing.  A wrong sign, factor or
    decay rate in u or p leaves a residual of the size of the terms."""
    X = np.random.default_rng(0).uniform(-1.0, 1.0, (50, 3))
    t, h, H = 0.3, 1e-5, 1e-3

    def U(Y, s):
        return S.beltrami_u(Y, s, rho, mu)

    def P(Y, s):
        return S.beltrami_p(Y, s, rho, mu)

    G, gp, lap = np.zeros((50, 3, 3)), np.zeros((50, 3)), np.zeros((50, 3))
    for j in range(3):
        e, E = np.eye(3)[j] * h, np.eye(3)[j] * H
        G[:, :, j] = (U(X + e, t) - U(X - e, t)) / (2 * h)
        gp[:, j] = (P(X + e, t) - P(X - e, t)) / (2 * h)
        lap += (U(X + E, t) - 2 * U(X, t) + U(X - E, t)) / H ** 2
    dudt = (U(X, t + h) - U(X, t - h)) / (2 * h)
    adv = np.einsum("nij,nj->ni", G, U(X, t))
    terms = [rho * dudt, rho * adv, mu * lap, gp]
    scale = sum(np.abs(v).max() for v in terms)
    assert np.abs(np.trace(G, axis1=1, axis2=2)).max() <= 1e-9 * np.abs(G).max()
    assert np.abs(G - S.beltrami_grad_u(X, t, rho, mu)).max() <= 1e-8 * np.abs(G).max()
    assert np.abs(terms[0] + terms[1] - terms[2] + terms[3]).max() <= 1e-6 * scale


def test_poiseuille_flow_solves_navier_stokes():
    """The steady pipe flow: divergence-free, no advection ((u . grad) u = 0 for an axial field that
    varies across the pipe only), -mu lap u + grad p = 0 inside the pipe, p = 0 at the outlet, and
    flow rate pi R^2 U / 2 (the unit-flow-rate parabolic profile scaled by it)."""
    R, Lp, U, mu = 1.0, 10.0, 20.0, 0.035
    rng = np.random.default_rng(1)
    r, th = 0.9 * R * np.sqrt(rng.uniform(size=40)), rng.uniform(0, 2 * np.pi, 40)
    X = np.stack([r * np.cos(th), r * np.sin(th), rng.uniform(0.5, Lp - 0.5, 40)], 1)
    h, H = 1e-6, 1e-3
    G, gp, lap = np.zeros((40, 3, 3)), np.zeros((40, 3)), np.zeros((40, 3))
    for j in range(3):
        e, E = np.eye(3)[j] * h, np.eye(3)[j] * H
        G[:, :, j] = (S.poiseuille_u(X + e, R, U) - S.poiseuille_u(X - e, R, U)) / (2 * h)
        gp[:, j] = (S.poiseuille_p(X + e, R, Lp, U, mu) - S.poiseuille_p(X - e, R, Lp, U, mu)) / (2 * h)
        lap += (S.poiseuille_u(X + E, R, U) - 2 * S.poiseuille_u(X, R, U) + S.poiseuille_u(X - E, R, U)) / H ** 2
    u = S.poiseuille_u(X, R, U)
    assert np.abs(np.trace(G, axis1=1, axis2=2)).max() <= 1e-8 * U
    assert np.abs(np.einsum("nij,nj->ni", G, u)).max() <= 1e-8 * U * U
    assert np.abs(-mu * lap + gp).max() <= 1e-6 * np.abs(gp).max()
    assert np.abs(S.poiseuille_p(np.array([[0.3, 0.2, Lp]]), R, Lp, U, mu)).max() == 0.0
    # flow rate through a cross-section (polar quadrature, exact for the quadratic profile)
    rq, wq = np.polynomial.legendre.leggauss(4)
    rr = 0.5 * R * (rq + 1.0)
    q = np.sum(0.5 * R * wq * 2 * np.pi * rr * S.poiseuille_u(np.stack([rr, 0 * rr, 0 * rr + 1.0], 1), R, U)[:, 2])
    assert q == pytest.approx(np.pi * R ** 2 * U / 2.0, rel=1e-12)


def test_zero_net_flux_correction_of_all_dirichlet_data():
    """Beltrami data on the whole boundary of the Kuhn cube: after the correction the discrete net
    flux of the piecewise-linear data (each face's area vector times the mean of its three nodal
    values) is zero.  The correction is small, because the exact field is divergence-free and the
    flux of the P1 interpolant only carries its interpolation error."""
    m = S.cube_kuhn(6)
    bd = np.unique(m.bfaces)
    g = S.beltrami_u(m.nodes, 0.01)

    def flux(values):
        full = np.zeros_like(m.nodes)
        full[bd] = values
        x = m.nodes[m.bfaces]
        area_vec = 0.5 * np.cross(x[:, 1] - x[:, 0], x[:, 2] - x[:, 0])
        # outward: the cube's centre lies on the inner side of every face
        inward = np.einsum("ij,ij->i", area_vec, x.mean(axis=1) - 0.5) < 0
        area_vec[inward] *= -1
        return np.sum(area_vec * full[m.bfaces].mean(axis=1))

    before = flux(g[bd])
    fixed = S.zero_net_flux(m.nodes, m.bfaces, bd, g[bd])
    scale = np.sum(np.abs(g[bd])) / bd.size
    assert abs(before) > 1e-8 * scale                    # the P1 data alone are not flux-free
    assert abs(flux(fixed)) <= 1e-13 * scale
    assert np.abs(fixed - g[bd]).max() <= 1e-2 * np.abs(g[bd]).max()
