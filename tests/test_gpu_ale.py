"""GPU tests of the moving-domain (ALE) path of Sections 2.1-2.3 against the oracle.

* Lifting (Eq. lifting, harmonic extension on the reference mesh): the device's conjugate-gradient
  solution matches the oracle's sparse direct solve within 1e-8 of the largest displacement.
* A step on a deforming cylinder (the configuration x^ + d^{n+1}, u* = u^EXT - u_ALE with u_ALE the
  BDF derivative of the displacement, Neumann loads on the moved outlet faces) matches the oracle's
  step(..., d_hist=...) within 1e-6 relative L2, in FP64 and mixed precision; so does a fully
  implicit step (Newton) on the same moving mesh.
* Galilean invariance on the device: on a domain translating at constant velocity v, with history
  v + w and Dirichlet data shifted by v, the step gives v + the fixed-domain step for w and the same
  pressure (1e-8)."""
import dataclasses
import math

import numpy as np
import pytest

from synthetic import cylinder
from tests import cases as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2304_12032_gb300 import build

    build.build()


L_CYL = 3.0


def _case(order=2, seed=13):
    m = cylinder(1.0, L_CYL, n_tets=3000, seed=seed)
    V = m.n_nodes
    rng = np.random.default_rng(19)
    r2 = m.nodes[:, 0] ** 2 + m.nodes[:, 1] ** 2
    inflow = np.zeros((V, 3))
    inflow[:, 2] = 20.0 * np.clip(1.0 - r2, 0.0, None)
    uh = np.stack([inflow + rng.standard_normal((V, 3)) for _ in range(order)])
    ph = np.stack([rng.standard_normal(V) for _ in range(order)])
    bcs = [dict(tag=0, kind="nodal"), dict(tag=1, kind="nodal"),
           dict(tag=2, kind="neumann", time="constant", p=(2.0,))]
    return C.Case(m, 1.06, 0.035, 1e-3, order, bcs, [], uh, ph, 0.05, 2, 0, (0.0, 0.0, 0.0),
                  nodal={0: np.zeros((V, 3)), 1: inflow})


def _dfield(X, s):
    # a smooth deformation: radial bulge and axial stretch, amplitude s
    w = np.sin(math.pi * X[:, 2] / L_CYL)
    return s * np.stack([0.04 * w * X[:, 0], 0.04 * w * X[:, 1], 0.02 * X[:, 2] * w], axis=1)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _ale_inputs(case):
    X = case.mesh.nodes
    bd = np.unique(case.mesh.bfaces.ravel())
    d_hist = [_dfield(X, 0.9 - 0.1 * j) for j in range(case.order)]
    return bd, _dfield(X[bd], 1.0), d_hist


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_deforming_mesh_step_matches_oracle(precision):
    import oracle as O

    case = _case()
    bd, dbd, d_hist = _ale_inputs(case)
    prob = C.oracle_problem(case)
    d1 = O.lifting(case.mesh, bd, dbd)
    ref = O.step(case.mesh, prob, list(case.u_hist), list(case.p_hist), case.t0 + case.dt, nodal=case.nodal,
                 d_hist=[d1] + d_hist).x.reshape(-1, 4)
    opts = dict(gmres_rtol=1e-12, gmres_max_iters=3000) if precision == "fp64" else \
        dict(precision="mixed", smoother_bf16=1, gmres_rtol=1e-10)
    _, _, st = C.gpu_state(case, **opts)
    st.set_displacement(d_hist)
    st.set_boundary_displacement(bd, dbd)
    stats = st.step()
    u, p = st.get()
    d, its = st.get_displacement()
    assert np.abs(d - d1).max() <= 1e-8 * np.abs(d1).max(), (np.abs(d - d1).max(), its)
    assert its > 0
    assert _rel(u, ref[:, :3]) <= 1e-6 and _rel(p, ref[:, 3]) <= 1e-6, (precision, _rel(u, ref[:, :3]),
                                                                        _rel(p, ref[:, 3]), stats)
    # the motion matters: the fixed-mesh step differs
    fixed = O.step(case.mesh, prob, list(case.u_hist), list(case.p_hist), case.t0 + case.dt,
                   nodal=case.nodal).x.reshape(-1, 4)
    assert _rel(fixed[:, :3], ref[:, :3]) > 1e-4


def test_deforming_mesh_implicit_step_matches_oracle():
    import oracle as O

    case = _case()
    bd, dbd, d_hist = _ale_inputs(case)
    prob = C.oracle_problem(case)
    d1 = O.lifting(case.mesh, bd, dbd)
    ref = O.implicit_step(case.mesh, prob, list(case.u_hist), list(case.p_hist), case.t0 + case.dt,
                          nodal=case.nodal, d_hist=[d1] + d_hist).x.reshape(-1, 4)
    _, _, st = C.gpu_state(case, implicit=1, newton_rtol=1e-9, gmres_rtol=1e-12, gmres_max_iters=3000)
    st.set_displacement(d_hist)
    st.set_boundary_displacement(bd, dbd)
    stats = st.step()
    u, p = st.get()
    assert _rel(u, ref[:, :3]) <= 1e-6 and _rel(p, ref[:, 3]) <= 1e-6, (_rel(u, ref[:, :3]), _rel(p, ref[:, 3]),
                                                                        stats, st.newton_residuals())
    assert stats["newton_iterations"] >= 1


def test_translating_domain_is_the_fixed_domain_step_plus_v():
    case = _case()
    V = case.mesh.n_nodes
    v = np.array([0.3, -0.2, 0.5])
    shift = np.broadcast_to(v, (V, 3))
    _, _, fixed = C.gpu_state(case, gmres_rtol=1e-12, gmres_max_iters=3000)
    fixed.step()
    uf, pf = fixed.get()
    moving_case = dataclasses.replace(case, u_hist=case.u_hist + v, nodal={k: w + v for k, w in case.nodal.items()})
    _, _, st = C.gpu_state(moving_case, gmres_rtol=1e-12, gmres_max_iters=3000)
    t0, dt = case.t0, case.dt
    st.set_displacement([shift * (t0 - j * dt) for j in range(case.order)])
    bd = np.unique(case.mesh.bfaces.ravel())
    st.set_boundary_displacement(bd, np.broadcast_to(v * (t0 + dt), (bd.size, 3)))
    st.step()
    um, pm = st.get()
    d, _ = st.get_displacement()
    assert np.abs(d - v * (t0 + dt)).max() <= 1e-12
    assert np.abs(um - v - uf).max() <= 1e-8 * np.abs(uf).max()
    assert np.abs(pm - pf).max() <= 1e-8 * np.abs(pf).max()
