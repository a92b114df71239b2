"""GPU tests of the fully implicit formulation (Eq. u_star in its implicit form and the implicit LES
term of Section 2.3, linearised by Newton's method, Section 2.4).

* The analytic Jacobian the CUDA path assembles at an iterate U equals the oracle's Jacobian, the
  sum of central differences of the implicit element residual (which takes u* = u, tau_M(u*),
  tau_C(u*) and r_M(u, p) at U itself), within 1e-6 of each scalar row's largest entry (the
  differences' own error is about 1e-9 relative); the right-hand side J U - R(U) likewise, scaled
  by the row's largest entry times max |U|.  FP64 and double-float assembly, with and without a
  resistive surface, VMS-LES and SUPG-PSPG; in each launch shape (element colours, chunk colours,
  one persistent launch: the chunked kernels sum each row's Newton share over its blocks in a
  final pass per chunk).
* A whole implicit step through lfx_step matches the oracle's implicit_step (Newton with a direct
  solve from the semi-implicit solution) within 1e-6 relative L2, in FP64 and mixed precision; the
  Newton history reaches the tolerance in a few iterations with a first contraction below 1e-2."""
import dataclasses

import numpy as np
import pytest

from tests import cases as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2304_12032_gb300 import build

    build.build()


JAC = {
    "vessel_vms_riis_bdf2": lambda: C.vessel_case(3000, seed=21, order=2, riis=True),
    "vessel_vms_bdf1": lambda: C.vessel_case(3000, seed=21, order=1, riis=False),
    "bifurcation_supg_bdf3": lambda: dataclasses.replace(C.bifurcation_case(4000, seed=1004, order=3, stab=1)),
}


@pytest.mark.parametrize("shape", ["colors", "chunks", "persistent"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("which", list(JAC))
def test_newton_jacobian_matches_finite_differences_of_the_oracle(which, precision, shape):
    import oracle as O

    case = JAC[which]()
    V = case.mesh.n_nodes
    rng = np.random.default_rng(31)
    U = np.concatenate([case.u_hist[0], case.p_hist[0][:, None]], axis=1) + 0.5 * rng.standard_normal((V, 4))
    prob = C.oracle_problem(case)
    J, F = O.implicit_system(case.mesh, prob, list(case.u_hist), case.t0 + case.dt, U.ravel())
    opts = dict(assembly=shape) if precision == "fp64" else dict(precision="mixed", assembly=shape)
    mesh, _, st = C.gpu_state(case, **opts)
    blocks, rhs = st.debug_assemble_newton(U)
    rp, ci = mesh.pattern()
    ref = C.blocks_from_csr(J, rp, ci)
    scale = C.row_scale(J).reshape(-1, 4)
    rows = np.repeat(np.arange(V), np.diff(rp))
    err = np.abs(blocks - ref) / np.maximum(scale[rows][:, :, None], 1e-300)
    assert err.max() <= 1e-6, (which, precision, float(err.max()))
    rref = (J @ U.ravel() - F).reshape(-1, 4)
    rtol = scale * np.abs(U).max() * 20
    rerr = np.abs(rhs - rref) / np.maximum(rtol, 1e-300)
    assert rerr.max() <= 1e-6, (which, precision, float(rerr.max()))


STEP = {
    "vessel_vms_bdf1": lambda: C.vessel_case(3000, seed=21, order=1, riis=False),
    "vessel_vms_riis_bdf2": lambda: C.vessel_case(3000, seed=21, order=2, riis=True),
}


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("which", list(STEP))
def test_implicit_step_matches_oracle(which, precision):
    import oracle as O

    case = STEP[which]()
    prob = C.oracle_problem(case)
    ref = O.implicit_step(case.mesh, prob, list(case.u_hist), list(case.p_hist), case.t0 + case.dt).x.reshape(-1, 4)
    opts = dict(gmres_rtol=1e-12, gmres_max_iters=3000) if precision == "fp64" else \
        dict(precision="mixed", smoother_bf16=1, gmres_rtol=1e-11)
    _, _, st = C.gpu_state(case, implicit=1, newton_rtol=1e-9, **opts)
    stats = st.step()
    u, p = st.get()
    ru = np.linalg.norm(u - ref[:, :3]) / np.linalg.norm(ref[:, :3])
    rp_ = np.linalg.norm(p - ref[:, 3]) / np.linalg.norm(ref[:, 3])
    hist = st.newton_residuals()
    assert ru <= 1e-6 and rp_ <= 1e-6, (which, precision, ru, rp_, stats, hist)
    assert 1 <= stats["newton_iterations"] <= 5 and len(hist) == stats["newton_iterations"] + 1, (stats, hist)
    assert hist[-1] <= 1e-9 and hist[1] <= 1e-2 * hist[0], hist
    # the implicit solution differs from the semi-implicit one by far more than the tolerance
    semi = C.oracle_step(case).x.reshape(-1, 4)
    assert np.linalg.norm(semi[:, :3] - ref[:, :3]) > 1e-5 * np.linalg.norm(ref[:, :3])
