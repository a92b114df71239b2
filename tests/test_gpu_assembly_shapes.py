"""The three launch shapes of the semi-implicit assembly give the oracle's system: per-colour
launches of element colours, compact 32-element chunks reduced in shared memory (one launch per
chunk colour), and the chunks in one persistent cooperative launch whose colours are separated by
bounded grid-wide waits.  FP64 within 1e-12 of each scalar row's largest entry, double-float within
5e-11 (the tolerances of the assembly parity tests); the autotuner times all three and keeps one."""
import numpy as np
import pytest

from tests import cases as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2304_12032_gb300 import build

    build.build()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("shape", ["colors", "chunks", "persistent"])
def test_assembly_shapes_match_oracle(shape, precision):
    case = C.vessel_case(6000, seed=21)
    ost = C.oracle_step(case)
    opts = dict(assembly=shape, gmres_rtol=1e-12, gmres_max_iters=3000)
    if precision == "mixed":
        opts.update(precision="mixed", smoother_bf16=1, gmres_rtol=1e-10)
    mesh, prob, st = C.gpu_state(case, **opts)
    blocks, rhs = st.debug_assemble(apply_bcs=True)
    rp, ci = mesh.pattern()
    ref = C.blocks_from_csr(ost.A, rp, ci)
    scale = C.row_scale(ost.A).reshape(-1, 4)
    rows = np.repeat(np.arange(case.mesh.n_nodes), np.diff(rp))
    tol = (1e-12 if precision == "fp64" else 5e-11) * np.maximum(np.abs(ref), scale[rows][:, :, None])
    assert np.all(np.abs(blocks - ref) <= tol), (shape, precision)
    bref = ost.b.reshape(-1, 4)
    assert np.all(np.abs(rhs - bref) <= (1e-12 if precision == "fp64" else 5e-11) * np.abs(bref).max())
    stats = st.step()
    assert stats["assembly_mode"] == {"colors": 1, "chunks": 2, "persistent": 3}[shape]
    u, p = st.get()
    x = ost.x.reshape(-1, 4)
    assert np.linalg.norm(u - x[:, :3]) <= 1e-6 * np.linalg.norm(x[:, :3])
    assert np.linalg.norm(p - x[:, 3]) <= 1e-6 * np.linalg.norm(x[:, 3])


def test_autotuner_times_every_shape_and_keeps_one():
    case = C.vessel_case(6000, seed=22)
    _, prob, st = C.gpu_state(case, precision="mixed", smoother_bf16=1)
    assert prob.assembly_tuning()[0] == 0            # not tuned before the first assembly
    stats = st.step()
    mode, ms = prob.assembly_tuning()
    assert mode in (1, 2, 3) and stats["assembly_mode"] == mode
    assert set(ms) == {"colors", "chunks", "persistent"} and all(v > 0 for v in ms.values())
    assert ms[("colors", "chunks", "persistent")[mode - 1]] == min(ms.values())
    # a second state of the same problem reuses the choice
    from paper_2304_12032_gb300 import lfx as L

    st2 = L.State(prob, case.u_hist, case.p_hist, case.t0)
    assert st2.step()["assembly_mode"] == mode


def test_persistent_assembly_wait_that_runs_out_returns_timeout():
    """The persistent launch's grid-wide waits are bounded: with the first wait's target made
    unreachable (a count nothing reaches) the CTAs give up after their poll limit and return, the
    call reports LFX_ERR_TIMEOUT, and the context stays usable: the next step reassembles and
    matches a fresh state's step."""
    from paper_2304_12032_gb300 import lfx as L

    case = C.vessel_case(6000, seed=23)
    _, prob, st = C.gpu_state(case, assembly="persistent", gmres_rtol=1e-12, gmres_max_iters=3000)
    assert st.debug_persistent_timeout() == L.LFX_ERR_TIMEOUT
    assert b"gave up" in L.library().lfx_last_error()
    st.step()
    u, p = st.get()
    fresh = L.State(prob, case.u_hist, case.p_hist, case.t0)
    fresh.step()
    u1, p1 = fresh.get()
    assert np.allclose(u, u1, rtol=0, atol=1e-10 * np.abs(u1).max())
    assert np.allclose(p, p1, rtol=0, atol=1e-10 * np.abs(p1).max())
