"""The staged velocity smoothing pass of the BF16 aSIMPLE smoother (Section 2.4's velocity block,
smoothed by Chebyshev steps on F): persistent CTAs copy whole row tiles of F sub-block records
into shared memory with bulk asynchronous copies on an mbarrier, double-buffered, and each lane
then takes its row's blocks in the order of the plain pass.

* A mixed step with the staged pass against the oracle's step (1e-6, the mixed-step tolerance),
  and against the same step with the plain pass (the same sums in the same order: equal results
  up to the rounding of the solver's own reductions, 1e-9).
* A mesh with more tiles than resident CTAs (each CTA walks several tiles, so that both buffers
  are refilled) over three steps: staged and plain agree step by step, with the same Krylov
  iteration counts, and both stay within 1e-6 of the FP64 GPU step.
* The failure path: with every wait for a staged tile given no polls, one preconditioner
  application returns LFX_ERR_TIMEOUT, and the state's next step still equals a fresh state's."""
import numpy as np
import pytest

from tests import cases as C

pytestmark = pytest.mark.gpu

MIXED = dict(precision="mixed", smoother_bf16=1, gmres_rtol=1e-10)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2304_12032_gb300 import build

    build.build()


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_staged_pass_matches_oracle_and_plain_pass():
    case = C.vessel_case(6000, seed=23)
    ost = C.oracle_step(case)
    outs = {}
    for staged in (1, 0):
        _, _, st = C.gpu_state(case, staged_f=staged, **MIXED)
        stats = st.step()
        assert stats["converged"]
        outs[staged] = st.get()
    u, p = outs[1]
    xref = ost.x.reshape(-1, 4)
    assert _rel(u, xref[:, :3]) <= 1e-6
    assert _rel(p, xref[:, 3]) <= 1e-6
    assert _rel(u, outs[0][0]) <= 1e-9
    assert _rel(p, outs[0][1]) <= 1e-9


def test_staged_pass_with_several_tiles_per_cta():
    case = C.vessel_case(400000, seed=5, riis=False)
    V = case.mesh.n_nodes
    assert V > 152 * 8 * 32      # more 32-row tiles than the staged kernel's resident CTAs
    states = {}
    for key, opts in (("staged", dict(staged_f=1, **MIXED)), ("plain", dict(staged_f=0, **MIXED)),
                      ("fp64", dict(gmres_rtol=1e-10))):
        states[key] = C.gpu_state(case, **opts)[2]
    for k in range(3):
        its = {key: st.step()["iterations"] for key, st in states.items()}
        assert its["staged"] == its["plain"], (k, its)
        sol = {key: st.get() for key, st in states.items()}
        for i in range(2):
            assert _rel(sol["staged"][i], sol["plain"][i]) <= 1e-9, (k, i)
            assert _rel(sol["staged"][i], sol["fp64"][i]) <= 1e-6, (k, i)


def test_staged_wait_that_runs_out_returns_timeout():
    from paper_2304_12032_gb300 import lfx as L

    case = C.vessel_case(6000, seed=29)
    _, prob, st = C.gpu_state(case, **MIXED)
    assert st.debug_staged_timeout() == L.LFX_ERR_TIMEOUT
    assert b"gave up" in L.library().lfx_last_error()
    st.step()
    u, p = st.get()
    fresh = L.State(prob, case.u_hist, case.p_hist, case.t0)
    fresh.step()
    u1, p1 = fresh.get()
    assert np.allclose(u, u1, rtol=0, atol=1e-10 * np.abs(u1).max())
    assert np.allclose(p, p1, rtol=0, atol=1e-10 * np.abs(p1).max())
