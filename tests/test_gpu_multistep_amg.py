"""GPU tests of the parts of the step that a single-step, single-level comparison cannot see.

* Several steps in a row against the oracle (Eq. bdf): each oracle step starts from the oracle's
  own previous solutions, so a wrong level order in the history rotation of the CUDA path
  (BDF2, BDF3) shows from the second step on.  FP64 and mixed precision, 1e-6 relative L2 per
  step (the target accuracy).
* The Schur block's multilevel AMG (Section 2.4 names AMG among the block approximations of
  aSIMPLE) with a hierarchy of at least three levels: the device hierarchy satisfies the Galerkin
  relation A_{l+1} = P_l^T A_l P_l, one device V-cycle over levels 1..L-1 equals a numpy V-cycle
  over the downloaded operators (Chebyshev smoothing by Saad's Chebyshev acceleration with Jacobi
  scaling, lambda_max = the Gershgorin bound, coarsest level solved directly), and the whole solve
  and the mixed step still match the oracle.
* Failure paths through the C ABI: a solve that hits its cap returns LFX_ERR_NOT_CONVERGED with
  the state advanced; a non-finite history gives LFX_ERR_NONFINITE; a request larger than the
  serving budget gives LFX_ERR_BUDGET; an allocator that fails the k-th allocation gives
  LFX_ERR_OOM with every earlier allocation of the call released."""
import dataclasses

import numpy as np
import pytest

from tests import cases as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2304_12032_gb300 import build

    build.build()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


MULTI = {
    "vessel_vms_riis_bdf2": lambda: C.vessel_case(6000, seed=21, order=2),
    "bifurcation_supg_bdf3": lambda: C.bifurcation_case(8000, seed=1003, order=3),
}


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("which", list(MULTI))
def test_three_steps_match_the_oracle(which, precision):
    case = MULTI[which]()
    opts = dict(gmres_rtol=1e-12, gmres_max_iters=3000) if precision == "fp64" else \
        dict(precision="mixed", smoother_bf16=1, gmres_rtol=1e-10)
    _, _, st = C.gpu_state(case, **opts)
    cur = case
    for k in range(3):
        ref = C.oracle_step(cur).x.reshape(-1, 4)
        stats = st.step()
        u, p = st.get()
        ru, rp_ = _rel(u, ref[:, :3]), _rel(p, ref[:, 3])
        assert ru <= 1e-6 and rp_ <= 1e-6, (which, precision, k, ru, rp_, stats)
        assert stats["t"] == pytest.approx(cur.t0 + cur.dt)
        # the oracle's next step starts from its own solution: levels shift by one
        uh = np.concatenate([ref[None, :, :3], cur.u_hist[:-1]], axis=0)
        ph = np.concatenate([ref[None, :, 3], cur.p_hist[:-1]], axis=0)
        cur = dataclasses.replace(cur, u_hist=uh, p_hist=ph, t0=cur.t0 + cur.dt)


# ---------------------------------------------------------------------------- multilevel AMG
def _cheb(A, dinv, b, x0, lmax, ratio, steps):
    """Chebyshev acceleration (Saad, Iterative Methods, Alg. 12.1) of the Jacobi-scaled iteration
    for A x = b on the interval [lmax/ratio, lmax], from x0, `steps` steps."""
    lmin = lmax / ratio
    theta, delta = 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)
    sigma = theta / delta
    rho = 1.0 / sigma
    r = dinv * (b - A @ x0)
    d = r / theta
    x = x0 + d
    for _ in range(1, steps):
        rho_new = 1.0 / (2.0 * sigma - rho)
        r = r - dinv * (A @ d)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * r
        x = x + d
        rho = rho_new
    return x


def _gershgorin(A):
    d = A.diagonal()
    dinv = np.where(d != 0.0, 1.0 / np.where(d != 0.0, d, 1.0), 0.0)
    rows = np.asarray(abs(A).sum(axis=1)).ravel()
    return dinv, float(np.max(np.abs(dinv) * rows))


def _vcycle(ops, l, b, ratio, steps, alpha):
    A, P = ops[l]["A"], ops[l]["P"]
    if P is None:
        return np.linalg.solve(A.toarray(), b)
    dinv, lam = _gershgorin(A)
    x = _cheb(A, dinv, b, np.zeros_like(b), lam, ratio, steps)
    xc = _vcycle(ops, l + 1, P.T @ (b - A @ x), ratio, steps, alpha)
    x = x + alpha * (P @ xc)
    return _cheb(A, dinv, b, x, lam, ratio, steps)


AMG = {
    "vessel_vms_riis": lambda: C.vessel_case(6000, seed=21),
    "stenosis_womersley_riis": lambda: C.stenosis_case(8000, seed=3),
}


@pytest.mark.parametrize("s_steps", [1, 2])
@pytest.mark.parametrize("which", list(AMG))
def test_multilevel_schur_amg(which, s_steps):
    case = AMG[which]()
    ost = C.oracle_step(case)
    _, _, st = C.gpu_state(case, gmres_rtol=1e-12, gmres_max_iters=3000, amg_coarse_size=30, s_steps=s_steps)
    st.debug_assemble(apply_bcs=True)
    x, stats = st.debug_solve()
    levels = st.amg_levels()
    assert len(levels) >= 3, levels
    assert _rel(x, ost.x.reshape(-1, 4)) <= 1e-6, (which, stats)
    assert stats["iterations"] <= 120, (which, stats, levels)
    # the device hierarchy: shapes, Galerkin coarse operators, Chebyshev bounds
    L = len(levels)
    ops = [st.debug_amg_level(l) for l in range(L)]
    assert ops[0]["A"] is None and ops[0]["P"].shape == (levels[0][0], levels[1][0])
    for l in range(1, L):
        assert ops[l]["n"] == levels[l][0]
    for l in range(1, L - 1):
        A, P = ops[l]["A"], ops[l]["P"]
        assert A.nnz == levels[l][1] and P.shape == (levels[l][0], levels[l + 1][0])
        assert ops[l]["lam"] == pytest.approx(_gershgorin(A)[1], rel=1e-12)
        # every fine row is covered by the prolongator and every coarse unknown is used
        assert (np.diff(P.indptr) > 0).all() and np.unique(P.indices).size == P.shape[1]
        Ac = (P.T @ A @ P).tocsr()
        if ops[l + 1]["A"] is not None:
            D = (Ac - ops[l + 1]["A"]).toarray()
            assert np.abs(D).max() <= 1e-11 * abs(Ac).max()
        else:
            ops[l + 1]["A"] = Ac            # the coarsest operator lives on the device only as its inverse
    # one device V-cycle over levels 1..L-1 against the numpy V-cycle
    b1 = np.random.default_rng(7).standard_normal(levels[1][0])
    x1 = st.debug_amg_vcycle(b1)
    ref = _vcycle(ops, 1, b1, 30.0, s_steps, 1.0)
    assert _rel(x1, ref) <= 1e-10, (which, s_steps, _rel(x1, ref))


def test_mixed_step_with_multilevel_amg_matches_oracle():
    case = AMG["stenosis_womersley_riis"]()
    ost = C.oracle_step(case)
    _, _, st = C.gpu_state(case, precision="mixed", smoother_bf16=1, gmres_rtol=1e-10, amg_coarse_size=30)
    stats = st.step()
    assert len(st.amg_levels()) >= 3
    u, p = st.get()
    ref = ost.x.reshape(-1, 4)
    assert _rel(u, ref[:, :3]) <= 1e-6 and _rel(p, ref[:, 3]) <= 1e-6, stats


# ----------------------------------------------------------------------------- failure paths
def test_iteration_cap_returns_not_converged_and_advances_the_state():
    from paper_2304_12032_gb300 import lfx as L

    case = C.vessel_case(3000, seed=26)
    _, _, st = C.gpu_state(case, gmres_max_iters=1, gmres_restart=8)
    u0, _ = st.get()
    stats = st.step(allow_not_converged=True)
    assert stats["status"] == L.LFX_ERR_NOT_CONVERGED and not stats["converged"]
    assert stats["t"] == pytest.approx(case.t0 + case.dt)
    u1, p1 = st.get()
    assert np.isfinite(u1).all() and np.linalg.norm(u1 - u0) > 0      # the best iterate became level 0
    with pytest.raises(L.LfxError) as e:
        st.step()
    assert e.value.status == L.LFX_ERR_NOT_CONVERGED


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_nonfinite_history_returns_nonfinite(precision):
    from paper_2304_12032_gb300 import lfx as L

    case = C.vessel_case(3000, seed=27)
    uh = case.u_hist.copy()
    uh[0, 5, 1] = np.nan
    case = dataclasses.replace(case, u_hist=uh)
    opts = {} if precision == "fp64" else dict(precision="mixed")
    _, _, st = C.gpu_state(case, **opts)
    with pytest.raises(L.LfxError) as e:
        st.step()
    assert e.value.status == L.LFX_ERR_NONFINITE


def test_request_above_the_budget_is_refused():
    from paper_2304_12032_gb300 import lfx as L

    case = C.vessel_case(3000, seed=28)
    _, prob, _ = C.gpu_state(case)
    need = L.problem_state_bytes(prob)
    srv = L.Server(need // 2, n_workers=1)
    try:
        with pytest.raises(L.LfxError) as e:
            srv.submit(prob, case.u_hist, case.p_hist, case.t0, 1)
        assert e.value.status == L.LFX_ERR_BUDGET
    finally:
        srv.close()


def test_failing_allocator_gives_oom_and_releases_everything():
    import gc

    import torch
    from paper_2304_12032_gb300 import lfx as L

    case = C.vessel_case(3000, seed=29)
    live, calls = {}, {"n": 0, "fail_at": -1}
    dev = torch.cuda.current_device()

    def _alloc(nbytes, ctx):
        calls["n"] += 1
        if calls["n"] == calls["fail_at"]:
            return None
        p = torch.cuda.caching_allocator_alloc(int(nbytes), dev)
        live[p] = nbytes
        return p

    def _free(ptr, ctx):
        if ptr in live:
            del live[ptr]
            torch.cuda.caching_allocator_delete(ptr)

    fa, ff = L.ALLOC_FN(_alloc), L.FREE_FN(_free)
    lib = L.library()
    L._check(lib.lfx_set_allocator(fa, ff, None))
    try:
        mesh, prob, st = C.gpu_state(case)
        del st
        before = dict(live)
        # a state needs many allocations: fail the 1st, a middle one and a late one
        for k in (1, 7, 20):
            calls["n"], calls["fail_at"] = 0, k
            with pytest.raises(L.LfxError) as e:
                L.State(prob, case.u_hist, case.p_hist, case.t0)
            assert e.value.status == L.LFX_ERR_OOM, k
            assert live.keys() == before.keys(), (k, len(live), len(before))
        calls["fail_at"] = -1
        st = L.State(prob, case.u_hist, case.p_hist, case.t0)
        st.step()
        del st
        assert live.keys() == before.keys()
        # the mesh and problem go back through the same allocator (the hook stays alive until then;
        # the exception info holds the failed constructor's frame, which holds the problem)
        del prob, mesh, e
        gc.collect()
        assert not live, len(live)
    finally:
        L._check(lib.lfx_set_allocator(L.ALLOC_FN(), L.FREE_FN(), None))
        torch.cuda.synchronize()
