"""Batching (several meshes assembled and solved as one disconnected system) and serving
(continuous batching by the native request loop): each simulation's result must equal its solo
run within the solution tolerance (1e-6 relative L2), and the solo run must match the oracle."""
import math
import time

import numpy as np
import pytest

from synthetic import batch, bifurcation, cylinder
from tests import cases as C

RHO, MU, DT = 1.06, 0.035, 1e-3


def _members():
    return [cylinder(1.0, 3.0, n_tets=4000, seed=31), bifurcation(n_tets=6000, seed=1001, angle_deg=40.0),
            cylinder(0.6, 2.0, n_tets=3000, seed=33)]


def _bcs(i, m, stride=10):
    if "bifurcation" in m.name:
        return [dict(tag=0 + stride * i, kind="noslip"),
                dict(tag=1 + stride * i, kind="dirichlet", profile="uniform", time="constant", p=(8.0,)),
                dict(tag=2 + stride * i, kind="neumann", time="constant", p=(0.0,)),
                dict(tag=3 + stride * i, kind="neumann", time="constant", p=(0.0,))]
    R = m.meta["radius"]
    Q = 15.0 * math.pi * R * R / 2
    return [dict(tag=0 + stride * i, kind="noslip"),
            dict(tag=1 + stride * i, kind="dirichlet", profile="parabolic", time="constant", p=(Q,), radius=R),
            dict(tag=2 + stride * i, kind="neumann", time="constant", p=(0.0,))]


def _hist(m, seed):
    rng = np.random.default_rng(seed)
    V = m.n_nodes
    return np.stack([rng.standard_normal((V, 3)) for _ in range(2)]), np.stack([rng.standard_normal(V) for _ in range(2)])


def test_batch_components_detected_on_cpu():
    from paper_2304_12032_gb300 import build as B

    B.build()
    from paper_2304_12032_gb300 import lfx as L

    ms = _members()
    u = batch(ms)
    info = L.Mesh.from_synthetic(u).info()
    assert info["n_components"] == 3
    rp, ci = L.Mesh.from_synthetic(u).pattern()
    offs = u.meta["node_offsets"]
    comp = np.searchsorted(offs, np.arange(u.n_nodes), side="right") - 1
    rows = np.repeat(np.arange(u.n_nodes), np.diff(rp))
    assert np.array_equal(comp[rows], comp[ci])          # no coupling between members


# (precision, one Arnoldi process per member or the union as one Krylov system, Schur smoother)
BATCH_MODES = {"fp64-segmented": dict(batch_segmented=1), "fp64-union": dict(batch_segmented=0),
               "mixed-segmented": dict(batch_segmented=1, precision="mixed", smoother_bf16=1),
               "fp64-segmented-chebyshev": dict(batch_segmented=1, s_smoother="chebyshev")}


@pytest.mark.gpu
@pytest.mark.parametrize("mode", list(BATCH_MODES))
def test_batched_step_equals_solo_runs(mode):
    opts = dict(BATCH_MODES[mode], gmres_rtol=1e-10)
    ms = _members()
    u = batch(ms)
    offs = u.meta["node_offsets"]
    hs = [_hist(m, 100 + i) for i, m in enumerate(ms)]
    uh = np.concatenate([h[0] for h in hs], axis=1)
    ph = np.concatenate([h[1] for h in hs], axis=1)
    bcs = sum((_bcs(i, m) for i, m in enumerate(ms)), [])
    case = C.Case(u, RHO, MU, DT, 2, bcs, [], uh, ph, 0.0)
    _, _, st = C.gpu_state(case, **opts)
    sb = st.step()
    ub, pb = st.get()
    solo_its = []
    for i, m in enumerate(ms):
        solo = C.Case(m, RHO, MU, DT, 2, _bcs(0, m), [], hs[i][0], hs[i][1], 0.0)
        _, _, s1 = C.gpu_state(solo, **opts)
        solo_its.append(s1.step()["iterations"])
        u1, p1 = s1.get()
        sl = slice(offs[i], offs[i + 1])
        ru = np.linalg.norm(ub[sl] - u1) / np.linalg.norm(u1)
        rp = np.linalg.norm(pb[sl] - p1) / np.linalg.norm(p1)
        assert ru <= 1e-6 and rp <= 1e-6, (i, ru, rp)
        if i == 0:
            ref = C.oracle_step(solo).x.reshape(-1, 4)
            assert np.linalg.norm(u1 - ref[:, :3]) / np.linalg.norm(ref[:, :3]) <= 1e-6
    if opts["batch_segmented"] and opts.get("s_smoother") == "chebyshev":
        # with the same preconditioner on every member, each member takes about the steps it takes
        # alone (the Chebyshev eigenvalue bounds are the union's, hence the slack); the union as one
        # Krylov system takes about twice the largest count here.  (With the Schur AMG the union's
        # hierarchy is deeper than a small member's, whose coarse level is S itself.)
        assert sb["iterations"] <= 1.25 * max(solo_its) + 4, (sb["iterations"], solo_its)


@pytest.mark.gpu
def test_server_admits_by_budget_and_results_match_solo():
    from paper_2304_12032_gb300 import lfx as L

    ms = _members()
    cases = [C.Case(m, RHO, MU, DT, 2, _bcs(0, m), [], *_hist(m, 200 + i), 0.0) for i, m in enumerate(ms)]
    handles = [C.gpu_state(c, gmres_rtol=1e-10) for c in cases]
    need = [L.problem_state_bytes(h[1]) for h in handles]
    # room for about two simulations at a time: the third must wait for memory
    srv = L.Server(int(sorted(need)[-1] + sorted(need)[-2] + 1), n_workers=2)
    tickets = [srv.submit(h[1], c.u_hist, c.p_hist, c.t0, 3) for c, h in zip(cases, handles)]
    saw_wait = srv.stats()["waiting"] > 0
    t0 = time.time()
    while not all(srv.poll(t)[0] for t in tickets):
        saw_wait |= srv.stats()["waiting"] > 0
        assert time.time() - t0 < 300
        time.sleep(0.01)
    stats = srv.stats()
    assert saw_wait and stats["max_active"] <= 2
    assert len(stats["latency_ms"]) == 9
    for c, h, t in zip(cases, handles, tickets):
        u, p = srv.result(t)
        st = h[2]
        for _ in range(3):
            st.step()
        u1, p1 = st.get()
        # independent states: same kernels, same reductions -> identical results
        assert np.allclose(u, u1, rtol=0, atol=1e-12 * np.abs(u1).max())
        assert np.allclose(p, p1, rtol=0, atol=1e-12 * np.abs(p1).max())
    srv.close()


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_step_of_independent_states_equals_solo_steps(precision):
    """lfx_batch_step: independent states on their own streams stepped concurrently (one host
    thread each) give exactly their solo results (no reduction is shared between states)."""
    import torch

    from paper_2304_12032_gb300 import build as B

    B.build()
    from paper_2304_12032_gb300 import lfx as L

    extra = dict(precision="mixed", smoother_bf16=1) if precision == "mixed" else {}
    ms = _members()
    probs, hists = [], []
    for i, m in enumerate(ms):
        mesh = L.Mesh.from_synthetic(m)
        bcs = [L.BC(tag=b["tag"], kind=b["kind"], profile=b.get("profile", "uniform"), time=b.get("time", "constant"),
                    p=b.get("p", (0.0,)), radius=b.get("radius", 1.0)) for b in _bcs(0, m, 0)]
        probs.append(L.Problem(mesh, RHO, MU, DT, 2, bcs, [], L.default_options(gmres_rtol=1e-10, **extra)))
        hists.append(_hist(m, 50 + i))
    solo = []
    for p, (uh, ph) in zip(probs, hists):
        st = L.State(p, uh, ph, 0.0)
        st.step()
        st.step()
        solo.append(st.get())
    streams = [torch.cuda.Stream() for _ in probs]
    states = [L.State(p, uh, ph, 0.0, stream=s) for p, (uh, ph), s in zip(probs, hists, streams)]
    for _ in range(2):
        stats = L.batch_step(states)
        assert len(stats) == len(states) and all(s["converged"] for s in stats)
    for st, (us, ps) in zip(states, solo):
        u, p = st.get()
        assert np.array_equal(u, us) and np.array_equal(p, ps)
