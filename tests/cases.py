"""Shared test workloads: each case is plain data (a synthetic mesh, physics, boundary
conditions, seeded history fields) turned into either the oracle's problem or the GPU
library's handles.  Nothing here computes any part of the method."""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

from synthetic import (beltrami_p, beltrami_u, bifurcation, cube_kuhn, cylinder, stenosis, zero_net_flux)


@dataclasses.dataclass
class Case:
    mesh: object
    rho: float
    mu: float
    dt: float
    order: int
    bcs: list                  # list of dicts: tag, kind, profile, time, p, a, b, theta, radius
    riis: list                 # list of dicts: resistance, eps, center, normal, radius
    u_hist: np.ndarray         # [order, V, 3]
    p_hist: np.ndarray         # [order, V]
    t0: float = 0.0
    stab: int = 2
    diffusion: int = 0
    f: tuple = (0.0, 0.0, 0.0)
    pin_node: int = -1
    pin_value: float = 0.0
    nodal: Optional[dict] = None     # tag -> [V,3] values for NODAL conditions


def beltrami_case(n=4, seed=11, order=1, dt=1e-3, stab=2):
    m = cube_kuhn(n, seed=seed)
    X = m.nodes
    uh = np.stack([beltrami_u(X, -k * dt) for k in range(order)])
    ph = np.stack([beltrami_p(X, -k * dt) for k in range(order)])
    bd = np.unique(m.bfaces.ravel())
    ue = beltrami_u(X, dt)
    ue[bd] = zero_net_flux(X, m.bfaces, bd, ue[bd])
    bcs = [dict(tag=t, kind="nodal") for t in range(1, 7)]
    return Case(m, 1.0, 1.0, dt, order, bcs, [], uh, ph, 0.0, stab, 0, (0.0, 0.0, 0.0), 0,
                float(beltrami_p(X[:1], dt)[0]), {t: ue for t in range(1, 7)})


def vessel_case(n_tets=6000, seed=21, order=2, stab=2, diffusion=0, riis=True, neumann_h=3.0, backflow=0.0,
                resistance=0.0):
    """Cylinder R=1, L=3 with a parabolic pulsatile inlet, a Neumann outlet with nonzero h
    (and inertial backflow stabilisation when backflow > 0: the random history flows back in
    near the outlet rim), a disk-shaped resistive surface at mid-length and random seeded
    history fields.  With resistance > 0 the outlet is a resistance condition instead, with
    p_0 = neumann_h and C_R = resistance."""
    R, L = 1.0, 3.0
    m = cylinder(R, L, n_tets=n_tets, seed=seed)
    rng = np.random.default_rng(seed)
    V = m.n_nodes
    base = np.zeros((V, 3))
    base[:, 2] = 20.0 * np.clip(1 - (m.nodes[:, 0] ** 2 + m.nodes[:, 1] ** 2) / R ** 2, 0, None)
    uh = np.stack([base + 2.0 * rng.standard_normal((V, 3)) for _ in range(order)])
    ph = np.stack([4 * 0.035 * 20 * (L - m.nodes[:, 2]) + 0.5 * rng.standard_normal(V) for _ in range(order)])
    bcs = [dict(tag=0, kind="noslip"),
           dict(tag=1, kind="dirichlet", profile="parabolic", time="pulsatile", p=(5.0, 30.0, 0.8),
                radius=R),
           dict(tag=2, kind="neumann", time="constant", p=(neumann_h,), beta=backflow)]
    if resistance > 0.0:
        bcs[2] = dict(tag=2, kind="resistance", time="constant", p=(neumann_h,), resistance=resistance)
    rs = [dict(resistance=1e4, eps=0.25, center=(0.0, 0.0, L / 2), normal=(0.0, 0.0, 1.0), radius=0.6)] if riis else []
    return Case(m, 1.06, 0.035, 1e-3, order, bcs, rs, uh, ph, 0.1, stab, diffusion, (0.0, 0.0, 0.0))


def stenosis_case(n_tets=8000, seed=3, order=2, harmonics=3):
    """The stenosis-with-valve workload at small size: cosine stenosis (75 % area reduction), Womersley inlet
    with a Fourier flow rate (period 1 s), a disk resistive surface downstream, VMS-LES."""
    R, L = 1.0, 10.0
    m = stenosis(R, L, n_tets=n_tets, seed=seed)
    rng = np.random.default_rng(seed)
    V = m.n_nodes
    uh = np.stack([rng.standard_normal((V, 3)) for _ in range(order)])
    ph = np.stack([rng.standard_normal(V) for _ in range(order)])
    qpk = math.pi * R * R * 33.0
    a = [0.5 * qpk] + [(-0.5 * qpk if k == 1 else 0.1 * qpk / k) for k in range(1, harmonics + 1)]
    b = [0.0] + [0.05 * qpk * k for k in range(1, harmonics + 1)]
    bcs = [dict(tag=0, kind="noslip"),
           dict(tag=1, kind="dirichlet", profile="womersley", time="fourier", p=(1.0,), a=a, b=b, radius=R),
           dict(tag=2, kind="neumann", time="constant", p=(0.0,))]
    rs = [dict(resistance=1e4, eps=0.3, center=(0.0, 0.0, 5.0), normal=(0.0, 0.0, 1.0), radius=0.5)]
    return Case(m, 1.06, 0.035, 5e-4, order, bcs, rs, uh, ph, 0.37, 2, 0, (0.0, 0.0, 0.0))


def bifurcation_case(n_tets=8000, seed=1003, order=3, stab=1):
    m = bifurcation(n_tets=n_tets, seed=seed, angle_deg=55.0)
    rng = np.random.default_rng(seed)
    V = m.n_nodes
    uh = np.stack([rng.standard_normal((V, 3)) * 5.0 for _ in range(order)])
    ph = np.stack([rng.standard_normal(V) for _ in range(order)])
    bcs = [dict(tag=0, kind="noslip"),
           dict(tag=1, kind="dirichlet", profile="uniform", time="ramp", p=(0.0, 15.0, 0.0, 0.05)),
           dict(tag=2, kind="neumann", time="constant", p=(0.0,)),
           dict(tag=3, kind="neumann", time="constant", p=(1.5,))]
    return Case(m, 1.06, 0.035, 1e-3, order, bcs, [], uh, ph, 0.01, stab, 1, (0.1, -0.2, 0.3))


# ------------------------------------------------------------------------------- oracle side
def oracle_problem(case: Case):
    import oracle as O

    prm = O.Params(rho=case.rho, mu=case.mu, dt=case.dt, bdf_order=case.order, stab=case.stab,
                   diffusion=case.diffusion, f=case.f)
    bcs = []
    for b in case.bcs:
        kind = b["kind"]
        time = b.get("time", "constant")
        p = b.get("p", (0.0,))
        if time == "constant":
            tp = {"value": p[0]}
        elif time == "pulsatile":
            tp = {"gmin": p[0], "gmax": p[1], "period": p[2]}
        elif time == "ramp":
            tp = {"g0": p[0], "g1": p[1], "t0": p[2], "tL": p[3]}
        else:
            tp = {"period": p[0], "a": list(b.get("a", [0.0])), "b": list(b.get("b", [0.0]))}
        bcs.append(O.BC(tag=b["tag"], kind=kind, time=time, tparams=tp, space=b.get("profile", "uniform"),
                        radius=b.get("radius", 1.0), theta=b.get("theta", 1.0), beta=b.get("beta", 0.0),
                        resistance=b.get("resistance", 0.0)))
    riis = [O.RIIS(r["resistance"], r["eps"], O.disk_sdf(case.mesh.nodes, r["center"], r["normal"], r["radius"]))
            for r in case.riis]
    return O.Problem(prm, bcs, riis, pin_node=case.pin_node)


def oracle_step(case: Case, solver=None):
    import oracle as O

    prob = oracle_problem(case)
    return O.step(case.mesh, prob, list(case.u_hist), list(case.p_hist), case.t0 + case.dt,
                  nodal=case.nodal, pin_value=case.pin_value, solver=solver)


# ------------------------------------------------------------------------------- GPU side
def gpu_state(case: Case, **opts):
    from paper_2304_12032_gb300 import lfx as L

    mesh = L.Mesh.from_synthetic(case.mesh)
    o = L.default_options(stab=case.stab, diffusion=case.diffusion, f=case.f,
                          pin_pressure_node=case.pin_node, **opts)
    bcs = [L.BC(tag=b["tag"], kind=b["kind"], profile=b.get("profile", "uniform"), time=b.get("time", "constant"),
                p=b.get("p", (0.0,)), a=b.get("a", ()), b=b.get("b", ()), theta=b.get("theta", 1.0),
                radius=b.get("radius", 1.0), beta=b.get("beta", 0.0),
                resistance=b.get("resistance", 0.0)) for b in case.bcs]
    riis = [L.RIIS(r["resistance"], r["eps"], r["center"], r["normal"], r["radius"]) for r in case.riis]
    prob = L.Problem(mesh, case.rho, case.mu, case.dt, case.order, bcs, riis, o)
    st = L.State(prob, case.u_hist, case.p_hist, case.t0)
    if case.nodal:
        for tag, vals in case.nodal.items():
            st.set_dirichlet_nodal(tag, vals)
    if case.pin_node >= 0:
        st.set_pressure_pin(case.pin_value)
    return mesh, prob, st


def blocks_from_csr(A, rp, ci):
    """Blocks [nnzb,4,4] of a scalar CSR matrix at the block pattern (rp, ci)."""
    nnzb = ci.size
    rows = np.repeat(np.arange(rp.size - 1), np.diff(rp))
    R = (4 * rows[:, None, None] + np.arange(4)[None, :, None]).repeat(4, axis=2)
    C = (4 * ci[:, None, None] + np.arange(4)[None, None, :]).repeat(4, axis=1)
    vals = np.asarray(A.tocsr()[R.ravel(), C.ravel()]).ravel()
    return vals.reshape(nnzb, 4, 4)


def row_scale(A):
    """max |A_ij| over each scalar row."""
    A = A.tocsr()
    a = np.abs(A.data)
    out = np.zeros(A.shape[0])
    nz = np.diff(A.indptr) > 0
    out[nz] = np.maximum.reduceat(a, A.indptr[:-1][nz])
    return out
