"""The host set-up of the Schur AMG hierarchy (Section 2.4 lists AMG among the approximations of the
aSIMPLE blocks), run on the host alone through lfx_debug_amg_host, without a GPU.

The input is the oracle's assembled FP64 system of a vessel step, as 4x4 blocks on the mesh pattern.
The checks use numpy/scipy, independent of the library's set-up code:
* level 0 is S = C - D diag(F)^-1 G (entrywise, to 1e-12 of |C| + |D| |diag(F)^-1| |G|);
* the finest prolongator has the smoothed-aggregation form P = (I - w D^-1 S) P_tent.  Here P_tent
  maps each node to one aggregate, and every aggregate is connected in the mesh node graph.
  w = 4 / (3 lam), with lam an estimate of lambda_max(D^-1 S) from a power iteration: it lies
  within [0.75, 1.1] of the exact value, and the damped Jacobi step is stable on every mode
  (w lambda_max < 2);
* every coarse operator is the Galerkin product P^T A P (to 1e-12 of |P|^T |A| |P|);
* each level's Chebyshev bound is the Gershgorin bound max_i |a_ii|^-1 sum_k |a_ik|;
* the coarsest level is below amg_coarse_size and the one above it is not; its dense inverse
  inverts it;
* two set-ups give the same bits (the host threads split rows, not sums).
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

from tests import cases as C


@pytest.fixture(scope="module")
def L():
    from paper_2304_12032_gb300 import build as B

    B.build()
    from paper_2304_12032_gb300 import lfx

    lfx.library()
    return lfx


@pytest.fixture(scope="module")
def system(L):
    case = C.vessel_case(6000, seed=21)
    ost = C.oracle_step(case)
    mesh = L.Mesh.from_synthetic(case.mesh)
    rp, ci = mesh.pattern()
    rows = np.repeat(np.arange(rp.size - 1), np.diff(rp))
    dg = np.flatnonzero(ci == rows).astype(np.int32)
    blocks = C.blocks_from_csr(ost.A, rp, ci)
    return rp.astype(np.int32), ci, dg, blocks, ost.A.tocsr()


COARSE = 50


@pytest.fixture(scope="module")
def levels(L, system):
    rp, ci, dg, blocks, _ = system
    return L.debug_amg_host(rp, ci, dg, blocks, L.default_options(amg_coarse_size=COARSE))


def _schur_parts(K):
    V = K.shape[0] // 4
    u = (4 * np.arange(V)[:, None] + np.arange(3)[None, :]).ravel()
    p = 4 * np.arange(V) + 3
    F, G, D, Cp = K[u][:, u], K[u][:, p], K[p][:, u], K[p][:, p]
    dF = F.diagonal()
    inv = np.where(dF != 0.0, 1.0 / np.where(dF != 0.0, dF, 1.0), 0.0)
    return Cp, D, sp.diags(inv), G


def test_level_zero_is_the_explicit_schur_complement(levels, system):
    Cp, D, Dinv, G = _schur_parts(system[4])
    ref = (Cp - D @ Dinv @ G).toarray()
    bound = (abs(Cp) + abs(D) @ abs(Dinv) @ abs(G)).toarray()
    S = levels[0]["A"].toarray()
    assert np.all(np.abs(S - ref) <= 1e-12 * bound + 1e-300)


def test_hierarchy_shape(levels):
    n = [lv["n"] for lv in levels]
    assert len(n) >= 3
    assert all(a > b for a, b in zip(n, n[1:]))
    assert n[-1] <= COARSE < n[-2]
    for lv, nxt in zip(levels, levels[1:]):
        P = lv["P"].tocsc()
        assert P.shape == (lv["n"], nxt["n"])
        assert np.all(np.diff(P.indptr) > 0)            # every aggregate holds at least one node


def test_finest_prolongator_is_smoothed_aggregation(levels, system):
    S, P = levels[0]["A"].tocsr(), levels[0]["P"].tocsr()
    V = S.shape[0]
    agg = np.asarray(P.argmax(axis=1)).ravel()
    Pt = sp.csr_matrix((np.ones(V), agg, np.arange(V + 1)), shape=P.shape)
    M = sp.diags(1.0 / S.diagonal()) @ S @ Pt
    X = Pt - P
    w = X.multiply(M).sum() / M.multiply(M).sum()
    assert w > 0.0
    assert abs(X - w * M).max() <= 1e-13 * abs(P).max()
    # w = 4 / (3 lam) with lam an estimate of lambda_max(D^-1 S) (1.1 x 15 power-iteration steps):
    # near the exact value, and the damped Jacobi step stable on every mode (w lambda_max < 2)
    lam_used = 4.0 / (3.0 * w)
    d = S.diagonal()
    lam_exact = np.max(np.abs(np.linalg.eigvals((S.toarray().T / d).T)))
    assert 0.75 * lam_exact <= lam_used <= 1.1 * lam_exact
    assert w * lam_exact < 2.0
    # every aggregate is connected in the mesh node graph
    rp, ci = system[0], system[1]
    graph = sp.csr_matrix((np.ones(ci.size), ci, rp), shape=(V, V))
    for a in range(P.shape[1]):
        members = np.flatnonzero(agg == a)
        k, _ = csg.connected_components(graph[members][:, members], directed=False)
        assert k == 1, a


def test_coarse_operators_are_galerkin_products(levels):
    for lv, nxt in zip(levels, levels[1:]):
        A, P = lv["A"], lv["P"]
        ref = (P.T @ A @ P).toarray()
        bound = (abs(P).T @ abs(A) @ abs(P)).toarray()
        assert np.all(np.abs(nxt["A"].toarray() - ref) <= 1e-12 * bound.max())


def test_chebyshev_bounds_are_gershgorin(levels):
    for lv in levels[:-1]:
        A = lv["A"].tocsr()
        g = np.max(np.asarray(abs(A).sum(axis=1)).ravel() / np.abs(A.diagonal()))
        assert lv["lam"] == pytest.approx(g, rel=1e-14)
    assert levels[-1]["lam"] == 0.0


def test_coarsest_level_inverse(levels):
    last = levels[-1]
    A = last["A"].toarray()
    assert np.abs(last["coarse_inv"] @ A - np.eye(last["n"])).max() <= 1e-10


def test_set_up_is_deterministic(L, system, levels):
    rp, ci, dg, blocks, _ = system
    again = L.debug_amg_host(rp, ci, dg, blocks, L.default_options(amg_coarse_size=COARSE))
    for a, b in zip(levels, again):
        assert (a["A"] != b["A"]).nnz == 0 and a["lam"] == b["lam"]
        if a["P"] is not None:
            assert (a["P"] != b["P"]).nnz == 0


def test_invalid_input_is_rejected(L, system):
    rp, ci, dg, blocks, _ = system
    lib = L.library()
    sz = np.zeros(5, dtype=np.int64)

    def call(rp_, ci_, dg_, level=0):
        return lib.lfx_debug_amg_host(int(rp_.size - 1), L._i(rp_), L._i(ci_), L._i(dg_), L._d(blocks), None,
                                      level, sz.ctypes.data_as(L._LP), None, None, None, None, None, None, None,
                                      None)

    assert call(rp, ci, dg) == L.LFX_OK
    bad = dg.copy()
    bad[3] = rp[3] if ci[rp[3]] != 3 else rp[3] + 1       # not the diagonal block of row 3
    assert call(rp, ci, bad) == L.LFX_ERR_INVALID_ARG
    badc = ci.copy()
    badc[7] = rp.size + 3                                  # column out of range
    assert call(rp, badc, dg) == L.LFX_ERR_INVALID_ARG
    assert call(rp, ci, dg, level=int(sz[0])) == L.LFX_ERR_INVALID_ARG     # one beyond the last level
