"""The allocation-free aSIMPLE entry point (lfx_asimple_apply_noalloc).

It serves callers that cannot allocate device memory while they run (for example a solver
embedded in a framework that owns all device memory through its own pool, or a time-critical loop
that must not pay for an allocation): its work arrays live in a fixed static device array.  Here it is called through the C ABI on a matrix
held in caller-owned device buffers, twice in a row, and each result is compared with the
preconditioner of the allocating entry point (lfx_debug_precond) on the same matrix, within
the tolerance of the preconditioner parity tests.  The file sorts last so that a run stopping
at the first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

from tests import cases as C

pytestmark = pytest.mark.gpu

CHEB = dict(s_smoother="chebyshev", s_steps=6, s_ratio=30.0)


def _diag_and_transpose(rp, ci):
    V = rp.size - 1
    rows = np.repeat(np.arange(V), np.diff(rp))
    key = rows.astype(np.int64) * V + ci
    order = np.argsort(key)
    tkey = ci.astype(np.int64) * V + rows
    trans = order[np.searchsorted(key[order], tkey)]    # position of block (j,i)
    diag = np.empty(V, dtype=np.int64)                  # position of block (i,i)
    hit = np.nonzero(rows == ci)[0]
    diag[rows[hit]] = hit
    return diag.astype(np.int32), trans.astype(np.int32)


def test_noalloc_preconditioner_matches_allocating_one():
    import torch

    from paper_2304_12032_gb300 import build

    build.build()
    from paper_2304_12032_gb300 import lfx as L

    case = C.vessel_case(6000, seed=41)
    mesh, prob, st = C.gpu_state(case, **CHEB)
    blocks, _ = st.debug_assemble(apply_bcs=True)
    rp, ci = mesh.pattern()
    V = case.mesh.n_nodes
    diag, trans = _diag_and_transpose(rp, ci)
    dev = torch.device("cuda", 0)
    t_rp = torch.tensor(rp.astype(np.int32), device=dev)
    t_ci = torch.tensor(ci, device=dev)
    t_dg = torch.tensor(diag, device=dev)
    t_tr = torch.tensor(trans, device=dev)
    t_bl = torch.tensor(blocks.reshape(-1), dtype=torch.float64, device=dev)
    opts = L.default_options(**CHEB)
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(9)
    for call in range(2):
        r = rng.standard_normal((V, 4))
        z_ref, _, _ = st.debug_precond(r)
        t_r = torch.tensor(r.reshape(-1), dtype=torch.float64, device=dev)
        t_z = torch.full_like(t_r, float("nan"))
        rc = L.library().lfx_asimple_apply_noalloc(
            V, ctypes.c_void_p(t_rp.data_ptr()), ctypes.c_void_p(t_ci.data_ptr()),
            ctypes.c_void_p(t_dg.data_ptr()), ctypes.c_void_p(t_tr.data_ptr()), ctypes.c_void_p(t_bl.data_ptr()),
            ctypes.c_void_p(t_r.data_ptr()), ctypes.c_void_p(t_z.data_ptr()), ctypes.byref(opts),
            ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, L.library().lfx_last_error()
        torch.cuda.synchronize()
        z = t_z.cpu().numpy().reshape(V, 4)
        assert np.all(np.isfinite(z)), call
        assert np.linalg.norm(z - z_ref) <= 1e-10 * np.linalg.norm(z_ref), call
        assert np.abs(z - z_ref).max() <= 1e-9 * np.abs(z_ref).max(), call


def test_noalloc_rejects_oversized_matrix():
    from paper_2304_12032_gb300 import build

    build.build()
    from paper_2304_12032_gb300 import lfx as L

    one = ctypes.c_void_p(1)   # never dereferenced: the size check comes first
    rc = L.library().lfx_asimple_apply_noalloc(65537, one, one, one, one, one, one, one, None, None)
    assert rc == L.LFX_ERR_INVALID_ARG
    assert b"65536" in L.library().lfx_last_error()
