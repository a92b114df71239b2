"""Mixed-precision path: the matrix assembled in double-float arithmetic (pairs of FP32 numbers,
48-bit significand) and the outer operator's compensated SpMV, against the FP64 oracle.

Tolerances.  The double-float unit roundoff is u = 2^-47 ~ 7.1e-15 per operation (measured on
random operands: add 7.1e-15, mul 1.2e-14, rsqrt 2.1e-14), against 2^-53 ~ 1.1e-16 for FP64.
The FP64 assembly test allows 1e-12 of the row scale (about 9000 FP64 roundoffs); here the
same allowance in units of u is 9000 u ~ 6e-11, and 5e-11 is used.  The SpMV is checked twice:
against the product of the downloaded double-float matrix (only the SpMV's own rounding, a
compensated dot product: about u times the row sums of |A||x|, allowed 1e-12), and against the
oracle's matrix (adds the entries' assembly error, allowed 1e-10 of the FP64 test's scale)."""
import numpy as np
import pytest

from tests import cases as C
from tests.test_gpu_parity import CASES

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2304_12032_gb300 import build

    build.build()


@pytest.fixture(scope="module", params=list(CASES))
def mixed_pair(request):
    case = CASES[request.param]()
    ost = C.oracle_step(case)
    mesh, prob, st = C.gpu_state(case, precision="mixed", smoother_bf16=1, gmres_rtol=1e-10)
    return request.param, case, ost, mesh, prob, st


def test_dd_assembly_matches_oracle(mixed_pair):
    name, case, ost, mesh, prob, st = mixed_pair
    blocks, rhs = st.debug_assemble(apply_bcs=True)
    rp, ci = mesh.pattern()
    ref = C.blocks_from_csr(ost.A, rp, ci)
    scale = C.row_scale(ost.A).reshape(-1, 4)
    rows = np.repeat(np.arange(case.mesh.n_nodes), np.diff(rp))
    tol = 5e-11 * np.maximum(np.abs(ref), scale[rows][:, :, None])
    err = np.abs(blocks - ref)
    assert np.all(err <= tol), (name, float((err / np.maximum(tol, 1e-300)).max()))
    # and far below FP32: the worst error in units of the row scale is reported on failure
    rel = float((err / np.maximum(scale[rows][:, :, None], 1e-300)).max())
    assert rel < 1e-11, (name, rel)
    bref = ost.b.reshape(-1, 4)
    btol = 5e-11 * np.maximum(np.abs(bref), np.abs(bref).max())
    assert np.all(np.abs(rhs - bref) <= btol), (name, float(np.abs(rhs - bref).max()))


def test_dd_spmv(mixed_pair):
    name, case, ost, mesh, prob, st = mixed_pair
    blocks, _ = st.debug_assemble(apply_bcs=True)
    rp, ci = mesh.pattern()
    V = case.mesh.n_nodes
    x = np.random.default_rng(7).standard_normal((V, 4))
    y = st.debug_spmv(x)
    # product of the downloaded (hi + lo) matrix in FP64, and the row sums of |A||x|
    rows = np.repeat(np.arange(V), np.diff(rp))
    contrib = np.einsum("kij,kj->ki", blocks, x[ci])
    absc = np.einsum("kij,kj->ki", np.abs(blocks), np.abs(x[ci]))
    yown = np.zeros((V, 4))
    aabs = np.zeros((V, 4))
    np.add.at(yown, rows, contrib)
    np.add.at(aabs, rows, absc)
    assert np.all(np.abs(y - yown) <= 1e-12 * aabs + 1e-300), (name, float(np.abs(y - yown).max()))
    yref = (ost.A @ x.ravel()).reshape(-1, 4)
    scale = C.row_scale(ost.A).reshape(-1, 4) * np.abs(x).max() * 20
    assert np.all(np.abs(y - yref) <= 1e-10 * np.maximum(scale, np.abs(yref))), name
