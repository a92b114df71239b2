"""CPU checks of the C ABI: the library builds and loads, exports every entry point declared in
include/lfx.h, its struct layouts match the binding, and the host-side mesh set-up (validation,
pattern, colouring) is right.  No kernel runs here."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2304_12032_gb300 import build as B
from synthetic import cube_kuhn, cylinder

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    B.build()
    from paper_2304_12032_gb300 import lfx

    lfx.library()
    return lfx


def _declared():
    txt = open(os.path.join(ROOT, "include", "lfx.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = set(re.findall(r"\b(lfx_[a-z0-9_]+)\s*\(", txt))
    return sorted(n for n in names if not n.endswith("_fn"))


def test_every_declared_symbol_is_exported(L):
    lib = L.library()
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert len(_declared()) >= 20


def test_binding_covers_header(L):
    assert set(_declared()) <= set(L._SIGS), set(_declared()) - set(L._SIGS)


@pytest.mark.parametrize("name", ["lfx_time_law", "lfx_bc", "lfx_riis", "lfx_options", "lfx_mesh_info",
                                  "lfx_step_stats"])
def test_struct_layouts(L, name):
    assert L.library().lfx_sizeof(name.encode()) == ctypes.sizeof(getattr(L, name))


def test_options_defaults(L):
    o = L.default_options()
    assert o.stab == 2 and o.diffusion == 0 and o.c_r == 30.0 and o.pin_pressure_node == -1
    assert o.gmres_restart == 64 and o.f_steps == 6 and o.f_ratio == 60.0 and o.s_smoother == 2 and o.s_steps == 1
    assert o.reorthogonalize == 0 and o.inner_adaptive == 1 and o.batch_segmented == 1


def _status(L, nodes, tets, bf, tg):
    h = L._P()
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    bf = np.ascontiguousarray(bf, dtype=np.int32)
    tg = np.ascontiguousarray(tg, dtype=np.int32)
    rc = L.library().lfx_mesh_create(L._d(nodes), nodes.shape[0], L._i(tets), tets.shape[0], L._i(bf), L._i(tg),
                                     bf.shape[0], ctypes.byref(h))
    if rc == 0:
        L.library().lfx_mesh_destroy(h)
    return rc


def test_mesh_validation_errors(L):
    m = cube_kuhn(2)
    assert _status(L, m.nodes, m.tets, m.bfaces, m.btags) == L.LFX_OK
    bad = m.tets.copy()
    bad[3, 2] = m.n_nodes + 5
    assert _status(L, m.nodes, bad, m.bfaces, m.btags) == L.LFX_ERR_BAD_MESH
    flat = m.tets.copy()
    flat[0, 3] = flat[0, 2]                                   # repeated vertex: zero volume
    assert _status(L, m.nodes, flat, m.bfaces, m.btags) == L.LFX_ERR_BAD_MESH
    extra = np.vstack([m.nodes, [[5.0, 5.0, 5.0]]])           # node in no tetrahedron
    assert _status(L, extra, m.tets, m.bfaces, m.btags) == L.LFX_ERR_BAD_MESH
    bf = m.bfaces.copy()
    bf[0] = [0, 1, m.n_nodes - 1]                              # not a face of any tetrahedron
    assert _status(L, m.nodes, m.tets, bf, m.btags) == L.LFX_ERR_BAD_MESH
    nanx = m.nodes.copy()
    nanx[4, 1] = np.nan
    assert _status(L, nanx, m.tets, m.bfaces, m.btags) == L.LFX_ERR_BAD_MESH
    h = L._P()
    assert L.library().lfx_mesh_create(None, 0, None, 0, None, None, 0, ctypes.byref(h)) == L.LFX_ERR_INVALID_ARG
    assert b"null" in L.library().lfx_last_error().lower() or L.library().lfx_last_error()


def test_flipped_tets_are_counted(L):
    m = cube_kuhn(3, seed=4)
    t = m.tets.copy()
    t[::5, [2, 3]] = t[::5, [3, 2]]
    mesh = L.Mesh(m.nodes, t, m.bfaces, m.btags)
    assert mesh.info()["n_flipped"] == len(t[::5])


def _adjacency(m):
    pairs = np.concatenate([np.stack([m.tets[:, a], m.tets[:, b]], 1) for a in range(4) for b in range(4)])
    key = np.unique(pairs[:, 0].astype(np.int64) * m.n_nodes + pairs[:, 1])
    return key // m.n_nodes, key % m.n_nodes


@pytest.mark.parametrize("which", ["cube", "cylinder"])
def test_pattern_and_colouring(L, which):
    m = cube_kuhn(5, seed=3) if which == "cube" else cylinder(1.0, 2.0, n_tets=5000, seed=9)
    mesh = L.Mesh.from_synthetic(m)
    info = mesh.info()
    rp, ci = mesh.pattern()
    r, c = _adjacency(m)
    assert info["nnz_blocks"] == r.size
    assert np.array_equal(np.repeat(np.arange(m.n_nodes), np.diff(rp)), r)
    assert np.array_equal(ci, c)
    col = mesh.colors()
    assert col.min() == 0 and col.max() == info["n_colors"] - 1
    # no two elements of one colour share a node
    for k in range(info["n_colors"]):
        nodes = m.tets[col == k].ravel()
        assert np.unique(nodes).size == nodes.size
    assert info["n_colors"] <= 80


def test_colouring_balanced_to_assembly_waves(L):
    """At 1M tets the colours span several waves of the assembly kernel (GB300: 152 SMs x 3 CTAs x
    32 elements = 14,592 elements, the value used when no device answers).  The colours are
    rebalanced so that the waves launched, sum_c ceil(|c| / W), come within two of the work,
    ceil(T / W), and the colouring stays valid."""
    m = cylinder(1.0, 10.0, n_tets=1_000_000, seed=2)
    mesh = L.Mesh.from_synthetic(m)
    col = mesh.colors()
    T, W = m.n_tets, 152 * 3 * 32
    sizes = np.bincount(col)
    assert sizes.min() > 0
    waves = int(np.ceil(sizes / W).sum())
    assert waves <= -(-T // W) + 2, (waves, sizes.tolist())
    key = np.unique(np.stack([np.repeat(col, 4), m.tets.ravel()], 1), axis=0)
    assert key.shape[0] == 4 * T       # no node carries two elements of one colour


@pytest.mark.parametrize("bc", [dict(tag=0, kind="noslip", beta=1.0), dict(tag=2, kind="neumann", beta=-0.5),
                                dict(tag=2, kind="neumann", resistance=0.3), dict(tag=2, kind="resistance", resistance=-1.0)])
def test_outlet_condition_arguments_are_checked_before_allocation(L, bc):
    """Backflow stabilisation only on Neumann tags, the resistance coefficient only on resistance
    tags, both non-negative: rejected as invalid arguments before any device memory is touched
    (so on a host without a GPU as well)."""
    m = cylinder(1.0, 2.0, n_tets=3000, seed=9)
    mesh = L.Mesh.from_synthetic(m)
    with pytest.raises(L.LfxError) as err:
        L.Problem(mesh, 1.06, 0.035, 1e-3, 2, [L.BC(**bc)], [])
    assert err.value.status == L.LFX_ERR_INVALID_ARG
