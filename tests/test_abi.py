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


def test_no_fallback_without_the_library(L, monkeypatch, tmp_path):
    """Without liblfx.so the binding raises instead of computing anything another way."""
    monkeypatch.setattr(L, "_lib", None)
    monkeypatch.setattr(L, "LIB_PATH", str(tmp_path / "liblfx.so"))
    m = cube_kuhn(2)
    with pytest.raises(ImportError):
        L.Mesh(m.nodes, m.tets, m.bfaces, m.btags)
    with pytest.raises(ImportError):
        L.default_options()


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


def _shape_quality(nodes, tets):
    """6 sqrt2 |K| / e_rms^3: 1 for a regular tetrahedron, 0 for a flat one."""
    x = nodes[tets]
    det = np.einsum("ij,ij->i", np.cross(x[:, 1] - x[:, 0], x[:, 2] - x[:, 0]), x[:, 3] - x[:, 0])
    e2 = sum(((x[:, a] - x[:, b]) ** 2).sum(1) for a in range(4) for b in range(a + 1, 4))
    return np.abs(det) / 6.0 * 6.0 * np.sqrt(2.0) / np.sqrt(e2 / 6.0) ** 3


def test_mesh_info_counts_components_and_badly_shaped_elements(L):
    # three pieces: a Kuhn cube, a shifted copy of it, and a pair of tetrahedra sharing a face, one
    # of them a sliver (quality about 0.05, below the default threshold 0.1)
    c = cube_kuhn(2)
    pair_nodes = np.array([[10.0, 0, 0], [11.0, 0, 0], [10.0, 1.0, 0], [10.3, 0.3, 0.5], [10.3, 0.3, -0.02]])
    nodes = np.vstack([c.nodes, c.nodes + [3.0, 0, 0], pair_nodes])
    V = c.n_nodes
    pair = np.array([[0, 1, 2, 3], [0, 2, 1, 4]]) + 2 * V
    tets = np.vstack([c.tets, c.tets + V, pair]).astype(np.int32)
    bfaces = np.vstack([c.bfaces, c.bfaces + V]).astype(np.int32)
    btags = np.concatenate([c.btags, c.btags]).astype(np.int32)
    q = _shape_quality(nodes, tets)
    assert q[-1] < 0.1 < q[:-1].min()
    info = L.Mesh(nodes, tets, bfaces, btags).info()
    assert info["n_components"] == 3
    assert info["n_bad_elements"] == int((q < 0.1).sum()) == 1
    assert info["n_tets"] == len(tets) and info["n_flipped"] == 0
    # the synthetic cylinder has none below the threshold
    m = cylinder(1.0, 4.0, n_tets=20000, seed=3)
    assert L.Mesh(m.nodes, m.tets, m.bfaces, m.btags).info()["n_bad_elements"] == int(
        (_shape_quality(m.nodes, m.tets) < 0.1).sum())


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
    ceil(T / W), and the colouring stays valid.  The chunk colours of the chunked assembly come
    within two waves of 456 chunks (one 32-element chunk per CTA) of theirs."""
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
    # the chunk colours of the chunked assembly, balanced to waves of 456 chunks (152 x 3 CTAs)
    ch = mesh.chunks()
    csz = np.diff(ch["chunk_color_off"])
    nch = int(csz.sum())
    assert csz.min() > 0 and nch == ch["chunk_elem_off"].size - 1
    assert int(np.ceil(csz / 456).sum()) <= -(-nch // 456) + 2, csz.tolist()


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


@pytest.mark.parametrize("opt", [dict(staged_f=2), dict(assembly=7), dict(assembly=-1), dict(implicit=2),
                                 dict(implicit=1, newton_max_iters=0), dict(implicit=1, newton_rtol=0.0),
                                 dict(gmres_restart=0), dict(f_steps=0), dict(s_smoother=5), dict(precision=3),
                                 dict(stab=3), dict(diffusion=-1)])
def test_options_are_checked_before_allocation(L, opt):
    """Options out of range are rejected as invalid arguments before any device memory is touched
    (so on a host without a GPU as well)."""
    m = cylinder(1.0, 2.0, n_tets=3000, seed=9)
    mesh = L.Mesh.from_synthetic(m)
    bcs = [L.BC(tag=0, kind="noslip"), L.BC(tag=1, kind="dirichlet"), L.BC(tag=2, kind="neumann")]
    with pytest.raises(L.LfxError) as err:
        L.Problem(mesh, 1.06, 0.035, 1e-3, 2, bcs, [], L.default_options(**opt))
    assert err.value.status == L.LFX_ERR_INVALID_ARG


def test_host_arguments_rejected_without_a_gpu(L):
    """Arguments the host can reject by themselves: a server without a positive budget or with a
    worker count outside 1..64, one allocator function without the other, queries on NULL handles,
    unknown struct names, more than eight resistive surfaces, and the allocation-free
    preconditioner's size and smoother limits."""
    lib = L.library()
    h = L._P()
    for budget, workers in ((0, 4), (-1, 4), (1 << 30, 0), (1 << 30, 65)):
        assert lib.lfx_server_create(budget, workers, ctypes.byref(h)) == L.LFX_ERR_INVALID_ARG
    assert lib.lfx_server_create(1 << 30, 4, None) == L.LFX_ERR_INVALID_ARG
    done = ctypes.c_int32()
    assert lib.lfx_server_poll(None, 0, ctypes.byref(done), None, None) == L.LFX_ERR_INVALID_ARG
    fa = L.ALLOC_FN(lambda n, ctx: None)
    assert lib.lfx_set_allocator(fa, L.FREE_FN(), None) == L.LFX_ERR_INVALID_ARG
    assert b"both" in lib.lfx_last_error()
    assert lib.lfx_set_allocator(L.ALLOC_FN(), L.FREE_FN(), None) == L.LFX_OK      # back to cudaMalloc
    info = L.lfx_mesh_info()
    assert lib.lfx_mesh_get_info(None, ctypes.byref(info)) == L.LFX_ERR_INVALID_ARG
    assert lib.lfx_sizeof(b"no_such_struct") == -1
    m = cylinder(1.0, 2.0, n_tets=3000, seed=9)
    mesh = L.Mesh.from_synthetic(m)
    disks = [L.RIIS(center=(0.0, 0.0, 1.0), normal=(0.0, 0.0, 1.0), radius=0.5, resistance=1e3, eps=0.05)] * 9
    with pytest.raises(L.LfxError) as err:
        L.Problem(mesh, 1.06, 0.035, 1e-3, 2, [L.BC(tag=0, kind="noslip")], disks)
    assert err.value.status == L.LFX_ERR_INVALID_ARG
    # the allocation-free preconditioner: at most 65,536 block rows, Jacobi or Chebyshev smoothers only
    # (the arguments are checked before any pointer is used, so host stand-ins serve here)
    dummy = np.zeros(8)
    ptr = dummy.ctypes.data

    def noalloc(n, opt=None):
        return lib.lfx_asimple_apply_noalloc(n, ptr, ptr, ptr, ptr, ptr, ptr, ptr,
                                             ctypes.byref(opt) if opt is not None else None, None)

    assert noalloc(0) == L.LFX_ERR_INVALID_ARG
    assert noalloc(65537) == L.LFX_ERR_INVALID_ARG
    assert b"65536" in lib.lfx_last_error()
    assert noalloc(100, L.default_options(s_smoother="amg")) == L.LFX_ERR_INVALID_ARG
    assert noalloc(100, L.default_options(s_smoother="chebyshev", f_steps=0)) == L.LFX_ERR_INVALID_ARG
    assert lib.lfx_asimple_apply_noalloc(100, None, ptr, ptr, ptr, ptr, ptr, ptr, None, None) == L.LFX_ERR_INVALID_ARG


def test_implicit_formulation_rejects_outlet_terms_before_allocation(L):
    m = cylinder(1.0, 2.0, n_tets=3000, seed=9)
    mesh = L.Mesh.from_synthetic(m)
    for outlet in (L.BC(tag=2, kind="resistance", resistance=10.0), L.BC(tag=2, kind="neumann", beta=1.0)):
        bcs = [L.BC(tag=0, kind="noslip"), L.BC(tag=1, kind="dirichlet"), outlet]
        with pytest.raises(L.LfxError) as err:
            L.Problem(mesh, 1.06, 0.035, 1e-3, 2, bcs, [], L.default_options(implicit=1))
        assert err.value.status == L.LFX_ERR_INVALID_ARG
        assert b"implicit" in L.library().lfx_last_error()


@pytest.mark.parametrize("which", ["cylinder", "bifurcation"])
def test_chunk_tables(L, which):
    """The chunked assembly's tables (host, no GPU): every element in exactly one chunk of at most 32;
    chunks of one colour share no node; every (element, a, b) block contribution appears exactly once
    in its chunk's passes, in a run whose matrix block is (node a, node b); runs do not straddle
    passes; each block has exactly one first-writer run, the one in the lowest chunk colour."""
    from synthetic import bifurcation

    m = cylinder(1.0, 3.0, n_tets=20000, seed=7) if which == "cylinder" else bifurcation(n_tets=20000, seed=1002)
    mesh = L.Mesh.from_synthetic(m)
    ch = mesh.chunks()
    T = m.n_tets
    eo, off, coff = ch["elem_old"], ch["chunk_elem_off"], ch["chunk_color_off"]
    assert np.array_equal(np.sort(eo), np.arange(T)) and off[0] == 0 and off[-1] == T
    assert np.diff(off).max() <= 32 and np.diff(off).min() >= 1
    tets = m.tets[eo]                                      # internal element -> caller nodes
    nch = off.size - 1
    ccol = np.zeros(nch, np.int64)
    for c in range(coff.size - 1):
        ccol[coff[c]:coff[c + 1]] = c
        nodes = [np.unique(tets[off[k]:off[k + 1]].ravel()) for k in range(coff[c], coff[c + 1])]
        alln = np.concatenate(nodes)
        assert np.unique(alln).size == alln.size, c           # no node in two chunks of one colour
    pcode, poff, roff, meta = ch["pass_code"], ch["chunk_pass_off"], ch["pass_run_off"], ch["run_meta"]
    PS = pcode.shape[1]
    first_of = {}
    for k in range(nch):
        seen = np.zeros((off[k + 1] - off[k], 4, 4), np.int64)
        for p in range(poff[k], poff[k + 1]):
            codes = pcode[p]
            covered = np.zeros(PS, bool)
            for r in range(roff[p], roff[p + 1]):
                st0, ln = int(meta[r]) & 0xff, (int(meta[r]) >> 8) & 63
                assert ln >= 1 and st0 + ln <= PS and not covered[st0:st0 + ln].any()
                covered[st0:st0 + ln] = True
                cc = codes[st0:st0 + ln].astype(np.int64)
                le, a, b = cc >> 4, (cc >> 2) & 3, cc & 3
                rows = tets[off[k] + le, a]
                cols = tets[off[k] + le, b]
                assert (rows == ch["run_row"][r]).all() and (cols == ch["run_col"][r]).all()
                assert bool(int(meta[r]) >> 15) == bool((a == b).all()) and (a == b).all() == (a == b).any()
                np.add.at(seen, (le, a, b), 1)
                if (int(meta[r]) >> 14) & 1:
                    key = (int(ch["run_row"][r]), int(ch["run_col"][r]))
                    assert key not in first_of
                    first_of[key] = ccol[k]
            assert (codes[~covered] == 0xffff).all()
        assert (seen == 1).all(), k
    # one first writer per block, in the lowest chunk colour touching it
    lowest = {}
    for k in range(nch):
        for p in range(poff[k], poff[k + 1]):
            for r in range(roff[p], roff[p + 1]):
                key = (int(ch["run_row"][r]), int(ch["run_col"][r]))
                lowest[key] = min(lowest.get(key, 1 << 30), ccol[k])
    assert first_of == lowest


@pytest.mark.parametrize("which", ["cylinder", "bifurcation"])
def test_row_tiles(L, which):
    """The staged velocity pass's row tiles (host, no GPU): consecutive block rows from 0 to n_nodes,
    each within both limits (rows, blocks = the rows' pattern lengths), and greedy: no tile but the
    last could take its successor's first row without breaking a limit; the internal row order is a
    permutation of the caller's nodes."""
    from synthetic import bifurcation

    m = cylinder(1.0, 3.0, n_tets=20000, seed=7) if which == "cylinder" else bifurcation(n_tets=20000, seed=1002)
    mesh = L.Mesh.from_synthetic(m)
    t = mesh.row_tiles()
    rp, _ = mesh.pattern()
    V = m.n_nodes
    node = t["row_node"]
    assert np.array_equal(np.sort(node), np.arange(V))
    length = (rp[1:] - rp[:-1])[node]               # blocks of each internal row
    tr = t["tile_row"]
    assert tr.size >= 2 and tr[0] == 0 and tr[-1] == V and np.all(np.diff(tr) >= 1)
    cum = np.concatenate([[0], np.cumsum(length)])
    rows = np.diff(tr)
    blocks = cum[tr[1:]] - cum[tr[:-1]]
    assert rows.max() <= t["max_rows"] and blocks.max() <= t["max_blocks"]
    nxt = tr[1:-1]                                  # first row of each following tile
    grow_rows = rows[:-1] + 1
    grow_blocks = blocks[:-1] + length[nxt]
    assert np.all((grow_rows > t["max_rows"]) | (grow_blocks > t["max_blocks"]))
