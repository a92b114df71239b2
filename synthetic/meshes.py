"""Seeded synthetic tetrahedral meshes shaped like the paper's test geometries.

The paper's meshes (the Zenodo parameter files, the aorta of Test III, the left atrium of
Test IV) are not available, so these generators stand in for them.  The tetrahedral meshes in
Table tab:mesh (Section 4) have 5.4-6.3 tetrahedra per vertex and edge ratios q of 1-17; a
jittered body-centred-cubic (BCC) point set tetrahedralised by Qhull (Delaunay) gives about
6 tetrahedra per vertex in the bulk, fewer at the boundary, and edge ratios of 1.2-3.

Every generator returns a :class:`Mesh` whose node and element order is shuffled by the seed
(so that a consumer cannot rely on a favourable input order), with positively oriented
tetrahedra and the boundary faces tagged as in Test II of Section 4.2: wall 0, inlet 1,
outlet 2 (outlets of a bifurcation are 2 and 3).  No finite-element arithmetic lives here.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

WALL, INLET, OUTLET, OUTLET2 = 0, 1, 2, 3


@dataclasses.dataclass
class Mesh:
    nodes: np.ndarray        # [V,3] float64
    tets: np.ndarray         # [T,4] int32, positively oriented
    bfaces: np.ndarray       # [F,3] int32, outward oriented (right-hand rule)
    btags: np.ndarray        # [F]   int32
    name: str = ""
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return int(self.nodes.shape[0])

    @property
    def n_tets(self) -> int:
        return int(self.tets.shape[0])

    def tag_nodes(self, tag: int) -> np.ndarray:
        """Sorted unique node indices lying on boundary faces with this tag."""
        return np.unique(self.bfaces[self.btags == tag].ravel())


# ----------------------------------------------------------------------------------------
# topology helpers (index bookkeeping only)
# ----------------------------------------------------------------------------------------
def _signed_volumes(nodes: np.ndarray, tets: np.ndarray) -> np.ndarray:
    x = nodes[tets]
    d1, d2, d3 = x[:, 1] - x[:, 0], x[:, 2] - x[:, 0], x[:, 3] - x[:, 0]
    return np.einsum("ij,ij->i", np.cross(d1, d2), d3) / 6.0


def _orient(nodes: np.ndarray, tets: np.ndarray) -> np.ndarray:
    tets = tets.copy()
    neg = _signed_volumes(nodes, tets) < 0
    tets[neg, 2], tets[neg, 3] = tets[neg, 3].copy(), tets[neg, 2].copy()
    return tets


_FACE_LOCAL = np.array([[1, 2, 3], [0, 3, 2], [0, 1, 3], [0, 2, 1]])  # outward for det>0


def _face_multiplicity(tets: np.ndarray) -> np.ndarray:
    """For each of the 4T faces (tet-major order), how many tetrahedra share it."""
    key = np.sort(tets[:, _FACE_LOCAL].reshape(-1, 3).astype(np.int64), axis=1)
    if key.size and key.max() < (1 << 21):
        k = (key[:, 0] << 42) | (key[:, 1] << 21) | key[:, 2]
        _, inv, cnt = np.unique(k, return_inverse=True, return_counts=True)
    else:
        _, inv, cnt = np.unique(key, axis=0, return_inverse=True, return_counts=True)
    return cnt[inv.ravel()]


def boundary_faces(nodes: np.ndarray, tets: np.ndarray) -> np.ndarray:
    """Faces that belong to exactly one tetrahedron, oriented outward (right-hand rule)."""
    faces = tets[:, _FACE_LOCAL].reshape(-1, 3)
    once = _face_multiplicity(tets) == 1
    bf = faces[once]
    # verify outward orientation against the opposite vertex
    opp = np.repeat(tets, 4, axis=0)[once]
    loc = np.tile(np.arange(4), tets.shape[0])[once]
    d = nodes[opp[np.arange(opp.shape[0]), loc]]
    a, b, c = nodes[bf[:, 0]], nodes[bf[:, 1]], nodes[bf[:, 2]]
    s = np.einsum("ij,ij->i", np.cross(b - a, c - a), d - a)
    flip = s > 0
    bf[flip, 1], bf[flip, 2] = bf[flip, 2].copy(), bf[flip, 1].copy()
    return bf.astype(np.int32)


def _quality(nodes: np.ndarray, tets: np.ndarray) -> np.ndarray:
    """Volume-to-rms-edge quality, 1 for a regular tetrahedron and 0 for a flat one."""
    x = nodes[tets]
    e2 = np.zeros(tets.shape[0])
    for i, j in ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)):
        e2 += np.sum((x[:, i] - x[:, j]) ** 2, axis=1)
    erms = np.sqrt(e2 / 6.0)
    return np.abs(_signed_volumes(nodes, tets)) * 6.0 * math.sqrt(2.0) / erms ** 3


def _shuffle(rng: np.random.Generator, nodes, tets):
    V, T = nodes.shape[0], tets.shape[0]
    pn = rng.permutation(V)           # new position -> old node
    inv = np.empty(V, dtype=np.int64)
    inv[pn] = np.arange(V)
    nodes = nodes[pn]
    tets = inv[tets]
    tets = tets[rng.permutation(T)]
    # random cyclic-preserving vertex rotation within each tet keeps orientation if even
    return nodes, tets


def _compact(nodes, tets):
    used = np.unique(tets.ravel())
    remap = -np.ones(nodes.shape[0], dtype=np.int64)
    remap[used] = np.arange(used.size)
    return nodes[used], remap[tets]


def _finish(name, nodes, tets, rng, classify, meta) -> Mesh:
    nodes, tets = _compact(nodes, tets)
    if rng is not None:
        nodes, tets = _shuffle(rng, nodes, tets)
    tets = _orient(nodes, tets).astype(np.int32)
    bf = boundary_faces(nodes, tets)
    tags = classify(nodes, bf).astype(np.int32)
    return Mesh(np.ascontiguousarray(nodes, dtype=np.float64), np.ascontiguousarray(tets),
                bf, tags, name, meta)


# ----------------------------------------------------------------------------------------
# structured cube (Test I / Beltrami)
# ----------------------------------------------------------------------------------------
def cube_kuhn(n: int, length: float = 1.0, origin=(0.0, 0.0, 0.0), seed: int | None = None) -> Mesh:
    """Unit-cube grid of n^3 hexahedra, each split into the 6 Kuhn tetrahedra that share the
    diagonal (0,0,0)-(1,1,1) of the cell; conforming across cells.  Boundary tags: face x=0 -> 1,
    x=L -> 2, y=0 -> 3, y=L -> 4, z=0 -> 5, z=L -> 6 (all are Dirichlet in the Beltrami case).
    ``seed`` (optional) shuffles node and element order."""
    m = n + 1
    g = np.arange(m, dtype=np.float64) * (length / n)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    nodes = np.stack([X.ravel(order="F"), Y.ravel(order="F"), Z.ravel(order="F")], axis=1)
    nodes += np.asarray(origin, dtype=np.float64)
    idx = lambda i, j, k: i + m * (j + m * k)
    ii, jj, kk = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ii, jj, kk = ii.ravel(), jj.ravel(), kk.ravel()
    tets = []
    for p in ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)):
        c = [np.zeros_like(ii), np.zeros_like(ii), np.zeros_like(ii)]
        verts = [idx(ii, jj, kk)]
        for ax in p[:2]:
            c[ax] = c[ax] + 1
            verts.append(idx(ii + c[0], jj + c[1], kk + c[2]))
        verts.append(idx(ii + 1, jj + 1, kk + 1))
        tets.append(np.stack(verts, axis=1))
    tets = np.concatenate(tets, axis=0)
    rng = np.random.default_rng(seed) if seed is not None else None
    o = np.asarray(origin, dtype=np.float64)

    def classify(nd, bf):
        x = nd[bf]  # [F,3,3]
        tag = np.full(bf.shape[0], -1)
        tol = 1e-9 * length
        for ax in range(3):
            lo = np.all(np.abs(x[:, :, ax] - o[ax]) < tol, axis=1)
            hi = np.all(np.abs(x[:, :, ax] - o[ax] - length) < tol, axis=1)
            tag[lo & (tag < 0)] = 1 + 2 * ax
            tag[hi & (tag < 0)] = 2 + 2 * ax
        assert np.all(tag >= 0)
        return tag

    return _finish(f"cube_kuhn_{n}", nodes, tets, rng, classify, {"n": n, "length": length})


def single_tet(seed: int, kind: str = "random") -> Mesh:
    """One tetrahedron: ``random`` (well shaped, random position and orientation), ``sliver``
    (nearly flat), or ``reference`` (the unit right simplex)."""
    rng = np.random.default_rng(seed)
    if kind == "reference":
        x = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=np.float64)
    elif kind == "sliver":
        x = np.array([[0, 0, 0], [1, 0, 0], [0.5, 0.9, 0.02], [0.5, 0.3, -0.03]], dtype=np.float64)
        q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
        x = x @ q.T * (0.5 + rng.random()) + rng.standard_normal(3)
    else:
        x = np.array([[0, 0, 0], [1, 0, 0], [0.5, 0.85, 0], [0.5, 0.3, 0.8]], dtype=np.float64)
        x += 0.15 * rng.standard_normal((4, 3))
        q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
        x = x @ q.T * (0.2 + rng.random()) + rng.standard_normal(3)
    tets = np.array([[0, 1, 2, 3]])
    return _finish(f"tet_{kind}_{seed}", x, tets, None,
                   lambda nd, bf: np.zeros(bf.shape[0], dtype=np.int32), {})


# ----------------------------------------------------------------------------------------
# jittered-BCC Delaunay meshes (vessels)
# ----------------------------------------------------------------------------------------
def _bcc_points(lo, hi, a, rng, jitter):
    axes = [np.arange(lo[d] - a, hi[d] + a, a) for d in range(3)]
    G = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, 3)
    P = np.concatenate([G, G + 0.5 * a], axis=0)
    P = P + jitter * a * rng.uniform(-1.0, 1.0, size=P.shape)
    return P


def _delaunay_clean(points, inside_centroid, qmin=0.05, max_passes=50):
    from scipy.spatial import Delaunay

    tri = Delaunay(points, qhull_options="Qbb Qc Qz Q12 Qt")
    tets = tri.simplices.astype(np.int64)
    c = points[tets].mean(axis=1)
    tets = tets[inside_centroid(c)]
    q = _quality(points, tets)
    tets = tets[q > 1e-9]
    # peel badly shaped tetrahedra that touch the boundary (surface slivers), repeatedly
    for _ in range(max_passes):
        on_bd = (_face_multiplicity(tets) == 1).reshape(-1, 4).any(axis=1)
        q = _quality(points, tets)
        bad = on_bd & (q < qmin)
        if not bad.any():
            break
        tets = tets[~bad]
    return tets


def _ring_points(R, z0, z1, h, rng, jitter):
    nth = max(8, int(round(2 * math.pi * R / h)))
    nz = max(2, int(round((z1 - z0) / (h * 0.866))) + 1)
    zs = np.linspace(z0, z1, nz)
    pts = []
    for k, z in enumerate(zs):
        th = (np.arange(nth) + 0.5 * (k % 2)) * (2 * math.pi / nth)
        if 0 < k < nz - 1:
            th = th + jitter * (2 * math.pi / nth) * rng.uniform(-1, 1, nth)
        pts.append(np.stack([R * np.cos(th), R * np.sin(th), np.full(nth, z)], axis=1))
    return np.concatenate(pts, axis=0)


def _disk_points(R, z, h, rng, jitter):
    pts = [np.zeros((1, 2))]
    nr = max(1, int(round(R / h)))
    for i in range(1, nr):
        r = R * i / nr
        nth = max(6, int(round(2 * math.pi * r / h)))
        th = (np.arange(nth) + rng.uniform()) * (2 * math.pi / nth)
        rr = r + jitter * h * rng.uniform(-0.5, 0.5, nth)
        pts.append(np.stack([rr * np.cos(th), rr * np.sin(th)], axis=1))
    p = np.concatenate(pts, axis=0)
    return np.concatenate([p, np.full((p.shape[0], 1), z)], axis=1)


def cylinder(radius: float = 1.0, length: float = 10.0, n_tets: int = 100_000, seed: int = 2,
             jitter: float = 0.2, radial_scale=None) -> Mesh:
    """Straight cylinder along z (inlet z=0 tag 1, outlet z=L tag 2, wall tag 0), about
    ``n_tets`` tetrahedra from a jittered BCC interior lattice plus wall and cap points.
    ``radial_scale(z)`` (optional) narrows the tube: the point set is mapped r -> r s(z) before
    the Delaunay tetrahedralisation, so every tetrahedron of the narrowed tube is valid."""
    rng = np.random.default_rng(seed)
    R, L = radius, length
    a = (12.0 * math.pi * R * R * L / n_tets) ** (1.0 / 3.0)
    h = 0.9 * a
    P = _bcc_points((-R, -R, 0.0), (R, R, L), a, rng, jitter)
    r = np.hypot(P[:, 0], P[:, 1])
    keep = (r < R - 0.45 * h) & (P[:, 2] > 0.45 * h) & (P[:, 2] < L - 0.45 * h)
    P = P[keep]
    wall = _ring_points(R, 0.0, L, h, rng, 0.15)
    cap0 = _disk_points(R, 0.0, h, rng, 0.3)
    cap1 = _disk_points(R, L, h, rng, 0.3)
    cap0 = cap0[np.hypot(cap0[:, 0], cap0[:, 1]) < R - 0.4 * h]
    cap1 = cap1[np.hypot(cap1[:, 0], cap1[:, 1]) < R - 0.4 * h]
    pts = np.concatenate([P, wall, cap0, cap1], axis=0)
    sc = (lambda z: np.ones_like(z)) if radial_scale is None else radial_scale
    if radial_scale is not None:
        f = sc(pts[:, 2])
        pts = pts.copy()
        pts[:, 0] *= f
        pts[:, 1] *= f

    def inside(c):
        return (np.hypot(c[:, 0], c[:, 1]) < R * sc(c[:, 2])) & (c[:, 2] > 0) & (c[:, 2] < L)

    tets = _delaunay_clean(pts, inside)

    def classify(nd, bf):
        z = nd[bf][:, :, 2]
        tol = 1e-9 * L
        tag = np.full(bf.shape[0], WALL)
        tag[np.all(np.abs(z) < tol, axis=1)] = INLET
        tag[np.all(np.abs(z - L) < tol, axis=1)] = OUTLET
        return tag

    return _finish(f"cylinder_{n_tets}_{seed}", pts, tets, rng, classify,
                   {"radius": R, "length": L, "spacing": a, "seed": seed})


def stenosis(radius: float = 1.0, length: float = 10.0, n_tets: int = 400_000, seed: int = 3,
             z_center: float = 3.0, half_length: float = 1.0, severity: float = 0.25) -> Mesh:
    """Cylinder with an axisymmetric cosine stenosis: radius R s(z), s = 1 - severity (1 + cos(pi
    (z - z_center)/half_length)) inside |z - z_center| <= half_length.  severity = 0.25 gives a throat
    of half the radius, i.e. a 75 % area reduction.  The cylinder's point set is mapped and then
    tetrahedralised, so the elements are valid Delaunay tetrahedra of the narrowed tube."""

    def scale(z):
        s = np.ones_like(z)
        w = np.abs(z - z_center) <= half_length
        s[w] = 1.0 - severity * (1.0 + np.cos(math.pi * (z[w] - z_center) / half_length))
        return s

    m = cylinder(radius, length, n_tets, seed, radial_scale=scale)
    meta = dict(m.meta)
    meta.update(z_center=z_center, half_length=half_length, severity=severity)
    return Mesh(m.nodes, m.tets, m.bfaces, m.btags, f"stenosis_{n_tets}_{seed}", meta)


def _seg_cyl_sdf(p, a, b, r):
    """Signed distance (approximate outside the rims) to the flat-capped cylinder a->b."""
    ab = b - a
    L = np.linalg.norm(ab)
    t = ab / L
    ap = p - a
    s = ap @ t
    radial = np.linalg.norm(ap - np.outer(s, t), axis=1) - r
    axial = np.abs(s - 0.5 * L) - 0.5 * L
    return np.maximum(radial, axial), s, L


def bifurcation(n_tets: int = 100_000, seed: int = 1000, angle_deg: float = 50.0,
                r0: float = 0.6, r1: float = 0.45, r2: float = 0.4, trunk_len: float | None = None,
                branch_len: float | None = None) -> Mesh:
    """Y-bifurcation: a trunk along +z from the origin (inlet, tag 1) splitting at its end into two
    branches at +-angle/2 in the x-z plane (outlets, tags 2 and 3); wall tag 0."""
    rng = np.random.default_rng(seed)
    trunk_len = trunk_len if trunk_len is not None else 6.0 * r0
    branch_len = branch_len if branch_len is not None else 5.0 * max(r1, r2)
    th = math.radians(angle_deg) / 2.0
    A0, B0 = np.array([0.0, 0, 0]), np.array([0.0, 0, trunk_len])
    d1 = np.array([math.sin(th), 0, math.cos(th)])
    d2 = np.array([-math.sin(th), 0, math.cos(th)])
    # branches start slightly inside the trunk so that the union is watertight
    B1 = B0 + branch_len * d1
    B2 = B0 + branch_len * d2
    A1 = B0 - 0.5 * r0 * d1
    A2 = B0 - 0.5 * r0 * d2
    comps = [(A0, B0 + 0.2 * r0 * np.array([0, 0, 1.0]), r0), (A1, B1, r1), (A2, B2, r2)]
    vol = sum(math.pi * r * r * np.linalg.norm(b - a) for a, b, r in comps) * 0.92
    a = (12.0 * vol / n_tets) ** (1.0 / 3.0)
    h = 0.9 * a

    def sdf(p):
        return np.min(np.stack([_seg_cyl_sdf(p, aa, bb, rr)[0] for aa, bb, rr in comps]), axis=0)

    allp = np.concatenate([np.stack(c[:2]) for c in comps])
    R = max(r0, r1, r2)
    lo, hi = allp.min(axis=0) - R, allp.max(axis=0) + R
    P = _bcc_points(lo, hi, a, rng, 0.2)
    P = P[sdf(P) < -0.45 * h]
    surf = []
    for k, (aa, bb, rr) in enumerate(comps):
        t = (bb - aa) / np.linalg.norm(bb - aa)
        u = np.cross(t, [0.0, 1.0, 0.0] if abs(t[1]) < 0.9 else [1.0, 0, 0])
        u /= np.linalg.norm(u)
        v = np.cross(t, u)
        Lc = np.linalg.norm(bb - aa)
        loc = _ring_points(rr, 0.0, Lc, h, rng, 0.15)
        caps = []
        if k == 0:
            caps.append(_disk_points(rr - 0.4 * h, 0.0, h, rng, 0.3))
        else:
            caps.append(_disk_points(rr - 0.4 * h, Lc, h, rng, 0.3))
        loc = np.concatenate([loc] + caps, axis=0)
        world = aa + loc[:, :1] * u + loc[:, 1:2] * v + loc[:, 2:3] * t
        surf.append(world)
    S = np.concatenate(surf, axis=0)
    S = S[sdf(S) > -0.3 * h]          # drop wall points buried inside another branch
    S = S[sdf(S) < 0.3 * h]
    pts = np.concatenate([P, S], axis=0)
    tets = _delaunay_clean(pts, lambda c: sdf(c) < 0.0, qmin=0.08)
    # keep the largest connected component only (drop stray tets at the junction)
    tets = _largest_component(tets)
    caps_def = [(A0, -(B0 - A0) / np.linalg.norm(B0 - A0), r0, INLET),
                (B1, d1, r1, OUTLET), (B2, d2, r2, OUTLET2)]

    def classify(nd, bf):
        x = nd[bf]
        tag = np.full(bf.shape[0], WALL)
        tol = 1e-6 * a
        for c, nrm, rr, tg in caps_def:
            dist = np.abs(np.einsum("fkj,j->fk", x - c, nrm))
            rad = np.linalg.norm((x - c) - np.einsum("fk,j->fkj", np.einsum("fkj,j->fk", x - c, nrm), nrm), axis=2)
            on = np.all(dist < tol, axis=1) & np.all(rad < rr + tol, axis=1)
            tag[on] = tg
        return tag

    return _finish(f"bifurcation_{n_tets}_{seed}", pts, tets, rng, classify,
                   {"angle_deg": angle_deg, "r": (r0, r1, r2), "spacing": a, "seed": seed,
                    "inlet_center": A0.tolist(), "inlet_normal": (-(B0 - A0) / np.linalg.norm(B0 - A0)).tolist(),
                    "outlet_centers": [B1.tolist(), B2.tolist()]})


def _largest_component(tets):
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components

    T = tets.shape[0]
    faces = tets[:, _FACE_LOCAL].reshape(-1, 3)
    key = np.sort(faces, axis=1)
    _, inv = np.unique(key, axis=0, return_inverse=True)
    inv = inv.ravel()
    owner = np.repeat(np.arange(T), 4)
    order = np.argsort(inv, kind="stable")
    si, so = inv[order], owner[order]
    same = si[1:] == si[:-1]
    r, c = so[1:][same], so[:-1][same]
    g = coo_matrix((np.ones(r.size), (r, c)), shape=(T, T))
    n, lab = connected_components(g, directed=False)
    if n == 1:
        return tets
    big = np.argmax(np.bincount(lab))
    return tets[lab == big]


# ----------------------------------------------------------------------------------------
# statistics in the form of Table tab:mesh (Section 4)
# ----------------------------------------------------------------------------------------
def mesh_stats(m: Mesh) -> dict:
    x = m.nodes[m.tets]
    el = []
    for i, j in ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)):
        el.append(np.linalg.norm(x[:, i] - x[:, j], axis=1))
    el = np.stack(el, axis=1)
    hK = el.max(axis=1)
    q = el.max(axis=1) / el.min(axis=1)
    return {
        "n_tets": m.n_tets, "n_nodes": m.n_nodes, "tets_per_vertex": m.n_tets / m.n_nodes,
        "h_min": float(hK.min()), "h_avg": float(hK.mean()), "h_max": float(hK.max()),
        "q_min": float(q.min()), "q_avg": float(q.mean()), "q_max": float(q.max()),
        "quality_min": float(_quality(m.nodes, m.tets).min()),
        "n_bfaces": int(m.bfaces.shape[0]),
    }


def batch(meshes, tag_stride: int = 10) -> Mesh:
    """Several independent meshes as one disconnected mesh: node and element indices offset,
    boundary tag t of mesh i becomes t + tag_stride * i.  Returns the union with
    meta['node_offsets'] (len n+1) for slicing per-mesh fields."""
    nodes, tets, bf, tg, offs = [], [], [], [], [0]
    for i, m in enumerate(meshes):
        o = offs[-1]
        nodes.append(m.nodes)
        tets.append(m.tets.astype(np.int64) + o)
        bf.append(m.bfaces.astype(np.int64) + o)
        tg.append(m.btags.astype(np.int64) + tag_stride * i)
        offs.append(o + m.n_nodes)
    return Mesh(np.concatenate(nodes), np.concatenate(tets).astype(np.int32), np.concatenate(bf).astype(np.int32),
                np.concatenate(tg).astype(np.int32), "batch_%d" % len(meshes),
                {"node_offsets": offs, "tag_stride": tag_stride, "names": [m.name for m in meshes]})
