"""Oracle, global part (test infrastructure only; see the package docstring).

Plain numpy/scipy FP64 implementation of everything around the element integrals of
``lfx_oracle.c``: BDF coefficients (Eq. bdf), boundary data (Section 2.2), global assembly of
Eq. (fullydiscrete_ns_ale_riis_vmsles_quasistatic_unified) into a scalar CSR matrix with 4
unknowns per node (u_x, u_y, u_z, p), Dirichlet rows, the direct solve, one time step, and the
error norms of Eq. (errors).

Readings of the paper used here (it is silent on them):
  * BDF/EXT coefficients: the standard ones of order 1-3 (alpha = 1, 3/2, 11/6).
  * Dirichlet imposition: the constrained row is replaced by s * e_r with right-hand side
    s * g, s = |A_rr| of the assembled row (1 if that is 0); columns are not eliminated.
    At nodes shared by several tags no-slip beats other Dirichlet data, which beats Neumann.
  * Parabolic/uniform profiles: centre = area-weighted barycentre of the tagged faces, n = the
    normalised area-weighted outward normal of those faces.
  * Neumann data: h(t) enters as -(h n, v) on the tagged faces (P1: A_f/3 per vertex).
  * Inertial backflow stabilisation (Section 2.2.2, beta > 0 on a Neumann tag): semi-implicit
    like the rest of the step, the term beta rho/2 |u* . n|_- (u, v) with u* = u^EXT moves to the
    matrix as c(x) (u, v)_Gamma, c = -beta rho/2 min(u* . n, 0) >= 0, integrated with the
    degree-2 rule of the three edge midpoints (weights A_f/3).
  * Resistance condition (Section 2.2.3, u_ALE = 0): implicit in u, the flux term becomes the
    rank-one matrix C_R w w^T with w_{4a+i} = int_Gamma phi_a n_i (so w . u is the exact flux of
    a P1 velocity), and p_0(t) enters as -(p_0 n, v) like Neumann data.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
from typing import Callable, Optional, Sequence

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

__all__ = [
    "Params", "BC", "RIIS", "Problem", "load_library", "bdf_coefficients", "element",
    "element_residual", "element_batch", "geometry", "tau", "qp_coefficients", "assemble", "time_law", "boundary_geometry",
    "dirichlet_data", "neumann_rhs", "apply_dirichlet", "solve_direct", "Step",
    "step", "relative_errors", "disk_sdf", "block_of", "womersley_profile", "backflow_matrix",
    "resistance_vectors", "resistance_terms", "set_threads", "lifting", "ale_velocity", "implicit_step", "ImplicitStep", "implicit_system",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lfx_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liblfx_oracle.so")
_lib = None
MAX_RIIS = 8


def build_library(force: bool = False) -> str:
    """Compile ``lfx_oracle.c`` with gcc (plain -O2, no fast-math) into ``oracle/_build``."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-fno-fast-math", "-fopenmp",
                               "-ffp-contract=off", "-D_DEFAULT_SOURCE", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _CParams(ctypes.Structure):
    _fields_ = [("rho", ctypes.c_double), ("mu", ctypes.c_double), ("dt", ctypes.c_double),
                ("alpha", ctypes.c_double), ("sigma", ctypes.c_double), ("c_r", ctypes.c_double),
                ("f", ctypes.c_double * 3), ("n_riis", ctypes.c_int32), ("stab", ctypes.c_int32),
                ("diffusion", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("riis_r", ctypes.c_double * MAX_RIIS), ("riis_eps", ctypes.c_double * MAX_RIIS)]


def load_library():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build_library())
        dp = ctypes.POINTER(ctypes.c_double)
        _lib.orc_element.argtypes = [ctypes.POINTER(_CParams), dp, dp, dp, dp, dp, dp, dp, dp]
        _lib.orc_element.restype = ctypes.c_int
        _lib.orc_element_residual.argtypes = [ctypes.POINTER(_CParams), dp, dp, dp, dp, dp, dp, dp, dp]
        _lib.orc_element_residual.restype = ctypes.c_int
        _lib.orc_geometry.argtypes = [dp, dp, dp, dp, dp]
        _lib.orc_geometry.restype = ctypes.c_double
        _lib.orc_tau.argtypes = [ctypes.POINTER(_CParams), dp, dp, dp, dp, dp, dp]
        _lib.orc_tau.restype = None
        _lib.orc_delta.argtypes = [ctypes.c_double, ctypes.c_double]
        _lib.orc_delta.restype = ctypes.c_double
        _lib.orc_elements.argtypes = [ctypes.POINTER(_CParams), dp, ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_int64), ctypes.c_int64, dp, dp, dp, dp, dp,
                                      ctypes.c_int64, dp, dp]
        _lib.orc_elements.restype = ctypes.c_int
        _lib.orc_elements_implicit.argtypes = [ctypes.POINTER(_CParams), dp, ctypes.POINTER(ctypes.c_int32),
                                               ctypes.POINTER(ctypes.c_int64), ctypes.c_int64, dp, dp, dp, dp,
                                               ctypes.c_int64, ctypes.c_double, dp, dp]
        _lib.orc_elements_implicit.restype = ctypes.c_int
        _lib.orc_qp_coefficients.argtypes = [ctypes.POINTER(_CParams), dp, dp, dp, dp, dp, dp,
                                             ctypes.c_int, dp]
        _lib.orc_qp_coefficients.restype = ctypes.c_int
        _lib.orc_set_threads.argtypes = [ctypes.c_int]
        _lib.orc_set_threads.restype = ctypes.c_int
        _lib.orc_set_threads(1)          # one thread unless a caller asks for more
    return _lib


def set_threads(n: int) -> int:
    """Threads of the C element loops (results do not depend on it); returns the count in use."""
    return int(load_library().orc_set_threads(int(n)))


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ----------------------------------------------------------------------------------------
# problem description
# ----------------------------------------------------------------------------------------
@dataclasses.dataclass
class Params:
    """Physical and numerical parameters of one step (Sections 2.1-2.3)."""
    rho: float = 1.0
    mu: float = 1.0
    dt: float = 1e-3
    bdf_order: int = 1
    c_r: float = 30.0              # C_r of tau_M; the paper does not print it (reading: 60*2^(r-2), r=1)
    f: Sequence[float] = (0.0, 0.0, 0.0)
    stab: int = 2                  # 0 none, 1 SUPG-PSPG, 2 VMS-LES
    diffusion: int = 0             # 0 grad-grad, 1 symgrad-grad, 2 symgrad-symgrad

    def c_struct(self, riis: Sequence["RIIS"] = ()) -> _CParams:
        alpha = bdf_coefficients(self.bdf_order)[0]
        s = _CParams()
        s.rho, s.mu, s.dt, s.alpha, s.sigma, s.c_r = (self.rho, self.mu, self.dt, alpha,
                                                      float(self.bdf_order), self.c_r)
        for i in range(3):
            s.f[i] = self.f[i]
        s.n_riis, s.stab, s.diffusion = len(riis), self.stab, self.diffusion
        for k, r in enumerate(riis):
            s.riis_r[k], s.riis_eps[k] = r.resistance, r.eps
        return s


@dataclasses.dataclass
class BC:
    """Boundary condition on one tag (Section 2.2).

    kind: 'noslip' | 'dirichlet' (g = theta g(t) s(x)) | 'nodal' (values given per step) |
          'neumann' (sigma n = -h(t) n, plus beta rho/2 |u . n|_- u when beta > 0) |
          'resistance' (sigma n = -(p_0(t) + resistance * int u . n) n, p_0 from time/tparams).
    time: 'constant' {value} | 'pulsatile' {gmin, gmax, period} | 'ramp' {g0, g1, t0, tL} |
          'fourier' {period, a (cosine coefficients a_0..a_K), b (sine coefficients, b_0 unused)}.
    space: 'parabolic' {radius} | 'uniform' | 'womersley' {radius; time must be 'fourier'}.
    """
    tag: int
    kind: str
    time: str = "constant"
    tparams: dict = dataclasses.field(default_factory=lambda: {"value": 0.0})
    space: str = "uniform"
    radius: float = 1.0
    theta: float = 1.0
    beta: float = 0.0              # inertial backflow stabilisation on a Neumann tag (0: off)
    resistance: float = 0.0        # C_R of a resistance tag


@dataclasses.dataclass
class RIIS:
    """Static resistive immersed surface (Eq. riis) with u_Sigma = 0; its signed distance is
    given at the nodes and interpolated linearly inside each element."""
    resistance: float
    eps: float
    phi_nodal: np.ndarray


@dataclasses.dataclass
class Problem:
    params: Params
    bcs: list
    riis: list = dataclasses.field(default_factory=list)
    pin_node: int = -1             # pressure DoF fixed when every boundary is Dirichlet


def disk_sdf(X, center, normal, radius):
    """Signed distance to a flat open disk: the plane distance inside the rim radius, else the
    distance to the rim circle signed by the side of the plane (the disk-valve reading)."""
    X = np.asarray(X, dtype=np.float64)
    n = np.asarray(normal, dtype=np.float64)
    n = n / np.linalg.norm(n)
    d = X - np.asarray(center, dtype=np.float64)
    h = d @ n
    rad = np.linalg.norm(d - np.outer(h, n), axis=1)
    out = np.abs(h).copy()
    o = rad > radius
    out[o] = np.hypot(rad[o] - radius, h[o])
    return np.where(h >= 0, out, -out)


# ----------------------------------------------------------------------------------------
# Eq. (bdf): coefficients
# ----------------------------------------------------------------------------------------
def bdf_coefficients(order: int):
    """(alpha, beta, gamma): (alpha u^{n+1} - sum beta_j u^{n-j})/dt approximates du/dt at t^{n+1}
    to order sigma; sum gamma_j u^{n-j} extrapolates u^{n+1} to order sigma."""
    if order == 1:
        return 1.0, (1.0,), (1.0,)
    if order == 2:
        return 1.5, (2.0, -0.5), (2.0, -1.0)
    if order == 3:
        return 11.0 / 6.0, (3.0, -1.5, 1.0 / 3.0), (3.0, -3.0, 1.0)
    raise ValueError("BDF order must be 1, 2 or 3")


# ----------------------------------------------------------------------------------------
# element-level wrappers around the C routines
# ----------------------------------------------------------------------------------------
def geometry(x):
    """Returns (det J, grad phi [4,3], G [3,3], g [3], |K|) for the vertices x [4,3]."""
    lib = load_library()
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(12)
    gp, G, g, v = np.zeros(12), np.zeros(9), np.zeros(3), np.zeros(1)
    det = lib.orc_geometry(_dp(x), _dp(gp), _dp(G), _dp(g), _dp(v))
    return det, gp.reshape(4, 3), G.reshape(3, 3), g, float(v[0])


def tau(params: Params, G, g, us, deltas=(), riis=()):
    lib = load_library()
    cp = params.c_struct(riis)
    G = np.ascontiguousarray(G, dtype=np.float64).reshape(9)
    g = np.ascontiguousarray(g, dtype=np.float64)
    us = np.ascontiguousarray(us, dtype=np.float64)
    de = np.zeros(MAX_RIIS)
    de[:len(deltas)] = deltas
    tm, tc = np.zeros(1), np.zeros(1)
    lib.orc_tau(ctypes.byref(cp), _dp(G), _dp(g), _dp(us), _dp(de), _dp(tm), _dp(tc))
    return float(tm[0]), float(tc[0])


def _opt(a, size):
    return None if a is None else _dp(np.ascontiguousarray(a, dtype=np.float64).reshape(size))


def element(params: Params, x, ubdf, uext, pext, phinod=None, riis=(), uale=None):
    """Element matrix [16,16] and right-hand side [16] (local unknown 4a+c); uale [4][3] is the
    mesh velocity at the vertices (None: fixed mesh)."""
    lib = load_library()
    cp = params.c_struct(riis)
    args = [np.ascontiguousarray(a, dtype=np.float64).ravel() for a in (x, ubdf, uext, pext)]
    ph = np.zeros(4 * MAX_RIIS) if phinod is None else np.ascontiguousarray(phinod, dtype=np.float64).ravel()
    A, b = np.zeros(256), np.zeros(16)
    rc = lib.orc_element(ctypes.byref(cp), *[_dp(a) for a in args], _dp(ph), _opt(uale, 12), _dp(A), _dp(b))
    if rc != 0:
        raise ValueError("degenerate or inverted element")
    return A.reshape(16, 16), b


def qp_coefficients(params: Params, x, ubdf, uext, pext, q, phinod=None, riis=(), uale=None):
    """The coefficients of quadrature point q (0..3) of one element, as the element routines use
    them: dict with tau_m, tau_c, s = tau_M r_M(u^EXT, p^EXT) [3] (the LES factor), us = u* [3],
    sR = sum_k (R_k/eps_k) delta_k, m = rho u^BDF/dt + f [3], w = quadrature weight."""
    lib = load_library()
    cp = params.c_struct(riis)
    args = [np.ascontiguousarray(a, dtype=np.float64).ravel() for a in (x, ubdf, uext, pext)]
    ph = np.zeros(4 * MAX_RIIS) if phinod is None else np.ascontiguousarray(phinod, dtype=np.float64).ravel()
    out = np.zeros(13)
    rc = lib.orc_qp_coefficients(ctypes.byref(cp), *[_dp(a) for a in args], _dp(ph), _opt(uale, 12), int(q),
                                 _dp(out))
    if rc != 0:
        raise ValueError("degenerate or inverted element, or q outside 0..3")
    return {"tau_m": out[0], "tau_c": out[1], "s": out[2:5].copy(), "us": out[5:8].copy(), "sR": out[8],
            "m": out[9:12].copy(), "w": out[12]}


def element_residual(params: Params, x, ubdf, uext, pext, sol, phinod=None, riis=(), uale=None):
    lib = load_library()
    cp = params.c_struct(riis)
    args = [np.ascontiguousarray(a, dtype=np.float64).ravel() for a in (x, ubdf, uext, pext)]
    ph = np.zeros(4 * MAX_RIIS) if phinod is None else np.ascontiguousarray(phinod, dtype=np.float64).ravel()
    sol = np.ascontiguousarray(sol, dtype=np.float64).ravel()
    R = np.zeros(16)
    rc = lib.orc_element_residual(ctypes.byref(cp), *[_dp(a) for a in args], _dp(ph), _opt(uale, 12), _dp(sol),
                                  _dp(R))
    if rc != 0:
        raise ValueError("degenerate or inverted element")
    return R


def _riis_nodal(problem_riis, V):
    if not problem_riis:
        return np.zeros((1, V))
    return np.ascontiguousarray(np.stack([np.asarray(r.phi_nodal, dtype=np.float64) for r in problem_riis]))


def element_batch(params, nodes, tets, elems, ubdf, uext, pext, riis=(), uale=None):
    """Element matrices [n,16,16] and right-hand sides [n,16] for the listed elements."""
    lib = load_library()
    cp = params.c_struct(riis)
    V = nodes.shape[0]
    elems = np.ascontiguousarray(elems, dtype=np.int64)
    n = elems.size
    A, b = np.zeros((n, 256)), np.zeros((n, 16))
    ph = _riis_nodal(riis, V)
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    rc = lib.orc_elements(ctypes.byref(cp), _dp(np.ascontiguousarray(nodes, dtype=np.float64)),
                          tets.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                          elems.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), n,
                          _dp(np.ascontiguousarray(ubdf, dtype=np.float64)),
                          _dp(np.ascontiguousarray(uext, dtype=np.float64)),
                          _dp(np.ascontiguousarray(pext, dtype=np.float64)), _dp(ph), _opt(uale, 3 * V), V,
                          _dp(A), _dp(b))
    if rc != 0:
        raise ValueError(f"degenerate element at batch position {-1 - rc}")
    return A.reshape(n, 16, 16), b


# ----------------------------------------------------------------------------------------
# global assembly (scalar CSR, 4 unknowns per node, interleaved)
# ----------------------------------------------------------------------------------------
def assemble(params: Params, nodes, tets, ubdf, uext, pext, riis=(), chunk: int = 65536, uale=None):
    """Sum of element contributions: returns (A csr [4V,4V], b [4V]); uale [V,3] is the mesh
    velocity (None: fixed mesh)."""
    V, T = nodes.shape[0], tets.shape[0]
    N = 4 * V
    A = sp.csr_matrix((N, N))
    b = np.zeros(N)
    for s in range(0, T, chunk):
        e = np.arange(s, min(T, s + chunk))
        Ae, be = element_batch(params, nodes, tets, e, ubdf, uext, pext, riis, uale)
        dof = (4 * tets[e].astype(np.int64)[:, :, None] + np.arange(4)[None, None, :]).reshape(-1, 16)
        rows = np.broadcast_to(dof[:, :, None], Ae.shape).ravel()
        cols = np.broadcast_to(dof[:, None, :], Ae.shape).ravel()
        A = A + sp.coo_matrix((Ae.ravel(), (rows, cols)), shape=(N, N)).tocsr()
        np.add.at(b, dof.ravel(), be.ravel())
    A.sum_duplicates()
    A.sort_indices()
    return A, b


def block_of(A: sp.csr_matrix, a: int, b: int) -> np.ndarray:
    """The 4x4 block (node a, node b) of a scalar CSR matrix with interleaved unknowns."""
    return A[4 * a:4 * a + 4, 4 * b:4 * b + 4].toarray()


# ----------------------------------------------------------------------------------------
# boundary data (Section 2.2)
# ----------------------------------------------------------------------------------------
def time_law(kind: str, t: float, tp: dict) -> float:
    """g(t) of Section 2.2.1: constant, pulsatile, sinusoidal ramp, Fourier series."""
    if kind == "constant":
        return float(tp["value"])
    if kind == "pulsatile":
        return tp["gmin"] + (tp["gmax"] - tp["gmin"]) * 0.5 * (1.0 - math.cos(2.0 * math.pi * t / tp["period"]))
    if kind == "ramp":
        if t < tp["t0"]:
            return float(tp["g0"])
        if t < tp["t0"] + tp["tL"]:
            return tp["g0"] + 0.5 * (tp["g1"] - tp["g0"]) * (1.0 - math.cos(math.pi * (t - tp["t0"]) / tp["tL"]))
        return float(tp["g1"])
    if kind == "fourier":
        w = 2.0 * math.pi / tp["period"]
        a, bcoef = tp["a"], tp.get("b", [0.0] * len(tp["a"]))
        return float(a[0] + sum(a[k] * math.cos(k * w * t) + bcoef[k] * math.sin(k * w * t)
                                for k in range(1, len(a))))
    raise ValueError(kind)


def womersley_profile(r, radius, omega, nu):
    """Unit-flow-rate Womersley shape for angular frequency omega > 0 (Section 2.2.1, the
    inverse problem of [berselli2013exact] for one Fourier harmonic): the axial velocity
    W(r) = (1 - J0(i^{3/2} a r/R) / J0(i^{3/2} a)) / Q with a = R sqrt(omega/nu) and
    Q = pi R^2 (1 - 2 J1(z) / (z J0(z))), z = i^{3/2} a, so that the flux of W over the disk is 1.
    Returns complex W at radii r."""
    from scipy.special import jv

    z = np.exp(0.75j * np.pi) * radius * math.sqrt(omega / nu)
    shape = 1.0 - jv(0, z * np.asarray(r) / radius) / jv(0, z)
    flux = math.pi * radius ** 2 * (1.0 - 2.0 * jv(1, z) / (z * jv(0, z)))
    return shape / flux


def boundary_geometry(nodes, bfaces, btags, tag):
    """(barycentre, unit outward normal, area) of the faces with this tag, area weighted."""
    f = bfaces[btags == tag]
    x = nodes[f]
    cr = np.cross(x[:, 1] - x[:, 0], x[:, 2] - x[:, 0])
    area = 0.5 * np.linalg.norm(cr, axis=1)
    cen = (x.mean(axis=1) * area[:, None]).sum(axis=0) / area.sum()
    n = cr.sum(axis=0)
    return cen, n / np.linalg.norm(n), float(area.sum())


def dirichlet_data(mesh, problem: Problem, t: float, nodal: Optional[dict] = None):
    """Constrained velocity values at t: returns (nodes [k], values [k,3]) with the precedence
    no-slip > other Dirichlet (Section 2.2.1)."""
    V = mesh.nodes.shape[0]
    val = np.zeros((V, 3))
    pri = np.zeros(V, dtype=np.int8)
    for bc in problem.bcs:
        ids = np.unique(mesh.bfaces[mesh.btags == bc.tag].ravel())
        if bc.kind == "noslip":
            val[ids] = 0.0
            pri[ids] = 3
        elif bc.kind in ("dirichlet", "nodal"):
            sel = ids[pri[ids] < 2]
            if bc.kind == "nodal":
                vv = nodal[bc.tag]            # [V,3] full-size array of values for this tag
                val[sel] = vv[sel]
            else:
                cen, n, _ = boundary_geometry(mesh.nodes, mesh.bfaces, mesh.btags, bc.tag)
                g = bc.theta * time_law(bc.time, t, bc.tparams)
                if bc.space == "parabolic":
                    R = bc.radius
                    r2 = np.sum((mesh.nodes[sel] - cen) ** 2, axis=1)
                    s = -2.0 * (R * R - r2)[:, None] / (math.pi * R ** 4) * n[None, :]
                elif bc.space == "uniform":
                    s = -np.broadcast_to(n, (sel.size, 3))
                elif bc.space == "womersley":
                    # u = -n [a_0 W_0(r) + sum_k Re((a_k - i b_k) W_k(r) e^{i k w t})], W_0 parabolic
                    tp, R = bc.tparams, bc.radius
                    w = 2.0 * math.pi / tp["period"]
                    r = np.sqrt(np.sum((mesh.nodes[sel] - cen) ** 2, axis=1))
                    a, bb = tp["a"], tp.get("b", [0.0] * len(tp["a"]))
                    amp = a[0] * 2.0 * (R * R - r * r) / (math.pi * R ** 4)
                    for k in range(1, len(a)):
                        W = womersley_profile(r, R, k * w, problem.params.mu / problem.params.rho)
                        amp = amp + np.real((a[k] - 1j * bb[k]) * W * np.exp(1j * k * w * t))
                    val[sel] = -bc.theta * amp[:, None] * n[None, :]
                    pri[sel] = 2
                    continue
                else:
                    raise ValueError(bc.space)
                val[sel] = g * s
            pri[sel] = 2
    ids = np.nonzero(pri >= 2)[0]
    return ids, val[ids]


def neumann_rhs(mesh, problem: Problem, t: float) -> np.ndarray:
    """-(h(t) n, v) on Neumann faces, P1: each vertex gets A_f/3 of the face integral."""
    V = mesh.nodes.shape[0]
    r = np.zeros(4 * V)
    for bc in problem.bcs:
        if bc.kind != "neumann":
            continue
        h = time_law(bc.time, t, bc.tparams)
        if h == 0.0:
            continue
        f = mesh.bfaces[mesh.btags == bc.tag]
        x = mesh.nodes[f]
        cr = 0.5 * np.cross(x[:, 1] - x[:, 0], x[:, 2] - x[:, 0])   # area * outward unit normal
        for k in range(3):
            for i in range(3):
                np.add.at(r, 4 * f[:, k].astype(np.int64) + i, -h * cr[:, i] / 3.0)
    return r


def _face_area_vectors(nodes, faces):
    x = nodes[faces]
    return 0.5 * np.cross(x[:, 1] - x[:, 0], x[:, 2] - x[:, 0])    # A_f n_f per face


def backflow_matrix(mesh, problem: Problem, uext: np.ndarray) -> sp.csr_matrix:
    """Inertial backflow stabilisation on the Neumann tags with beta > 0 (Section 2.2.2):
    c(x) (u, v)_Gamma, c = -beta rho/2 min(u* . n, 0), edge-midpoint rule on each face."""
    V = mesh.nodes.shape[0]
    rows, cols, vals = [], [], []
    rho = problem.params.rho
    for bc in problem.bcs:
        if bc.kind != "neumann" or bc.beta <= 0.0:
            continue
        f = mesh.bfaces[mesh.btags == bc.tag].astype(np.int64)
        an = _face_area_vectors(mesh.nodes, f)
        area = np.linalg.norm(an, axis=1)
        n = an / area[:, None]
        for (i, j) in ((0, 1), (1, 2), (0, 2)):
            um = 0.5 * (uext[f[:, i]] + uext[f[:, j]])               # u* at the edge midpoint
            c = -bc.beta * rho / 2.0 * np.minimum(np.sum(um * n, axis=1), 0.0) * area / 3.0
            # phi = 1/2 at the edge's two vertices, 0 at the third
            for a in (i, j):
                for b in (i, j):
                    for comp in range(3):
                        rows.append(4 * f[:, a] + comp)
                        cols.append(4 * f[:, b] + comp)
                        vals.append(0.25 * c)
    if not rows:
        return sp.csr_matrix((4 * V, 4 * V))
    return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(4 * V, 4 * V)).tocsr()


def resistance_vectors(mesh, tag) -> np.ndarray:
    """w with w_{4a+i} = int_Gamma phi_a n_i over the faces of the tag (P1: A_f n_f / 3 per vertex)."""
    V = mesh.nodes.shape[0]
    f = mesh.bfaces[mesh.btags == tag].astype(np.int64)
    an = _face_area_vectors(mesh.nodes, f)
    w = np.zeros(4 * V)
    for k in range(3):
        for i in range(3):
            np.add.at(w, 4 * f[:, k] + i, an[:, i] / 3.0)
    return w


def resistance_terms(mesh, problem: Problem, t: float):
    """Resistance tags (Section 2.2.3): the rank-one matrices C_R w w^T (as a list of (C_R, w))
    and the right-hand side -p_0(t) w summed over the tags."""
    V = mesh.nodes.shape[0]
    terms, r = [], np.zeros(4 * V)
    for bc in problem.bcs:
        if bc.kind != "resistance":
            continue
        w = resistance_vectors(mesh, bc.tag)
        terms.append((bc.resistance, w))
        r -= time_law(bc.time, t, bc.tparams) * w
    return terms, r


def lifting(mesh, nodes_fixed, values, alpha=None):
    """Domain displacement by harmonic extension (Eq. lifting with sigma^L = grad d): P1 solution
    of -div(alpha grad d) = 0 in the reference domain, component by component, with d = values at
    nodes_fixed and zero normal flux elsewhere.  alpha [T] per element (None: 1).  Returns [V,3]."""
    X, tets = mesh.nodes, mesh.tets.astype(np.int64)
    V, T = X.shape[0], tets.shape[0]
    x = X[tets]                                                       # [T,4,3]
    J = np.stack([x[:, 1] - x[:, 0], x[:, 2] - x[:, 0], x[:, 3] - x[:, 0]], axis=2)   # columns
    vol = np.abs(np.linalg.det(J)) / 6.0
    Jinv = np.linalg.inv(J)                                           # rows: gradients of lambda_1..3
    g = np.concatenate([-Jinv.sum(axis=1, keepdims=True), Jinv], axis=1)   # [T,4,3] grad phi_a
    a = np.ones(T) if alpha is None else np.asarray(alpha, dtype=np.float64)
    Ke = (a * vol)[:, None, None] * np.einsum("tai,tbi->tab", g, g)
    rows = np.broadcast_to(tets[:, :, None], Ke.shape).ravel()
    cols = np.broadcast_to(tets[:, None, :], Ke.shape).ravel()
    K = sp.coo_matrix((Ke.ravel(), (rows, cols)), shape=(V, V)).tocsr()
    fixed = np.asarray(nodes_fixed, dtype=np.int64)
    free = np.setdiff1d(np.arange(V), fixed)
    d = np.zeros((V, 3))
    d[fixed] = values
    Kff = K[free][:, free].tocsc()
    rhs = -K[free][:, fixed] @ d[fixed]
    d[free] = np.column_stack([spla.spsolve(Kff, rhs[:, k]) for k in range(3)])
    return d


def ale_velocity(order: int, d_hist, dt: float):
    """Mesh velocity u_ALE^{n+1} = (alpha d^{n+1} - sum_j beta_j d^{n-j}) / dt, the BDF derivative of
    the displacement (Section 2.3), from d_hist = [d^{n+1}, d^n, d^{n-1}, ...] (order + 1 levels)."""
    alpha, beta, _ = bdf_coefficients(order)
    return (alpha * d_hist[0] - sum(beta[j] * d_hist[j + 1] for j in range(order))) / dt


def apply_dirichlet(A: sp.csr_matrix, b: np.ndarray, rows, values):
    """Replace each constrained row r by s e_r and b_r by s g_r, s = |A_rr| (1 if zero)."""
    A = A.tocsr(copy=True)
    A.sort_indices()
    b = b.copy()
    rows = np.asarray(rows, dtype=np.int64)
    values = np.asarray(values, dtype=np.float64)
    diag = A.diagonal()
    s = np.abs(diag[rows])
    s[s == 0.0] = 1.0
    N = A.shape[0]
    is_c = np.zeros(N, dtype=bool)
    is_c[rows] = True
    scale = np.zeros(N)
    scale[rows] = s
    r_of = np.repeat(np.arange(N), np.diff(A.indptr))
    hit = is_c[r_of]
    A.data[hit] = 0.0
    on_diag = hit & (A.indices == r_of)
    A.data[on_diag] = scale[r_of[on_diag]]
    missing = rows[~np.isin(rows, r_of[on_diag])]
    if missing.size:
        A = A + sp.coo_matrix((scale[missing], (missing, missing)), shape=A.shape).tocsr()
    b[rows] = s * values
    return A, b


def solve_direct(A, b):
    """Sparse LU (SuperLU) of the assembled system."""
    return spla.spsolve(A.tocsc(), b)


@dataclasses.dataclass
class Step:
    A: sp.csr_matrix          # after Dirichlet rows
    b: np.ndarray
    x: np.ndarray             # solution [4V]
    ubdf: np.ndarray
    uext: np.ndarray
    pext: np.ndarray


def step(mesh, problem: Problem, u_hist: Sequence[np.ndarray], p_hist: Sequence[np.ndarray],
         t_next: float, nodal: Optional[dict] = None, pin_value: float = 0.0,
         solver: Optional[Callable] = None, d_hist: Optional[Sequence[np.ndarray]] = None) -> Step:
    """One semi-implicit BDF step from t^n to t^{n+1} = t_next (Eq. fullydiscrete...).
    u_hist = [u^n, u^{n-1}, ...] ([V,3] each), p_hist likewise ([V]).  On a moving domain (ALE),
    d_hist = [d^{n+1}, d^n, ...] (order + 1 levels of nodal displacement from the reference mesh,
    e.g. from ``lifting``): the step is assembled on the configuration x^ + d^{n+1} with
    u* = u^EXT - u_ALE, u_ALE the BDF derivative of d (Eq. u_star, semi-implicit form)."""
    prm = problem.params
    alpha, beta, gamma = bdf_coefficients(prm.bdf_order)
    s = prm.bdf_order
    ubdf = sum(beta[j] * u_hist[j] for j in range(s))
    uext = sum(gamma[j] * u_hist[j] for j in range(s))
    pext = sum(gamma[j] * p_hist[j] for j in range(s))
    uale = None
    if d_hist is not None:
        uale = ale_velocity(s, d_hist, prm.dt)
        mesh = dataclasses.replace(mesh, nodes=mesh.nodes + d_hist[0])
    A, b = assemble(prm, mesh.nodes, mesh.tets, ubdf, uext, pext, problem.riis, uale=uale)
    b = b + neumann_rhs(mesh, problem, t_next)
    A = A + backflow_matrix(mesh, problem, uext)
    terms, rres = resistance_terms(mesh, problem, t_next)
    b = b + rres
    for cr, w in terms:                      # rank-one: dense over the tag's velocity DoFs
        nz = np.nonzero(w)[0]
        A = A + sp.coo_matrix((cr * np.outer(w[nz], w[nz]).ravel(),
                               (np.repeat(nz, nz.size), np.tile(nz, nz.size))), shape=A.shape).tocsr()
    ids, vals = dirichlet_data(mesh, problem, t_next, nodal)
    rows = (4 * ids[:, None] + np.arange(3)[None, :]).ravel()
    rv = vals.ravel()
    if problem.pin_node >= 0:
        rows = np.concatenate([rows, [4 * problem.pin_node + 3]])
        rv = np.concatenate([rv, [pin_value]])
    A, b = apply_dirichlet(A, b, rows, rv)
    x = (solver or solve_direct)(A, b)
    return Step(A, b, x, ubdf, uext, pext)


@dataclasses.dataclass
class ImplicitStep:
    x: np.ndarray             # solution [4V]
    residuals: list           # ||F|| before each Newton update and at the end
    scale: float              # ||b|| of the semi-implicit system at the same step (the tolerance's unit)


def implicit_step(mesh, problem: Problem, u_hist: Sequence[np.ndarray], p_hist: Sequence[np.ndarray],
                  t_next: float, nodal: Optional[dict] = None, pin_value: float = 0.0,
                  d_hist: Optional[Sequence[np.ndarray]] = None, tol: float = 1e-11, max_newton: int = 20,
                  h: float = 1e-6) -> ImplicitStep:
    """One step of the fully implicit formulation (Eq. u_star implicit, implicit LES term; Section
    2.4: linearised by Newton's method).  F(U) = sum_e R_e(U) - Neumann data, R_e the element
    residual with u* = u - u_ALE, tau_M(u*) and r_M(u, p) taken at U itself; Dirichlet rows
    F_r = s (U_r - g_r).  Newton from the semi-implicit solution, with element Jacobians by central
    differences of step h (the element residual depends only on the element's 16 unknowns), until
    ||F|| <= tol ||b_semi||.  Backflow stabilisation and resistance conditions are not included."""
    for bc in problem.bcs:
        if bc.kind == "resistance" or (bc.kind == "neumann" and bc.beta > 0.0):
            raise NotImplementedError("implicit_step: backflow or resistance conditions")
    prm = problem.params
    sgm = prm.bdf_order
    alpha, beta, gamma = bdf_coefficients(sgm)
    ubdf = sum(beta[j] * u_hist[j] for j in range(sgm))
    semi = step(mesh, problem, u_hist, p_hist, t_next, nodal, pin_value, d_hist=d_hist)
    U = semi.x.copy()
    uale = None
    if d_hist is not None:
        uale = ale_velocity(sgm, d_hist, prm.dt)
        mesh = dataclasses.replace(mesh, nodes=mesh.nodes + d_hist[0])
    V, T = mesh.nodes.shape[0], mesh.tets.shape[0]
    N = 4 * V
    bN = neumann_rhs(mesh, problem, t_next)
    ids, vals = dirichlet_data(mesh, problem, t_next, nodal)
    rows = (4 * ids[:, None] + np.arange(3)[None, :]).ravel()
    rv = vals.ravel()
    if problem.pin_node >= 0:
        rows = np.concatenate([rows, [4 * problem.pin_node + 3]])
        rv = np.concatenate([rv, [pin_value]])
    free = np.ones(N, dtype=bool)
    free[rows] = False
    scale = float(np.linalg.norm(semi.b))
    norms = []
    for it in range(max_newton + 1):
        Jg, F = _implicit_system(mesh, problem, ubdf, U, uale, h)
        F -= bN
        norm = float(np.sqrt(np.sum(F[free] ** 2) + np.sum((U[rows] - rv) ** 2)))
        norms.append(norm)
        if norm <= tol * scale or it == max_newton:
            break
        A, rhs = apply_dirichlet(Jg, -F, rows, rv - U[rows])
        U = U + solve_direct(A, rhs)
    return ImplicitStep(U, norms, scale)


def _implicit_system(mesh, problem: Problem, ubdf, U, uale=None, h: float = 1e-6):
    """Sum over the elements of the implicit element residuals R_e(U) and of their Jacobians by
    central differences of step h: (J csr [4V,4V], F [4V]), without boundary data."""
    prm = problem.params
    V, T = mesh.nodes.shape[0], mesh.tets.shape[0]
    N = 4 * V
    lib = load_library()
    cp = prm.c_struct(problem.riis)
    ph = _riis_nodal(problem.riis, V)
    tets = np.ascontiguousarray(mesh.tets, dtype=np.int32)
    elems = np.arange(T, dtype=np.int64)
    nodes = np.ascontiguousarray(mesh.nodes, dtype=np.float64)
    dof = (4 * tets.astype(np.int64)[:, :, None] + np.arange(4)[None, None, :]).reshape(-1, 16)
    jr = np.broadcast_to(dof[:, :, None], (T, 16, 16)).ravel()
    jc = np.broadcast_to(dof[:, None, :], (T, 16, 16)).ravel()
    Je, Re = np.zeros(T * 256), np.zeros(T * 16)
    rc = lib.orc_elements_implicit(ctypes.byref(cp), _dp(nodes), tets.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                   elems.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), T,
                                   _dp(np.ascontiguousarray(ubdf, dtype=np.float64)),
                                   _dp(np.ascontiguousarray(U, dtype=np.float64)), _dp(ph),
                                   _opt(uale, 3 * V), V, h, _dp(Je), _dp(Re))
    if rc != 0:
        raise ValueError(f"degenerate element at position {-1 - rc}")
    F = np.zeros(N)
    np.add.at(F, dof.ravel(), Re)
    return sp.coo_matrix((Je, (jr, jc)), shape=(N, N)).tocsr(), F


def implicit_system(mesh, problem: Problem, u_hist: Sequence[np.ndarray], t_next: float, U, h: float = 1e-6):
    """The Newton system of the fully implicit formulation at the iterate U [4V] on a fixed mesh:
    (J, F) with J the sum of the element Jacobians (central differences of step h) and
    F = sum_e R_e(U) - Neumann data at t_next, before Dirichlet rows."""
    prm = problem.params
    _, beta, _ = bdf_coefficients(prm.bdf_order)
    ubdf = sum(beta[j] * u_hist[j] for j in range(prm.bdf_order))
    J, F = _implicit_system(mesh, problem, ubdf, np.ascontiguousarray(U, dtype=np.float64).ravel(), None, h)
    return J, F - neumann_rhs(mesh, problem, t_next)


# ----------------------------------------------------------------------------------------
# Eq. (errors): relative L2 / H1-seminorm errors against a closed-form solution
# ----------------------------------------------------------------------------------------
def relative_errors(nodes, tets, u, p, u_ex: Callable, gradu_ex: Callable, p_ex: Callable,
                    p_mean_free: bool = False):
    """Relative errors e_L2^u, e_H1^u, e_L2^p of Eq. (errors) with the 4-point rule.
    p_mean_free compares p - mean(p) with p_ex - mean(p_ex) (pressure defined up to a constant)."""
    qa, qb = 0.5854101966249685, 0.1381966011250105
    x = nodes[tets]                                     # [T,4,3]
    J = np.stack([x[:, 1] - x[:, 0], x[:, 2] - x[:, 0], x[:, 3] - x[:, 0]], axis=2)  # [T,3,3]
    det = np.linalg.det(J)
    Ji = np.linalg.inv(J)
    gh = np.array([[-1, -1, -1], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]])
    gphi = np.einsum("tmk,am->tak", Ji, gh)             # grad phi_a [T,4,3]
    gu = np.einsum("tai,taj->tij", u[tets], gphi)       # grad u_h [T,3,3]
    w = det / 24.0
    eu = nu = eg = ng = ep = npn = 0.0
    pts, ph_vals, pex_vals, ws = [], [], [], []
    for q in range(4):
        lam = np.full(4, qb)
        lam[q] = qa
        xq = np.einsum("a,tai->ti", lam, x)
        uh = np.einsum("a,tai->ti", lam, u[tets])
        ue = u_ex(xq)
        ge = gradu_ex(xq)
        eu += np.sum(w * np.sum((uh - ue) ** 2, axis=1))
        nu += np.sum(w * np.sum(ue ** 2, axis=1))
        eg += np.sum(w * np.sum((gu - ge) ** 2, axis=(1, 2)))
        ng += np.sum(w * np.sum(ge ** 2, axis=(1, 2)))
        ph_vals.append(np.einsum("a,ta->t", lam, p[tets]))
        pex_vals.append(p_ex(xq))
        ws.append(w)
    ph_vals, pex_vals, ws = np.stack(ph_vals), np.stack(pex_vals), np.stack(ws)
    if p_mean_free:
        vol = ws.sum()
        ph_vals = ph_vals - (ws * ph_vals).sum() / vol
        pex_vals = pex_vals - (ws * pex_vals).sum() / vol
    ep = np.sum(ws * (ph_vals - pex_vals) ** 2)
    npn = np.sum(ws * pex_vals ** 2)
    return math.sqrt(eu / nu), math.sqrt(eg / ng), math.sqrt(ep / npn)
