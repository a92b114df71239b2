"""Thin ctypes binding of liblfx (include/lfx.h): the same entry points under the same names,
argument marshalling only.  Every step of the computation runs in the library's CUDA kernels;
there is no Python or CPU fallback: if the library is missing, importing the handles raises.

PyTorch is used only as plumbing: its CUDA caching allocator can back the library's device
allocations (``use_torch_allocator``) and its current stream can be handed to a state.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblfx.so")
_lib = None

# ----------------------------------------------------------------------------- C structs
MAX_FOURIER = 16
(LFX_OK, LFX_ERR_INVALID_ARG, LFX_ERR_BAD_MESH, LFX_ERR_OOM, LFX_ERR_NOT_CONVERGED,
 LFX_ERR_NONFINITE, LFX_ERR_CUDA, LFX_ERR_TIMEOUT, LFX_ERR_BUDGET) = (0, -1, -2, -3, -4, -5, -6, -7, -8)
TIME = {"constant": 0, "pulsatile": 1, "ramp": 2, "fourier": 3}
KIND = {"noslip": 0, "dirichlet": 1, "nodal": 2, "neumann": 3, "resistance": 4}
PROFILE = {"uniform": 0, "parabolic": 1, "womersley": 2}
PREC = {"fp64": 0, "mixed": 1}
ASM = {"auto": 0, "colors": 1, "chunks": 2, "persistent": 3}
SMOOTH = {"jacobi": 0, "chebyshev": 1, "amg": 2}


class lfx_time_law(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("n_harmonics", ctypes.c_int32), ("p", ctypes.c_double * 4),
                ("a", ctypes.c_double * (MAX_FOURIER + 1)), ("b", ctypes.c_double * (MAX_FOURIER + 1))]


class lfx_bc(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_int32), ("kind", ctypes.c_int32), ("profile", ctypes.c_int32),
                ("given_geometry", ctypes.c_int32), ("time", lfx_time_law), ("theta", ctypes.c_double),
                ("radius", ctypes.c_double), ("center", ctypes.c_double * 3), ("normal", ctypes.c_double * 3),
                ("beta", ctypes.c_double), ("resistance", ctypes.c_double)]


class lfx_riis(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("pad", ctypes.c_int32), ("resistance", ctypes.c_double),
                ("eps", ctypes.c_double), ("center", ctypes.c_double * 3), ("normal", ctypes.c_double * 3),
                ("radius", ctypes.c_double), ("sdf_nodal", ctypes.POINTER(ctypes.c_double))]


class lfx_options(ctypes.Structure):
    _fields_ = [("stab", ctypes.c_int32), ("diffusion", ctypes.c_int32), ("c_r", ctypes.c_double),
                ("f", ctypes.c_double * 3), ("pin_pressure_node", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("gmres_restart", ctypes.c_int32), ("gmres_max_iters", ctypes.c_int32),
                ("gmres_rtol", ctypes.c_double), ("reorthogonalize", ctypes.c_int32),
                ("f_smoother", ctypes.c_int32), ("f_steps", ctypes.c_int32),
                ("f_omega", ctypes.c_double), ("f_ratio", ctypes.c_double),
                ("s_smoother", ctypes.c_int32), ("s_steps", ctypes.c_int32),
                ("s_omega", ctypes.c_double), ("s_ratio", ctypes.c_double), ("n_power", ctypes.c_int32),
                ("smoother_bf16", ctypes.c_int32), ("outer_restart", ctypes.c_int32),
                ("outer_max_iters", ctypes.c_int32), ("inner_rtol", ctypes.c_double),
                ("inner_max_iters", ctypes.c_int32), ("bad_element_quality", ctypes.c_double),
                ("amg_refresh", ctypes.c_int32), ("amg_coarse_size", ctypes.c_int32),
                ("amg_theta", ctypes.c_double), ("amg_alpha", ctypes.c_double),
                ("batch_normalize", ctypes.c_int32), ("batch_segmented", ctypes.c_int32),
                ("inner_adaptive", ctypes.c_int32), ("implicit", ctypes.c_int32),
                ("newton_max_iters", ctypes.c_int32), ("assembly", ctypes.c_int32),
                ("newton_rtol", ctypes.c_double), ("staged_f", ctypes.c_int32), ("pad2", ctypes.c_int32)]


class lfx_mesh_info(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("n_tets", ctypes.c_int64), ("n_bfaces", ctypes.c_int64),
                ("nnz_blocks", ctypes.c_int64), ("n_colors", ctypes.c_int32), ("n_flipped", ctypes.c_int32),
                ("max_color_size", ctypes.c_int32), ("min_color_size", ctypes.c_int32),
                ("n_bad_elements", ctypes.c_int64), ("n_components", ctypes.c_int32), ("pad", ctypes.c_int32)]


class lfx_step_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("outer_iterations", ctypes.c_int32),
                ("rel_residual", ctypes.c_double), ("t", ctypes.c_double), ("ms_assembly", ctypes.c_float),
                ("ms_solve", ctypes.c_float), ("ms_total", ctypes.c_float), ("converged", ctypes.c_int32),
                ("ms_assembly_kernels", ctypes.c_float), ("n_assembly_launches", ctypes.c_int32),
                ("ms_spmv", ctypes.c_float), ("n_spmv", ctypes.c_int32), ("newton_iterations", ctypes.c_int32),
                ("ms_newton_assembly", ctypes.c_float), ("n_fpass", ctypes.c_int32),
                ("ms_fpass_median", ctypes.c_float), ("assembly_mode", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 2)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


_P = ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int32)
_LP = ctypes.POINTER(ctypes.c_int64)
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

_SIGS = {
    "lfx_last_error": ([], ctypes.c_char_p),
    "lfx_sizeof": ([ctypes.c_char_p], ctypes.c_int64),
    "lfx_launch_count": ([], ctypes.c_int64),
    "lfx_mesh_create": ([_DP, ctypes.c_int64, _IP, ctypes.c_int64, _IP, _IP, ctypes.c_int64,
                         ctypes.POINTER(_P)], ctypes.c_int32),
    "lfx_mesh_destroy": ([_P], None),
    "lfx_mesh_get_info": ([_P, ctypes.POINTER(lfx_mesh_info)], ctypes.c_int32),
    "lfx_mesh_get_pattern": ([_P, _LP, _IP], ctypes.c_int32),
    "lfx_mesh_get_colors": ([_P, _IP], ctypes.c_int32),
    "lfx_mesh_get_chunks": ([_P, _LP, _IP, _IP, _IP, _IP, ctypes.POINTER(ctypes.c_uint16), _IP,
                             ctypes.POINTER(ctypes.c_uint16), _IP, _IP], ctypes.c_int32),
    "lfx_mesh_get_row_tiles": ([_P, _LP, _IP, _IP], ctypes.c_int32),
    "lfx_options_default": ([ctypes.POINTER(lfx_options)], None),
    "lfx_problem_create": ([_P, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                            ctypes.POINTER(lfx_bc), ctypes.c_int32, ctypes.POINTER(lfx_riis), ctypes.c_int32,
                            ctypes.POINTER(lfx_options), ctypes.POINTER(_P)], ctypes.c_int32),
    "lfx_problem_destroy": ([_P], None),
    "lfx_problem_assembly_tuning": ([_P, _IP, ctypes.POINTER(ctypes.c_float)], ctypes.c_int32),
    "lfx_state_create": ([_P, _DP, _DP, ctypes.c_double, ctypes.POINTER(_P)], ctypes.c_int32),
    "lfx_state_destroy": ([_P], None),
    "lfx_set_stream": ([_P, _P], ctypes.c_int32),
    "lfx_set_dirichlet_nodal": ([_P, ctypes.c_int32, _DP], ctypes.c_int32),
    "lfx_set_pressure_pin": ([_P, ctypes.c_double], ctypes.c_int32),
    "lfx_step": ([_P, ctypes.POINTER(lfx_step_stats)], ctypes.c_int32),
    "lfx_state_get": ([_P, _DP, _DP], ctypes.c_int32),
    "lfx_state_newton_residuals": ([_P, _DP, ctypes.c_int32, _IP], ctypes.c_int32),
    "lfx_state_set_displacement": ([_P, _DP], ctypes.c_int32),
    "lfx_set_boundary_displacement": ([_P, ctypes.c_int64, _IP, _DP], ctypes.c_int32),
    "lfx_state_get_displacement": ([_P, _DP, _IP], ctypes.c_int32),
    "lfx_state_set": ([_P, _DP, _DP, ctypes.c_double], ctypes.c_int32),
    "lfx_debug_assemble": ([_P, ctypes.c_int32, _DP, _DP], ctypes.c_int32),
    "lfx_debug_spmv": ([_P, _DP, _DP], ctypes.c_int32),
    "lfx_debug_assemble_newton": ([_P, _DP, _DP, _DP], ctypes.c_int32),
    "lfx_debug_persistent_timeout": ([_P], ctypes.c_int32),
    "lfx_debug_staged_timeout": ([_P], ctypes.c_int32),
    "lfx_debug_precond": ([_P, _DP, _DP, _DP, _DP], ctypes.c_int32),
    "lfx_debug_solve": ([_P, _DP, ctypes.POINTER(lfx_step_stats)], ctypes.c_int32),
    "lfx_set_allocator": ([ALLOC_FN, FREE_FN, _P], ctypes.c_int32),
    "lfx_problem_state_bytes": ([_P, _LP], ctypes.c_int32),
    "lfx_server_create": ([ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(_P)], ctypes.c_int32),
    "lfx_server_submit": ([_P, _P, _DP, _DP, ctypes.c_double, ctypes.c_int32, _LP], ctypes.c_int32),
    "lfx_server_poll": ([_P, ctypes.c_int64, _IP, _IP, ctypes.POINTER(lfx_step_stats)], ctypes.c_int32),
    "lfx_server_result": ([_P, ctypes.c_int64, _DP, _DP], ctypes.c_int32),
    "lfx_server_stats": ([_P, ctypes.POINTER(ctypes.c_float), ctypes.c_int64, _LP, _LP, _LP, _LP], ctypes.c_int32),
    "lfx_server_destroy": ([_P], None),
    "lfx_batch_step": ([ctypes.POINTER(_P), ctypes.c_int32, ctypes.POINTER(lfx_step_stats)], ctypes.c_int32),
    "lfx_asimple_apply_noalloc": ([ctypes.c_int64, _P, _P, _P, _P, _P, _P, _P, ctypes.POINTER(lfx_options), _P],
                                  ctypes.c_int32),
    "lfx_state_device_bytes": ([_P, _LP], ctypes.c_int32),
    "lfx_debug_amg_level": ([_P, ctypes.c_int32, _LP, _IP, _IP, _DP, _IP, _IP, _DP, _DP], ctypes.c_int32),
    "lfx_debug_amg_vcycle": ([_P, _DP, _DP], ctypes.c_int32),
    "lfx_debug_amg_host": ([ctypes.c_int64, _IP, _IP, _IP, _DP, ctypes.POINTER(lfx_options), ctypes.c_int32, _LP,
                            _IP, _IP, _DP, _IP, _IP, _DP, _DP, _DP], ctypes.c_int32),
    "lfx_state_amg_levels": ([_P, _IP, _LP, _LP, ctypes.c_int32], ctypes.c_int32),
}


class LfxError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"lfx status {status}: {msg}")
        self.status = status


def library():
    """Load liblfx.so (built by paper_2304_12032_gb300.build); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"liblfx.so not built ({LIB_PATH}); run `python -m paper_2304_12032_gb300.build`")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
    return _lib


def _check(status, allow=()):
    if status != LFX_OK and status not in allow:
        raise LfxError(status, library().lfx_last_error().decode())
    return status


def _d(a):
    return a.ctypes.data_as(_DP)


def _i(a):
    return a.ctypes.data_as(_IP)


# ----------------------------------------------------------------------------- allocator hook
_alloc_keepalive = []


def use_torch_allocator():
    """Back every later device allocation of the library with PyTorch's caching allocator."""
    import torch

    dev = torch.cuda.current_device()

    def _alloc(nbytes, ctx):
        return torch.cuda.caching_allocator_alloc(int(nbytes), dev)

    def _free(ptr, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    fa, ff = ALLOC_FN(_alloc), FREE_FN(_free)
    _alloc_keepalive[:] = [fa, ff]
    _check(library().lfx_set_allocator(fa, ff, None))


def use_cuda_allocator():
    _check(library().lfx_set_allocator(ALLOC_FN(), FREE_FN(), None))
    _alloc_keepalive.clear()


# ----------------------------------------------------------------------------- options / BCs
def default_options(**kw) -> lfx_options:
    o = lfx_options()
    library().lfx_options_default(ctypes.byref(o))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = PREC[v]
        if k in ("f_smoother", "s_smoother") and isinstance(v, str):
            v = SMOOTH[v]
        if k == "assembly" and isinstance(v, str):
            v = ASM[v]
        if k == "f":
            for i in range(3):
                o.f[i] = v[i]
            continue
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


@dataclasses.dataclass
class BC:
    """Python form of lfx_bc (Section 2.2)."""
    tag: int
    kind: str                       # noslip | dirichlet | nodal | neumann | resistance
    profile: str = "uniform"        # uniform | parabolic | womersley
    time: str = "constant"          # constant | pulsatile | ramp | fourier
    p: Sequence[float] = (0.0,)     # time-law parameters (see lfx_time_law)
    a: Sequence[float] = ()         # Fourier cosine coefficients a_0..a_K
    b: Sequence[float] = ()         # Fourier sine coefficients (b_0 ignored)
    theta: float = 1.0
    radius: float = 1.0
    center: Optional[Sequence[float]] = None
    normal: Optional[Sequence[float]] = None
    beta: float = 0.0               # neumann: inertial backflow stabilisation (0: off)
    resistance: float = 0.0         # resistance: C_R (p holds the time law of p_0)

    def c(self) -> lfx_bc:
        s = lfx_bc()
        s.tag, s.kind, s.profile = self.tag, KIND[self.kind], PROFILE[self.profile]
        s.time.kind = TIME[self.time]
        for i, v in enumerate(self.p):
            s.time.p[i] = v
        K = max(len(self.a), len(self.b)) - 1
        s.time.n_harmonics = max(K, 0)
        for i, v in enumerate(self.a):
            s.time.a[i] = v
        for i, v in enumerate(self.b):
            s.time.b[i] = v
        s.theta, s.radius, s.beta, s.resistance = self.theta, self.radius, self.beta, self.resistance
        if self.center is not None and self.normal is not None:
            s.given_geometry = 1
            for i in range(3):
                s.center[i], s.normal[i] = self.center[i], self.normal[i]
        return s


@dataclasses.dataclass
class RIIS:
    """Python form of lfx_riis: a disk (center, normal, radius) or nodal signed distances."""
    resistance: float
    eps: float
    center: Sequence[float] = (0.0, 0.0, 0.0)
    normal: Sequence[float] = (0.0, 0.0, 1.0)
    radius: float = 1.0
    sdf_nodal: Optional[np.ndarray] = None


# ----------------------------------------------------------------------------- handles
def lfx_mesh_create(nodes, tets, bfaces, btags):
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    bfaces = np.ascontiguousarray(bfaces, dtype=np.int32)
    btags = np.ascontiguousarray(btags, dtype=np.int32)
    h = _P()
    _check(library().lfx_mesh_create(_d(nodes), nodes.shape[0], _i(tets), tets.shape[0], _i(bfaces), _i(btags),
                                     bfaces.shape[0], ctypes.byref(h)))
    return h


class Mesh:
    def __init__(self, nodes, tets, bfaces, btags):
        self.n_nodes = int(np.asarray(nodes).shape[0])
        self.h = lfx_mesh_create(nodes, tets, bfaces, btags)

    @classmethod
    def from_synthetic(cls, m):
        return cls(m.nodes, m.tets, m.bfaces, m.btags)

    def info(self) -> dict:
        i = lfx_mesh_info()
        _check(library().lfx_mesh_get_info(self.h, ctypes.byref(i)))
        return {k: getattr(i, k) for k, _ in i._fields_}

    def pattern(self):
        inf = self.info()
        rp = np.zeros(inf["n_nodes"] + 1, dtype=np.int64)
        ci = np.zeros(inf["nnz_blocks"], dtype=np.int32)
        _check(library().lfx_mesh_get_pattern(self.h, rp.ctypes.data_as(_LP), _i(ci)))
        return rp, ci

    def colors(self):
        c = np.zeros(self.info()["n_tets"], dtype=np.int32)
        _check(library().lfx_mesh_get_colors(self.h, _i(c)))
        return c

    def row_tiles(self) -> dict:
        """The staged velocity pass's row tiles (see lfx_mesh_get_row_tiles)."""
        lib = library()
        sz = np.zeros(3, dtype=np.int64)
        _check(lib.lfx_mesh_get_row_tiles(self.h, sz.ctypes.data_as(_LP), None, None))
        n = int(sz[0])
        tile_row = np.zeros(n + 1, np.int32)
        row_node = np.zeros(self.info()["n_nodes"], np.int32)
        _check(lib.lfx_mesh_get_row_tiles(self.h, sz.ctypes.data_as(_LP), _i(tile_row) if n else None, _i(row_node)))
        return {"tile_row": tile_row if n else np.zeros(0, np.int32), "row_node": row_node,
                "max_rows": int(sz[1]), "max_blocks": int(sz[2])}

    def chunks(self) -> dict:
        """The chunked assembly's tables (see lfx_mesh_get_chunks)."""
        lib = library()
        sz = np.zeros(5, dtype=np.int64)
        _check(lib.lfx_mesh_get_chunks(self.h, sz.ctypes.data_as(_LP), None, None, None, None, None, None, None,
                                       None, None))
        nch, ncc, npass, nrun, ps = (int(v) for v in sz)
        T = self.info()["n_tets"]
        out = {"elem_old": np.zeros(T, np.int32), "chunk_elem_off": np.zeros(nch + 1, np.int32),
               "chunk_color_off": np.zeros(ncc + 1, np.int32), "chunk_pass_off": np.zeros(nch + 1, np.int32),
               "pass_code": np.zeros((max(npass, 1), ps), np.uint16), "pass_run_off": np.zeros(npass + 1, np.int32),
               "run_meta": np.zeros(max(nrun, 1), np.uint16), "run_row": np.zeros(max(nrun, 1), np.int32),
               "run_col": np.zeros(max(nrun, 1), np.int32)}
        u16 = ctypes.POINTER(ctypes.c_uint16)
        _check(lib.lfx_mesh_get_chunks(self.h, sz.ctypes.data_as(_LP), _i(out["elem_old"]), _i(out["chunk_elem_off"]),
                                       _i(out["chunk_color_off"]), _i(out["chunk_pass_off"]),
                                       out["pass_code"].ctypes.data_as(u16), _i(out["pass_run_off"]),
                                       out["run_meta"].ctypes.data_as(u16), _i(out["run_row"]), _i(out["run_col"])))
        out["pass_code"] = out["pass_code"][:npass]
        for k in ("run_meta", "run_row", "run_col"):
            out[k] = out[k][:nrun]
        return out

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.lfx_mesh_destroy(self.h)
            self.h = None


def debug_amg_host(row_ptr, col_idx, diag_idx, blocks, options: Optional[lfx_options] = None):
    """The Schur AMG set-up on the host alone (lfx_debug_amg_host) for a 4x4 block-CSR system held in
    host memory: a list of levels, each a dict with n, A (scipy CSR; A_0 = S = C - D diag(F)^-1 G),
    P (scipy CSR n_l x n_{l+1}; None at the coarsest level), lam (Gershgorin bound of
    lambda_max(D^-1 A_l)) and, at the coarsest level, coarse_inv (its dense inverse)."""
    import scipy.sparse as sp

    lib = library()
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    dg = np.ascontiguousarray(diag_idx, dtype=np.int32)
    bl = np.ascontiguousarray(blocks, dtype=np.float64).reshape(-1, 16)
    n = int(rp.size - 1)
    opt = ctypes.byref(options) if options is not None else None
    levels, out = 1, []
    while len(out) < levels:
        level = len(out)
        sz = np.zeros(5, dtype=np.int64)
        lam = ctypes.c_double()
        _check(lib.lfx_debug_amg_host(n, _i(rp), _i(ci), _i(dg), _d(bl), opt, level, sz.ctypes.data_as(_LP), None,
                                      None, None, None, None, None, ctypes.byref(lam), None))
        levels, nl, nnz_a, nn, nnz_p = (int(v) for v in sz)
        last = level == levels - 1
        arp, aci, av = np.zeros(nl + 1, np.int32), np.zeros(max(nnz_a, 1), np.int32), np.zeros(max(nnz_a, 1))
        prp, pci, pv = np.zeros(nl + 1, np.int32), np.zeros(max(nnz_p, 1), np.int32), np.zeros(max(nnz_p, 1))
        inv = np.zeros((nl, nl)) if last else None
        _check(lib.lfx_debug_amg_host(n, _i(rp), _i(ci), _i(dg), _d(bl), opt, level, sz.ctypes.data_as(_LP),
                                      _i(arp), _i(aci), _d(av), _i(prp), _i(pci), _d(pv), ctypes.byref(lam),
                                      _d(inv) if last else None))
        A = sp.csr_matrix((av[:nnz_a], aci[:nnz_a], arp), shape=(nl, nl))
        P = None if last else sp.csr_matrix((pv[:nnz_p], pci[:nnz_p], prp), shape=(nl, nn))
        out.append({"n": nl, "A": A, "P": P, "lam": lam.value, "coarse_inv": inv})
    return out


class Problem:
    def __init__(self, mesh: Mesh, rho, mu, dt, bdf_order, bcs: Sequence[BC], riis: Sequence[RIIS] = (),
                 options: Optional[lfx_options] = None):
        self.mesh = mesh
        arr = (lfx_bc * max(1, len(bcs)))(*[b.c() for b in bcs])
        self._sdf = []
        rarr = (lfx_riis * max(1, len(riis)))()
        for k, r in enumerate(riis):
            s = rarr[k]
            s.resistance, s.eps, s.radius = r.resistance, r.eps, r.radius
            for i in range(3):
                s.center[i], s.normal[i] = r.center[i], r.normal[i]
            if r.sdf_nodal is not None:
                a = np.ascontiguousarray(r.sdf_nodal, dtype=np.float64)
                self._sdf.append(a)
                s.kind, s.sdf_nodal = 1, _d(a)
        self.options = options if options is not None else default_options()
        self.bdf_order = bdf_order
        self.h = _P()
        _check(library().lfx_problem_create(mesh.h, rho, mu, dt, bdf_order, arr, len(bcs), rarr, len(riis),
                                            ctypes.byref(self.options), ctypes.byref(self.h)))

    def assembly_tuning(self):
        """(launch shape in use, {shape: ms per assembly} of the autotuner's timings)."""
        mode = ctypes.c_int32()
        ms = (ctypes.c_float * 3)()
        _check(library().lfx_problem_assembly_tuning(self.h, ctypes.byref(mode), ms))
        names = ("colors", "chunks", "persistent")
        return mode.value, {names[i]: ms[i] for i in range(3) if ms[i] > 0}

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.lfx_problem_destroy(self.h)
            self.h = None


class State:
    def __init__(self, problem: Problem, u_hist, p_hist, t0=0.0, stream=None):
        self.problem = problem
        V = problem.mesh.n_nodes
        u = np.ascontiguousarray(np.asarray(u_hist, dtype=np.float64).reshape(problem.bdf_order, V, 3))
        p = np.ascontiguousarray(np.asarray(p_hist, dtype=np.float64).reshape(problem.bdf_order, V))
        self.V = V
        self.h = _P()
        _check(library().lfx_state_create(problem.h, _d(u), _d(p), t0, ctypes.byref(self.h)))
        if stream is not None:
            self.set_stream(stream)

    def set_stream(self, stream):
        ptr = getattr(stream, "cuda_stream", stream)
        _check(library().lfx_set_stream(self.h, ctypes.c_void_p(int(ptr) if ptr else 0)))

    def set_dirichlet_nodal(self, tag, u):
        u = np.ascontiguousarray(u, dtype=np.float64)
        _check(library().lfx_set_dirichlet_nodal(self.h, tag, _d(u)))

    def set_pressure_pin(self, value):
        _check(library().lfx_set_pressure_pin(self.h, float(value)))

    def step(self, allow_not_converged=False) -> dict:
        st = lfx_step_stats()
        rc = library().lfx_step(self.h, ctypes.byref(st))
        _check(rc, allow=(LFX_ERR_NOT_CONVERGED,) if allow_not_converged else ())
        d = st.as_dict()
        d["status"] = rc
        return d

    def set(self, u_hist, p_hist, t):
        u = np.ascontiguousarray(np.asarray(u_hist, dtype=np.float64).reshape(self.problem.bdf_order, self.V, 3))
        p = np.ascontiguousarray(np.asarray(p_hist, dtype=np.float64).reshape(self.problem.bdf_order, self.V))
        _check(library().lfx_state_set(self.h, _d(u), _d(p), float(t)))

    def get(self, u=None, p=None):
        """u [V][3], p [V] at the current time level; into the given C-contiguous float64 arrays
        (e.g. views of page-locked buffers, which the copy then reads by DMA) or new ones."""
        if u is None:
            u = np.zeros((self.V, 3))
        if p is None:
            p = np.zeros(self.V)
        for a, shape in ((u, (self.V, 3)), (p, (self.V,))):
            if a.dtype != np.float64 or a.shape != shape or not a.flags["C_CONTIGUOUS"]:
                raise ValueError(f"State.get: output must be C-contiguous float64 of shape {shape}")
        _check(library().lfx_state_get(self.h, _d(u), _d(p)))
        return u, p

    def set_displacement(self, d_hist):
        """Moving mesh: displacement levels d^n, d^{n-1}, ... ([bdf_order][V][3])."""
        d = np.ascontiguousarray(np.asarray(d_hist, dtype=np.float64).reshape(self.problem.bdf_order, self.V, 3))
        _check(library().lfx_state_set_displacement(self.h, _d(d)))

    def set_boundary_displacement(self, nodes, d):
        """The next step's displacement d [n][3] at the listed nodes (the lifting extends it)."""
        nodes = np.ascontiguousarray(nodes, dtype=np.int32)
        d = np.ascontiguousarray(np.asarray(d, dtype=np.float64).reshape(nodes.size, 3))
        _check(library().lfx_set_boundary_displacement(self.h, nodes.size, _i(nodes), _d(d)))

    def get_displacement(self):
        """(d [V][3] of the current time level, CG iterations of the last lifting)."""
        d = np.zeros((self.V, 3))
        it = ctypes.c_int32()
        _check(library().lfx_state_get_displacement(self.h, _d(d), ctypes.byref(it)))
        return d, it.value

    def newton_residuals(self):
        """||R(U_k)|| / ||b|| of the last step's Newton iterates (empty for semi-implicit steps)."""
        n = ctypes.c_int32()
        out = np.zeros(64)
        _check(library().lfx_state_newton_residuals(self.h, _d(out), 64, ctypes.byref(n)))
        return out[:min(n.value, 64)].copy()

    def device_bytes(self) -> int:
        b = ctypes.c_int64()
        _check(library().lfx_state_device_bytes(self.h, ctypes.byref(b)))
        return b.value

    def amg_levels(self):
        """[(rows, nonzeros)] of each level of the Schur multigrid hierarchy (empty before set-up)."""
        n = ctypes.c_int32()
        rows = np.zeros(16, dtype=np.int64)
        nnz = np.zeros(16, dtype=np.int64)
        _check(library().lfx_state_amg_levels(self.h, ctypes.byref(n), rows.ctypes.data_as(_LP),
                                              nnz.ctypes.data_as(_LP), 16))
        return [(int(rows[i]), int(nnz[i])) for i in range(min(n.value, 16))]

    # ---- building blocks, for parity tests
    def debug_assemble(self, apply_bcs=True):
        nnzb = self.problem.mesh.info()["nnz_blocks"]
        blocks = np.zeros((nnzb, 4, 4))
        rhs = np.zeros((self.V, 4))
        _check(library().lfx_debug_assemble(self.h, int(apply_bcs), _d(blocks), _d(rhs)))
        return blocks, rhs

    def debug_assemble_newton(self, U):
        """Jacobian blocks [nnzb,4,4] and right-hand side J U - R(U) [V,4] of the fully implicit
        formulation at the iterate U [V,4] (no Dirichlet rows)."""
        U = np.ascontiguousarray(U, dtype=np.float64).reshape(self.V, 4)
        nnzb = self.problem.mesh.info()["nnz_blocks"]
        blocks = np.zeros((nnzb, 4, 4))
        rhs = np.zeros((self.V, 4))
        _check(library().lfx_debug_assemble_newton(self.h, _d(U), _d(blocks), _d(rhs)))
        return blocks, rhs

    def debug_persistent_timeout(self):
        """Status of one persistent assembly whose first grid-wide wait is made to run out."""
        return library().lfx_debug_persistent_timeout(self.h)

    def debug_staged_timeout(self):
        """Status of one BF16 preconditioner application whose staged-tile waits are made to run out."""
        return library().lfx_debug_staged_timeout(self.h)

    def debug_spmv(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(self.V, 4)
        y = np.zeros((self.V, 4))
        _check(library().lfx_debug_spmv(self.h, _d(x), _d(y)))
        return y

    def debug_precond(self, r):
        r = np.ascontiguousarray(r, dtype=np.float64).reshape(self.V, 4)
        z = np.zeros((self.V, 4))
        lf, ls = ctypes.c_double(), ctypes.c_double()
        _check(library().lfx_debug_precond(self.h, _d(r), _d(z), ctypes.byref(lf), ctypes.byref(ls)))
        return z, lf.value, ls.value

    def debug_amg_level(self, level):
        """Level `level` of the device Schur AMG hierarchy (FP64 path): dict with n, A (scipy CSR,
        None at level 0 and at the coarsest level), P (scipy CSR n_l x n_{l+1}, None at the coarsest)
        and lam (Gershgorin bound of lambda_max(D^-1 A_l))."""
        import scipy.sparse as sp

        lib = library()
        sz = np.zeros(4, dtype=np.int64)
        lam = ctypes.c_double()
        _check(lib.lfx_debug_amg_level(self.h, int(level), sz.ctypes.data_as(_LP), None, None, None, None, None,
                                       None, ctypes.byref(lam)))
        n, nnz_a, nn, nnz_p = (int(v) for v in sz)
        arp, aci, av = np.zeros(n + 1, np.int32), np.zeros(max(nnz_a, 1), np.int32), np.zeros(max(nnz_a, 1))
        prp, pci, pv = np.zeros(n + 1, np.int32), np.zeros(max(nnz_p, 1), np.int32), np.zeros(max(nnz_p, 1))
        _check(lib.lfx_debug_amg_level(self.h, int(level), sz.ctypes.data_as(_LP), _i(arp), _i(aci), _d(av), _i(prp),
                                       _i(pci), _d(pv), ctypes.byref(lam)))
        A = sp.csr_matrix((av[:nnz_a], aci[:nnz_a], arp), shape=(n, n)) if nnz_a else None
        P = sp.csr_matrix((pv[:nnz_p], pci[:nnz_p], prp), shape=(n, nn)) if nnz_p else None
        return {"n": n, "A": A, "P": P, "lam": lam.value}

    def debug_amg_vcycle(self, b1):
        b1 = np.ascontiguousarray(b1, dtype=np.float64)
        x1 = np.zeros_like(b1)
        _check(library().lfx_debug_amg_vcycle(self.h, _d(b1), _d(x1)))
        return x1

    def debug_solve(self, allow_not_converged=False):
        x = np.zeros((self.V, 4))
        st = lfx_step_stats()
        rc = library().lfx_debug_solve(self.h, _d(x), ctypes.byref(st))
        _check(rc, allow=(LFX_ERR_NOT_CONVERGED,) if allow_not_converged else ())
        return x, st.as_dict()

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.lfx_state_destroy(self.h)
            self.h = None


class Server:
    """Continuous-batching request loop (lfx_server_*): admission by device-memory budget,
    resident states, round-robin stepping by native worker threads on separate streams."""

    def __init__(self, hbm_budget_bytes: int, n_workers: int = 4):
        self.h = _P()
        _check(library().lfx_server_create(int(hbm_budget_bytes), int(n_workers), ctypes.byref(self.h)))
        self._keep = {}

    def submit(self, problem: Problem, u_hist, p_hist, t0, n_steps) -> int:
        V = problem.mesh.n_nodes
        u = np.ascontiguousarray(np.asarray(u_hist, dtype=np.float64).reshape(problem.bdf_order, V, 3))
        p = np.ascontiguousarray(np.asarray(p_hist, dtype=np.float64).reshape(problem.bdf_order, V))
        t = ctypes.c_int64()
        _check(library().lfx_server_submit(self.h, problem.h, _d(u), _d(p), float(t0), int(n_steps), ctypes.byref(t)))
        self._keep[t.value] = (problem, V)
        return t.value

    def poll(self, ticket):
        done, steps = ctypes.c_int32(), ctypes.c_int32()
        st = lfx_step_stats()
        _check(library().lfx_server_poll(self.h, ticket, ctypes.byref(done), ctypes.byref(steps), ctypes.byref(st)))
        return bool(done.value), steps.value, st.as_dict()

    def result(self, ticket):
        problem, V = self._keep.pop(ticket)
        u, p = np.zeros((V, 3)), np.zeros(V)
        _check(library().lfx_server_result(self.h, ticket, _d(u), _d(p)))
        return u, p

    def stats(self, capacity=1 << 20):
        lat = np.zeros(capacity, dtype=np.float32)
        n, used, waiting, peak = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(library().lfx_server_stats(self.h, lat.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), capacity,
                                          ctypes.byref(n), ctypes.byref(used), ctypes.byref(waiting), ctypes.byref(peak)))
        return {"latency_ms": lat[:min(n.value, capacity)].copy(), "used_bytes": used.value,
                "waiting": waiting.value, "max_active": peak.value}

    def close(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.lfx_server_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()


def batch_step(states: Sequence[State], allow_not_converged=False):
    """lfx_batch_step: one step of every state, concurrently (each state on its own stream)."""
    n = len(states)
    arr = (_P * max(n, 1))(*[s.h for s in states])
    stats = (lfx_step_stats * max(n, 1))()
    rc = library().lfx_batch_step(arr, n, stats)
    _check(rc, allow=(LFX_ERR_NOT_CONVERGED,) if allow_not_converged else ())
    return [stats[i].as_dict() for i in range(n)]


def problem_state_bytes(problem: Problem) -> int:
    b = ctypes.c_int64()
    _check(library().lfx_problem_state_bytes(problem.h, ctypes.byref(b)))
    return b.value
