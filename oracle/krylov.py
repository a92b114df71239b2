"""Oracle, linear-algebra part (test infrastructure only; see the package docstring).

The paper solves the block system of Section 2.4 with GMRES preconditioned by aSIMPLE
[deparis2014parallel], the velocity and Schur blocks approximated by a black-box method.  This
module writes that preconditioner with Jacobi / Chebyshev smoothing (textbook forms from
[saad2003iterative], which the paper cites) and a flexible GMRES, in plain scipy, with the
assembled Schur approximation.  It is the "same algorithm" reference for the GPU
preconditioner and the timed CPU baseline; the accuracy reference for solutions is the
direct solve of ``core.solve_direct``.

Reading of aSIMPLE taken here (the paper gives only the name and the citation):
    with the block system [[F, G], [D, C]] (velocity rows first),
    D_F = diag(F) and S = C - D D_F^-1 G,
        z_u* ~= F^-1 r_u          (k_F smoothing steps from zero)
        z_p  ~= S^-1 (r_p - D z_u*) (k_S smoothing steps from zero)
        z_u  =  z_u* - D_F^-1 G z_p
Jacobi step: x <- x + omega D^-1 (b - M x).  Chebyshev: Saad's Chebyshev acceleration of
D^-1 M with spectrum [lmax/ratio, lmax].  lmax is a Gershgorin bound, which holds for every
eigenvalue: for F the largest absolute row sum of diag(F)^-1 F; for S the triangle-inequality
bound |dinvS_a| (sum_b |C_ab| + sum_(b,j) |D_a,(b,j)| |dinvF_(b,j)| sum_c |G_(b,j),c|), which
needs no explicit S.  (A power iteration from the all-ones vector, n_power > 0, is kept as an
option: on meshes with slivers it underestimates lmax and Chebyshev then amplifies the missed
modes.)
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp

__all__ = ["SmootherOpts", "ASimpleOpts", "split_blocks", "power_lambda_max", "jacobi",
           "chebyshev", "ASimple", "fgmres"]


@dataclasses.dataclass
class SmootherOpts:
    kind: str = "chebyshev"     # 'jacobi' | 'chebyshev'
    steps: int = 4              # number of smoothing steps (polynomial degree)
    omega: float = 0.7          # Jacobi damping
    ratio: float = 10.0         # Chebyshev: lmin = lmax / ratio
    n_power: int = 0            # 0: Gershgorin bound for lmax; > 0: power-iteration steps (x 1.1)


@dataclasses.dataclass
class ASimpleOpts:
    f: SmootherOpts = dataclasses.field(default_factory=lambda: SmootherOpts("chebyshev", 3, 0.7, 20.0, 0))
    s: SmootherOpts = dataclasses.field(default_factory=lambda: SmootherOpts("chebyshev", 6, 0.7, 30.0, 0))


def split_blocks(A: sp.csr_matrix):
    """F, G, D, C of the interleaved (u_x,u_y,u_z,p per node) system."""
    N = A.shape[0]
    V = N // 4
    vel = (4 * np.arange(V)[:, None] + np.arange(3)[None, :]).ravel()
    pre = 4 * np.arange(V) + 3
    A = A.tocsr()
    F = A[vel][:, vel].tocsr()
    G = A[vel][:, pre].tocsr()
    D = A[pre][:, vel].tocsr()
    C = A[pre][:, pre].tocsr()
    return F, G, D, C, vel, pre


def power_lambda_max(M, dinv, n_power):
    """Power iteration on D^-1 M from the normalised all-ones vector; returns ||D^-1 M v_k||."""
    v = np.ones(M.shape[0]) / math.sqrt(M.shape[0])
    lam = 0.0
    for _ in range(n_power):
        w = dinv * (M @ v)
        lam = float(np.linalg.norm(w))
        v = w / lam
    return lam


def jacobi(M, dinv, b, omega, steps):
    x = omega * dinv * b
    for _ in range(steps - 1):
        x = x + omega * dinv * (b - M @ x)
    return x


def chebyshev(M, dinv, b, lmin, lmax, steps):
    """Chebyshev acceleration (Saad, Alg. 12.1) for D^-1 M x = D^-1 b from x0 = 0."""
    theta = 0.5 * (lmax + lmin)
    delta = 0.5 * (lmax - lmin)
    sigma1 = theta / delta
    rho = 1.0 / sigma1
    r = dinv * b
    d = r / theta
    x = np.zeros_like(b)
    for k in range(steps):
        x = x + d
        if k == steps - 1:
            break
        r = r - dinv * (M @ d)
        rho_new = 1.0 / (2.0 * sigma1 - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * r
        rho = rho_new
    return x


class ASimple:
    """aSIMPLE preconditioner (reading in the module docstring) for one assembled system."""

    def __init__(self, A: sp.csr_matrix, opts: ASimpleOpts = ASimpleOpts()):
        self.opts = opts
        F, G, D, C, vel, pre = split_blocks(A)
        self.F, self.G, self.D, self.C, self.vel, self.pre = F, G, D, C, vel, pre
        dF = F.diagonal()
        self.dFinv = 1.0 / dF
        self.S = (C - D @ sp.diags(self.dFinv) @ G).tocsr()
        dS = self.S.diagonal()
        # a vanishing diagonal of S (no pressure stabilisation, all velocity neighbours
        # constrained) leaves that pressure unknown unsmoothed
        self.dSinv = np.divide(1.0, dS, out=np.zeros_like(dS), where=dS != 0.0)
        gsum = np.asarray(abs(G).sum(axis=1)).ravel()
        self.bound_f = float(np.max(np.abs(self.dFinv) * np.asarray(abs(F).sum(axis=1)).ravel()))
        self.bound_s = float(np.max(np.abs(self.dSinv) * (np.asarray(abs(C).sum(axis=1)).ravel()
                                                          + abs(D) @ (np.abs(self.dFinv) * gsum))))
        self.lam_f = self._lmax(F, self.dFinv, opts.f, self.bound_f)
        self.lam_s = self._lmax(self.S, self.dSinv, opts.s, self.bound_s)

    @staticmethod
    def _lmax(M, dinv, so, bound):
        if so.kind != "chebyshev":
            return None
        return power_lambda_max(M, dinv, so.n_power) * 1.1 if so.n_power > 0 else bound

    def _smooth(self, M, dinv, b, so: SmootherOpts, lam):
        if so.kind == "jacobi":
            return jacobi(M, dinv, b, so.omega, so.steps)
        return chebyshev(M, dinv, b, lam / so.ratio, lam, so.steps)

    def apply(self, r: np.ndarray) -> np.ndarray:
        ru, rp = r[self.vel], r[self.pre]
        zu = self._smooth(self.F, self.dFinv, ru, self.opts.f, self.lam_f)
        zp = self._smooth(self.S, self.dSinv, rp - self.D @ zu, self.opts.s, self.lam_s)
        zu = zu - self.dFinv * (self.G @ zp)
        z = np.empty_like(r)
        z[self.vel], z[self.pre] = zu, zp
        return z


def fgmres(A, b, x0=None, M=None, restart=30, tol=1e-10, maxiter=2000):
    """Right-preconditioned flexible GMRES (Saad, Alg. 9.6) with modified Gram-Schmidt and
    Givens rotations.  Stops when ||b - A x|| <= tol ||b||.  Returns (x, iterations, history)."""
    n = b.size
    x = np.zeros(n) if x0 is None else x0.copy()
    Mf = (lambda v: v) if M is None else M
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros(n), 0, [0.0]
    its, hist = 0, []
    while its < maxiter:
        r = b - A @ x
        beta = np.linalg.norm(r)
        hist.append(beta / bnorm)
        if beta <= tol * bnorm:
            break
        Vb = np.zeros((restart + 1, n))
        Z = np.zeros((restart, n))
        H = np.zeros((restart + 1, restart))
        cs, sn = np.zeros(restart), np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        Vb[0] = r / beta
        j_end = 0
        for j in range(restart):
            Z[j] = Mf(Vb[j])
            w = A @ Z[j]
            for i in range(j + 1):
                H[i, j] = w @ Vb[i]
                w = w - H[i, j] * Vb[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0:
                Vb[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = math.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            j_end = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) <= tol * bnorm or its >= maxiter:
                break
        y = np.zeros(j_end)
        for i in range(j_end - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:j_end] @ y[i + 1:j_end]) / H[i, i]
        x = x + Z[:j_end].T @ y
        if abs(g[j_end]) <= tol * bnorm:
            r = b - A @ x
            if np.linalg.norm(r) <= 10 * tol * bnorm:
                break
    return x, its, hist
