// Per-element, per-quadrature-point assembly of the linearised block system of Section 2.3,
// Eq. (fullydiscrete_ns_ale_riis_vmsles_quasistatic_unified), with the SUPG-PSPG, VMS and
// semi-implicit LES terms (Eqs. stabilization_form_*), tau_M / tau_C (Section 2.3), and the
// resistive term of Eq. (riis); plus the BDF/EXT fields (Eq. bdf) and the boundary data of
// Section 2.2.
//
// Layout: 4 unknowns per node interleaved (u_x, u_y, u_z, p); matrix in 4x4 block CSR, each
// block 16 values row-major (row = test component, column = trial component).  Elements of one
// colour share no node, so one launch per colour updates disjoint blocks without atomics.
//
// The arithmetic type R is FP64 (the FP64 path), FP32, or double-float (dd: FP32 pairs with a
// 48-bit significand, for the mixed-precision path: FP64-class accuracy on the FP32 pipes; its
// inputs arrive pre-split and the matrix is accumulated as FP32 high and low parts).
//
// One CTA of 128 threads works on 32 elements at a time:
//   phase 1: 4 threads per element, thread q evaluates quadrature point q (geometry, u*, tau_M,
//            tau_C, the LES vector tau_M r_M(u^EXT, p^EXT), ...) into shared memory;
//   phase 2: 16 threads per element, thread (a, b) forms block (a, b) and right-hand-side entry
//            (a, b) and adds them into global memory (read-modify-write of 128 B / 64 B).
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "dd.h"
#include "lfx_internal.h"
#include "kernels.h"
#include "pdl.h"

namespace lfx {

namespace {

constexpr int kCta = 128;
constexpr int kElems = 32;          // elements per CTA pass
constexpr double kQA = 0.58541019662496845446;   // (5 + 3 sqrt5) / 20
constexpr double kQB = 0.13819660112501051518;   // (5 - sqrt5) / 20

// Physical coefficients in the arithmetic type (split once on the host)
template <class R>
struct PhysR {
  R rho, mu, rho_dt, alpha, rho_alpha_dt, tau_t, cr_mu2, f[3];
};
template <class R>
PhysR<R> phys_r(const PhysParams &P) {
  PhysR<R> q;
  q.rho = R(P.rho);
  q.mu = R(P.mu);
  q.rho_dt = R(P.rho_dt);
  q.alpha = R(P.alpha);
  q.rho_alpha_dt = R(P.rho_alpha_dt);
  q.tau_t = R(P.tau_t);
  q.cr_mu2 = R(P.cr_mu2);
  for (int i = 0; i < 3; ++i) q.f[i] = R(P.f[i]);
  return q;
}

// four values of node n: FP64 and FP32 from the FP64 array, dd from the split arrays
template <class R>
__device__ __forceinline__ void ld_node(const D4 *d, const float4 *, const float4 *, int64_t n, R v[4]) {
  const D4 a = d[n];
  v[0] = (R)a.x;
  v[1] = (R)a.y;
  v[2] = (R)a.z;
  v[3] = (R)a.w;
}
template <>
__device__ __forceinline__ void ld_node<dd>(const D4 *, const float4 *hi, const float4 *lo, int64_t n, dd v[4]) {
  const float4 h = hi[n], l = lo[n];
  v[0] = dd(h.x, l.x);
  v[1] = dd(h.y, l.y);
  v[2] = dd(h.z, l.z);
  v[3] = dd(h.w, l.w);
}

// a compile-time constant in the arithmetic type (the split of a literal folds at compile time)
template <class R>
__device__ __forceinline__ R cst(double c) {
  return (R)c;
}
template <>
__device__ __forceinline__ dd cst<dd>(double c) {
  return dd((float)c, (float)(c - (double)(float)c));
}

// a * b + c (one fused double-float operation for dd; contracted to an FMA otherwise)
template <class R>
__device__ __forceinline__ R fmadd(R a, R b, R c) {
  return a * b + c;
}
// (for dd the one-pass form: products and sums of the element terms are judged against the terms'
// own magnitude, and it takes 15 FP32 operations instead of 27; the accumulation into the matrix
// keeps the exact sum, which measured faster on this GPU than the cheaper one as well)
template <>
__device__ __forceinline__ dd fmadd<dd>(dd a, dd b, dd c) {
  return fma_dd_fast(a, b, c);
}

// a + b where contributions are summed into a matrix entry, a right-hand side or an element sum:
// in double-float the accumulating sum, whose error is relative to the operands (the error model
// of recursive summation), not to the result
template <class R>
__device__ __forceinline__ R acc(R a, R b) {
  return a + b;
}
template <>
__device__ __forceinline__ dd acc<dd>(dd a, dd b) {
  return add_acc(a, b);
}

template <class R>
struct ElemShared {
  R gphi[kElems][12];      // grad phi_a, a = 0..3
  R w[kElems];             // |K| / 4 (quadrature weight)
  R Gm[kElems][9];         // metric tensor G = J^-T J^-1
  R GG[kElems];            // G : G
  R igg[kElems];           // 1 / (g . g), g = J^-T 1
  R cs[kElems][4];         // rho alpha / dt + sum_k (R_k/eps_k) delta_k at each qp
  R wtm[kElems][4];        // w tau_M
  R wtmr[kElems][4];       // w tau_M rho
  R wtc[kElems][4];        // w tau_C
  R adv[kElems][4][4];     // [q][a] = u*(x_q) . grad phi_a
  R wz[kElems][4][3];      // w rho tau_M (u* - tau_M r_M^EXT) (VMS + LES), 0 without VMS-LES
  R m[kElems][4][3];       // rho u^BDF / dt + f
  // per (qp, node) and per element sums (phase 1c)
  R E[kElems][4][4];       // [q][a] = w (phi_a(q) + tau_M rho adv_q(a))  (test-function weight)
  R cb[kElems][4][4];      // [q][b] = cs_q phi_b(q) + rho adv_q(b)     (trial-function residual)
  R mga[kElems][4][4];     // [q][a] = m_q . grad phi_a
  R wg[kElems][4][3];      // w grad phi_a
  R Svp[kElems][4], Ppv[kElems][4], Wv[kElems][4][3], Zv[kElems][3], TM[kElems], TC[kElems], muvol[kElems];
  int32_t eid[kElems];     // element of each slot (-1: none)
};

// Extra per-element data of the Newton linearisation of the fully implicit formulation (the
// residual's dependence on u* = u - u_ALE, tau_M(u*), tau_C(u*) and r_M(u, p) at the iterate):
template <class R>
struct ImplShared {
  R Gr[kElems][9];         // grad u of the iterate, (grad u)_ij = d_j u_i (constant on a P1 element)
  R uq[kElems][4][3];      // u*(x_q)
  R rq[kElems][4][3];      // r_M(u, p)(x_q)
  R tm[kElems][4];         // tau_M
  R tcr[kElems][4];        // tau_C / tau_M
  R kap[kElems][4][3];     // d tau_M / d u* = -tau_M^3 rho^2 G u*
  R Gga[kElems][4][3];     // (grad u)^T grad phi_a
};
template <class R, bool IMPL>
struct AsmShared {
  ElemShared<R> e;
};
template <class R>
struct AsmShared<R, true> {
  ElemShared<R> e;
  ImplShared<R> x;
};

// Geometry of one tetrahedron in precision G: grad phi_a = J^-T grad_ref phi_a, the metric
// tensor G = J^-T J^-1 (as its 9 entries), g = J^-T 1, |K| = det J / 6.
template <class G>
__device__ __forceinline__ void tet_geometry(const G x[4][3], G gp[12], G Gm[9], G gv[3], G &vol) {
  G J[3][3];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int r = 0; r < 3; ++r) J[r][c] = x[c + 1][r] - x[0][r];
  G c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  G c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  G c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  G det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
  G id = cst<G>(1.0) / det;
  // inverse: Ji[r][c]
  G Ji[3][3];
  Ji[0][0] = c00 * id;
  Ji[1][0] = c01 * id;
  Ji[2][0] = c02 * id;
  Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id;
  Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
  Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id;
  Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
  Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
  Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
  // grad phi_1..3 = rows of J^-1 transposed: (grad phi_a)_k = Ji[a-1][k]; phi_0 = -(sum)
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    gp[3 + k] = Ji[0][k];
    gp[6 + k] = Ji[1][k];
    gp[9 + k] = Ji[2][k];
    gp[k] = -(Ji[0][k] + Ji[1][k] + Ji[2][k]);
    gv[k] = Ji[0][k] + Ji[1][k] + Ji[2][k];
  }
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int l = 0; l < 3; ++l) Gm[3 * k + l] = Ji[0][k] * Ji[0][l] + Ji[1][k] * Ji[1][l] + Ji[2][k] * Ji[2][l];
  vol = det / cst<G>(6.0);
}

// Phase 1a (one thread per element): geometry in FP64 (FP64 assembly, or a badly shaped
// element in mixed assembly), else FP32.
template <class R>
__device__ void element_geometry(const AssembleArgs &A, int64_t e, R gpo[12], R Go[9], R &GGo, R &igg, R &w) {
  const int4 cn = A.conn[e];
  const int nd[4] = {cn.x, cn.y, cn.z, cn.w};
  const bool fp64_geom = std::is_same<R, double>::value || (A.bad && A.bad[e]);
  if (fp64_geom) {
    double x[4][3], gp[12], G[9], g[3], v;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const D4 p = A.xyz[nd[a]];
      x[a][0] = p.x;
      x[a][1] = p.y;
      x[a][2] = p.z;
    }
    tet_geometry<double>(x, gp, G, g, v);
#pragma unroll
    for (int k = 0; k < 12; ++k) gpo[k] = (R)gp[k];
#pragma unroll
    for (int k = 0; k < 9; ++k) Go[k] = (R)G[k];
    double gg = 0.0;
#pragma unroll
    for (int k = 0; k < 9; ++k) gg += G[k] * G[k];
    GGo = (R)gg;
    igg = (R)(1.0 / (g[0] * g[0] + g[1] * g[1] + g[2] * g[2]));
    w = (R)(0.25 * v);
  } else {
    // geometry in the arithmetic type (FP32, or dd from the split coordinates)
    R x[4][3], g[3], v;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      R p[4];
      ld_node<R>(A.xyz, A.xyz_hi, A.xyz_lo, nd[a], p);
      x[a][0] = p[0];
      x[a][1] = p[1];
      x[a][2] = p[2];
    }
    tet_geometry<R>(x, gpo, Go, g, v);
    GGo = cst<R>(0.0);
#pragma unroll
    for (int k = 0; k < 9; ++k) GGo = fmadd(Go[k], Go[k], GGo);
    igg = cst<R>(1.0) / (g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    w = cst<R>(0.25) * v;
  }
}

// value k of the geometry cache for element e
template <class R>
__device__ __forceinline__ R geo_value(const AssembleArgs &A, int k, int64_t e, int64_t T);
template <>
__device__ __forceinline__ double geo_value<double>(const AssembleArgs &A, int k, int64_t e, int64_t T) {
  return A.geo64[k * T + e];
}
template <>
__device__ __forceinline__ dd geo_value<dd>(const AssembleArgs &A, int k, int64_t e, int64_t T) {
  return dd(A.geo_hi[k * T + e], A.geo_lo[k * T + e]);
}
template <>
__device__ __forceinline__ float geo_value<float>(const AssembleArgs &A, int k, int64_t e, int64_t T) {
  return A.geo_hi[k * T + e];
}
template <class R>
__device__ __forceinline__ bool has_geo(const AssembleArgs &A) {
  return std::is_same<R, double>::value ? A.geo64 != nullptr : A.geo_hi != nullptr;
}

// Phase 1a: geometry of element e into shared memory (one thread per element), when there is no
// cache
template <class R>
__device__ void geom_phase(const AssembleArgs &A, int64_t e, int le, ElemShared<R> &sh) {
  R GG, igg, w;
  element_geometry<R>(A, e, sh.gphi[le], sh.Gm[le], GG, igg, w);
  sh.GG[le] = GG;
  sh.igg[le] = igg;
  sh.w[le] = w;
}

// Phase 1a from the cache: the CTA's threads load kGeoValues values of each of its elements
// (for a fixed value index, consecutive elements are consecutive in memory)
template <class R>
__device__ void geom_load(const AssembleArgs &A, int64_t T, ElemShared<R> &sh) {
  for (int idx = threadIdx.x; idx < kGeoValues * kElems; idx += kCta) {
    const int k = idx / kElems, le = idx % kElems;
    const int64_t e = sh.eid[le];
    if (e < 0) continue;
    const R v = geo_value<R>(A, k, e, T);
    if (k < 12) sh.gphi[le][k] = v;
    else if (k < 21) sh.Gm[le][k - 12] = v;
    else if (k == 21) sh.igg[le] = v;
    else if (k == 22) sh.w[le] = v;
    else sh.GG[le] = v;
  }
}

template <class R>
__global__ void geometry_kernel(AssembleArgs A, int64_t T, double *out64, float *out_hi, float *out_lo) {
  pdl_entry();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < T; e += (int64_t)gridDim.x * blockDim.x) {
    R gp[12], G[9], GG, igg, w, v[kGeoValues];
    element_geometry<R>(A, e, gp, G, GG, igg, w);
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = gp[k];
#pragma unroll
    for (int k = 0; k < 9; ++k) v[12 + k] = G[k];
    v[21] = igg;
    v[22] = w;
    v[23] = GG;
#pragma unroll
    for (int k = 0; k < kGeoValues; ++k) {
      if constexpr (std::is_same<R, double>::value) {
        out64[k * T + e] = v[k];
      } else if constexpr (std::is_same<R, dd>::value) {
        out_hi[k * T + e] = v[k].hi;
        out_lo[k * T + e] = v[k].lo;
      } else {
        out_hi[k * T + e] = v[k];
      }
    }
  }
}

// value of lane src (within the warp) among the lanes of mask
template <class R>
__device__ __forceinline__ R shfl_from(R v, int src, unsigned mask) {
  return __shfl_sync(mask, v, src);
}
template <>
__device__ __forceinline__ dd shfl_from<dd>(dd v, int src, unsigned mask) {
  return dd(__shfl_sync(mask, v.hi, src), __shfl_sync(mask, v.lo, src));
}

// Phase 1b for one (element, quadrature point): u*, u^BDF, tau_M and tau_C (FP64 for the FP64
// and FP32 kernels, dd for the dd kernel), the resistive coefficient (FP64), and the LES vector
// tau_M r_M(u^EXT, p^EXT).
template <class R, bool IMPL>
__device__ void qp_phase(const AssembleArgs &A, const PhysParams &P, const PhysR<R> &Q, int64_t e, int q,
                         int le, ElemShared<R> &sh, ImplShared<R> *ix) {
  const int4 cn = A.conn[e];
  const int nd[4] = {cn.x, cn.y, cn.z, cn.w};
  R ue[4][4], ub[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    ld_node<R>(A.xext, A.xext_hi, A.xext_lo, nd[a], ue[a]);
    ld_node<R>(A.ubdf, A.ubdf_hi, A.ubdf_lo, nd[a], ub[a]);
  }
  const R *gp = sh.gphi[le];
  // barycentric coordinates of point q: phi_a(x_q)
  R lam[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) lam[a] = (a == q) ? cst<R>(kQA) : cst<R>(kQB);
  // u^EXT(x_q), u^BDF(x_q), and the advection velocity u* = u^EXT - u_ALE (Eq. u_star; u_ALE = 0 on
  // a fixed mesh)
  R uq[3], us[3], ubq[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    uq[i] = fmadd(lam[3], ue[3][i], fmadd(lam[2], ue[2][i], fmadd(lam[1], ue[1][i], lam[0] * ue[0][i])));
    ubq[i] = fmadd(lam[3], ub[3][i], fmadd(lam[2], ub[2][i], fmadd(lam[1], ub[1][i], lam[0] * ub[0][i])));
    us[i] = uq[i];
  }
  if (A.uale) {
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const D4 v = A.uale[nd[a]];
      us[0] = us[0] - lam[a] * (R)v.x;
      us[1] = us[1] - lam[a] * (R)v.y;
      us[2] = us[2] - lam[a] * (R)v.z;
    }
  }
  R adv[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) adv[a] = fmadd(us[2], gp[3 * a + 2], fmadd(us[1], gp[3 * a + 1], us[0] * gp[3 * a]));
  // resistive coefficient sum_k (R_k/eps_k) delta_k and sum_k (R_k/eps_k)^2 delta_k^2
  double sR = 0.0, sR2 = 0.0;
  for (int k = 0; k < P.n_riis; ++k) {
    const double *ph = A.phi_riis + (int64_t)k * A.n_nodes;
    double phq = 0.0;
#pragma unroll
    for (int a = 0; a < 4; ++a) phq += ((a == q) ? kQA : kQB) * ph[nd[a]];
    // smoothed Dirac delta of Section 2.1.2: (1 + cos(pi phi/eps)) / (2 eps) inside |phi| <= eps
    const double dl = fabs(phq) > P.riis_eps[k] ? 0.0 : (1.0 + cos(P.riis_pi_eps[k] * phq)) * P.riis_inv2eps[k];
    const double c = P.riis_coef[k] * dl;
    sR += c;
    sR2 += c * c;
  }
  const R sRr = P.n_riis > 0 ? (R)sR : cst<R>(0.0);
  // tau_M, tau_C (Section 2.3)
  const R *Gm = sh.Gm[le];
  R taum, tauc;
  if constexpr (std::is_same<R, dd>::value) {
    R uGu = cst<R>(0.0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      R Gu = cst<R>(0.0);
#pragma unroll
      for (int l = 0; l < 3; ++l) Gu = fmadd(Gm[3 * k + l], us[l], Gu);
      uGu = fmadd(us[k], Gu, uGu);
    }
    R tsum = fmadd(Q.cr_mu2, sh.GG[le], fmadd(Q.rho * Q.rho, uGu, Q.tau_t));
    if (P.n_riis > 0) tsum += (R)sR2;
    taum = dd_rsqrt(tsum);                        // tau_M = tsum^-1/2
    tauc = tsum * taum * sh.igg[le];              // tau_C = 1/(tau_M g.g) = sqrt(tsum)/(g.g)
  } else {
    double uGu = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
#pragma unroll
      for (int l = 0; l < 3; ++l) uGu += (double)us[k] * (double)Gm[3 * k + l] * (double)us[l];
    }
    const double GG = (double)sh.GG[le];
    const double rho = P.rho;
    const double tsum = P.tau_t + rho * rho * uGu + P.cr_mu2 * GG + sR2;
    const double tm = rsqrt(tsum);
    taum = (R)tm;
    tauc = (R)(tsum * tm * (double)sh.igg[le]);
  }
  R z[3] = {cst<R>(0.0), cst<R>(0.0), cst<R>(0.0)};
  // grad p^EXT, constant on the element: the element's four threads (one per quadrature point, a
  // quad of lanes) each form one component (the fourth repeats the third) and exchange them
  R gpr[3];
  if (IMPL || P.stab >= 2) {
    const int c = q < 3 ? q : 2;
    R g = cst<R>(0.0);
#pragma unroll
    for (int a = 0; a < 4; ++a) g = fmadd(ue[a][3], gp[3 * a + c], g);
    const int base = threadIdx.x & 28;
    const unsigned mask = 0xFu << base;
#pragma unroll
    for (int i = 0; i < 3; ++i) gpr[i] = shfl_from<R>(g, base + i, mask);
  }
  if (IMPL) {
    // the iterate's strong residual r_M(u, p), grad u, and the derivative of tau_M in u*
    R rmv[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      R conv = cst<R>(0.0);
#pragma unroll
      for (int a = 0; a < 4; ++a) conv = fmadd(adv[a], ue[a][i], conv);
      rmv[i] = fmadd(sRr, uq[i], fmadd(Q.rho, conv, fmadd(Q.rho_dt, fmadd(Q.alpha, uq[i], -ubq[i]), gpr[i]))) - Q.f[i];
    }
    const R k3 = -(taum * taum * taum) * (Q.rho * Q.rho);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      R Gu = cst<R>(0.0);
#pragma unroll
      for (int l = 0; l < 3; ++l) Gu = fmadd(Gm[3 * k + l], us[l], Gu);
      ix->kap[le][q][k] = k3 * Gu;
      ix->uq[le][q][k] = us[k];
      ix->rq[le][q][k] = rmv[k];
    }
    ix->tm[le][q] = taum;
    ix->tcr[le][q] = tauc / taum;
    if (q == 0) {
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          R g = cst<R>(0.0);
#pragma unroll
          for (int a = 0; a < 4; ++a) g = fmadd(ue[a][i], gp[3 * a + j], g);
          ix->Gr[le][3 * i + j] = g;
        }
    }
  }
  if (P.stab >= 2) {
    // tau_M r_M(u^EXT, p^EXT) with the strong residual of Section 2.3 (-mu Lap u = 0 for P1)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      R conv = cst<R>(0.0);
#pragma unroll
      for (int a = 0; a < 4; ++a) conv = fmadd(adv[a], ue[a][i], conv);
      const R rm = fmadd(sRr, uq[i], fmadd(Q.rho, conv, fmadd(Q.rho_dt, fmadd(Q.alpha, uq[i], -ubq[i]), gpr[i]))) - Q.f[i];
      z[i] = Q.rho * taum * (us[i] - taum * rm);
    }
  }
  const R w = sh.w[le];
  const R wtm = w * taum;
  sh.cs[le][q] = Q.rho_alpha_dt + sRr;
  sh.wtm[le][q] = wtm;
  sh.wtmr[le][q] = wtm * Q.rho;
  sh.wtc[le][q] = w * tauc;
#pragma unroll
  for (int a = 0; a < 4; ++a) sh.adv[le][q][a] = adv[a];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    sh.wz[le][q][i] = w * z[i];
    sh.m[le][q][i] = fmadd(Q.rho_dt, ubq[i], Q.f[i]);
  }
}

// Phase 1c for one (element, node n): per-(qp, node) products and per-node sums over the
// quadrature points, shared by the 16 blocks of the element.
template <class R, bool IMPL>
__device__ void node_phase(const PhysParams &P, const PhysR<R> &Q, int n, int le, ElemShared<R> &sh,
                           ImplShared<R> *ix) {
  if (IMPL) {
    const R *g = sh.gphi[le] + 3 * n;
#pragma unroll
    for (int j = 0; j < 3; ++j)
      ix->Gga[le][n][j] = fmadd(ix->Gr[le][6 + j], g[2], fmadd(ix->Gr[le][3 + j], g[1], ix->Gr[le][j] * g[0]));
  }
  const R w = sh.w[le];
  const R rho = Q.rho;
  const R *gn = sh.gphi[le] + 3 * n;
  const R wA = w * cst<R>(kQA), wB = w * cst<R>(kQB);
  R svp = cst<R>(0.0), ppv = svp, wv0 = svp, wv1 = svp, wv2 = svp;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const R pn = (n == q) ? cst<R>(kQA) : cst<R>(kQB);
    const R wpn = (n == q) ? wA : wB;
    const R an = sh.adv[le][q][n];
    const R cbq = fmadd(rho, an, sh.cs[le][q] * pn);
    const R *mq = sh.m[le][q];
    sh.cb[le][q][n] = cbq;
    sh.E[le][q][n] = (P.stab >= 1) ? fmadd(sh.wtmr[le][q], an, wpn) : wpn;
    sh.mga[le][q][n] = fmadd(mq[2], gn[2], fmadd(mq[1], gn[1], mq[0] * gn[0]));
    svp = fmadd(sh.wtmr[le][q], an, svp);
    ppv = fmadd(sh.wtm[le][q], cbq, ppv);
    wv0 = fmadd(sh.wz[le][q][0], cbq, wv0);
    wv1 = fmadd(sh.wz[le][q][1], cbq, wv1);
    wv2 = fmadd(sh.wz[le][q][2], cbq, wv2);
  }
  sh.Svp[le][n] = svp;
  sh.Ppv[le][n] = ppv;
  sh.Wv[le][n][0] = wv0;
  sh.Wv[le][n][1] = wv1;
  sh.Wv[le][n][2] = wv2;
#pragma unroll
  for (int k = 0; k < 3; ++k) sh.wg[le][n][k] = w * gn[k];
  if (n == 0) {
    R tmw = cst<R>(0.0), tcw = tmw, z0 = tmw, z1 = tmw, z2 = tmw;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      tmw = acc(tmw, sh.wtm[le][q]);
      tcw = acc(tcw, sh.wtc[le][q]);
      z0 = acc(z0, sh.wz[le][q][0]);
      z1 = acc(z1, sh.wz[le][q][1]);
      z2 = acc(z2, sh.wz[le][q][2]);
    }
    sh.TM[le] = tmw;
    sh.TC[le] = tcw;
    sh.Zv[le][0] = z0;
    sh.Zv[le][1] = z1;
    sh.Zv[le][2] = z2;
    sh.muvol[le] = Q.mu * (cst<R>(4.0) * w);
  }
}

template <class S> struct Vec16;
template <> struct Vec16<double> {
  static __device__ __forceinline__ void add(double *dst, const double v[16]) {
    double2 *p = reinterpret_cast<double2 *>(dst);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      double2 o = p[k];
      o.x += v[2 * k];
      o.y += v[2 * k + 1];
      p[k] = o;
    }
  }
};
template <> struct Vec16<float> {
  static __device__ __forceinline__ void add(float *dst, const float v[16]) {
    float4 *p = reinterpret_cast<float4 *>(dst);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float4 o = p[k];
      o.x += v[4 * k];
      o.y += v[4 * k + 1];
      o.z += v[4 * k + 2];
      o.w += v[4 * k + 3];
      p[k] = o;
    }
  }
};

// Phase 2 for one (element, a, b): block (a, b) and right-hand-side entry 4a+b.
// dd values across the 4 lanes (a, b = 0..3) of one block row: sum over b
template <class R>
__device__ __forceinline__ R quad_sum(R v, unsigned mask) {
#pragma unroll
  for (int o = 1; o < 4; o <<= 1) v += __shfl_xor_sync(mask, v, o);
  return v;
}
template <>
__device__ __forceinline__ dd quad_sum<dd>(dd v, unsigned mask) {
#pragma unroll
  for (int o = 1; o < 4; o <<= 1) v += dd(__shfl_xor_sync(mask, v.hi, o), __shfl_xor_sync(mask, v.lo, o));
  return v;
}

// Newton terms of block (a, b) of the fully implicit formulation: the derivatives of the element
// residual through u* (advection velocity and SUPG / VMS test functions), tau_M(u*), tau_C(u*) and
// the second r_M factor of the LES term, which the semi-implicit matrix assembled at the iterate
// (u^EXT = u, p^EXT = p) leaves out; added to blk.  Returns in ext[i] this block's own share
// (X_ab U_b)_i of the right-hand side J U - R(U) = b(U) + X U (the caller sums it over b).
template <class R>
__device__ void newton_block(const AssembleArgs &A, const PhysParams &P, const PhysR<R> &Q, int64_t e, int le,
                             int a, int b, const ElemShared<R> &sh, const ImplShared<R> &ix, R blk[16], R ext[4]) {
  const R *ga = sh.gphi[le] + 3 * a;
  const R *gb = sh.gphi[le] + 3 * b;
  const R *Gr = ix.Gr[le];
  const R *Gga = ix.Gga[le][a];
  const R rho = Q.rho, w = sh.w[le];
  const R divu = Gr[0] + Gr[4] + Gr[8];
  const R z0 = cst<R>(0.0);
  R Sal = z0, Dd = z0, Yc = z0, Mhk[9], Tv[3] = {z0, z0, z0}, Zb[3] = {z0, z0, z0}, Zp[3] = {z0, z0, z0};
#pragma unroll
  for (int k = 0; k < 9; ++k) Mhk[k] = z0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const R pa = (a == q) ? cst<R>(kQA) : cst<R>(kQB);
    const R pb = (b == q) ? cst<R>(kQA) : cst<R>(kQB);
    const R wpb = w * pb;
    const R *r = ix.rq[le][q], *u = ix.uq[le][q], *kp = ix.kap[le][q];
    const R tm = ix.tm[le][q], rt = rho * tm;
    const R rga = fmadd(r[2], ga[2], fmadd(r[1], ga[1], r[0] * ga[0]));
    const R adva = sh.adv[le][q][a];
    R al = rho * pa;                                    // Galerkin (grad u) phi_b e_j
    R h[3] = {z0, z0, z0};
    if (P.stab >= 1) {
      al = fmadd(rho * rt, adva, al);                   // SUPG: r_M's (grad u) part
      const R c1 = -(ix.tcr[le][q] * divu), c2 = rho * adva;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        h[i] = fmadd(c1, ga[i], c2 * r[i]);              // tau_C(u*) and SUPG tau_M(u*)
        Tv[i] = fmadd(wpb * rt, r[i], Tv[i]);            // SUPG test function (u* . grad) v
      }
#pragma unroll
      for (int j = 0; j < 3; ++j) Zp[j] = fmadd(wpb, fmadd(rt, Gga[j], kp[j] * rga), Zp[j]);   // PSPG
    }
    if (P.stab >= 2) {
      al = al - rho * rt * tm * rga;                    // LES: r_M's (grad u) part
      const R c3 = rho * rga, t2 = tm + tm;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        h[i] = fmadd(c3, u[i] - t2 * r[i], h[i]);       // VMS/LES tau_M(u*)
        Zb[i] = fmadd(pb * rho, sh.wz[le][q][i], Zb[i]);   // VMS/LES: second factor's (grad u) part
      }
      const R gam = -(w * rt * tm * rga);
      Dd = fmadd(wpb, rt * rga, fmadd(gam, sh.cb[le][q][b], Dd));   // VMS u* and LES r_M(u) identity parts
      Yc += gam;
    }
    Sal = fmadd(wpb, al, Sal);
    if (P.stab >= 1) {
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const R wh = wpb * h[i];
#pragma unroll
        for (int j = 0; j < 3; ++j) Mhk[3 * i + j] = fmadd(wh, kp[j], Mhk[3 * i + j]);
      }
    }
  }
  // U at node b of the iterate, for the right-hand-side share
  const int4 cn = A.conn[e];
  const int nb = (b == 0) ? cn.x : ((b == 1) ? cn.y : ((b == 2) ? cn.z : cn.w));
  R Ub[4];
  ld_node<R>(A.xext, A.xext_hi, A.xext_lo, nb, Ub);
  R ev[4] = {z0, z0, z0, z0};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      R x = fmadd(Sal, Gr[3 * i + j], Mhk[3 * i + j]);
      x = fmadd(Tv[i], ga[j], x);
      x = fmadd(Zb[i], Gga[j], x);
      if (i == j) x += Dd;
      blk[4 * i + j] += x;
      ev[i] = fmadd(x, Ub[j], ev[i]);
    }
    const R y = Yc * gb[i];
    blk[4 * i + 3] += y;
    ev[i] = fmadd(y, Ub[3], ev[i]);
    blk[12 + i] += Zp[i];
    ev[3] = fmadd(Zp[i], Ub[i], ev[3]);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) ext[i] = ev[i];
}

// Right-hand-side entry (a, i) of element slot le: (f + rho u^BDF/dt, v) with the SUPG, VMS and
// LES test functions (velocity rows), PSPG (pressure row)
template <class R>
__device__ __forceinline__ R rhs_value(const PhysParams &P, const ElemShared<R> &sh, int le, int a, int i) {
  R rhs = cst<R>(0.0);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const R Eqa = sh.E[le][q][a];
    if (i < 3) rhs = fmadd(sh.m[le][q][i], Eqa, fmadd(sh.wz[le][q][i], sh.mga[le][q][a], rhs));
    else if (P.stab >= 1) rhs = fmadd(sh.wtm[le][q], sh.mga[le][q][a], rhs);
  }
  return rhs;
}

// Block (a, b) of element slot le (row = test component, column = trial component)
template <class R>
__device__ __forceinline__ void block_values(const PhysParams &P, int le, int a, int b, const ElemShared<R> &sh,
                                             R blk[16]) {
  const R *ga = sh.gphi[le] + 3 * a;
  const R *gb = sh.gphi[le] + 3 * b;
  const R gab = fmadd(ga[2], gb[2], fmadd(ga[1], gb[1], ga[0] * gb[0]));
  // velocity-velocity scalar: sum_q E_q(a) cb_q(b) = mass/dt + resistive + Galerkin advection
  // + SUPG (Eq. fullydiscrete..., Eq. stabilization_form_SUPG)
  R Mab = cst<R>(0.0);
#pragma unroll
  for (int q = 0; q < 4; ++q) Mab = fmadd(sh.E[le][q][a], sh.cb[le][q][b], Mab);
  const R muvol = sh.muvol[le];
  const R TC = (P.stab >= 1) ? sh.TC[le] : cst<R>(0.0);
  const R *Wv = sh.Wv[le][b];
  const R dg = fmadd(muvol, gab, Mab);                          // + grad-grad diffusion
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const R tci = TC * ga[i];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      R v = fmadd(tci, gb[j], Wv[i] * ga[j]);                   // tau_C div-div + VMS/LES
      if (i == j) v = acc(v, dg);
      if (P.diffusion != 0) v = fmadd(muvol * ga[j], gb[i], v); // symmetric-gradient part
      blk[4 * i + j] = v;
    }
  }
  const R *wga = sh.wg[le][a], *wgb = sh.wg[le][b];
  if (P.stab >= 1) {
    const R svp = sh.Svp[le][a], ppv = sh.Ppv[le][b];
    const R *Zv = sh.Zv[le];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      blk[4 * i + 3] = fmadd(Zv[i], gab, fmadd(svp, gb[i], -wga[i]));   // -(p, div v) + SUPG + VMS/LES
      blk[12 + i] = fmadd(ppv, ga[i], wgb[i]);                         // (div u, q) + PSPG
    }
    blk[15] = sh.TM[le] * gab;                                          // PSPG
  } else {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      blk[4 * i + 3] = -wga[i];
      blk[12 + i] = wgb[i];
    }
    blk[15] = cst<R>(0.0);
  }
}

template <class R, class S, bool IMPL>
__device__ void block_phase(const AssembleArgs &A, const PhysParams &P, const PhysR<R> &Q, int64_t e, int le,
                            int a, int b, const ElemShared<R> &sh, const ImplShared<R> *ix, S *vals) {
  const int i_rhs = b;   // this thread also forms right-hand-side entry (a, i_rhs)
  R blk[16];
  block_values<R>(P, le, a, b, sh, blk);
  R rhs = rhs_value<R>(P, sh, le, a, i_rhs);
  if (IMPL) {
    // the row's share sum_b (X_ab U_b): the quad of lanes of blocks (a, 0..3) sums it
    R ext[4];
    newton_block<R>(A, P, Q, e, le, a, b, sh, *ix, blk, ext);
    const unsigned mask = 0xFu << (threadIdx.x & 28);
#pragma unroll
    for (int i = 0; i < 4; ++i) ext[i] = quad_sum<R>(ext[i], mask);
    rhs += (i_rhs == 0) ? ext[0] : ((i_rhs == 1) ? ext[1] : ((i_rhs == 2) ? ext[2] : ext[3]));
  }
  const int32_t s = A.slot[e * 16 + 4 * a + b];
  const int4 cn = A.conn[e];
  const int na = (a == 0) ? cn.x : ((a == 1) ? cn.y : ((a == 2) ? cn.z : cn.w));
  const int64_t ir = 4 * (int64_t)na + i_rhs;
  // the block's (and the row's) first writer stores instead of reading back zeros
  const uint32_t fm = A.first ? (uint32_t)A.first[e] : 0u;
  const bool bfirst = (fm >> (4 * a + b)) & 1u, rfirst = (fm >> (5 * a)) & 1u;
  if constexpr (std::is_same<R, dd>::value) {
    // dd accumulation into the high (vals) and low parts, with the exact sum: the accumulating
    // sum, which the chunked kernels use, ran this kernel 3.4x slower on a 1M-tet mesh (same
    // registers, no spills; cause not identified), so it is not used here
    float4 *ph = reinterpret_cast<float4 *>(vals + (int64_t)s * 16);
    float4 *pl = reinterpret_cast<float4 *>(A.vals_lo + (int64_t)s * 16);
    if (bfirst) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        ph[k] = make_float4(blk[4 * k].hi, blk[4 * k + 1].hi, blk[4 * k + 2].hi, blk[4 * k + 3].hi);
        pl[k] = make_float4(blk[4 * k].lo, blk[4 * k + 1].lo, blk[4 * k + 2].lo, blk[4 * k + 3].lo);
      }
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        float4 h = ph[k], l = pl[k];
        const dd v0 = dd(h.x, l.x) + blk[4 * k], v1 = dd(h.y, l.y) + blk[4 * k + 1];
        const dd v2 = dd(h.z, l.z) + blk[4 * k + 2], v3 = dd(h.w, l.w) + blk[4 * k + 3];
        ph[k] = make_float4(v0.hi, v1.hi, v2.hi, v3.hi);
        pl[k] = make_float4(v0.lo, v1.lo, v2.lo, v3.lo);
      }
    }
    const dd r = rfirst ? rhs : dd(A.rhs_hi[ir], A.rhs_lo[ir]) + rhs;
    A.rhs_hi[ir] = r.hi;
    A.rhs_lo[ir] = r.lo;
  } else {
    S out[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) out[k] = (S)blk[k];
    if (bfirst) {
#pragma unroll
      for (int k = 0; k < 16; ++k) vals[(int64_t)s * 16 + k] = out[k];
    } else {
      Vec16<S>::add(vals + (int64_t)s * 16, out);
    }
    A.rhs[ir] = rfirst ? (double)rhs : A.rhs[ir] + (double)rhs;
  }
}

// CTAs per SM the register allocation must allow for the double-float kernel: 3 (164 registers)
// measured faster than 4 (128 registers) and 5 (96, with spills) once the element terms used the
// one-pass multiply-add
template <class R> struct MinCtas { static constexpr int value = 1; };
#ifndef LFX_ASM_DD_MIN_CTAS
#define LFX_ASM_DD_MIN_CTAS 3
#endif
template <> struct MinCtas<dd> { static constexpr int value = LFX_ASM_DD_MIN_CTAS; };

template <class R, class S, bool IMPL>
__global__ void __launch_bounds__(kCta, IMPL ? 1 : MinCtas<R>::value) assemble_color_kernel(AssembleArgs A, PhysParams P,
                                                              PhysR<R> Q, int64_t e0, int64_t e1, S *vals) {
  pdl_entry();
  __shared__ AsmShared<R, IMPL> shm;
  ElemShared<R> &sh = shm.e;
  ImplShared<R> *ix = nullptr;
  if constexpr (IMPL) ix = &shm.x;
  const int t = threadIdx.x;
  for (int64_t base = e0 + (int64_t)blockIdx.x * kElems; base < e1; base += (int64_t)gridDim.x * kElems) {
    if (t < kElems) sh.eid[t] = base + t < e1 ? (A.elist ? A.elist[base + t] : (int32_t)(base + t)) : -1;
    __syncthreads();
    if (has_geo<R>(A)) geom_load<R>(A, A.n_elems, sh);
    else if (t < kElems && sh.eid[t] >= 0) geom_phase<R>(A, sh.eid[t], t, sh);
    __syncthreads();
    const int le = t >> 2, q = t & 3;
    const bool live = sh.eid[le] >= 0;
    if (live) qp_phase<R, IMPL>(A, P, Q, sh.eid[le], q, le, sh, ix);
    __syncthreads();
    if (live) node_phase<R, IMPL>(P, Q, q, le, sh, ix);
    __syncthreads();
#pragma unroll 1
    for (int pass = 0; pass < kElems * 16 / kCta; ++pass) {
      const int le2 = pass * (kCta / 16) + (t >> 4);
      const int64_t e = sh.eid[le2];
      if (e >= 0) block_phase<R, S, IMPL>(A, P, Q, e, le2, (t >> 2) & 3, t & 3, sh, ix, vals);
    }
    __syncthreads();
  }
}

// ---- chunked assembly: one CTA per chunk of kElems elements at a time.  The element phases are
// those of the colour kernel; the 16 x kElems block contributions are then formed one pass of kCta
// slots at a time into shared memory (slot code le << 4 | a << 2 | b, runs of slots sharing one
// matrix block, no run straddling two passes), and each run is summed there and written to its
// block once: 16 threads per run, one value each (a store for the block's first-writing chunk, an
// add otherwise).  Diagonal runs (a == b) also carry the rows' right-hand sides.  Chunks of one
// colour share no node, so concurrent CTAs never write the same block or row.
constexpr int kStage = 17;          // staging row: 16 values + 1 to spread shared-memory banks
__device__ __forceinline__ void prefetch_l2(const void *p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}
constexpr int kChunkMaxRuns = 4 * kCta;   // a chunk's slots, the most runs it can have
struct ChunkNoImpl {};
template <class R>
struct ChunkImpl {
  ImplShared<R> x;
  R ext[kElems][4][4][4];   // [element][a][b][i]: block (a, b)'s share (X_ab U_b)_i of row a's right-hand side
};
template <class R, bool IMPL = false>
struct ChunkShared {
  ElemShared<R> e;
  R stage[kCta][kStage];
  R rst[kCta][4];
  // the chunk's tables, staged at its start (runs numbered from the chunk's first run)
  uint16_t code[kChunkMaxPasses * kCta];
  uint16_t meta[kChunkMaxRuns];
  int32_t block[kChunkMaxRuns], node[kChunkMaxRuns];
  int32_t run_off[kChunkMaxPasses + 1], ndiag[kChunkMaxPasses];
  typename std::conditional<IMPL, ChunkImpl<R>, ChunkNoImpl>::type n;   // Newton data (IMPL)
};

// Four consecutive matrix values or one node's four right-hand-side entries (16-byte aligned): their
// old values are loaded ahead of the stores, so that a thread's loads of several items are in
// flight together; a store for the first writer, an add otherwise.
template <class S, class R> struct AccumOut;
template <>
struct AccumOut<double, double> {
  struct Old {
    double2 a, b;
  };
  static __device__ __forceinline__ double *at(const AssembleArgs &A, double *vals, int64_t k, bool is_rhs) {
    return is_rhs ? A.rhs + k : vals + k;
  }
  // (L2 only: in the persistent launch another SM may have written the value since this SM last
  // cached it)
  static __device__ __forceinline__ Old load(const AssembleArgs &A, double *vals, int64_t k, bool is_rhs) {
    const double2 *p = reinterpret_cast<const double2 *>(at(A, vals, k, is_rhs));
    return Old{__ldcg(p), __ldcg(p + 1)};
  }
  static __device__ __forceinline__ void store(const AssembleArgs &A, double *vals, int64_t k, bool is_rhs,
                                               const double v[4], const Old &o, bool first) {
    double2 *p = reinterpret_cast<double2 *>(at(A, vals, k, is_rhs));
    if (first) {
      p[0] = make_double2(v[0], v[1]);
      p[1] = make_double2(v[2], v[3]);
    } else {
      p[0] = make_double2(o.a.x + v[0], o.a.y + v[1]);
      p[1] = make_double2(o.b.x + v[2], o.b.y + v[3]);
    }
  }
};
template <>
struct AccumOut<float, dd> {
  struct Old {
    float4 hi, lo;
  };
  static __device__ __forceinline__ Old load(const AssembleArgs &A, float *vals, int64_t k, bool is_rhs) {
    const float4 *h = reinterpret_cast<const float4 *>(is_rhs ? A.rhs_hi + k : vals + k);
    const float4 *l = reinterpret_cast<const float4 *>(is_rhs ? A.rhs_lo + k : A.vals_lo + k);
    return Old{__ldcg(h), __ldcg(l)};
  }
  static __device__ __forceinline__ void store(const AssembleArgs &A, float *vals, int64_t k, bool is_rhs,
                                               const dd v[4], const Old &o, bool first) {
    float4 *h = reinterpret_cast<float4 *>(is_rhs ? A.rhs_hi + k : vals + k);
    float4 *l = reinterpret_cast<float4 *>(is_rhs ? A.rhs_lo + k : A.vals_lo + k);
    dd r[4] = {v[0], v[1], v[2], v[3]};
    if (!first) {
      r[0] = acc(dd(o.hi.x, o.lo.x), v[0]);
      r[1] = acc(dd(o.hi.y, o.lo.y), v[1]);
      r[2] = acc(dd(o.hi.z, o.lo.z), v[2]);
      r[3] = acc(dd(o.hi.w, o.lo.w), v[3]);
    }
    *h = make_float4(r[0].hi, r[1].hi, r[2].hi, r[3].hi);
    *l = make_float4(r[0].lo, r[1].lo, r[2].lo, r[3].lo);
  }
};
constexpr int kItemsInFlight = 2;   // reduction items (four values each) per thread loaded together (1 and 4 were slower)

// Geometry of the elements e0..e1-1 of a chunk from the cache (the CTA's threads load kGeoValues
// values of each; for a fixed value index, consecutive elements are consecutive in memory)
template <class R>
__device__ void geom_load_range(const AssembleArgs &A, int64_t T, int64_t e0, int64_t e1, ElemShared<R> &sh) {
  for (int idx = threadIdx.x; idx < kGeoValues * kElems; idx += kCta) {
    const int k = idx / kElems, le = idx % kElems;
    const int64_t e = e0 + le;
    if (e >= e1) continue;
    const R v = geo_value<R>(A, k, e, T);
    if (k < 12) sh.gphi[le][k] = v;
    else if (k < 21) sh.Gm[le][k - 12] = v;
    else if (k == 21) sh.igg[le] = v;
    else if (k == 22) sh.w[le] = v;
    else sh.GG[le] = v;
  }
}

// The chunks c0 + blockIdx.x, c0 + blockIdx.x + gridDim.x, ... (< c1).  Each chunk's slot codes,
// run tables and pass offsets are staged in shared memory at its start with loads that do not
// wait on one another (its geometry loads among them), and the next chunk's offsets are loaded
// while this one is processed, so that no phase waits on a chain of dependent global loads; its
// node fields and geometry are prefetched into L2 during this chunk's first pass, its tables
// during the second.
template <class R, class S, bool IMPL>
__device__ __forceinline__ void chunk_range(const AssembleArgs &A, const PhysParams &P, const PhysR<R> &Q,
                                            const ChunkArgs &C, int64_t c0, int64_t c1, S *vals,
                                            ChunkShared<R, IMPL> &cs) {
  ElemShared<R> &sh = cs.e;
  ImplShared<R> *ix = nullptr;
  if constexpr (IMPL) ix = &cs.n.x;
  const int t = threadIdx.x;
  int64_t ch = c0 + blockIdx.x;
  int32_t e0 = 0, e1 = 0, p0 = 0, p1 = 0, rb = 0, re = 0;
  if (ch < c1) {
    e0 = C.elem_off[ch];
    e1 = C.elem_off[ch + 1];
    p0 = C.pass_off[ch];
    p1 = C.pass_off[ch + 1];
    rb = C.run_off[p0];
    re = C.run_off[p1];
  }
  for (; ch < c1; ch += gridDim.x) {
    const int64_t chn = ch + gridDim.x;
    int32_t ne0 = 0, ne1 = 0, np0 = 0, np1 = 0;
    if (chn < c1) {
      ne0 = C.elem_off[chn];
      ne1 = C.elem_off[chn + 1];
      np0 = C.pass_off[chn];
      np1 = C.pass_off[chn + 1];
    }
    // the next chunk's nodes, for the L2 prefetch of its node data during this chunk's passes
    int4 ncn = make_int4(0, 0, 0, 0);
    const bool nlive = chn < c1 && t < kElems && ne0 + t < ne1;
    if (nlive) ncn = A.conn[ne0 + t];
    const int npass = p1 - p0, nrun = re - rb;
    for (int i = t; i < npass * kCta; i += kCta) cs.code[i] = C.code[(int64_t)p0 * kCta + i];
    for (int i = t; i < nrun; i += kCta) {
      cs.meta[i] = C.meta[rb + i];
      cs.block[i] = C.block[rb + i];
      cs.node[i] = C.node[rb + i];
    }
    if (t <= npass) cs.run_off[t] = C.run_off[p0 + t] - rb;
    if (t < npass) cs.ndiag[t] = C.ndiag[p0 + t];
    if (t < kElems) sh.eid[t] = e0 + t < e1 ? (int32_t)(e0 + t) : -1;
    if (has_geo<R>(A)) geom_load_range<R>(A, A.n_elems, e0, e1, sh);
    else if (t < kElems && e0 + t < e1) geom_phase<R>(A, e0 + t, t, sh);
    __syncthreads();
    // the blocks (and rows) this chunk adds to, into L2 ahead of its reduction phases
    for (int r = t; r < nrun; r += kCta) {
      const uint32_t meta = cs.meta[r];
      if ((meta >> 14) & 1) continue;
      const int64_t k = (int64_t)cs.block[r] * 16;
      prefetch_l2(vals + k);
      if (std::is_same<R, dd>::value) prefetch_l2(A.vals_lo + k);
      if (meta >> 15) {
        const int64_t rr = 4 * (int64_t)cs.node[r];
        if (std::is_same<R, dd>::value) {
          prefetch_l2(A.rhs_hi + rr);
          prefetch_l2(A.rhs_lo + rr);
        } else {
          prefetch_l2(A.rhs + rr);
        }
      }
    }
    const int le = t >> 2, q = t & 3;
    const bool live = sh.eid[le] >= 0;
    if (live) qp_phase<R, IMPL>(A, P, Q, sh.eid[le], q, le, sh, ix);
    __syncthreads();
    if (live) node_phase<R, IMPL>(P, Q, q, le, sh, ix);
    // the next chunk's run range (its pass offsets have arrived by now)
    int32_t nrb = 0, nre = 0;
    if (chn < c1) {
      nrb = C.run_off[np0];
      nre = C.run_off[np1];
    }
    __syncthreads();
    for (int pi = 0; pi < npass; ++pi) {
      const uint16_t code = cs.code[pi * kCta + t];
      if (code != 0xffffu) {
        const int l2 = code >> 4, a = (code >> 2) & 3, b = code & 3;
        R blk[16];
        block_values<R>(P, l2, a, b, sh, blk);
        if constexpr (IMPL) {
          R ev[4];
          newton_block<R>(A, P, Q, e0 + l2, l2, a, b, sh, *ix, blk, ev);
#pragma unroll
          for (int i = 0; i < 4; ++i) cs.n.ext[l2][a][b][i] = ev[i];
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) cs.stage[t][k] = blk[k];
        if (a == b) {
#pragma unroll
          for (int i = 0; i < 4; ++i) cs.rst[t][i] = rhs_value<R>(P, sh, l2, a, i);
        }
      }
      if (pi == 0) {
        // the next chunk's node fields and geometry into L2 while this chunk computes
        if (nlive) {
          const int nn[4] = {ncn.x, ncn.y, ncn.z, ncn.w};
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            if (std::is_same<R, dd>::value) {
              prefetch_l2(A.xext_hi + nn[a]);
              prefetch_l2(A.xext_lo + nn[a]);
              prefetch_l2(A.ubdf_hi + nn[a]);
              prefetch_l2(A.ubdf_lo + nn[a]);
            } else {
              prefetch_l2(A.xext + nn[a]);
              prefetch_l2(A.ubdf + nn[a]);
            }
          }
        }
        if (chn < c1 && has_geo<R>(A) && t < 2 * kGeoValues) {
          const int k = t >> 1;
          const int64_t at = (int64_t)k * A.n_elems + ne0 + ((t & 1) ? ne1 - ne0 - 1 : 0);
          if (std::is_same<R, dd>::value) {
            prefetch_l2(A.geo_hi + at);
            prefetch_l2(A.geo_lo + at);
          } else {
            prefetch_l2(A.geo64 + at);
          }
        }
      }
      if (pi == 1 && chn < c1) {
        // the next chunk's slot codes and run tables into L2 (128-byte lines, one per thread)
        const char *base[4] = {reinterpret_cast<const char *>(C.code + (int64_t)np0 * kCta),
                               reinterpret_cast<const char *>(C.meta + nrb), reinterpret_cast<const char *>(C.block + nrb),
                               reinterpret_cast<const char *>(C.node + nrb)};
        const int64_t bytes[4] = {(int64_t)(np1 - np0) * kCta * 2, (int64_t)(nre - nrb) * 2, (int64_t)(nre - nrb) * 4,
                                  (int64_t)(nre - nrb) * 4};
        int idx = t;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int64_t first = reinterpret_cast<uintptr_t>(base[q]) >> 7;
          const int64_t last = bytes[q] > 0 ? (reinterpret_cast<uintptr_t>(base[q]) + bytes[q] - 1) >> 7 : first - 1;
          const int nl = (int)(last - first + 1);
          if (idx >= 0 && idx < nl) prefetch_l2(reinterpret_cast<const void *>((first + idx) << 7));
          idx -= nl;
        }
      }
      __syncthreads();
      const int r0 = cs.run_off[pi], nr = cs.run_off[pi + 1] - r0, nd = cs.ndiag[pi];
      const int items = 4 * nr + nd;     // a block's values in four quarters; a diagonal run's rhs row
      using Out = AccumOut<S, R>;
      for (int jb = t; jb < items; jb += kCta * kItemsInFlight) {
        int64_t where[kItemsInFlight];
        bool is_rhs[kItemsInFlight], first[kItemsInFlight];
        typename Out::Old old[kItemsInFlight];
        R sum[kItemsInFlight][4];
#pragma unroll
        for (int i = 0; i < kItemsInFlight; ++i) {
          const int j = jb + i * kCta;
          where[i] = -1;
          if (j >= items) continue;
          const bool blk_item = j < 4 * nr;
          const int run = r0 + (blk_item ? j >> 2 : j - 4 * nr);
          const int v0 = blk_item ? 4 * (j & 3) : 0;
          const uint32_t meta = cs.meta[run];
          first[i] = (meta >> 14) & 1;
          is_rhs[i] = !blk_item;
          where[i] = blk_item ? (int64_t)cs.block[run] * 16 + v0 : 4 * (int64_t)cs.node[run];
          if (!first[i]) old[i] = Out::load(A, vals, where[i], is_rhs[i]);
          const int st0 = meta & 0xff, len = (meta >> 8) & 63;
#pragma unroll
          for (int v = 0; v < 4; ++v) sum[i][v] = blk_item ? cs.stage[st0][v0 + v] : cs.rst[st0][v];
          for (int k = 1; k < len; ++k) {
#pragma unroll
            for (int v = 0; v < 4; ++v) sum[i][v] = acc(sum[i][v], blk_item ? cs.stage[st0 + k][v0 + v] : cs.rst[st0 + k][v]);
          }
        }
#pragma unroll
        for (int i = 0; i < kItemsInFlight; ++i)
          if (where[i] >= 0) Out::store(A, vals, where[i], is_rhs[i], sum[i], old[i], first[i]);
      }
      __syncthreads();   // (the last one also frees the staged tables for the next chunk)
    }
    if constexpr (IMPL) {
      // Newton right-hand side: every node row of the chunk (one diagonal run each) gains the
      // shares sum_b (X_ab U_b) of the elements of its run, added once to the row
      using Out = AccumOut<S, R>;
      for (int pi = 0; pi < npass; ++pi) {
        const int r0 = cs.run_off[pi], nd = cs.ndiag[pi];
        for (int j = t; j < nd; j += kCta) {
          const uint32_t meta = cs.meta[r0 + j];
          const int st0 = meta & 0xff, len = (meta >> 8) & 63;
          R sum[4];
          for (int k = 0; k < len; ++k) {
            const uint16_t code = cs.code[pi * kCta + st0 + k];
            const int l2 = code >> 4, a = (code >> 2) & 3;
#pragma unroll
            for (int bb = 0; bb < 4; ++bb)
#pragma unroll
              for (int i = 0; i < 4; ++i) sum[i] = (k == 0 && bb == 0) ? cs.n.ext[l2][a][0][i] : acc(sum[i], cs.n.ext[l2][a][bb][i]);
          }
          const int64_t where = 4 * (int64_t)cs.node[r0 + j];
          const typename Out::Old old = Out::load(A, vals, where, true);
          Out::store(A, vals, where, true, sum, old, false);
        }
      }
      __syncthreads();
    }
    e0 = ne0;
    e1 = ne1;
    p0 = np0;
    p1 = np1;
    rb = nrb;
    re = nre;
  }
}

// one launch per chunk colour (IMPL: the Newton system of the fully implicit step)
template <class R, class S, bool IMPL>
__global__ void __launch_bounds__(kCta, IMPL ? 1 : MinCtas<R>::value) assemble_chunk_kernel(AssembleArgs A, PhysParams P,
                                                                                          PhysR<R> Q, ChunkArgs C,
                                                                                          int64_t c0, int64_t c1,
                                                                                          S *vals) {
  pdl_entry();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  chunk_range<R, S, IMPL>(A, P, Q, C, c0, c1, vals, *reinterpret_cast<ChunkShared<R, IMPL> *>(smem_raw));
}

// Grid-wide barrier of a co-resident (cooperatively launched) grid on a counter that only grows:
// every CTA adds one and waits until the count reaches target = (barrier index + 1) x grid size.
// The wait is bounded: after kBarrierSpins polls it sets *err and gives up, and so does every CTA
// that finds *err set, so that no CTA waits on one that has left.  Returns false on failure.
constexpr unsigned kBarrierSpins = 1u << 24;
__device__ __forceinline__ bool grid_barrier(unsigned *count, unsigned target, int *err, unsigned max_spins) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(count, 1u);
    unsigned spins = 0;
    int good = 1;
    while (true) {
      unsigned seen;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(seen) : "l"(count) : "memory");
      if (seen >= target) break;
      if (*(volatile int *)err != 0 || ++spins > max_spins) {
        atomicExch(err, 1);
        good = 0;
        break;
      }
      __nanosleep(64);
    }
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

// every chunk colour in one cooperative launch, colours separated by grid-wide barriers (a test
// can pass unreachable > 0 with a small max_spins to make the first wait run out)
template <class R, class S, bool IMPL>
__global__ void __launch_bounds__(kCta, IMPL ? 1 : MinCtas<R>::value) assemble_chunks_persistent_kernel(
    AssembleArgs A, PhysParams P, PhysR<R> Q, ChunkArgs C, const int32_t *color_off, int n_colors, S *vals,
    unsigned *barrier, int *err, unsigned unreachable, unsigned max_spins) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ChunkShared<R, IMPL> &cs = *reinterpret_cast<ChunkShared<R, IMPL> *>(smem_raw);
  for (int c = 0; c < n_colors; ++c) {
    chunk_range<R, S, IMPL>(A, P, Q, C, color_off[c], color_off[c + 1], vals, cs);
    if (c + 1 < n_colors &&
        !grid_barrier(barrier, (unsigned)(c + 1) * gridDim.x + unreachable, err, max_spins))
      return;
  }
}

__device__ __forceinline__ void split4(const D4 &v, float4 &hi, float4 &lo) {
  const dd a(v.x), b(v.y), c(v.z), d(v.w);
  hi = make_float4(a.hi, b.hi, c.hi, d.hi);
  lo = make_float4(a.lo, b.lo, c.lo, d.lo);
}

__global__ void bdf_kernel(int64_t V, int order, const D4 *h0, const D4 *h1,
                           const D4 *h2, double b0, double b1, double b2, double g0, double g1,
                           double g2, D4 *xext, D4 *ubdf, float4 *xe_hi, float4 *xe_lo,
                           float4 *ub_hi, float4 *ub_lo) {
  pdl_entry();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < V; i += (int64_t)gridDim.x * blockDim.x) {
    D4 a = h0[i];
    D4 e = D4{g0 * a.x, g0 * a.y, g0 * a.z, g0 * a.w};
    D4 u = D4{b0 * a.x, b0 * a.y, b0 * a.z, 0.0};
    if (order >= 2) {
      D4 c = h1[i];
      e.x += g1 * c.x; e.y += g1 * c.y; e.z += g1 * c.z; e.w += g1 * c.w;
      u.x += b1 * c.x; u.y += b1 * c.y; u.z += b1 * c.z;
    }
    if (order >= 3) {
      D4 c = h2[i];
      e.x += g2 * c.x; e.y += g2 * c.y; e.z += g2 * c.z; e.w += g2 * c.w;
      u.x += b2 * c.x; u.y += b2 * c.y; u.z += b2 * c.z;
    }
    xext[i] = e;
    ubdf[i] = u;
    if (xe_hi) {
      split4(e, xe_hi[i], xe_lo[i]);
      split4(u, ub_hi[i], ub_lo[i]);
    }
  }
}

__global__ void dd_combine_kernel(int64_t n, const float *hi, const float *lo, double *out) {
  pdl_entry();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (double)hi[i] + (double)lo[i];
}

// apply_dirichlet_kernel on a double-float matrix: the diagonal scale s = |A_rr| is taken from
// hi + lo in FP64 and stored split
__global__ void apply_dirichlet_dd_kernel(int64_t nd, const int32_t *dnode, const D4 *g, int32_t pin_node,
                                          double pin_value, const int32_t *rowptr, const int32_t *diag,
                                          float *hi, float *lo, double *rhs, double *x0) {
  pdl_entry();
  const int64_t total = 3 * nd + (pin_node >= 0 ? 1 : 0);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    int node, c;
    double gv;
    if (k < 3 * nd) {
      const int64_t d = k / 3;
      c = (int)(k - 3 * d);
      node = dnode[d];
      const D4 gg = g[d];
      gv = (c == 0) ? gg.x : ((c == 1) ? gg.y : gg.z);
    } else {
      node = pin_node;
      c = 3;
      gv = pin_value;
    }
    const int64_t di = (int64_t)diag[node] * 16 + 5 * c;
    double s = fabs((double)hi[di] + (double)lo[di]);
    if (s == 0.0) s = 1.0;
    for (int32_t kb = rowptr[node]; kb < rowptr[node + 1]; ++kb) {
      const int64_t o = (int64_t)kb * 16 + 4 * c;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        hi[o + j] = 0.0f;
        lo[o + j] = 0.0f;
      }
    }
    const dd sd(s);
    hi[di] = sd.hi;
    lo[di] = sd.lo;
    rhs[4 * (int64_t)node + c] = s * gv;
    x0[4 * (int64_t)node + c] = gv;
  }
}

// comp_scale_kernel on a double-float matrix (products in dd)
__global__ void comp_scale_dd_kernel(int64_t V, int n_comp, const int32_t *comp_off, const double *scale,
                                     const int32_t *rowptr, float *hi, float *lo, double *rhs) {
  pdl_entry();
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < 4 * V; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = k >> 2;
    const int i = (int)(k & 3);
    int lo_c = 0, hi_c = n_comp - 1;
    while (lo_c < hi_c) {
      const int mid = (lo_c + hi_c + 1) / 2;
      if (comp_off[mid] <= r) lo_c = mid;
      else hi_c = mid - 1;
    }
    const double sc = scale[lo_c];
    const dd scd(sc);
    for (int32_t kb = rowptr[r]; kb < rowptr[r + 1]; ++kb) {
      const int64_t o = (int64_t)kb * 16 + 4 * i;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const dd v = dd(hi[o + j], lo[o + j]) * scd;
        hi[o + j] = v.hi;
        lo[o + j] = v.lo;
      }
    }
    rhs[k] *= sc;
  }
}

// g at Dirichlet node d: sum_h coef[bc(d)][h] * S[h][d] + coef_nodal[bc(d)] * N[d]
// (Section 2.2.1: g = theta g(t) s(x); NODAL conditions carry their values in N)
__global__ void dirichlet_values_kernel(int64_t nd, int H, const int32_t *bc_of,
                                        const double *S /* [H][nd][3] */, DirCoef C,
                                        const double *N /* [nd][3] */, int nb, D4 *g) {
  pdl_entry();
  for (int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; d < nd; d += (int64_t)gridDim.x * blockDim.x) {
    const int bc = bc_of[d];
    double v[3] = {0.0, 0.0, 0.0};
    for (int h = 0; h < H; ++h) {
      const double c = C.c[bc * H + h];
      if (c == 0.0) continue;
#pragma unroll
      for (int i = 0; i < 3; ++i) v[i] += c * S[((int64_t)h * nd + d) * 3 + i];
    }
    const double cn = C.c[nb * H + bc];
    if (cn != 0.0) {
#pragma unroll
      for (int i = 0; i < 3; ++i) v[i] += cn * N[3 * d + i];
    }
    g[d] = D4{v[0], v[1], v[2], 0.0};
  }
}

// -(h n, v) on Neumann faces, precomputed per node as vec = sum_faces A_f n_f / 3
__global__ void neumann_kernel(int64_t n, const int32_t *node, const int32_t *bc_of,
                               const double *vec /* [n][3] */, DirCoef C, double *rhs) {
  pdl_entry();
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const double h = C.c[bc_of[k]];
    const int64_t r = 4 * (int64_t)node[k];
#pragma unroll
    for (int i = 0; i < 3; ++i) rhs[r + i] -= h * vec[3 * k + i];
  }
}

// Row replacement for constrained unknowns: row r -> s e_r, rhs_r -> s g, x0_r -> g, with
// s = |A_rr| (1 if zero).  Thread per constrained (node, component).
template <class S>
__global__ void apply_dirichlet_kernel(int64_t nd, const int32_t *dnode, const D4 *g,
                                       int32_t pin_node, double pin_value,
                                       const int32_t *rowptr, const int32_t *diag, S *vals,
                                       double *rhs, double *x0) {
  pdl_entry();
  const int64_t total = 3 * nd + (pin_node >= 0 ? 1 : 0);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    int node, c;
    double gv;
    if (k < 3 * nd) {
      const int64_t d = k / 3;
      c = (int)(k - 3 * d);
      node = dnode[d];
      const D4 gg = g[d];
      gv = (c == 0) ? gg.x : ((c == 1) ? gg.y : gg.z);
    } else {
      node = pin_node;
      c = 3;
      gv = pin_value;
    }
    S *dblk = vals + (int64_t)diag[node] * 16;
    double s = fabs((double)dblk[5 * c]);
    if (s == 0.0) s = 1.0;
    for (int32_t kb = rowptr[node]; kb < rowptr[node + 1]; ++kb) {
      S *blk = vals + (int64_t)kb * 16 + 4 * c;
      blk[0] = S(0); blk[1] = S(0); blk[2] = S(0); blk[3] = S(0);
    }
    dblk[5 * c] = (S)s;
    rhs[4 * (int64_t)node + c] = s * gv;
    x0[4 * (int64_t)node + c] = gv;
  }
}

// ||rhs|| of each component (one CTA per component, contiguous node range, fixed order)
__global__ void comp_norm_kernel(const int32_t *comp_off, const double *rhs, double *scale) {
  pdl_entry();
  __shared__ double red[256];
  const int c = blockIdx.x;
  const int64_t i0 = 4 * (int64_t)comp_off[c], i1 = 4 * (int64_t)comp_off[c + 1];
  double s = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) s += rhs[i] * rhs[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) scale[c] = red[0] > 0.0 ? 1.0 / sqrt(red[0]) : 1.0;
}

// rows of component c (matrix and right-hand side) multiplied by scale[c]; thread per scalar row
template <class S>
__global__ void comp_scale_kernel(int64_t V, int n_comp, const int32_t *comp_off, const double *scale,
                                  const int32_t *rowptr, S *vals, double *rhs) {
  pdl_entry();
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < 4 * V; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = k >> 2;
    const int i = (int)(k & 3);
    int lo = 0, hi = n_comp - 1;             // component containing node r
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if (comp_off[mid] <= r) lo = mid;
      else hi = mid - 1;
    }
    const double sc = scale[lo];
    for (int32_t kb = rowptr[r]; kb < rowptr[r + 1]; ++kb) {
      S *blk = vals + (int64_t)kb * 16 + 4 * i;
      blk[0] = (S)(sc * (double)blk[0]);
      blk[1] = (S)(sc * (double)blk[1]);
      blk[2] = (S)(sc * (double)blk[2]);
      blk[3] = (S)(sc * (double)blk[3]);
    }
    rhs[k] *= sc;
  }
}

inline int grid_for(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  if (g > 152 * 32) g = 152 * 32;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

lfx_status launch_bdf(cudaStream_t st, int64_t V, int order, const D4 *h0, const D4 *h1,
                      const D4 *h2, const double beta[3], const double gamma[3],
                      D4 *xext, D4 *ubdf, float4 *xe_hi, float4 *xe_lo, float4 *ub_hi, float4 *ub_lo) {
  note_launches(1);
  pdl_launch(bdf_kernel, grid_for(V, 256), 256, 0, st, V, order, h0, h1, h2, beta[0], beta[1], beta[2],
                                               gamma[0], gamma[1], gamma[2], xext, ubdf, xe_hi, xe_lo,
                                               ub_hi, ub_lo);
  LFX_CUDA_TRY(cudaGetLastError());
  return LFX_OK;
}

lfx_status launch_dd_combine(cudaStream_t st, int64_t n, const float *hi, const float *lo, double *out) {
  if (n == 0) return LFX_OK;
  note_launches(1);
  pdl_launch(dd_combine_kernel, grid_for(n, 256), 256, 0, st, n, hi, lo, out);
  LFX_CUDA_TRY(cudaGetLastError());
  return LFX_OK;
}

lfx_status launch_apply_dirichlet_dd(cudaStream_t st, int64_t nd, const int32_t *dnode, const D4 *g,
                                     int32_t pin_node, double pin_value, const int32_t *rowptr,
                                     const int32_t *diag, float *hi, float *lo, double *rhs, double *x0) {
  const int64_t total = 3 * nd + (pin_node >= 0 ? 1 : 0);
  if (total == 0) return LFX_OK;
  note_launches(1);
  pdl_launch(apply_dirichlet_dd_kernel, grid_for(total, 128), 128, 0, st, nd, dnode, g, pin_node, pin_value, rowptr, diag,
                                                                   hi, lo, rhs, x0);
  LFX_CUDA_TRY(cudaGetLastError());
  return LFX_OK;
}

lfx_status launch_comp_normalize_dd(cudaStream_t st, int64_t V, int n_comp, const int32_t *comp_off,
                                    double *scale, const int32_t *rowptr, float *hi, float *lo, double *rhs) {
  pdl_launch(comp_norm_kernel, n_comp, 256, 0, st, comp_off, rhs, scale);
  pdl_launch(comp_scale_dd_kernel, grid_for(4 * V, 256), 256, 0, st, V, n_comp, comp_off, scale, rowptr, hi, lo, rhs);
  note_launches(2);
  LFX_CUDA_TRY(cudaGetLastError());
  return LFX_OK;
}

template <class R, class S, bool IMPL>
lfx_status launch_chunks_impl(cudaStream_t st, const AssembleArgs &A, const PhysParams &P, const ChunkArgs &C,
                              const int32_t *chunk_color_off, int n_colors, S *vals) {
  const PhysR<R> Q = phys_r<R>(P);
  const size_t smem = sizeof(ChunkShared<R, IMPL>);
  int dev = 0, nsm = 152, per_sm = 1;
  LFX_CUDA_TRY(cudaGetDevice(&dev));
  static int attr_dev = -1;   // the attribute is per device: set again after a device switch
  if (attr_dev != dev) {
    LFX_CUDA_TRY(cudaFuncSetAttribute(assemble_chunk_kernel<R, S, IMPL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    attr_dev = dev;
  }
  LFX_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  LFX_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, assemble_chunk_kernel<R, S, IMPL>, kCta, smem));
  const int64_t resident = (int64_t)nsm * std::max(per_sm, 1);
  for (int c = 0; c < n_colors; ++c) {
    const int64_t c0 = chunk_color_off[c], c1 = chunk_color_off[c + 1];
    if (c1 <= c0) continue;
    const int grid = (int)std::min<int64_t>(c1 - c0, resident);
    pdl_launch(assemble_chunk_kernel<R, S, IMPL>, grid, kCta, smem, st, A, P, Q, C, c0, c1, vals);
    note_launches(1);
  }
  LFX_CUDA_TRY(cudaGetLastError());
  return LFX_OK;
}

template <class R, class S>
lfx_status launch_assemble_chunks(cudaStream_t st, const AssembleArgs &A, const PhysParams &P, const ChunkArgs &C,
                                  const int32_t *chunk_color_off, int n_colors, S *vals, bool newton) {
  return newton ? launch_chunks_impl<R, S, true>(st, A, P, C, chunk_color_off, n_colors, vals)
                : launch_chunks_impl<R, S, false>(st, A, P, C, chunk_color_off, n_colors, vals);
}
template lfx_status launch_assemble_chunks<double, double>(cudaStream_t, const AssembleArgs &, const PhysParams &,
                                                           const ChunkArgs &, const int32_t *, int, double *, bool);
template lfx_status launch_assemble_chunks<dd, float>(cudaStream_t, const AssembleArgs &, const PhysParams &,
                                                      const ChunkArgs &, const int32_t *, int, float *, bool);

template <class R, class S, bool IMPL>
lfx_status launch_persistent_impl(cudaStream_t st, const AssembleArgs &A, const PhysParams &P, const ChunkArgs &C,
                                  const int32_t *d_chunk_color_off, int n_colors, S *vals, unsigned *barrier, int *err,
                                  bool force_timeout) {
  const PhysR<R> Q = phys_r<R>(P);
  const size_t smem = sizeof(ChunkShared<R, IMPL>);
  int dev = 0, nsm = 152, per_sm = 0, coop = 0;
  LFX_CUDA_TRY(cudaGetDevice(&dev));
  static int attr_dev = -1;   // the attribute is per device: set again after a device switch
  if (attr_dev != dev) {
    LFX_CUDA_TRY(cudaFuncSetAttribute(assemble_chunks_persistent_kernel<R, S, IMPL>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr_dev = dev;
  }
  LFX_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  LFX_CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  LFX_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, assemble_chunks_persistent_kernel<R, S, IMPL>,
                                                              kCta, smem));
  if (!coop || per_sm < 1) {
    set_error("persistent assembly: cooperative launch unavailable");
    return LFX_ERR_CUDA;
  }
  LFX_CUDA_TRY(cudaMemsetAsync(barrier, 0, sizeof(unsigned), st));
  LFX_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
  const int grid = nsm * per_sm;
  unsigned unreachable = force_timeout ? 1u : 0u, max_spins = force_timeout ? (1u << 12) : kBarrierSpins;
  void *args[] = {(void *)&A, (void *)&P, (void *)&Q, (void *)&C, (void *)&d_chunk_color_off, (void *)&n_colors,
                  (void *)&vals, (void *)&barrier, (void *)&err, (void *)&unreachable, (void *)&max_spins};
  LFX_CUDA_TRY(cudaLaunchCooperativeKernel((void *)assemble_chunks_persistent_kernel<R, S, IMPL>, dim3(grid), dim3(kCta),
                                           args, smem, st));
  note_launches(1);
  return LFX_OK;
}

template <class R, class S>
lfx_status launch_assemble_persistent(cudaStream_t st, const AssembleArgs &A, const PhysParams &P, const ChunkArgs &C,
                                      const int32_t *d_chunk_color_off, int n_colors, S *vals, unsigned *barrier,
                                      int *err, bool force_timeout, bool newton) {
  return newton ? launch_persistent_impl<R, S, true>(st, A, P, C, d_chunk_color_off, n_colors, vals, barrier, err,
                                                     force_timeout)
                : launch_persistent_impl<R, S, false>(st, A, P, C, d_chunk_color_off, n_colors, vals, barrier, err,
                                                      force_timeout);
}
template lfx_status launch_assemble_persistent<double, double>(cudaStream_t, const AssembleArgs &, const PhysParams &,
                                                               const ChunkArgs &, const int32_t *, int, double *,
                                                               unsigned *, int *, bool, bool);
template lfx_status launch_assemble_persistent<dd, float>(cudaStream_t, const AssembleArgs &, const PhysParams &,
                                                          const ChunkArgs &, const int32_t *, int, float *, unsigned *,
                                                          int *, bool, bool);

int64_t assemble_chunk_wave() {
  int dev = 0, v = 0, sms = 152, per_sm = LFX_ASM_DD_MIN_CTAS;
  if (cudaGetDevice(&dev) == cudaSuccess &&
      cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0) {
    sms = v;
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, assemble_chunk_kernel<dd, float, false>, kCta,
                                                      sizeof(ChunkShared<dd, false>)) == cudaSuccess && b > 0)
      per_sm = b;
  }
  (void)cudaGetLastError();
  return (int64_t)sms * per_sm;
}

template <class R, class S>
lfx_status launch_assemble(cudaStream_t st, const AssembleArgs &A, const PhysParams &P,
                           const int32_t *color_off, int n_colors, S *vals, bool newton) {
  const PhysR<R> Q = phys_r<R>(P);
  for (int c = 0; c < n_colors; ++c) {
    const int64_t e0 = color_off[c], e1 = color_off[c + 1];
    if (e1 <= e0) continue;
    int64_t chunks = (e1 - e0 + kElems - 1) / kElems;
    int grid = (int)(chunks < 152 * 8 ? chunks : 152 * 8);
    if (newton)
      pdl_launch(assemble_color_kernel<R, S, true>, grid, kCta, 0, st, A, P, Q, e0, e1, vals);
    else
      pdl_launch(assemble_color_kernel<R, S, false>, grid, kCta, 0, st, A, P, Q, e0, e1, vals);
    note_launches(1);
  }
  LFX_CUDA_TRY(cudaGetLastError());
  return LFX_OK;
}

namespace {
__global__ void node_scatter_kernel(int64_t V, const int32_t *node_old, const double *u, const double *p, D4 *dst) {
  pdl_entry();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < V; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = node_old[i];
    dst[i] = D4{u[3 * o], u[3 * o + 1], u[3 * o + 2], p[o]};
  }
}
__global__ void node_gather_kernel(int64_t V, const int32_t *node_old, const D4 *src, double *u, double *p) {
  pdl_entry();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < V; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = node_old[i];
    const D4 v = src[i];
    u[3 * o] = v.x;
    u[3 * o + 1] = v.y;
    u[3 * o + 2] = v.z;
    p[o] = v.w;
  }
}
}  // namespace

lfx_status launch_node_scatter(cudaStream_t st, int64_t V, const int32_t *node_old, const double *u, const double *p,
                               D4 *dst) {
  if (V == 0) return LFX_OK;
  pdl_launch(node_scatter_kernel, grid_for(V, 256), 256, 0, st, V, node_old, u, p, dst);
  note_launches(1);
  LFX_CUDA_TRY(cudaGetLastError());
  return LFX_OK;
}
lfx_status launch_node_gather(cudaStream_t st, int64_t V, const int32_t *node_old, const D4 *src, double *u,
                              double *p) {
  if (V == 0) return LFX_OK;
  pdl_launch(node_gather_kernel, grid_for(V, 256), 256, 0, st, V, node_old, src, u, p);
  note_launches(1);
  LFX_CUDA_TRY(cudaGetLastError());
  return LFX_OK;
}

namespace {
__global__ void backflow_edge_kernel(int64_t n_edges, const int32_t *ij, const double *an, const double *coef,
                                     const int32_t *slot4, const D4 *xext, double *acc) {
  pdl_entry();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_edges; e += (int64_t)gridDim.x * blockDim.x) {
    const D4 ui = xext[ij[2 * e]], uj = xext[ij[2 * e + 1]];
    const double un = 0.5 * ((ui.x + uj.x) * an[3 * e] + (ui.y + uj.y) * an[3 * e + 1] + (ui.z + uj.z) * an[3 * e + 2]);
    const double c = -coef[e] * fmin(un, 0.0) / 3.0 * 0.25;
    if (c == 0.0) continue;
#pragma unroll
    for (int t = 0; t < 4; ++t) atomicAdd(acc + slot4[4 * e + t], c);
  }
}
__global__ void backflow_apply_kernel(int64_t n_blocks, const int32_t *blk, const double *acc, double *vals64,
                                      float *hi, float *lo) {
  pdl_entry();
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_blocks; k += (int64_t)gridDim.x * blockDim.x) {
    const double v = acc[k];
    const int64_t s = blk[k];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int64_t q = 16 * s + 5 * d;   // diagonal entry (d, d) of the block
      if (vals64) {
        vals64[q] += v;
      } else {
        const dd r = dd(hi[q], lo[q]) + dd(v);
        hi[q] = r.hi;
        lo[q] = r.lo;
      }
    }
  }
}
}  // namespace

lfx_status launch_backflow(cudaStream_t st, int64_t n_edges, const int32_t *ij, const double *an, const double *coef,
                           const int32_t *slot4, const D4 *xext, int64_t n_blocks, const int32_t *blk, double *acc,
                           double *vals64, float *hi, float *lo) {
  if (n_edges == 0) return LFX_OK;
  LFX_CUDA_TRY(cudaMemsetAsync(acc, 0, sizeof(double) * (size_t)n_blocks, st));
  pdl_launch(backflow_edge_kernel, grid_for(n_edges, 256), 256, 0, st, n_edges, ij, an, coef, slot4, xext, acc);
  pdl_launch(backflow_apply_kernel, grid_for(n_blocks, 256), 256, 0, st, n_blocks, blk, (const double *)acc, vals64,
             hi, lo);
  note_launches(2);
  LFX_CUDA_TRY(cudaGetLastError());
  return LFX_OK;
}

int64_t assemble_wave_elements() {
  int dev = 0, v = 0, sms = 152, per_sm = LFX_ASM_DD_MIN_CTAS;
  if (cudaGetDevice(&dev) == cudaSuccess &&
      cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0) {
    sms = v;
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, assemble_color_kernel<dd, float, false>, kCta, 0) == cudaSuccess &&
        b > 0)
      per_sm = b;
  }
  (void)cudaGetLastError();   // a host without a device leaves a (non-sticky) error behind
  return (int64_t)sms * per_sm * kElems;
}

template <class R>
lfx_status launch_geometry(cudaStream_t st, const AssembleArgs &A, int64_t T, double *out64, float *out_hi,
                           float *out_lo) {
  if (T == 0) return LFX_OK;
  note_launches(1);
  pdl_launch(geometry_kernel<R>, grid_for(T, 128), 128, 0, st, A, T, out64, out_hi, out_lo);
  LFX_CUDA_TRY(cudaGetLastError());
  return LFX_OK;
}
template lfx_status launch_geometry<double>(cudaStream_t, const AssembleArgs &, int64_t, double *, float *, float *);
template lfx_status launch_geometry<dd>(cudaStream_t, const AssembleArgs &, int64_t, double *, float *, float *);

template lfx_status launch_assemble<double, double>(cudaStream_t, const AssembleArgs &, const PhysParams &,
                                                    const int32_t *, int, double *, bool);
template lfx_status launch_assemble<dd, float>(cudaStream_t, const AssembleArgs &, const PhysParams &,
                                               const int32_t *, int, float *, bool);

lfx_status launch_dirichlet_values(cudaStream_t st, int64_t nd, int H, const int32_t *bc_of,
                                   const double *S, const DirCoef &C, const double *N, int nb, D4 *g) {
  if (nd == 0) return LFX_OK;
  note_launches(1);
  pdl_launch(dirichlet_values_kernel, grid_for(nd, 256), 256, 0, st, nd, H, bc_of, S, C, N, nb, g);
  LFX_CUDA_TRY(cudaGetLastError());
  return LFX_OK;
}

lfx_status launch_neumann(cudaStream_t st, int64_t n, const int32_t *node, const int32_t *bc_of,
                          const double *vec, const DirCoef &C, double *rhs) {
  if (n == 0) return LFX_OK;
  note_launches(1);
  pdl_launch(neumann_kernel, grid_for(n, 256), 256, 0, st, n, node, bc_of, vec, C, rhs);
  LFX_CUDA_TRY(cudaGetLastError());
  return LFX_OK;
}

lfx_status launch_comp_normalize(cudaStream_t st, int64_t V, int n_comp, const int32_t *comp_off, double *scale,
                                 const int32_t *rowptr, double *vals, double *rhs) {
  pdl_launch(comp_norm_kernel, n_comp, 256, 0, st, comp_off, rhs, scale);
  pdl_launch(comp_scale_kernel<double>, grid_for(4 * V, 256), 256, 0, st, V, n_comp, comp_off, scale, rowptr, vals, rhs);
  note_launches(2);
  LFX_CUDA_TRY(cudaGetLastError());
  return LFX_OK;
}

template <class S>
lfx_status launch_apply_dirichlet(cudaStream_t st, int64_t nd, const int32_t *dnode, const D4 *g,
                                  int32_t pin_node, double pin_value, const int32_t *rowptr,
                                  const int32_t *diag, S *vals, double *rhs, double *x0) {
  int64_t total = 3 * nd + (pin_node >= 0 ? 1 : 0);
  if (total == 0) return LFX_OK;
  note_launches(1);
  pdl_launch(apply_dirichlet_kernel<S>, grid_for(total, 128), 128, 0, st, nd, dnode, g, pin_node, pin_value,
                                                                  rowptr, diag, vals, rhs, x0);
  LFX_CUDA_TRY(cudaGetLastError());
  return LFX_OK;
}
template lfx_status launch_apply_dirichlet<double>(cudaStream_t, int64_t, const int32_t *, const D4 *,
                                                   int32_t, double, const int32_t *, const int32_t *,
                                                   double *, double *, double *);
template lfx_status launch_apply_dirichlet<float>(cudaStream_t, int64_t, const int32_t *, const D4 *,
                                                  int32_t, double, const int32_t *, const int32_t *,
                                                  float *, double *, double *);

}  // namespace lfx
