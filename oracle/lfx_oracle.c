/*
 * Oracle (test infrastructure only): plain, slow, FP64 element routines for one semi-implicit
 * BDF step of the P1-P1 VMS-LES Navier-Stokes discretisation of Section 2.3, Eq.
 * (fullydiscrete_ns_ale_riis_vmsles_quasistatic_unified).  Only the tests, the smoke check and
 * the CPU-baseline leg of the benchmark may load this library; the CUDA path shares no code
 * with it.  Everything is written loop by loop from the weak form, with no blocking, fusion
 * or reordering, so that each term can be checked against the paper by eye.
 *
 * Local unknown numbering: 4*a + c, node a in 0..3, c = 0,1,2 velocity components, c = 3
 * pressure.  Element matrix A[16][16] row-major (row = test function, column = trial function).
 *
 * Readings of the paper taken here (where it is silent or ambiguous):
 *  - Reference element: unit right simplex, phi_0 = 1-xi-eta-zeta, phi_1 = xi, phi_2 = eta,
 *    phi_3 = zeta; J = [x1-x0 | x2-x0 | x3-x0]; G = J^-T J^-1, g = J^-T (1,1,1)  (Sec. 2.3,
 *    definitions after the tau formulas).
 *  - Quadrature: 4-point degree-2 symmetric rule, barycentric (a,b,b,b) and permutations with
 *    a = (5+3 sqrt5)/20, b = (5-sqrt5)/20, weights |K|/4.
 *  - Semi-implicit advection velocity u* = u^EXT (no ALE, u_ALE = 0).
 *  - (grad v)_ij = d v_i / d x_j; SUPG uses the advective derivative (u*.grad)v; the VMS term uses
 *    sum_i u*_i d_j v_i (the transposed, cross-stress form); (a (x) b, grad v) = sum_ij a_i b_j d_j v_i.
 *  - -mu Laplacian(u) vanishes for P1 (strong residual r_M, Sec. 2.3).
 *  - RIIS level set: the P1 interpolant of nodal signed distances; u_Sigma = 0.
 *  - r_M(u^EXT, p^EXT) in the LES term keeps its time-derivative part (alpha u^EXT - u^BDF)/dt.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAX_RIIS 8

typedef struct {
  double rho, mu, dt;
  double alpha;        /* alpha_BDF */
  double sigma;        /* sigma_BDF, the BDF order, used squared in tau_M */
  double c_r;          /* C_r in tau_M */
  double f[3];         /* constant body force */
  int32_t n_riis;
  int32_t stab;        /* 0 Galerkin only, 1 SUPG-PSPG, 2 VMS-LES */
  int32_t diffusion;   /* 0 grad-grad, 1 symgrad-grad, 2 symgrad-symgrad */
  int32_t pad;
  double riis_r[ORC_MAX_RIIS];    /* R_k */
  double riis_eps[ORC_MAX_RIIS];  /* epsilon_k */
} orc_params;

/* ---- geometry (Sec. 2.3: J, G = J^-T J^-1, g = J^-T 1) ---------------------------------- */
double orc_geometry(const double x[12], double gradphi[12], double G[9], double g[3],
                    double *volume) {
  double J[3][3];   /* J[r][c] = d x_r / d xi_c */
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) J[r][c] = x[3 * (c + 1) + r] - x[r];
  double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1])
             - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0])
             + J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  double Ji[3][3];  /* J^-1 by cofactors */
  Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
  Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
  Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
  Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
  /* reference gradients of phi_0..phi_3 */
  const double gh[4][3] = {{-1, -1, -1}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  for (int a = 0; a < 4; ++a)
    for (int k = 0; k < 3; ++k) {   /* grad phi_a = J^-T gh_a : (J^-T)_{k m} = Ji[m][k] */
      double s = 0;
      for (int m = 0; m < 3; ++m) s += Ji[m][k] * gh[a][m];
      gradphi[3 * a + k] = s;
    }
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l) {
      double s = 0;
      for (int m = 0; m < 3; ++m) s += Ji[m][k] * Ji[m][l];
      G[3 * k + l] = s;
    }
  for (int k = 0; k < 3; ++k) g[k] = Ji[0][k] + Ji[1][k] + Ji[2][k];
  if (volume) *volume = det / 6.0;
  return det;
}

/* ---- quadrature: barycentric coordinates of the 4 points, weight = |K|/4 ---------------- */
static void qp_bary(int q, double lam[4]) {
  const double qa = 0.58541019662496845446, qb = 0.13819660112501051518;
  for (int a = 0; a < 4; ++a) lam[a] = (a == q) ? qa : qb;
}

/* smoothed Dirac delta of Sec. 2.1.2 */
double orc_delta(double phi, double eps) {
  if (fabs(phi) > eps) return 0.0;
  return (1.0 + cos(M_PI * phi / eps)) / (2.0 * eps);
}

/* tau_M and tau_C of Sec. 2.3 */
void orc_tau(const orc_params *P, const double G[9], const double g[3], const double us[3],
             const double *delta, double *tau_m, double *tau_c) {
  double uGu = 0, GG = 0, gg = 0;
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l) {
      uGu += us[k] * G[3 * k + l] * us[l];
      GG += G[3 * k + l] * G[3 * k + l];
    }
  for (int k = 0; k < 3; ++k) gg += g[k] * g[k];
  double s = P->sigma * P->sigma * P->rho * P->rho / (P->dt * P->dt)
           + P->rho * P->rho * uGu + P->c_r * P->mu * P->mu * GG;
  for (int k = 0; k < P->n_riis; ++k) {
    double c = P->riis_r[k] / P->riis_eps[k] * delta[k];
    s += c * c;
  }
  *tau_m = 1.0 / sqrt(s);
  *tau_c = 1.0 / (*tau_m * gg);
}

/* Per-quadrature-point coefficients shared by the matrix and the residual routines. */
typedef struct {
  double w, phi[4], us[3], ubdf[3], m[3], sR, tau_m, tau_c, s[3];
} qp_data;

static void element_qp(const orc_params *P, const double x[12], const double gradphi[12],
                       const double G[9], const double g[3], double vol, const double ubdf[12],
                       const double uext[12], const double pext[4], const double *phinod,
                       const double *uale, int q, qp_data *d) {
  double lam[4];
  qp_bary(q, lam);
  d->w = vol / 4.0;
  for (int a = 0; a < 4; ++a) d->phi[a] = lam[a];
  double ue[3] = {0, 0, 0};
  for (int i = 0; i < 3; ++i) {
    d->us[i] = 0; d->ubdf[i] = 0;
    for (int a = 0; a < 4; ++a) {
      d->us[i] += lam[a] * uext[3 * a + i];
      d->ubdf[i] += lam[a] * ubdf[3 * a + i];
    }
    ue[i] = d->us[i];            /* u^EXT at the point */
  }
  /* u* = u^EXT - u_ALE (semi-implicit, Eq. u_star); u_ALE = 0 on a fixed mesh (uale NULL) */
  if (uale)
    for (int i = 0; i < 3; ++i)
      for (int a = 0; a < 4; ++a) d->us[i] -= lam[a] * uale[3 * a + i];
  double delta[ORC_MAX_RIIS];
  d->sR = 0;
  for (int k = 0; k < P->n_riis; ++k) {
    double ph = 0;
    for (int a = 0; a < 4; ++a) ph += lam[a] * phinod[4 * k + a];
    delta[k] = orc_delta(ph, P->riis_eps[k]);
    d->sR += P->riis_r[k] / P->riis_eps[k] * delta[k];
  }
  orc_tau(P, G, g, d->us, delta, &d->tau_m, &d->tau_c);
  for (int i = 0; i < 3; ++i) d->m[i] = P->rho * d->ubdf[i] / P->dt + P->f[i];
  /* strong momentum residual at (u^EXT, p^EXT): rho((alpha u - u^BDF)/dt + (u*.grad)u) + grad p
     + R u - f ; grad u^EXT and grad p^EXT are constant on a P1 element */
  for (int i = 0; i < 3; ++i) {
    double adv = 0, gp = 0;
    for (int a = 0; a < 4; ++a) {
      double ua = 0;
      for (int j = 0; j < 3; ++j) ua += d->us[j] * gradphi[3 * a + j];
      adv += ua * uext[3 * a + i];
      gp += pext[a] * gradphi[3 * a + i];
    }
    double rm = P->rho * ((P->alpha * ue[i] - d->ubdf[i]) / P->dt + adv) + gp + d->sR * ue[i] - P->f[i];
    d->s[i] = d->tau_m * rm;
  }
}

/* Per-quadrature-point coefficients of one element, for the tests that pin them one by one:
 * out[0] = tau_M, out[1] = tau_C, out[2..4] = tau_M r_M(u^EXT, p^EXT) (the LES factor),
 * out[5..7] = u*, out[8] = sum_k (R_k/eps_k) delta_k, out[9..11] = m = rho u^BDF/dt + f,
 * out[12] = the quadrature weight. */
int orc_qp_coefficients(const orc_params *P, const double x[12], const double ubdf[12],
                        const double uext[12], const double pext[4], const double *phinod,
                        const double *uale, int q, double out[13]) {
  double gp[12], G[9], g[3], vol;
  double det = orc_geometry(x, gp, G, g, &vol);
  if (!(det > 0) || q < 0 || q > 3) return -1;
  qp_data d;
  element_qp(P, x, gp, G, g, vol, ubdf, uext, pext, phinod, uale, q, &d);
  out[0] = d.tau_m;
  out[1] = d.tau_c;
  for (int i = 0; i < 3; ++i) {
    out[2 + i] = d.s[i];
    out[5 + i] = d.us[i];
    out[9 + i] = d.m[i];
  }
  out[8] = d.sR;
  out[12] = d.w;
  return 0;
}

/* ---- element matrix and right-hand side ------------------------------------------------ */
int orc_element(const orc_params *P, const double x[12], const double ubdf[12],
                const double uext[12], const double pext[4], const double *phinod,
                const double *uale, double A[256], double b[16]) {
  double gp[12], G[9], g[3], vol;
  double det = orc_geometry(x, gp, G, g, &vol);
  if (!(det > 0)) return -1;
  memset(A, 0, 256 * sizeof(double));
  memset(b, 0, 16 * sizeof(double));
  const double rho = P->rho, mu = P->mu, ca = P->rho * P->alpha / P->dt;
  for (int q = 0; q < 4; ++q) {
    qp_data d;
    element_qp(P, x, gp, G, g, vol, ubdf, uext, pext, phinod, uale, q, &d);
    const double w = d.w;
    for (int a = 0; a < 4; ++a) {
      const double *ga = gp + 3 * a;
      const double ua = d.us[0] * ga[0] + d.us[1] * ga[1] + d.us[2] * ga[2];   /* u*.grad phi_a */
      const double mga = d.m[0] * ga[0] + d.m[1] * ga[1] + d.m[2] * ga[2];
      /* right-hand side */
      for (int i = 0; i < 3; ++i) {
        double r = d.phi[a] * d.m[i];                                  /* (f + rho u^BDF/dt, v) */
        if (P->stab >= 1) r += d.tau_m * d.m[i] * rho * ua;           /* SUPG */
        if (P->stab >= 2) {
          r += rho * d.tau_m * d.us[i] * mga;                          /* VMS */
          r -= rho * d.tau_m * d.s[i] * mga;                           /* LES */
        }
        b[4 * a + i] += w * r;
      }
      if (P->stab >= 1) b[4 * a + 3] += w * d.tau_m * mga;             /* PSPG */
      for (int bb = 0; bb < 4; ++bb) {
        const double *gb = gp + 3 * bb;
        const double ub = d.us[0] * gb[0] + d.us[1] * gb[1] + d.us[2] * gb[2];
        const double gab = ga[0] * gb[0] + ga[1] * gb[1] + ga[2] * gb[2];
        const double cb = (ca + d.sR) * d.phi[bb] + rho * ub;         /* r~_M of u = phi_b e_j, per comp */
        for (int i = 0; i < 3; ++i) {
          for (int j = 0; j < 3; ++j) {
            double v = 0;
            if (i == j) {
              v += (ca + d.sR) * d.phi[a] * d.phi[bb];                 /* mass/dt + resistive */
              v += rho * d.phi[a] * ub;                                /* (rho (u*.grad) u, v) */
              v += mu * gab;                                           /* grad-grad diffusion */
            }
            if (P->diffusion != 0) v += mu * ga[j] * gb[i];            /* symmetric-gradient part */
            if (P->stab >= 1) {
              if (i == j) v += d.tau_m * rho * ua * cb;                /* SUPG */
              v += d.tau_c * ga[i] * gb[j];                            /* (tau_C div u, div v) */
            }
            if (P->stab >= 2) {
              v += rho * d.tau_m * d.us[i] * cb * ga[j];               /* VMS */
              v -= rho * d.tau_m * d.s[i] * cb * ga[j];                /* LES */
            }
            A[16 * (4 * a + i) + 4 * bb + j] += w * v;
          }
          /* velocity test, pressure trial */
          double v = -d.phi[bb] * ga[i];                               /* -(p, div v) */
          if (P->stab >= 1) v += d.tau_m * rho * ua * gb[i];           /* SUPG */
          if (P->stab >= 2) {
            v += rho * d.tau_m * d.us[i] * gab;                        /* VMS */
            v -= rho * d.tau_m * d.s[i] * gab;                         /* LES */
          }
          A[16 * (4 * a + i) + 4 * bb + 3] += w * v;
        }
        /* pressure test */
        for (int j = 0; j < 3; ++j) {
          double v = d.phi[a] * gb[j];                                 /* (div u, q) */
          if (P->stab >= 1) v += d.tau_m * cb * ga[j];                 /* PSPG */
          A[16 * (4 * a + 3) + 4 * bb + j] += w * v;
        }
        if (P->stab >= 1) A[16 * (4 * a + 3) + 4 * bb + 3] += w * d.tau_m * gab;   /* PSPG */
      }
    }
  }
  return 0;
}

/* ---- element residual written from the strong residual at each quadrature point --------
 * R(sol) = A sol - b, computed without forming A: the fields u_h, p_h of the local solution are
 * evaluated at the point, r_M and r_C are formed as vectors, and each term of the weak form is
 * tested against every basis function.  Used by the finite-difference checks of orc_element. */
int orc_element_residual(const orc_params *P, const double x[12], const double ubdf[12],
                         const double uext[12], const double pext[4], const double *phinod,
                         const double *uale, const double sol[16], double R[16]) {
  double gp[12], G[9], g[3], vol;
  double det = orc_geometry(x, gp, G, g, &vol);
  if (!(det > 0)) return -1;
  memset(R, 0, 16 * sizeof(double));
  double gu[3][3] = {{0}}, gpr[3] = {0}, divu = 0;
  for (int a = 0; a < 4; ++a)
    for (int i = 0; i < 3; ++i) {
      for (int j = 0; j < 3; ++j) gu[i][j] += sol[4 * a + i] * gp[3 * a + j];
      gpr[i] += sol[4 * a + 3] * gp[3 * a + i];
    }
  divu = gu[0][0] + gu[1][1] + gu[2][2];
  for (int q = 0; q < 4; ++q) {
    qp_data d;
    element_qp(P, x, gp, G, g, vol, ubdf, uext, pext, phinod, uale, q, &d);
    double u[3] = {0, 0, 0}, p = 0;
    for (int a = 0; a < 4; ++a) {
      for (int i = 0; i < 3; ++i) u[i] += d.phi[a] * sol[4 * a + i];
      p += d.phi[a] * sol[4 * a + 3];
    }
    double adv[3], rm[3];
    for (int i = 0; i < 3; ++i) {
      adv[i] = gu[i][0] * d.us[0] + gu[i][1] * d.us[1] + gu[i][2] * d.us[2];
      rm[i] = P->rho * (P->alpha * u[i] - d.ubdf[i]) / P->dt + P->rho * adv[i] + gpr[i]
            + d.sR * u[i] - P->f[i];
    }
    for (int a = 0; a < 4; ++a) {
      const double *ga = gp + 3 * a;
      const double ua = d.us[0] * ga[0] + d.us[1] * ga[1] + d.us[2] * ga[2];
      const double rga = rm[0] * ga[0] + rm[1] * ga[1] + rm[2] * ga[2];
      for (int i = 0; i < 3; ++i) {
        double r = 0;
        /* Galerkin: rho (alpha u - u^BDF)/dt + rho (u*.grad) u + R u - f, tested with phi_a e_i */
        r += d.phi[a] * (P->rho * (P->alpha * u[i] - d.ubdf[i]) / P->dt + P->rho * adv[i]
                         + d.sR * u[i] - P->f[i]);
        double dif = gu[i][0] * ga[0] + gu[i][1] * ga[1] + gu[i][2] * ga[2];     /* grad u : grad v */
        if (P->diffusion != 0)                                                   /* + (grad u)^T : grad v */
          dif += gu[0][i] * ga[0] + gu[1][i] * ga[1] + gu[2][i] * ga[2];
        r += P->mu * dif;
        r -= p * ga[i];                                                          /* -(p, div v) */
        if (P->stab >= 1) {
          r += d.tau_m * rm[i] * P->rho * ua;                                    /* SUPG */
          r += d.tau_c * divu * ga[i];
        }
        if (P->stab >= 2) {
          r += P->rho * d.tau_m * d.us[i] * rga;                                 /* VMS */
          r -= P->rho * d.s[i] * d.tau_m * rga;                                  /* LES */
        }
        R[4 * a + i] += d.w * r;
      }
      double rq = d.phi[a] * divu;
      if (P->stab >= 1) rq += d.tau_m * rga;                                     /* PSPG */
      R[4 * a + 3] += d.w * rq;
    }
  }
  return 0;
}

/* Threads of the element loops below (OpenMP builds; each element is computed on its own, so the
 * results do not depend on the count).  Returns the count in use (1 without OpenMP). */
int orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* ---- batch driver: element matrices for a list of elements of a global mesh ------------ */
int orc_elements(const orc_params *P, const double *nodes, const int32_t *tets,
                 const int64_t *elems, int64_t n, const double *ubdf, const double *uext,
                 const double *pext, const double *phinod /* [n_riis][V] */,
                 const double *uale /* [V][3] mesh velocity, or NULL */, int64_t n_nodes,
                 double *A /* [n][256] */, double *b /* [n][16] */) {
  int err = 0;
#pragma omp parallel for schedule(static)
  for (int64_t t = 0; t < n; ++t) {
    const int32_t *v = tets + 4 * elems[t];
    double x[12], ub[12], ue[12], ua[12], pe[4], ph[4 * ORC_MAX_RIIS];
    for (int a = 0; a < 4; ++a) {
      for (int i = 0; i < 3; ++i) {
        x[3 * a + i] = nodes[3 * (int64_t)v[a] + i];
        ub[3 * a + i] = ubdf[3 * (int64_t)v[a] + i];
        ue[3 * a + i] = uext[3 * (int64_t)v[a] + i];
        ua[3 * a + i] = uale ? uale[3 * (int64_t)v[a] + i] : 0.0;
      }
      pe[a] = pext[v[a]];
      for (int k = 0; k < P->n_riis; ++k) ph[4 * k + a] = phinod[k * n_nodes + v[a]];
    }
    if (orc_element(P, x, ub, ue, pe, ph, uale ? ua : NULL, A + 256 * t, b + 16 * t) != 0) {
#pragma omp critical
      if (err == 0 || -1 - (int)t > err) err = -1 - (int)t;
    }
  }
  return err;
}

/* ---- fully implicit formulation (Eq. u_star, implicit; implicit LES term) ---------------
 * The residual of one element when the advection velocity and the LES residual are taken at the
 * unknown itself: the semi-implicit residual with u^EXT, p^EXT replaced by the element's own
 * solution, so that u* = u - u_ALE, tau_M = tau_M(u*) and every r_M is r_M(u, p). */
int orc_element_residual_implicit(const orc_params *P, const double x[12], const double ubdf[12],
                                  const double sol[16], const double *phinod, const double *uale,
                                  double R[16]) {
  double ue[12], pe[4];
  for (int a = 0; a < 4; ++a) {
    for (int i = 0; i < 3; ++i) ue[3 * a + i] = sol[4 * a + i];
    pe[a] = sol[4 * a + 3];
  }
  return orc_element_residual(P, x, ubdf, ue, pe, phinod, uale, sol, R);
}

/* Residuals R [n][16] and their Jacobians J [n][16][16] by central differences of step h in each
 * of the 16 local unknowns, for a list of elements of a global mesh at the global solution
 * sol [V][4] (the building blocks of Newton's method for the implicit formulation). */
int orc_elements_implicit(const orc_params *P, const double *nodes, const int32_t *tets,
                          const int64_t *elems, int64_t n, const double *ubdf, const double *sol,
                          const double *phinod, const double *uale, int64_t n_nodes, double h,
                          double *J, double *R) {
  int err = 0;
#pragma omp parallel for schedule(static)
  for (int64_t t = 0; t < n; ++t) {
    const int32_t *v = tets + 4 * elems[t];
    double x[12], ub[12], ua[12], s[16], ph[4 * ORC_MAX_RIIS];
    for (int a = 0; a < 4; ++a) {
      for (int i = 0; i < 3; ++i) {
        x[3 * a + i] = nodes[3 * (int64_t)v[a] + i];
        ub[3 * a + i] = ubdf[3 * (int64_t)v[a] + i];
        ua[3 * a + i] = uale ? uale[3 * (int64_t)v[a] + i] : 0.0;
      }
      for (int c = 0; c < 4; ++c) s[4 * a + c] = sol[4 * (int64_t)v[a] + c];
      for (int k = 0; k < P->n_riis; ++k) ph[4 * k + a] = phinod[k * n_nodes + v[a]];
    }
    const double *uap = uale ? ua : NULL;
    if (orc_element_residual_implicit(P, x, ub, s, ph, uap, R + 16 * t) != 0) {
#pragma omp critical
      if (err == 0 || -1 - (int)t > err) err = -1 - (int)t;
      continue;
    }
    for (int k = 0; k < 16; ++k) {
      double sp[16], sm[16], Rp[16], Rm[16];
      memcpy(sp, s, sizeof sp);
      memcpy(sm, s, sizeof sm);
      sp[k] += h;
      sm[k] -= h;
      orc_element_residual_implicit(P, x, ub, sp, ph, uap, Rp);
      orc_element_residual_implicit(P, x, ub, sm, ph, uap, Rm);
      for (int i = 0; i < 16; ++i) J[256 * t + 16 * i + k] = (Rp[i] - Rm[i]) / (2.0 * h);
    }
  }
  return err;
}
