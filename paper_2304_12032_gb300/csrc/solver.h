// aSIMPLE preconditioner and restarted GMRES on the device (Section 2.4).
#pragma once

#include <cmath>

#include "kernels.h"

namespace lfx {

constexpr int kMaxRestart = 64;
constexpr int kMaxSmooth = 32;

struct SmootherConfig {
  int f_kind = LFX_SMOOTH_CHEBYSHEV, f_steps = 3;
  double f_omega = 0.7, f_ratio = 8.0;
  int s_kind = LFX_SMOOTH_CHEBYSHEV, s_steps = 6;
  double s_omega = 0.7, s_ratio = 30.0;
  int n_power = 10;
};

// Device-resident smoothing coefficients (Chebyshev from lambda_max, or constant Jacobi).
struct SmoothCoef {
  double lam_f, lam_s;            // power-iteration estimates (before the 1.1 safety factor)
  double f_init, s_init;          // first step: d_0 = init * diag^-1 b
  double f_c1[kMaxSmooth], f_c2[kMaxSmooth];
  double s_c1[kMaxSmooth], s_c2[kMaxSmooth];
};

// Device-resident GMRES status and small dense data (Hessenberg, Givens, g).
struct KState {
  int done;                       // cycle finished (converged, full, or failed)
  int j;                          // Arnoldi steps completed in this cycle
  int total;                      // steps over all cycles
  int flag;                       // 0 running/full, 1 converged, 2 non-finite
  double bnorm, tol_abs, beta, res, scale;
  double H[kMaxRestart * (kMaxRestart + 1)];   // column-major, ld = kMaxRestart + 1
  double g[kMaxRestart + 1], cs[kMaxRestart], sn[kMaxRestart], y[kMaxRestart];
  double hcol[kMaxRestart + 1], hwork[kMaxRestart + 1];
};

template <class S, class T>
struct ASimple {
  int64_t V = 0;
  SmootherConfig cfg;
  DBuf dinvF, dinvS, X, D0, D1, R, W, coef, part;
  lfx_status init(int64_t V, const SmootherConfig &cfg);
  lfx_status setup(cudaStream_t st, const BsrView<S> &A);
  lfx_status apply(cudaStream_t st, const BsrView<S> &A, const T *r, T *z, const KState *ks);
  lfx_status lambdas(double *lf, double *ls) const;
  size_t device_bytes() const;
};

template <class S, class T>
struct Gmres {
  int64_t V = 0, n = 0;
  int restart = 40;
  int nblk_dot = 0;
  DBuf basis, zbasis, work, part, part_n, state;
  int *pinned = nullptr;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  Gmres() = default;
  Gmres(const Gmres &) = delete;
  ~Gmres();
  lfx_status init(int64_t V, int restart);
  lfx_status solve(cudaStream_t st, const BsrView<S> &A, ASimple<S, T> &pc, const T *b, T *x,
                   double rtol, int maxit, bool cgs2, int *its_out, double *res_out);
  size_t device_bytes() const;
};

}  // namespace lfx
