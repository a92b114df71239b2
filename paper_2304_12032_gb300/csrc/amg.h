// Smoothed-aggregation AMG for the pressure Schur approximation (host set-up, device V-cycle).
#pragma once

#include <stdint.h>

#include <vector>

#include "lfx_internal.h"

namespace lfx {

struct CsrHost {
  int64_t n = 0, m = 0;          // rows, columns
  std::vector<int32_t> rp, ci;
  std::vector<double> v;
};

struct AmgParams {
  int coarse_size = 400;         // dense solve below this many unknowns
  int max_levels = 8;
  double theta = 0.08;           // strength threshold below the finest level
};

struct AmgHost {
  std::vector<CsrHost> A;        // A[0] = S (finest), ..., A[L-1] coarsest
  std::vector<CsrHost> P, R;     // P[l]: n_l x n_{l+1}, R[l] = P[l]^T
  std::vector<std::vector<double>> dinv;   // 1/diag(A_l), l < L-1
  std::vector<double> lam;       // Gershgorin bound of lambda_max(D^-1 A_l), l < L-1
  std::vector<double> coarse_inv;
  int64_t nc = 0;
};

CsrHost schur_explicit(int64_t V, const std::vector<int32_t> &rp, const std::vector<int32_t> &ci,
                       const std::vector<int32_t> &diag, const double *vals);
lfx_status amg_setup_host(CsrHost S0, const std::vector<int32_t> &node_rp,
                          const std::vector<int32_t> &node_ci, const AmgParams &prm, AmgHost &H);

}  // namespace lfx
