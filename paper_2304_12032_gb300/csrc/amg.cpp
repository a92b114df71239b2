// Host set-up of a smoothed-aggregation algebraic multigrid hierarchy for the Schur
// approximation S = C - D diag(F)^-1 G of the aSIMPLE preconditioner (Section 2.4 names AMG
// as one of the approximations of the velocity and Schur blocks).  Built from the assembled
// block matrix (downloaded once per set-up); applied on the device by the V-cycle in solver.cu.
//
// Steps: explicit S (distance-2 pattern); greedy aggregation (the mesh node graph on the
// finest level, strength-filtered matrix graphs below); tentative piecewise-constant
// prolongator smoothed by one damped Jacobi step, P = (I - w D^-1 A) P_tent,
// w = 4 / (3 lambda_max(D^-1 A)); Galerkin coarse operators P^T A P; dense inverse at the
// coarsest level.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <numeric>
#include <thread>

#include "amg.h"

namespace lfx {

namespace {

// Host threads of the set-up: the row-independent parts (sparse products, the explicit Schur
// complement, the power iteration) run on contiguous row ranges; every row is computed exactly
// as in a serial pass, so results do not depend on the thread count.
int setup_threads(int64_t rows) {
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  return (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)hw, 32, rows / 64}));
}

template <class F>
void parallel_ranges(int64_t n, int T, F fn) {
  if (T <= 1) {
    fn(0, int64_t{0}, n);
    return;
  }
  std::vector<std::thread> th;
  for (int t = 1; t < T; ++t) th.emplace_back(fn, t, n * t / T, n * (t + 1) / T);
  fn(0, int64_t{0}, n / T);
  for (auto &x : th) x.join();
}

// per-thread work space of a row-wise sparse product: a dense marker/accumulator over the
// columns and the thread's rows in CSR pieces
struct RowWork {
  std::vector<int64_t> mark;
  std::vector<double> acc;
  std::vector<int32_t> cols, ci, len;
  std::vector<double> v;
  void add(int64_t row, int32_t c, double val) {
    if (mark[c] != row) {
      mark[c] = row;
      acc[c] = 0.0;
      cols.push_back(c);
    }
    acc[c] += val;
  }
  void flush() {   // the marked row, columns sorted
    std::sort(cols.begin(), cols.end());
    for (int32_t c : cols) {
      ci.push_back(c);
      v.push_back(acc[c]);
    }
    len.push_back((int32_t)cols.size());
    cols.clear();
  }
};

// n x m CSR matrix whose row i is produced by row(i, work) (RowWork::add calls, then flush)
template <class RowFn>
CsrHost build_rows(int64_t n, int64_t m, RowFn row) {
  const int T = setup_threads(n);
  std::vector<RowWork> w(T);
  parallel_ranges(n, T, [&](int t, int64_t r0, int64_t r1) {
    RowWork &k = w[t];
    k.mark.assign(m, -1);
    k.acc.assign(m, 0.0);
    for (int64_t i = r0; i < r1; ++i) {
      row(i, k);
      k.flush();
    }
  });
  CsrHost C;
  C.n = n;
  C.m = m;
  C.rp.assign(n + 1, 0);
  size_t nnz = 0;
  for (auto &k : w) nnz += k.ci.size();
  C.ci.reserve(nnz);
  C.v.reserve(nnz);
  int64_t r = 0;
  for (auto &k : w) {
    for (int32_t l : k.len) {
      C.rp[r + 1] = C.rp[r] + l;
      ++r;
    }
    C.ci.insert(C.ci.end(), k.ci.begin(), k.ci.end());
    C.v.insert(C.v.end(), k.v.begin(), k.v.end());
  }
  return C;
}

// C = A * B (Gustavson, dense marker per thread)
CsrHost multiply(const CsrHost &A, const CsrHost &B) {
  return build_rows(A.n, B.m, [&](int64_t i, RowWork &w) {
    for (int32_t k = A.rp[i]; k < A.rp[i + 1]; ++k) {
      const int32_t a = A.ci[k];
      const double av = A.v[k];
      for (int32_t q = B.rp[a]; q < B.rp[a + 1]; ++q) w.add(i, B.ci[q], av * B.v[q]);
    }
  });
}

CsrHost transpose(const CsrHost &A) {
  CsrHost T;
  T.n = A.m;
  T.m = A.n;
  T.rp.assign(A.m + 1, 0);
  for (int32_t c : A.ci) T.rp[c + 1]++;
  for (int64_t i = 0; i < A.m; ++i) T.rp[i + 1] += T.rp[i];
  T.ci.resize(A.ci.size());
  T.v.resize(A.v.size());
  std::vector<int32_t> f(T.rp.begin(), T.rp.end() - 1);
  for (int64_t i = 0; i < A.n; ++i)
    for (int32_t k = A.rp[i]; k < A.rp[i + 1]; ++k) {
      const int32_t p = f[A.ci[k]]++;
      T.ci[p] = (int32_t)i;
      T.v[p] = A.v[k];
    }
  return T;
}

std::vector<double> diag_of(const CsrHost &A) {
  std::vector<double> d(A.n, 0.0);
  for (int64_t i = 0; i < A.n; ++i)
    for (int32_t k = A.rp[i]; k < A.rp[i + 1]; ++k)
      if (A.ci[k] == i) d[i] += A.v[k];
  return d;
}

std::vector<double> safe_inverse(const std::vector<double> &d) {
  std::vector<double> r(d.size());
  for (size_t i = 0; i < d.size(); ++i) r[i] = d[i] != 0.0 ? 1.0 / d[i] : 0.0;
  return r;
}

// power iteration on D^-1 A from the normalised ones vector (rows in parallel; the norm is summed
// over fixed chunks of rows in chunk order, independent of the thread count)
double lambda_max(const CsrHost &A, const std::vector<double> &dinv, int iters) {
  std::vector<double> v(A.n, 1.0 / std::sqrt((double)A.n)), w(A.n);
  constexpr int64_t kChunk = 4096;
  const int64_t nch = (A.n + kChunk - 1) / kChunk;
  std::vector<double> part(nch);
  const int T = setup_threads(A.n);
  double lam = 1.0;
  for (int it = 0; it < iters; ++it) {
    parallel_ranges(nch, T, [&](int, int64_t c0, int64_t c1) {
      for (int64_t c = c0; c < c1; ++c) {
        double nrm = 0.0;
        for (int64_t i = c * kChunk; i < std::min(A.n, (c + 1) * kChunk); ++i) {
          double s = 0.0;
          for (int32_t k = A.rp[i]; k < A.rp[i + 1]; ++k) s += A.v[k] * v[A.ci[k]];
          w[i] = dinv[i] * s;
          nrm += w[i] * w[i];
        }
        part[c] = nrm;
      }
    });
    double nrm = 0.0;
    for (double p : part) nrm += p;
    lam = std::sqrt(nrm);
    if (!(lam > 0)) return 1.0;
    for (int64_t i = 0; i < A.n; ++i) v[i] = w[i] / lam;
  }
  return lam;
}

// Greedy aggregation: a node whose neighbours are all free starts an aggregate with them;
// remaining nodes join a neighbouring aggregate, or start their own.
int64_t aggregate(int64_t n, const std::vector<int32_t> &rp, const std::vector<int32_t> &ci,
                  std::vector<int32_t> &agg) {
  agg.assign(n, -1);
  int64_t na = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (agg[i] >= 0) continue;
    bool free_all = true;
    for (int32_t k = rp[i]; k < rp[i + 1] && free_all; ++k)
      if (agg[ci[k]] >= 0) free_all = false;
    if (!free_all) continue;
    agg[i] = (int32_t)na;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) agg[ci[k]] = (int32_t)na;
    ++na;
  }
  for (int64_t i = 0; i < n; ++i) {
    if (agg[i] >= 0) continue;
    int32_t a = -1;
    for (int32_t k = rp[i]; k < rp[i + 1] && a < 0; ++k)
      if (agg[ci[k]] >= 0) a = agg[ci[k]];
    agg[i] = a >= 0 ? a : (int32_t)na++;
  }
  return na;
}

// strong-connection graph |a_ij| >= theta sqrt(|a_ii a_jj|), i != j
void strength_graph(const CsrHost &A, const std::vector<double> &d, double theta, std::vector<int32_t> &rp,
                    std::vector<int32_t> &ci) {
  rp.assign(A.n + 1, 0);
  ci.clear();
  for (int64_t i = 0; i < A.n; ++i) {
    for (int32_t k = A.rp[i]; k < A.rp[i + 1]; ++k) {
      const int32_t j = A.ci[k];
      if (j == i) continue;
      if (std::fabs(A.v[k]) >= theta * std::sqrt(std::fabs(d[i] * d[j]))) ci.push_back(j);
    }
    rp[i + 1] = (int32_t)ci.size();
  }
}


// Spin barrier for a fixed team of host threads (sense reversal; yields while waiting).
class SpinBarrier {
 public:
  explicit SpinBarrier(int n) : n_(n) {}
  void wait() {
    const int gen = gen_.load(std::memory_order_acquire);
    if (count_.fetch_add(1, std::memory_order_acq_rel) + 1 == n_) {
      count_.store(0, std::memory_order_relaxed);
      gen_.fetch_add(1, std::memory_order_acq_rel);
      return;
    }
    for (int spins = 0; gen_.load(std::memory_order_acquire) == gen; ++spins)
      if (spins > 64) std::this_thread::yield();
  }

 private:
  const int n_;
  std::atomic<int> count_{0}, gen_{0};
};

// M^-1 into I (I = identity on entry, M destroyed): for pivot c, the pivot row is found, swapped
// and scaled by one thread, then every other row r subtracts M[r][c] times it, rows split among
// the team.  Columns k < c of M are already zero outside their pivot rows and are skipped.
void gauss_jordan_inverse(int64_t n, std::vector<double> &M, std::vector<double> &I) {
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const int T = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)hw, 32, n / 64}));
  SpinBarrier bar(T);
  auto team = [&](int tid) {
    const int64_t r0 = n * tid / T, r1 = n * (tid + 1) / T;
    for (int64_t c = 0; c < n; ++c) {
      if (tid == 0) {
        int64_t p = c;
        for (int64_t r = c + 1; r < n; ++r)
          if (std::fabs(M[r * n + c]) > std::fabs(M[p * n + c])) p = r;
        // singular coarsest operator (e.g. a pure-Neumann pressure): regularise this pivot
        if (M[p * n + c] == 0.0) M[p * n + c] = 1.0;
        if (p != c)
          for (int64_t k = 0; k < n; ++k) {
            std::swap(M[p * n + k], M[c * n + k]);
            std::swap(I[p * n + k], I[c * n + k]);
          }
        const double piv = 1.0 / M[c * n + c];
        for (int64_t k = c; k < n; ++k) M[c * n + k] *= piv;
        for (int64_t k = 0; k < n; ++k) I[c * n + k] *= piv;
      }
      bar.wait();
      const double *mc = &M[c * n], *ic = &I[c * n];
      for (int64_t r = r0; r < r1; ++r) {
        if (r == c) continue;
        const double f = M[r * n + c];
        if (f == 0.0) continue;
        double *mr = &M[r * n], *ir = &I[r * n];
        for (int64_t k = c; k < n; ++k) mr[k] -= f * mc[k];
        for (int64_t k = 0; k < n; ++k) ir[k] -= f * ic[k];
      }
      bar.wait();
    }
  };
  if (T == 1) {
    team(0);
    return;
  }
  std::vector<std::thread> th;
  for (int t = 1; t < T; ++t) th.emplace_back(team, t);
  team(0);
  for (auto &t : th) t.join();
}
}  // namespace

// Explicit S = C - D diag(F)^-1 G from 4x4 blocks (row-major, [i][j], F = [0..2][0..2],
// G = [0..2][3], D = [3][0..2], C = [3][3]).
CsrHost schur_explicit(int64_t V, const std::vector<int32_t> &rp, const std::vector<int32_t> &ci,
                       const std::vector<int32_t> &diag, const double *vals) {
  std::vector<double> dinvF(3 * V);
  for (int64_t b = 0; b < V; ++b)
    for (int j = 0; j < 3; ++j) {
      const double f = vals[16 * (int64_t)diag[b] + 5 * j];
      dinvF[3 * b + j] = f != 0.0 ? 1.0 / f : 0.0;
    }
  return build_rows(V, V, [&](int64_t a, RowWork &w) {
    for (int32_t k = rp[a]; k < rp[a + 1]; ++k) {
      const int32_t b = ci[k];
      const double *blk = vals + 16 * (int64_t)k;
      w.add(a, b, blk[15]);
      for (int j = 0; j < 3; ++j) {
        const double d = blk[12 + j] * dinvF[3 * b + j];
        if (d == 0.0) continue;
        for (int32_t k2 = rp[b]; k2 < rp[b + 1]; ++k2) {
          const double g = vals[16 * (int64_t)k2 + 4 * j + 3];
          if (g != 0.0) w.add(a, ci[k2], -d * g);
        }
      }
    }
  });
}

lfx_status amg_setup_host(CsrHost S0, const std::vector<int32_t> &node_rp,
                          const std::vector<int32_t> &node_ci, const AmgParams &prm, AmgHost &H) {
  H = AmgHost();
  CsrHost A = std::move(S0);
  bool finest = true;
  while (A.n > prm.coarse_size && (int)H.P.size() < prm.max_levels - 1) {
    std::vector<double> d = diag_of(A), dinv = safe_inverse(d);
    std::vector<int32_t> grp, gci, agg;
    if (finest) {
      // mesh node graph without the diagonal
      grp.assign(A.n + 1, 0);
      for (int64_t i = 0; i < A.n; ++i) {
        for (int32_t k = node_rp[i]; k < node_rp[i + 1]; ++k)
          if (node_ci[k] != i) gci.push_back(node_ci[k]);
        grp[i + 1] = (int32_t)gci.size();
      }
    } else {
      strength_graph(A, d, prm.theta, grp, gci);
    }
    const int64_t na = aggregate(A.n, grp, gci, agg);
    if (na >= A.n || na < 1) break;   // no coarsening possible
    CsrHost Pt;
    Pt.n = A.n;
    Pt.m = na;
    Pt.rp.resize(A.n + 1);
    Pt.ci.resize(A.n);
    Pt.v.assign(A.n, 1.0);
    for (int64_t i = 0; i <= A.n; ++i) Pt.rp[i] = (int32_t)i;
    for (int64_t i = 0; i < A.n; ++i) Pt.ci[i] = agg[i];
    const double lam = lambda_max(A, dinv, 15) * 1.1;
    const double w = 4.0 / (3.0 * lam);
    CsrHost AP = multiply(A, Pt);   // (I - w D^-1 A) Pt = Pt - w D^-1 (A Pt)
    CsrHost P = build_rows(A.n, na, [&](int64_t i, RowWork &rw) {
      for (int32_t k = AP.rp[i]; k < AP.rp[i + 1]; ++k) rw.add(i, AP.ci[k], -w * dinv[i] * AP.v[k]);
      rw.add(i, agg[i], 1.0);
    });
    CsrHost R = transpose(P);
    CsrHost Ac = multiply(R, multiply(A, P));
    H.A.push_back(std::move(A));
    H.P.push_back(std::move(P));
    H.R.push_back(std::move(R));
    A = std::move(Ac);
    finest = false;
  }
  H.A.push_back(A);
  // dense inverse of the coarsest operator (Gauss-Jordan with partial pivoting); the row updates
  // of each pivot step are shared among host threads
  const int64_t n = A.n;
  H.nc = n;
  std::vector<double> M(n * n, 0.0), I(n * n, 0.0);
  for (int64_t i = 0; i < n; ++i) {
    I[i * n + i] = 1.0;
    for (int32_t k = A.rp[i]; k < A.rp[i + 1]; ++k) M[i * n + A.ci[k]] += A.v[k];
  }
  gauss_jordan_inverse(n, M, I);
  H.coarse_inv = std::move(I);
  H.lam.clear();
  for (size_t l = 0; l + 1 < H.A.size(); ++l) {
    // Gershgorin bound of D^-1 A_l for the Chebyshev interval of the level smoother
    std::vector<double> dinv = safe_inverse(diag_of(H.A[l]));
    double g = 0.0;
    for (int64_t i = 0; i < H.A[l].n; ++i) {
      double s = 0.0;
      for (int32_t k = H.A[l].rp[i]; k < H.A[l].rp[i + 1]; ++k) s += std::fabs(H.A[l].v[k]);
      g = std::max(g, std::fabs(dinv[i]) * s);
    }
    H.dinv.push_back(dinv);
    H.lam.push_back(g > 0 ? g : 1.0);
  }
  return LFX_OK;
}

}  // namespace lfx
