// aSIMPLE preconditioner and restarted GMRES on the device (Section 2.4).
#pragma once

#include <cuda_bf16.h>

#include <cmath>
#include <functional>
#include <vector>

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
  // FP32 copies, read by the FP32 kernels (a double -> float conversion takes an FP64 issue slot,
  // at 1/64 of the FP32 rate on this GPU)
  float f_initf, s_initf;
  float f_c1f[kMaxSmooth], f_c2f[kMaxSmooth];
  float s_c1f[kMaxSmooth], s_c2f[kMaxSmooth];
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

// Independent problems solved together: node ranges of the components of a block-diagonal
// system, cut into tasks of at most kSegNodes nodes (one CTA each) that never straddle two
// components.  Device arrays.
constexpr int64_t kSegNodes = 2048;
struct SegTasks {
  const int64_t *lo, *hi;     // [n_task] node range of each task
  const int32_t *seg;         // [n_task] component of each task
  const int32_t *task_off;    // [n_seg + 1] first task of each component
  int n_task, n_seg;
};

// Rank-one terms of the operator (resistance conditions, Section 2.2.3): y += sum_t cr[t] w_t
// (w_t . x).  The dot product runs over every node of tag t (dot_off[t] .. dot_off[t+1] of
// dot_node, three components each in dot_w); the update over the listed rows only (ax_*: the
// tag's nodes that are not Dirichlet rows).  Device arrays.
struct Rank1View {
  int n_tags;
  const double *cr;
  const int32_t *dot_off, *dot_node;
  const double *dot_w;
  int64_t n_ax;
  const int32_t *ax_node, *ax_tag;
  const double *ax_w;
};

struct AmgHost;

// One explicit level (l >= 1) of the Schur AMG hierarchy on the device, and the transfer
// operators from level l to l+1 (also for l = 0).
struct AmgDevLevel {
  int64_t n = 0, nnext = 0;
  DBuf rp, ci, v, dinv;          // A_l (l >= 1)
  DBuf Prp, Pci, Pv;             // P_l: n_l x n_{l+1}
  DBuf Rrp, Rci, Rv;             // R_l = P_l^T
  DBuf x, b, r, d0, d1, rr;      // work vectors (l >= 1)
  double lam = 0.0;              // Gershgorin bound of lambda_max(D^-1 A_l) (l < L-1)
  double init = 0.0;             // Chebyshev coefficients of this level (host-computed)
  double c1[kMaxSmooth] = {}, c2[kMaxSmooth] = {};
};

template <class S, class T>
struct ASimple {
  int64_t V = 0;
  SmootherConfig cfg;
  DBuf dinvF, dinvS, X, D0, D1, R, W, coef, part;
  // Schur AMG (cfg.s_kind == LFX_SMOOTH_AMG)
  std::vector<AmgDevLevel> amg;
  DBuf Bs, rr0, coarse_inv, coarse_args;
  DBuf sF, sG, sDC;                // sub-blocks stored apart (setup_split)
  int64_t nnz_split = 0;
  bool split = false;
  // Staged velocity smoothing pass (BF16 sub-blocks): the pattern's row tiles (device, [n_ftile+1]
  // row offsets; none: the plain pass runs), and a device error word the pass sets when a wait for
  // a staged tile gives up, with its page-locked host copy
  const int32_t *ftile = nullptr;
  int n_ftile = 0;
  DBuf berr;
  int *berr_host = nullptr;
  void set_tiles(const int32_t *d_tile_row, int n_tiles) {
    ftile = d_tile_row;
    n_ftile = n_tiles;
  }
  // queues the copy of the error word to the host (and its reset) on st; after st has reached it,
  // bulk_failed() says whether a wait gave up since the previous check
  lfx_status queue_bulk_check(cudaStream_t st);
  bool bulk_failed();
  // tests: make every wait of the staged pass run out at once (then the pass sets the error word)
  bool force_bulk_timeout = false;
  int64_t nc = 0;
  std::vector<int64_t> lvl_rows, lvl_nnz;   // hierarchy shape (rows, nonzeros of A_l per level)
  int coop_grid = 0;   // > 0: the coarse V-cycle runs as one cooperative launch of this many CTAs
  bool amg_ready = false;
  double amg_alpha = 1.0;
  // CUDA-event timing of the plain F passes (velocity smoothing steps 2 .. f_steps-1, the fused
  // first step excluded) of the first application after each reset of n_fev, kept until read_f_timing
  std::vector<cudaEvent_t> fev;
  int n_fev = 0;
  bool time_f = false;   // off unless the owner asks (the events are created on first use)
  lfx_status read_f_timing(float *median_ms_per_pass, int *passes);
  ASimple() = default;
  ASimple(const ASimple &) = delete;
  ~ASimple();
  lfx_status upload_amg(const AmgHost &H);
  lfx_status vcycle(cudaStream_t st, int l, const KState *ks);
  // The V-cycle below level 0 (levels 1 .. L-1) for amg[1].b: one cooperative launch, or the
  // level-by-level launches; its result is at coarse_x().
  lfx_status coarse_cycle(cudaStream_t st, const KState *ks);
  const T *coarse_x() const;
  size_t amg_bytes() const;
  lfx_status init(int64_t V, const SmootherConfig &cfg);
  // Work arrays carved from caller-provided device memory (no allocation); zeroed on st.
  static size_t scratch_bytes(int64_t V);
  lfx_status init_borrowed(int64_t V, const SmootherConfig &cfg, void *base, size_t cap, cudaStream_t st);
  // Set-up on the full blocks A (the smoother then reads A's 4x4 blocks on every pass) ...
  lfx_status setup(cudaStream_t st, const BsrView<S> &A);
  // ... or on a copy of the FP64 blocks A64 converted to S with F, G and (D, C) stored apart, so
  // that each pass reads only the sub-block it needs (nnzb = number of blocks).
  lfx_status setup_split(cudaStream_t st, const BsrView<double> &A64, int64_t nnzb);
  lfx_status setup_split(cudaStream_t st, const BsrView<float> &A32, int64_t nnzb);
  // z = P^-1 r; with a split set-up only A's pattern (rowptr, col, diag, trans) is used.
  lfx_status apply(cudaStream_t st, const BsrView<S> &A, const T *r, T *z, const KState *ks);
  lfx_status lambdas(double *lf, double *ls) const;
  size_t device_bytes() const;

 private:
  template <class View>
  lfx_status setup_view(cudaStream_t st, const View &A);
  template <class View>
  bool use_staged(const View &A) const;
  template <class View>
  lfx_status launch_staged(cudaStream_t st, const View &A, bool first, int k, const T *d_old, T *d_new, const T *b0,
                           const KState *ks);
  template <class Src>
  lfx_status setup_split_from(cudaStream_t st, const BsrView<Src> &A, int64_t nnzb);
  template <class View>
  lfx_status apply_view(cudaStream_t st, const View &A, const T *r, T *z, const KState *ks);
};

// z = M^-1 v on the solver's stream; kernels may return early once ks->done is set.
template <class T>
using PrecFn = std::function<lfx_status(cudaStream_t, const T *v, T *z, const KState *ks)>;

// dst[i] = (B) src[i] for i < n (precision conversion of vectors or matrix values);
// skipped when ks says the calling solve is already finished.
template <class A, class B>
lfx_status launch_convert(cudaStream_t st, const A *src, B *dst, int64_t n, const KState *ks);

template <class S, class T>
struct Gmres {
  int64_t V = 0, n = 0;
  int restart = 40;
  int nblk_dot = 0;
  DBuf basis, zbasis, work, part, part_n, state;
  int *pinned = nullptr;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  // CUDA-event timing of the Arnoldi SpMV launches (accumulated until read_spmv_timing)
  std::vector<cudaEvent_t> tev;
  int n_tev = 0, n_spmv_calls = 0;
  lfx_status read_spmv_timing(float *ms, int *count);
  Gmres() = default;
  Gmres(const Gmres &) = delete;
  ~Gmres();
  lfx_status init(int64_t V, int restart);
  // Solve A x = b to ||b - A x|| <= rtol ||b|| starting from x (zeroed first if x_zero).
  // lag = Arnoldi steps the host may queue beyond the last convergence flag it has read.
  lfx_status solve(cudaStream_t st, const BsrView<S> &A, const PrecFn<T> &pc, const T *b, T *x,
                   double rtol, int maxit, bool cgs2, int lag, bool x_zero, int *its_out,
                   double *res_out);
  // From now on solve the components [comp_off[c], comp_off[c+1]) (node ranges; A must be block
  // diagonal over them and the preconditioner must not couple them) as separate problems: one
  // Arnoldi process per component, each stopped by its own test ||b_c - A x_c|| <= rtol ||b_c||.
  // *its_out is then the largest step count, *res_out the largest relative residual.
  lfx_status set_segments(const std::vector<int32_t> &comp_off);
  // Tolerance for the inner solve that preconditions this (flexible) solve's next step, from the
  // progress so far: with r the residual estimate and tol the target, 1/2 sqrt(tol / r) at a
  // cycle's first step (two steps of inner accuracy eta reach tol) and 1/2 tol / r after (this
  // step reaches it); the tightest over the running components; within [lo, hi].  Reads the
  // status from the device (synchronises st).
  lfx_status inner_tolerance(cudaStream_t st, double lo, double hi, double *eta);
  // Include rank-one terms in every product with A (single systems only).
  lfx_status set_rank1(const Rank1View &r);
  // One cycle from x = 0, as the preconditioner of a flexible outer solve, without waiting for the
  // device: the tolerance is eta ||b|| with eta = rtol, or (outer != null) the rule of
  // inner_tolerance evaluated on the device from the outer's status; no confirmation of the true
  // residual (the outer solve tests its own).  The step count lands in *its_pinned (page-locked
  // host memory) once the stream reaches it.  Needs maxit <= restart and one component.
  lfx_status solve_inner(cudaStream_t st, const BsrView<S> &A, const PrecFn<T> &pc, const T *b, T *x, double rtol,
                         const KState *outer, double lo, double hi, int maxit, bool cgs2, int lag, int *its_pinned);
  bool segmented() const { return n_seg > 1; }
  size_t device_bytes() const;

 private:
  Rank1View r1{};
  DBuf r1_s;   // the dot products w_t . x
  void apply_rank1(cudaStream_t st, const T *x, T *y, double sign, const KState *ks);
  lfx_status residual(cudaStream_t st, const BsrView<S> &A, const T *x, const T *b, T *w, double *pn, int *ng);
  lfx_status timed_spmv(cudaStream_t st, const BsrView<S> &A, const T *z, T *w, const KState *ks);
  lfx_status arnoldi_cycle(cudaStream_t st, const BsrView<S> &A, const PrecFn<T> &pc, int m, int maxit, bool cgs2,
                           int lag);
  int n_seg = 0;
  SegTasks tasks{};
  DBuf seg_lo, seg_hi, seg_id, seg_toff, seg_state, seg_part, seg_pn;
  lfx_status solve_seg(cudaStream_t st, const BsrView<S> &A, const PrecFn<T> &pc, const T *b, T *x,
                       double rtol, int maxit, bool cgs2, int lag, bool x_zero, int *its_out, double *res_out);
};

}  // namespace lfx
