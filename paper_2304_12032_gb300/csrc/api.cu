// C ABI of liblfx (declared in include/lfx.h): mesh / problem / state handles, boundary data
// preprocessing (Section 2.2), one time step (Section 2.3 assembly + Section 2.4 solve), and
// the parity/debug entry points.  Host code only; kernels live in assemble.cu and solver.cu.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <unordered_map>
#include <string>
#include <vector>

#include "kernels.h"
#include "lfx_internal.h"
#include "amg.h"
#include "solver.h"

namespace lfx {

// ------------------------------------------------------------------------------ errors
static thread_local std::string g_err;
void set_error(const char *fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
}
void clear_error() { g_err.clear(); }

static std::atomic<int64_t> g_launches{0};
void note_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// ------------------------------------------------------------------------------ allocator
static lfx_alloc_fn g_alloc = nullptr;
static lfx_free_fn g_free = nullptr;
static void *g_alloc_ctx = nullptr;

void *dalloc(size_t bytes, DFree *how) {
  void *p = nullptr;
  if (g_alloc) {
    p = g_alloc(bytes, g_alloc_ctx);
    if (!p) {
      set_error("device allocation of %zu bytes failed (user allocator)", bytes);
      return nullptr;
    }
    if ((reinterpret_cast<uintptr_t>(p) & 15u) != 0) {
      // the kernels load 16-byte vectors and copy 16-byte units from every buffer
      if (g_free) g_free(p, g_alloc_ctx);
      set_error("user allocator returned %p, not aligned to 16 bytes", p);
      return nullptr;
    }
    if (how) *how = DFree{g_free, g_alloc_ctx};
    return p;
  }
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    return nullptr;
  }
  if (how) *how = DFree{};
  return p;
}
void dfree(void *p, const DFree &how) {
  if (!p) return;
  if (how.fn) how.fn(p, how.ctx);
  else cudaFree(p);
}

// ------------------------------------------------------------------------------ time laws
// g(t) of Section 2.2.1
static double time_law(const lfx_time_law &L, double t) {
  switch (L.kind) {
    case LFX_TIME_CONSTANT: return L.p[0];
    case LFX_TIME_PULSATILE: return L.p[0] + (L.p[1] - L.p[0]) * 0.5 * (1.0 - std::cos(2.0 * M_PI * t / L.p[2]));
    case LFX_TIME_RAMP:
      if (t < L.p[2]) return L.p[0];
      if (t < L.p[2] + L.p[3]) return L.p[0] + 0.5 * (L.p[1] - L.p[0]) * (1.0 - std::cos(M_PI * (t - L.p[2]) / L.p[3]));
      return L.p[1];
    case LFX_TIME_FOURIER: {
      const double w = 2.0 * M_PI / L.p[0];
      double g = L.a[0];
      for (int k = 1; k <= L.n_harmonics; ++k) g += L.a[k] * std::cos(k * w * t) + L.b[k] * std::sin(k * w * t);
      return g;
    }
  }
  return 0.0;
}

}  // namespace lfx

using namespace lfx;

// ================================================================================ problem
struct lfx_problem {
  const lfx_mesh *mesh = nullptr;
  PhysParams P{};
  int bdf_order = 1;
  double beta[3] = {0, 0, 0}, gamma[3] = {0, 0, 0};
  lfx_options opt{};
  std::vector<lfx_bc> bcs;
  // Dirichlet data: g(d) = sum_h c[bc(d)][h] S[h][d] + nodal(d)  (internal node ids)
  int H = 1;
  std::vector<int32_t> dir_node, dir_bc;
  std::vector<int32_t> dir_pos_of_node;   // [V] -> index into dir_node, -1 if free
  DBuf d_dir_node, d_dir_bc, d_S;
  // Neumann data: rhs(node) -= h(t) * vec(node) per Neumann BC
  std::vector<int32_t> neu_node, neu_bc;
  DBuf d_neu_node, d_neu_bc, d_neu_vec;
  // inertial backflow stabilisation: one task per edge of a face of a Neumann tag with beta > 0
  // (nodes i, j; the face's area vector A_f n_f; beta rho / 2; the compact indices of blocks
  // (i,i), (i,j), (j,i), (j,j)); the compact blocks' matrix slots and FP64 accumulators
  int64_t n_bf_edges = 0, n_bf_blocks = 0;
  DBuf d_bf_ij, d_bf_an, d_bf_coef, d_bf_slot4, d_bf_blk, d_bf_acc;
  // resistance tags: rank-one terms C_R w w^T of the operator (see Rank1View)
  int n_r1_tags = 0;
  int64_t n_r1_ax = 0;
  DBuf d_r1_cr, d_r1_off, d_r1_node, d_r1_w, d_r1_ax_node, d_r1_ax_tag, d_r1_ax_w;
  Rank1View rank1() const {
    return Rank1View{n_r1_tags, d_r1_cr.as<double>(), d_r1_off.as<int32_t>(), d_r1_node.as<int32_t>(),
                     d_r1_w.as<double>(), n_r1_ax, d_r1_ax_node.as<int32_t>(), d_r1_ax_tag.as<int32_t>(),
                     d_r1_ax_w.as<double>()};
  }
  // faces of Neumann tags (internal numbering) and their BC index: the loads on a moving mesh
  int64_t n_neu_faces = 0;
  DBuf d_neu_faces, d_neu_face_bc;
  // RIIS nodal signed distances [n_riis][V]
  DBuf d_phi;
  DBuf d_bad;
  // element geometry computed once per problem (fixed mesh): FP64 (geo64) or double-float
  // (geo_hi + geo_lo) [kGeoValues][T]
  DBuf geo64, geo_hi, geo_lo;
  int32_t pin_node = -1;   // internal
  int64_t n_bad = 0;
  // assembly launch shape (LFX_ASM_*): options.assembly, or the autotuner's choice (0 until tuned),
  // with the tuning times (ms per assembly: colours, chunks, persistent) and the device copy of the
  // chunk colour offsets the persistent launch reads
  std::mutex tune_mu;
  int asm_mode = 0, asm_mode_newton = 0;   // launch shapes of the semi-implicit and Newton systems
  float asm_ms[3] = {0.0f, 0.0f, 0.0f}, asm_ms_newton[3] = {0.0f, 0.0f, 0.0f};
  DBuf d_chunk_color_off;
  size_t device_bytes() const {
    return d_dir_node.bytes + d_dir_bc.bytes + d_S.bytes + d_neu_node.bytes + d_neu_bc.bytes +
           d_neu_vec.bytes + d_phi.bytes + d_bad.bytes + geo64.bytes + geo_hi.bytes + geo_lo.bytes +
           d_bf_ij.bytes + d_bf_an.bytes + d_bf_coef.bytes + d_bf_slot4.bytes + d_bf_blk.bytes + d_bf_acc.bytes +
           d_r1_cr.bytes + d_r1_off.bytes + d_r1_node.bytes + d_r1_w.bytes + d_r1_ax_node.bytes + d_r1_ax_tag.bytes +
           d_r1_ax_w.bytes + d_neu_faces.bytes + d_neu_face_bc.bytes;
  }
};

// ================================================================================ state
struct lfx_state {
  lfx_problem *pb = nullptr;
  cudaStream_t stream = nullptr;
  int sigma = 1;
  DBuf hist[3];            // D4 [V]; level l = hist[(head + l) % sigma]
  mutable DBuf io_u, io_p;  // caller-layout staging on the device: u [sigma][V][3], p [sigma][V]
  int head = 0;
  DBuf xsol, ubdf, rhs, gdir, nodal, comp_scale;
  DBuf vals64, vals32, nopat;   // nopat: empty (pattern-only views)
  ASimple<double, double> pc64;
  Gmres<double, double> gm64;
  // mixed precision: the matrix is assembled in double-float arithmetic as FP32 high parts
  // (vals32, also the inner solve's operator) and low parts (vals_lo); the outer FGMRES runs on
  // hi + lo with FP64 vectors
  DBuf vals_lo, rhs_hi, rhs_lo, xe_hi, xe_lo, ub_hi, ub_lo, xs_hi, xs_lo;
  Gmres<DDMat, double> gmdd;
  // mixed precision: FP32 inner Krylov with an FP32 or BF16-storage aSIMPLE
  ASimple<float, float> pc32;
  ASimple<__nv_bfloat16, float> pcbf;
  Gmres<float, float> gm32;
  DBuf r32, z32;
  int inner_total = 0;
  int *inner_its = nullptr;      // page-locked: step counts of the inner solves of one outer solve
  int inner_cap = 0, n_inner = 0;
  double t = 0.0, pin_value = 0.0;
  bool assembled = false;
  int amg_age = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr, ea0 = nullptr, ea1 = nullptr;
  int n_asm_launch = 0;
  // fully implicit formulation: residual vector, norm partials, Newton history of the last step
  DBuf fres, npart;
  std::vector<double> newton_res;
  // moving domain (ALE): displacement levels d^n, d^{n-1}, ... (level l = dhist[(dhead + l) % sigma]),
  // the next level d^{n+1}, u_ALE, the moved coordinates and their element geometry, the lifting
  // Laplacian and its CG work arrays, and the next step's prescribed displacements
  bool ale = false, have_bnd = false;
  int dhead = 0, lifting_iters = 0;
  DBuf dhist[3], dnew, uale, xyz, xyz_hi, xyz_lo, geo64, geo_hi, geo_lo;
  DBuf lapK, lapDinv, lapFixed, lapR, lapZ, lapP, lapAp, lapPart, lapCg, bnd_node, bnd_val;
  // persistent assembly: grid-barrier counter and error word (device), the error word's host copy
  DBuf asm_sync;
  int *asm_err_host = nullptr;
  int asm_mode_used = 0;
  bool force_timeout = false;   // tests: make the persistent assembly's first grid-wide wait run out
  int64_t n_bnd = 0;
  D4 *dlevel(int l) { return dhist[(dhead + l) % sigma].as<D4>(); }
  ~lfx_state() {
    if (ea0) cudaEventDestroy(ea0);
    if (ea1) cudaEventDestroy(ea1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e2) cudaEventDestroy(e2);
    if (inner_its) cudaFreeHost(inner_its);
    if (asm_err_host) cudaFreeHost(asm_err_host);
  }
  D4 *level(int l) { return hist[(head + l) % sigma].as<D4>(); }
  template <class S>
  BsrView<S> view(const DBuf &v) const {
    const Mesh &m = pb->mesh->m;
    return BsrView<S>{m.V, m.d_rowptr.as<int32_t>(), m.d_col.as<int32_t>(), m.d_diag.as<int32_t>(),
                      m.d_trans.as<int32_t>(), v.as<S>()};
  }
  BsrView<DDMat> view_dd() const {
    const Mesh &m = pb->mesh->m;
    return BsrView<DDMat>{m.V, m.d_rowptr.as<int32_t>(), m.d_col.as<int32_t>(), m.d_diag.as<int32_t>(),
                          m.d_trans.as<int32_t>(), vals32.as<float>(), vals_lo.as<float>(),
                          xs_hi.as<float4>(), xs_lo.as<float4>()};
  }
  bool mixed() const { return pb->opt.precision == LFX_PREC_MIXED; }
  BsrView<double> view64() const {
    const Mesh &m = pb->mesh->m;
    return BsrView<double>{m.V, m.d_rowptr.as<int32_t>(), m.d_col.as<int32_t>(), m.d_diag.as<int32_t>(),
                           m.d_trans.as<int32_t>(), vals64.as<double>()};
  }
};

extern "C" {

const char *lfx_last_error(void) { return g_err.c_str(); }

int64_t lfx_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

int64_t lfx_sizeof(const char *type_name) {
  if (!type_name) return -1;
  const std::string t(type_name);
  if (t == "lfx_time_law") return sizeof(lfx_time_law);
  if (t == "lfx_bc") return sizeof(lfx_bc);
  if (t == "lfx_riis") return sizeof(lfx_riis);
  if (t == "lfx_options") return sizeof(lfx_options);
  if (t == "lfx_mesh_info") return sizeof(lfx_mesh_info);
  if (t == "lfx_step_stats") return sizeof(lfx_step_stats);
  return -1;
}

lfx_status lfx_set_allocator(lfx_alloc_fn alloc, lfx_free_fn free_fn, void *ctx) {
  if ((alloc == nullptr) != (free_fn == nullptr)) {
    set_error("lfx_set_allocator: give both functions or neither");
    return LFX_ERR_INVALID_ARG;
  }
  g_alloc = alloc;
  g_free = free_fn;
  g_alloc_ctx = ctx;
  return LFX_OK;
}

// ---------------------------------------------------------------------------------- mesh
lfx_status lfx_mesh_create(const double *nodes, int64_t n_nodes, const int32_t *tets, int64_t n_tets,
                           const int32_t *bfaces, const int32_t *boundary_tags, int64_t n_bfaces,
                           lfx_mesh **out) {
  clear_error();
  if (!out) {
    set_error("lfx_mesh_create: out is NULL");
    return LFX_ERR_INVALID_ARG;
  }
  *out = nullptr;
  std::unique_ptr<lfx_mesh> h(new (std::nothrow) lfx_mesh);
  if (!h) return LFX_ERR_OOM;
  LFX_TRY(build_mesh(nodes, n_nodes, tets, n_tets, bfaces, boundary_tags, n_bfaces, h->m));
  *out = h.release();
  return LFX_OK;
}

void lfx_mesh_destroy(lfx_mesh *mesh) { delete mesh; }

// default shape-quality threshold below which an element keeps FP64 geometry in mixed assembly
constexpr double kDefaultBadElementQuality = 0.1;

lfx_status lfx_mesh_get_info(const lfx_mesh *mesh, lfx_mesh_info *info) {
  if (!mesh || !info) {
    set_error("lfx_mesh_get_info: NULL argument");
    return LFX_ERR_INVALID_ARG;
  }
  const Mesh &m = mesh->m;
  info->n_nodes = m.V;
  info->n_tets = m.T;
  info->n_bfaces = m.F;
  info->nnz_blocks = m.nnzb;
  info->n_colors = (int32_t)m.color_off.size() - 1;
  info->n_flipped = m.n_flipped;
  int mx = 0, mn = INT32_MAX;
  for (size_t c = 0; c + 1 < m.color_off.size(); ++c) {
    int s = m.color_off[c + 1] - m.color_off[c];
    mx = std::max(mx, s);
    mn = std::min(mn, s);
  }
  info->max_color_size = mx;
  info->min_color_size = mn;
  int64_t n_bad = 0;
  for (const double q : m.quality) n_bad += q < kDefaultBadElementQuality ? 1 : 0;
  info->n_bad_elements = n_bad;
  info->n_components = m.n_comp;
  return LFX_OK;
}

// user-ordered pattern: row i (caller), columns = caller ids of the internal row, sorted
static void user_pattern(const Mesh &m, std::vector<int64_t> &rp, std::vector<int32_t> &ci,
                         std::vector<int64_t> &internal_block) {
  rp.assign(m.V + 1, 0);
  ci.resize(m.nnzb);
  internal_block.resize(m.nnzb);
  for (int64_t i = 0; i < m.V; ++i) {
    const int32_t r = m.node_new[i];
    rp[i + 1] = rp[i] + (m.row_ptr[r + 1] - m.row_ptr[r]);
  }
  std::vector<std::pair<int32_t, int64_t>> tmp;
  for (int64_t i = 0; i < m.V; ++i) {
    const int32_t r = m.node_new[i];
    tmp.clear();
    for (int32_t k = m.row_ptr[r]; k < m.row_ptr[r + 1]; ++k) tmp.push_back({m.node_old[m.col_idx[k]], k});
    std::sort(tmp.begin(), tmp.end());
    for (size_t q = 0; q < tmp.size(); ++q) {
      ci[rp[i] + q] = tmp[q].first;
      internal_block[rp[i] + q] = tmp[q].second;
    }
  }
}

lfx_status lfx_mesh_get_pattern(const lfx_mesh *mesh, int64_t *row_ptr, int32_t *col_idx) {
  if (!mesh || !row_ptr || !col_idx) {
    set_error("lfx_mesh_get_pattern: NULL argument");
    return LFX_ERR_INVALID_ARG;
  }
  std::vector<int64_t> rp, ib;
  std::vector<int32_t> ci;
  user_pattern(mesh->m, rp, ci, ib);
  std::copy(rp.begin(), rp.end(), row_ptr);
  std::copy(ci.begin(), ci.end(), col_idx);
  return LFX_OK;
}

lfx_status lfx_mesh_get_colors(const lfx_mesh *mesh, int32_t *colors) {
  if (!mesh || !colors) {
    set_error("lfx_mesh_get_colors: NULL argument");
    return LFX_ERR_INVALID_ARG;
  }
  const Mesh &m = mesh->m;
  for (size_t c = 0; c + 1 < m.color_off.size(); ++c)
    for (int32_t i = m.color_off[c]; i < m.color_off[c + 1]; ++i) colors[m.elem_old[m.color_elems[i]]] = (int32_t)c;
  return LFX_OK;
}

lfx_status lfx_mesh_get_row_tiles(const lfx_mesh *mesh, int64_t sizes[3], int32_t *tile_row, int32_t *row_node) {
  if (!mesh || !sizes) {
    set_error("lfx_mesh_get_row_tiles: NULL argument");
    return LFX_ERR_INVALID_ARG;
  }
  const Mesh &m = mesh->m;
  sizes[0] = m.ftile_row.empty() ? 0 : (int64_t)m.ftile_row.size() - 1;
  sizes[1] = kFTileRows;
  sizes[2] = kFTileBlocks;
  if (tile_row) std::copy(m.ftile_row.begin(), m.ftile_row.end(), tile_row);
  if (row_node) std::copy(m.node_old.begin(), m.node_old.end(), row_node);
  return LFX_OK;
}

lfx_status lfx_mesh_get_chunks(const lfx_mesh *mesh, int64_t sizes[5], int32_t *elem_old, int32_t *chunk_elem_off,
                               int32_t *chunk_color_off, int32_t *chunk_pass_off, uint16_t *pass_code,
                               int32_t *pass_run_off, uint16_t *run_meta, int32_t *run_row, int32_t *run_col) {
  if (!mesh || !sizes) {
    set_error("lfx_mesh_get_chunks: NULL argument");
    return LFX_ERR_INVALID_ARG;
  }
  const Mesh &m = mesh->m;
  sizes[0] = (int64_t)m.chunk_elem_off.size() - 1;
  sizes[1] = (int64_t)m.chunk_color_off.size() - 1;
  sizes[2] = (int64_t)m.pass_ndiag.size();
  sizes[3] = (int64_t)m.run_block.size();
  sizes[4] = 4 * kChunkElems;
  auto put = [](auto *dst, const auto &v) {
    if (dst) std::copy(v.begin(), v.end(), dst);
  };
  put(elem_old, m.elem_old);
  put(chunk_elem_off, m.chunk_elem_off);
  put(chunk_color_off, m.chunk_color_off);
  put(chunk_pass_off, m.chunk_pass_off);
  put(pass_code, m.pass_code);
  put(pass_run_off, m.pass_run_off);
  put(run_meta, m.run_meta);
  if (run_row && run_col) {
    // block index -> (row, column) in the caller's node numbering
    std::vector<int32_t> row_of(m.nnzb);
    for (int64_t i = 0; i < m.V; ++i)
      for (int32_t k = m.row_ptr[i]; k < m.row_ptr[i + 1]; ++k) row_of[k] = (int32_t)i;
    for (size_t r = 0; r < m.run_block.size(); ++r) {
      run_row[r] = m.node_old[row_of[m.run_block[r]]];
      run_col[r] = m.node_old[m.col_idx[m.run_block[r]]];
    }
  }
  return LFX_OK;
}

// ------------------------------------------------------------------------------- problem
void lfx_options_default(lfx_options *o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->stab = LFX_STAB_VMS_LES;
  o->diffusion = LFX_DIFF_GRAD_GRAD;
  o->c_r = 30.0;
  o->pin_pressure_node = -1;
  o->precision = LFX_PREC_FP64;
  o->gmres_restart = 64;
  o->gmres_max_iters = 1000;
  o->gmres_rtol = 1e-10;
  o->reorthogonalize = 0;
  o->f_smoother = LFX_SMOOTH_CHEBYSHEV;
  o->f_steps = 6;
  o->f_omega = 0.7;
  o->f_ratio = 60.0;
  o->s_smoother = LFX_SMOOTH_AMG;
  o->s_steps = 1;
  o->s_omega = 0.7;
  o->s_ratio = 30.0;
  o->n_power = 0;
  o->smoother_bf16 = 0;
  o->outer_restart = 8;
  o->outer_max_iters = 40;
  o->inner_rtol = 1e-4;
  o->inner_max_iters = 60;
  o->bad_element_quality = kDefaultBadElementQuality;
  o->amg_refresh = 0;
  o->amg_coarse_size = 2000;
  o->amg_theta = 0.08;
  o->amg_alpha = 1.0;
  o->batch_normalize = 1;
  o->batch_segmented = 1;
  o->inner_adaptive = 1;
  o->implicit = 0;
  o->newton_max_iters = 10;
  o->assembly = LFX_ASM_AUTO;
  o->newton_rtol = 1e-10;
  o->staged_f = 1;
}

// barycentre, unit outward normal, area of the faces carrying `tag` (area weighted)
static bool tag_geometry(const Mesh &m, int tag, double c[3], double n[3], double *area) {
  double A = 0, cs[3] = {0, 0, 0}, ns[3] = {0, 0, 0};
  for (int64_t f = 0; f < m.F; ++f) {
    if (m.btags[f] != tag) continue;
    const double *a = &m.xyz[3 * (int64_t)m.bfaces[3 * f]], *b = &m.xyz[3 * (int64_t)m.bfaces[3 * f + 1]],
                 *d = &m.xyz[3 * (int64_t)m.bfaces[3 * f + 2]];
    double u[3], v[3], cr[3];
    for (int k = 0; k < 3; ++k) {
      u[k] = b[k] - a[k];
      v[k] = d[k] - a[k];
    }
    cr[0] = u[1] * v[2] - u[2] * v[1];
    cr[1] = u[2] * v[0] - u[0] * v[2];
    cr[2] = u[0] * v[1] - u[1] * v[0];
    const double ar = 0.5 * std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    A += ar;
    for (int k = 0; k < 3; ++k) {
      cs[k] += ar * (a[k] + b[k] + d[k]) / 3.0;
      ns[k] += cr[k];
    }
  }
  if (A <= 0) return false;
  const double nn = std::sqrt(ns[0] * ns[0] + ns[1] * ns[1] + ns[2] * ns[2]);
  for (int k = 0; k < 3; ++k) {
    c[k] = cs[k] / A;
    n[k] = ns[k] / nn;
  }
  if (area) *area = A;
  return true;
}

// Womersley unit-flow-rate profile for harmonic k (omega_k = k w), radius R, nu = mu/rho:
// W_k(r) = [1 - J0(i^{3/2} a r/R) / J0(i^{3/2} a)] / Q_k, a = R sqrt(omega_k / nu), Q_k its flux.
static std::complex<double> bessel_j0(std::complex<double> z) {
  std::complex<double> term(1.0, 0.0), sum(1.0, 0.0);
  const std::complex<double> q = -0.25 * z * z;
  for (int m = 1; m < 400; ++m) {
    term *= q / double(m * m);
    sum += term;
    if (std::abs(term) < 1e-17 * std::abs(sum)) break;
  }
  return sum;
}
static std::complex<double> bessel_j1(std::complex<double> z) {
  std::complex<double> term = 0.5 * z, sum = term;
  const std::complex<double> q = -0.25 * z * z;
  for (int m = 1; m < 400; ++m) {
    term *= q / double(m * (m + 1));
    sum += term;
    if (std::abs(term) < 1e-17 * std::abs(sum)) break;
  }
  return sum;
}

lfx_status lfx_problem_create(const lfx_mesh *mesh, double rho, double mu, double dt, int32_t bdf_order,
                              const lfx_bc *bcs, int32_t n_bcs, const lfx_riis *riis, int32_t n_riis,
                              const lfx_options *opt, lfx_problem **out) {
  clear_error();
  if (!mesh || !out || !(rho > 0) || !(mu > 0) || !(dt > 0) || bdf_order < 1 || bdf_order > 3 ||
      n_bcs < 0 || (n_bcs > 0 && !bcs) || n_riis < 0 || n_riis > kMaxRiis || (n_riis > 0 && !riis)) {
    set_error("lfx_problem_create: invalid argument");
    return LFX_ERR_INVALID_ARG;
  }
  // each boundary condition on its own, before anything is allocated
  for (int32_t b = 0; b < n_bcs; ++b) {
    const lfx_bc &bc = bcs[b];
    if (bc.kind < 0 || bc.kind > 4 || bc.profile < 0 || bc.profile > 2 || bc.time.n_harmonics < 0 ||
        bc.time.n_harmonics > LFX_MAX_FOURIER || !(bc.beta >= 0.0) || (bc.beta != 0.0 && bc.kind != LFX_BC_NEUMANN) ||
        !(bc.resistance >= 0.0) || (bc.resistance != 0.0 && bc.kind != LFX_BC_RESISTANCE)) {
      set_error("lfx_problem_create: invalid boundary condition %d (kind, profile, harmonics, beta or resistance)", b);
      return LFX_ERR_INVALID_ARG;
    }
  }
  *out = nullptr;
  std::unique_ptr<lfx_problem> pb(new (std::nothrow) lfx_problem);
  if (!pb) return LFX_ERR_OOM;
  if (opt) pb->opt = *opt;
  else lfx_options_default(&pb->opt);
  lfx_options &o = pb->opt;
  // the options, too, are checked before anything is allocated on the device
  if (o.stab < 0 || o.stab > 2 || o.diffusion < 0 || o.diffusion > 2 || o.gmres_restart < 1 ||
      o.gmres_restart > kMaxRestart || o.f_steps < 1 || o.f_steps > kMaxSmooth || o.s_steps < 1 ||
      o.s_steps > kMaxSmooth || o.precision < 0 || o.precision > 1 || o.n_power < 0 || o.f_smoother < 0 ||
      o.f_smoother > 1 || o.s_smoother < 0 || o.s_smoother > 2) {
    set_error("lfx_problem_create: option out of range (restart <= %d, smoothing steps <= %d)", kMaxRestart,
              kMaxSmooth);
    return LFX_ERR_INVALID_ARG;
  }
  if (o.staged_f < 0 || o.staged_f > 1) {
    set_error("lfx_problem_create: staged_f must be 0 or 1");
    return LFX_ERR_INVALID_ARG;
  }
  if (o.assembly < LFX_ASM_AUTO || o.assembly > LFX_ASM_PERSISTENT) {
    set_error("lfx_problem_create: assembly must be one of LFX_ASM_*");
    return LFX_ERR_INVALID_ARG;
  }
  if (o.implicit < 0 || o.implicit > 1 || (o.implicit && (o.newton_max_iters < 1 || !(o.newton_rtol > 0.0)))) {
    set_error("lfx_problem_create: implicit must be 0 or 1, with newton_max_iters >= 1 and newton_rtol > 0");
    return LFX_ERR_INVALID_ARG;
  }
  if (o.implicit)
    for (int32_t b = 0; b < n_bcs; ++b)
      if (bcs[b].kind == LFX_BC_RESISTANCE || (bcs[b].kind == LFX_BC_NEUMANN && bcs[b].beta > 0.0)) {
        set_error("lfx_problem_create: the fully implicit formulation is not available with backflow "
                  "stabilisation or resistance conditions (boundary condition %d)", b);
        return LFX_ERR_INVALID_ARG;
      }
  const Mesh &m = mesh->m;
  if (!m.uploaded) {
    // device copies are made on first use, so that mesh set-up itself needs no GPU
    Mesh &mm = const_cast<lfx_mesh *>(mesh)->m;
    LFX_TRY(upload_mesh(mm));
    mm.uploaded = true;
  }
  pb->mesh = mesh;
  // physics (Section 2.1.2, Eq. bdf)
  PhysParams &P = pb->P;
  P.rho = rho;
  P.mu = mu;
  P.dt = dt;
  pb->bdf_order = bdf_order;
  static const double alph[3] = {1.0, 1.5, 11.0 / 6.0};
  static const double bet[3][3] = {{1.0, 0, 0}, {2.0, -0.5, 0}, {3.0, -1.5, 1.0 / 3.0}};
  static const double gam[3][3] = {{1.0, 0, 0}, {2.0, -1.0, 0}, {3.0, -3.0, 1.0}};
  P.alpha = alph[bdf_order - 1];
  P.sigma = (double)bdf_order;
  for (int k = 0; k < 3; ++k) {
    pb->beta[k] = bet[bdf_order - 1][k];
    pb->gamma[k] = gam[bdf_order - 1][k];
  }
  P.c_r = o.c_r;
  for (int k = 0; k < 3; ++k) P.f[k] = o.f[k];
  P.stab = o.stab;
  P.diffusion = o.diffusion;
  P.n_riis = n_riis;
  for (int k = 0; k < n_riis; ++k) {
    if (!(riis[k].resistance >= 0) || !(riis[k].eps > 0) ||
        (riis[k].kind == LFX_RIIS_SDF_NODAL && !riis[k].sdf_nodal) || riis[k].kind < 0 || riis[k].kind > 1) {
      set_error("lfx_problem_create: invalid RIIS surface %d", k);
      return LFX_ERR_INVALID_ARG;
    }
    P.riis_r[k] = riis[k].resistance;
    P.riis_eps[k] = riis[k].eps;
  }
  P.rho_dt = rho / dt;
  P.rho_alpha_dt = rho * P.alpha / dt;
  P.tau_t = P.sigma * P.sigma * rho * rho / (dt * dt);
  P.cr_mu2 = P.c_r * mu * mu;
  for (int k = 0; k < n_riis; ++k) {
    P.riis_coef[k] = P.riis_r[k] / P.riis_eps[k];
    P.riis_pi_eps[k] = M_PI / P.riis_eps[k];
    P.riis_inv2eps[k] = 0.5 / P.riis_eps[k];
  }
  pb->bcs.assign(bcs, bcs + n_bcs);
  const int64_t V = m.V;

  // ---- Dirichlet nodes and their BC (precedence: no-slip > Dirichlet/nodal)
  std::vector<int> pri(V, 0), owner(V, -1);
  for (int b = 0; b < n_bcs; ++b) {
    const lfx_bc &bc = bcs[b];
    if (bc.kind < 0 || bc.kind > 4 || bc.profile < 0 || bc.profile > 2) {
      set_error("lfx_problem_create: invalid boundary condition %d", b);
      return LFX_ERR_INVALID_ARG;
    }
    if (bc.kind == LFX_BC_DIRICHLET && bc.profile == LFX_PROFILE_WOMERSLEY && bc.time.kind != LFX_TIME_FOURIER) {
      set_error("lfx_problem_create: the Womersley profile needs a Fourier time law (Section 2.2.1)");
      return LFX_ERR_INVALID_ARG;
    }
    if (bc.time.n_harmonics < 0 || bc.time.n_harmonics > LFX_MAX_FOURIER) {
      set_error("lfx_problem_create: too many Fourier harmonics");
      return LFX_ERR_INVALID_ARG;
    }
    if (!(bc.beta >= 0.0) || (bc.beta != 0.0 && bc.kind != LFX_BC_NEUMANN)) {
      set_error("lfx_problem_create: backflow stabilisation beta must be >= 0, and only on Neumann tags");
      return LFX_ERR_INVALID_ARG;
    }
    if (!(bc.resistance >= 0.0) || (bc.resistance != 0.0 && bc.kind != LFX_BC_RESISTANCE)) {
      set_error("lfx_problem_create: the resistance coefficient must be >= 0, and only on resistance tags");
      return LFX_ERR_INVALID_ARG;
    }
    if (bc.kind == LFX_BC_NEUMANN || bc.kind == LFX_BC_RESISTANCE) continue;
    const int p = bc.kind == LFX_BC_NOSLIP ? 3 : 2;
    for (int64_t f = 0; f < m.F; ++f) {
      if (m.btags[f] != bc.tag) continue;
      for (int k = 0; k < 3; ++k) {
        const int32_t nd = m.bfaces[3 * f + k];
        if (p > pri[nd]) {
          pri[nd] = p;
          owner[nd] = b;
        }
      }
    }
  }
  int H = 1;
  for (int b = 0; b < n_bcs; ++b)
    if (bcs[b].kind == LFX_BC_DIRICHLET && bcs[b].profile == LFX_PROFILE_WOMERSLEY)
      H = std::max(H, 1 + 2 * bcs[b].time.n_harmonics);
  pb->H = H;
  if ((int64_t)n_bcs * (H + 1) > kMaxDirCoef) {
    set_error("lfx_problem_create: too many boundary-condition terms");
    return LFX_ERR_INVALID_ARG;
  }
  pb->dir_pos_of_node.assign(V, -1);
  for (int64_t i = 0; i < V; ++i)
    if (owner[i] >= 0) {
      pb->dir_pos_of_node[i] = (int32_t)pb->dir_node.size();
      pb->dir_node.push_back((int32_t)i);
      pb->dir_bc.push_back(owner[i]);
    }
  const int64_t nd = (int64_t)pb->dir_node.size();
  std::vector<double> S((size_t)H * nd * 3, 0.0);
  for (int b = 0; b < n_bcs; ++b) {
    const lfx_bc &bc = bcs[b];
    if (bc.kind != LFX_BC_DIRICHLET) continue;
    double c[3], n[3];
    if (bc.given_geometry) {
      const double nn = std::sqrt(bc.normal[0] * bc.normal[0] + bc.normal[1] * bc.normal[1] + bc.normal[2] * bc.normal[2]);
      for (int k = 0; k < 3; ++k) {
        c[k] = bc.center[k];
        n[k] = bc.normal[k] / nn;
      }
    } else if (!tag_geometry(m, bc.tag, c, n, nullptr)) {
      set_error("lfx_problem_create: no boundary faces carry tag %d", bc.tag);
      return LFX_ERR_INVALID_ARG;
    }
    const double R = bc.radius;
    for (int64_t d = 0; d < nd; ++d) {
      if (pb->dir_bc[d] != b) continue;
      const double *x = &m.xyz[3 * (int64_t)pb->dir_node[d]];
      double r2 = 0.0;
      for (int k = 0; k < 3; ++k) r2 += (x[k] - c[k]) * (x[k] - c[k]);
      if (bc.profile == LFX_PROFILE_UNIFORM) {
        for (int k = 0; k < 3; ++k) S[((size_t)0 * nd + d) * 3 + k] = -n[k];
      } else if (bc.profile == LFX_PROFILE_PARABOLIC) {
        const double s = -2.0 * (R * R - r2) / (M_PI * R * R * R * R);
        for (int k = 0; k < 3; ++k) S[((size_t)0 * nd + d) * 3 + k] = s * n[k];
      } else {
        // Womersley: harmonic 0 is the parabolic unit-flux profile; harmonic k >= 1 contributes
        // Re[(a_k - i b_k) W_k(r) e^{i k w t}] with W_k of unit flux (stored as Re W_k, Im W_k).
        const double s0 = -2.0 * (R * R - r2) / (M_PI * R * R * R * R);
        for (int k = 0; k < 3; ++k) S[((size_t)0 * nd + d) * 3 + k] = s0 * n[k];
        const double w = 2.0 * M_PI / bc.time.p[0], nu = mu / rho;
        const double r = std::sqrt(r2);
        const std::complex<double> i32 = std::exp(std::complex<double>(0.0, 0.75 * M_PI));  // i^{3/2}
        for (int h = 1; h <= bc.time.n_harmonics; ++h) {
          const double a = R * std::sqrt(h * w / nu);
          const std::complex<double> z = i32 * a;
          const std::complex<double> j0 = bessel_j0(z), j1 = bessel_j1(z);
          // velocity shape 1 - J0(z r/R)/J0(z); its flux over the disk: pi R^2 (1 - 2 J1(z)/(z J0(z)))
          const std::complex<double> shape = 1.0 - bessel_j0(z * (r / R)) / j0;
          const std::complex<double> flux = M_PI * R * R * (1.0 - 2.0 * j1 / (z * j0));
          const std::complex<double> W = shape / flux;
          for (int k = 0; k < 3; ++k) {
            S[((size_t)(2 * h - 1) * nd + d) * 3 + k] = -W.real() * n[k];
            S[((size_t)(2 * h) * nd + d) * 3 + k] = -W.imag() * n[k];
          }
        }
      }
    }
  }
  LFX_TRY(pb->d_dir_node.alloc(sizeof(int32_t) * nd));
  LFX_TRY(pb->d_dir_bc.alloc(sizeof(int32_t) * nd));
  LFX_TRY(pb->d_S.alloc(sizeof(double) * S.size()));
  if (nd) {
    LFX_CUDA_TRY(cudaMemcpy(pb->d_dir_node.p, pb->dir_node.data(), sizeof(int32_t) * nd, cudaMemcpyHostToDevice));
    LFX_CUDA_TRY(cudaMemcpy(pb->d_dir_bc.p, pb->dir_bc.data(), sizeof(int32_t) * nd, cudaMemcpyHostToDevice));
    LFX_CUDA_TRY(cudaMemcpy(pb->d_S.p, S.data(), sizeof(double) * S.size(), cudaMemcpyHostToDevice));
  }

  // ---- Neumann load vectors: sum over the tag's faces of A_f n_f / 3 at each face vertex
  {
    std::vector<std::vector<double>> acc(n_bcs);
    std::vector<double> vec;
    std::vector<int32_t> r1_off(1, 0), r1_node, ax_node, ax_tag;
    std::vector<double> r1_w, ax_w, r1_cr;
    for (int b = 0; b < n_bcs; ++b) {
      if (bcs[b].kind != LFX_BC_NEUMANN && bcs[b].kind != LFX_BC_RESISTANCE) continue;
      std::vector<double> nv((size_t)V * 3, 0.0);
      std::vector<char> hit(V, 0);
      for (int64_t f = 0; f < m.F; ++f) {
        if (m.btags[f] != bcs[b].tag) continue;
        const int32_t *fv = &m.bfaces[3 * f];
        const double *a = &m.xyz[3 * (int64_t)fv[0]], *bb = &m.xyz[3 * (int64_t)fv[1]], *c = &m.xyz[3 * (int64_t)fv[2]];
        double u[3], v[3], cr[3];
        for (int k = 0; k < 3; ++k) {
          u[k] = bb[k] - a[k];
          v[k] = c[k] - a[k];
        }
        cr[0] = u[1] * v[2] - u[2] * v[1];
        cr[1] = u[2] * v[0] - u[0] * v[2];
        cr[2] = u[0] * v[1] - u[1] * v[0];
        for (int q = 0; q < 3; ++q) {
          hit[fv[q]] = 1;
          for (int k = 0; k < 3; ++k) nv[3 * (int64_t)fv[q] + k] += 0.5 * cr[k] / 3.0;
        }
      }
      for (int64_t i = 0; i < V; ++i)
        if (hit[i]) {
          pb->neu_node.push_back((int32_t)i);
          pb->neu_bc.push_back(b);
          for (int k = 0; k < 3; ++k) vec.push_back(nv[3 * i + k]);
        }
      if (bcs[b].kind == LFX_BC_RESISTANCE) {
        // rank-one term: w . x over every node of the tag; the update skips Dirichlet rows
        const int32_t t = (int32_t)r1_cr.size();
        r1_cr.push_back(bcs[b].resistance);
        for (int64_t i = 0; i < V; ++i) {
          if (!hit[i]) continue;
          r1_node.push_back((int32_t)i);
          for (int k = 0; k < 3; ++k) r1_w.push_back(nv[3 * i + k]);
          if (pri[i] < 2) {
            ax_node.push_back((int32_t)i);
            ax_tag.push_back(t);
            for (int k = 0; k < 3; ++k) ax_w.push_back(nv[3 * i + k]);
          }
        }
        r1_off.push_back((int32_t)r1_node.size());
      }
    }
    pb->n_r1_tags = (int)r1_cr.size();
    pb->n_r1_ax = (int64_t)ax_node.size();
    if (pb->n_r1_tags > 0) {
      auto up = [](DBuf &d, const void *src, size_t bytes) -> lfx_status {
        LFX_TRY(d.alloc(std::max<size_t>(bytes, 8)));
        if (bytes) LFX_CUDA_TRY(cudaMemcpy(d.p, src, bytes, cudaMemcpyHostToDevice));
        return LFX_OK;
      };
      LFX_TRY(up(pb->d_r1_cr, r1_cr.data(), sizeof(double) * r1_cr.size()));
      LFX_TRY(up(pb->d_r1_off, r1_off.data(), sizeof(int32_t) * r1_off.size()));
      LFX_TRY(up(pb->d_r1_node, r1_node.data(), sizeof(int32_t) * r1_node.size()));
      LFX_TRY(up(pb->d_r1_w, r1_w.data(), sizeof(double) * r1_w.size()));
      LFX_TRY(up(pb->d_r1_ax_node, ax_node.data(), sizeof(int32_t) * ax_node.size()));
      LFX_TRY(up(pb->d_r1_ax_tag, ax_tag.data(), sizeof(int32_t) * ax_tag.size()));
      LFX_TRY(up(pb->d_r1_ax_w, ax_w.data(), sizeof(double) * ax_w.size()));
    }
    {
      std::vector<int32_t> fl, fb;
      for (int b = 0; b < n_bcs; ++b) {
        if (bcs[b].kind != LFX_BC_NEUMANN) continue;
        for (int64_t f = 0; f < m.F; ++f) {
          if (m.btags[f] != bcs[b].tag) continue;
          for (int k = 0; k < 3; ++k) fl.push_back(m.bfaces[3 * f + k]);
          fb.push_back(b);
        }
      }
      pb->n_neu_faces = (int64_t)fb.size();
      LFX_TRY(pb->d_neu_faces.alloc(sizeof(int32_t) * std::max<size_t>(fl.size(), 1)));
      LFX_TRY(pb->d_neu_face_bc.alloc(sizeof(int32_t) * std::max<size_t>(fb.size(), 1)));
      if (!fb.empty()) {
        LFX_CUDA_TRY(cudaMemcpy(pb->d_neu_faces.p, fl.data(), sizeof(int32_t) * fl.size(), cudaMemcpyHostToDevice));
        LFX_CUDA_TRY(cudaMemcpy(pb->d_neu_face_bc.p, fb.data(), sizeof(int32_t) * fb.size(), cudaMemcpyHostToDevice));
      }
    }
    const int64_t nn = (int64_t)pb->neu_node.size();
    LFX_TRY(pb->d_neu_node.alloc(sizeof(int32_t) * nn));
    LFX_TRY(pb->d_neu_bc.alloc(sizeof(int32_t) * nn));
    LFX_TRY(pb->d_neu_vec.alloc(sizeof(double) * 3 * nn));
    if (nn) {
      LFX_CUDA_TRY(cudaMemcpy(pb->d_neu_node.p, pb->neu_node.data(), sizeof(int32_t) * nn, cudaMemcpyHostToDevice));
      LFX_CUDA_TRY(cudaMemcpy(pb->d_neu_bc.p, pb->neu_bc.data(), sizeof(int32_t) * nn, cudaMemcpyHostToDevice));
      LFX_CUDA_TRY(cudaMemcpy(pb->d_neu_vec.p, vec.data(), sizeof(double) * 3 * nn, cudaMemcpyHostToDevice));
    }
  }

  // ---- inertial backflow stabilisation (Section 2.2.2): tasks per face edge
  {
    auto block_of = [&](int32_t r, int32_t c) -> int32_t {
      const auto b0 = m.col_idx.begin() + m.row_ptr[r], b1 = m.col_idx.begin() + m.row_ptr[r + 1];
      const auto it = std::lower_bound(b0, b1, c);
      return (it != b1 && *it == c) ? (int32_t)(it - m.col_idx.begin()) : -1;
    };
    std::vector<int32_t> ij, slot4, blk;
    std::vector<double> an, coef;
    std::unordered_map<int32_t, int32_t> compact;
    for (int b = 0; b < n_bcs; ++b) {
      if (bcs[b].kind != LFX_BC_NEUMANN || bcs[b].beta <= 0.0) continue;
      for (int64_t f = 0; f < m.F; ++f) {
        if (m.btags[f] != bcs[b].tag) continue;
        const int32_t *fv = &m.bfaces[3 * f];
        const double *x0 = &m.xyz[3 * (int64_t)fv[0]], *x1 = &m.xyz[3 * (int64_t)fv[1]], *x2 = &m.xyz[3 * (int64_t)fv[2]];
        double u[3], v[3];
        for (int k = 0; k < 3; ++k) {
          u[k] = x1[k] - x0[k];
          v[k] = x2[k] - x0[k];
        }
        const double a[3] = {0.5 * (u[1] * v[2] - u[2] * v[1]), 0.5 * (u[2] * v[0] - u[0] * v[2]),
                             0.5 * (u[0] * v[1] - u[1] * v[0])};
        const int e[3][2] = {{0, 1}, {1, 2}, {0, 2}};
        for (int q = 0; q < 3; ++q) {
          const int32_t i = fv[e[q][0]], j = fv[e[q][1]];
          ij.push_back(i);
          ij.push_back(j);
          for (int k = 0; k < 3; ++k) an.push_back(a[k]);
          coef.push_back(bcs[b].beta * rho / 2.0);
          const int32_t pr[4][2] = {{i, i}, {i, j}, {j, i}, {j, j}};
          for (int t = 0; t < 4; ++t) {
            const int32_t s = block_of(pr[t][0], pr[t][1]);
            if (s < 0) {
              set_error("lfx_problem_create: boundary face edge outside the block pattern");
              return LFX_ERR_BAD_MESH;
            }
            auto ins = compact.emplace(s, (int32_t)blk.size());
            if (ins.second) blk.push_back(s);
            slot4.push_back(ins.first->second);
          }
        }
      }
    }
    pb->n_bf_edges = (int64_t)coef.size();
    pb->n_bf_blocks = (int64_t)blk.size();
    if (pb->n_bf_edges > 0) {
      LFX_TRY(pb->d_bf_ij.alloc(sizeof(int32_t) * ij.size()));
      LFX_TRY(pb->d_bf_an.alloc(sizeof(double) * an.size()));
      LFX_TRY(pb->d_bf_coef.alloc(sizeof(double) * coef.size()));
      LFX_TRY(pb->d_bf_slot4.alloc(sizeof(int32_t) * slot4.size()));
      LFX_TRY(pb->d_bf_blk.alloc(sizeof(int32_t) * blk.size()));
      LFX_TRY(pb->d_bf_acc.alloc(sizeof(double) * blk.size()));
      LFX_CUDA_TRY(cudaMemcpy(pb->d_bf_ij.p, ij.data(), sizeof(int32_t) * ij.size(), cudaMemcpyHostToDevice));
      LFX_CUDA_TRY(cudaMemcpy(pb->d_bf_an.p, an.data(), sizeof(double) * an.size(), cudaMemcpyHostToDevice));
      LFX_CUDA_TRY(cudaMemcpy(pb->d_bf_coef.p, coef.data(), sizeof(double) * coef.size(), cudaMemcpyHostToDevice));
      LFX_CUDA_TRY(cudaMemcpy(pb->d_bf_slot4.p, slot4.data(), sizeof(int32_t) * slot4.size(), cudaMemcpyHostToDevice));
      LFX_CUDA_TRY(cudaMemcpy(pb->d_bf_blk.p, blk.data(), sizeof(int32_t) * blk.size(), cudaMemcpyHostToDevice));
    }
  }

  // ---- RIIS nodal signed distances (internal numbering)
  {
    std::vector<double> phi((size_t)std::max(1, n_riis) * V, 0.0);
    for (int k = 0; k < n_riis; ++k) {
      const lfx_riis &s = riis[k];
      for (int64_t i = 0; i < V; ++i) {
        double val;
        if (s.kind == LFX_RIIS_SDF_NODAL) {
          val = s.sdf_nodal[m.node_old[i]];
        } else {
          const double *x = &m.xyz[3 * i];
          const double nn = std::sqrt(s.normal[0] * s.normal[0] + s.normal[1] * s.normal[1] + s.normal[2] * s.normal[2]);
          double d[3], h = 0.0;
          for (int q = 0; q < 3; ++q) {
            d[q] = x[q] - s.center[q];
            h += d[q] * s.normal[q] / nn;
          }
          double rad2 = 0.0;
          for (int q = 0; q < 3; ++q) {
            const double t = d[q] - h * s.normal[q] / nn;
            rad2 += t * t;
          }
          const double rad = std::sqrt(rad2);
          double dist = std::fabs(h);
          if (rad > s.radius) dist = std::hypot(rad - s.radius, h);
          val = h >= 0 ? dist : -dist;
        }
        phi[(size_t)k * V + i] = val;
      }
    }
    LFX_TRY(pb->d_phi.alloc(sizeof(double) * phi.size()));
    LFX_CUDA_TRY(cudaMemcpy(pb->d_phi.p, phi.data(), sizeof(double) * phi.size(), cudaMemcpyHostToDevice));
  }

  // ---- elements that keep FP64 geometry in mixed assembly
  {
    std::vector<uint8_t> bad(m.T, 0);
    for (int64_t e = 0; e < m.T; ++e)
      if (m.quality[e] < o.bad_element_quality) {
        bad[e] = 1;
        ++pb->n_bad;
      }
    LFX_TRY(pb->d_bad.alloc(m.T));
    LFX_CUDA_TRY(cudaMemcpy(pb->d_bad.p, bad.data(), m.T, cudaMemcpyHostToDevice));
  }
  if (o.pin_pressure_node >= 0) {
    if (o.pin_pressure_node >= V) {
      set_error("lfx_problem_create: pin_pressure_node out of range");
      return LFX_ERR_INVALID_ARG;
    }
    pb->pin_node = m.node_new[o.pin_pressure_node];
  }
  // ---- element geometry, once: the mesh does not move, so every step reuses it
  {
    AssembleArgs A{};
    A.conn = m.d_conn.as<int4>();
    A.xyz = m.d_xyz.as<D4>();
    A.xyz_hi = m.d_xyz_hi.as<float4>();
    A.xyz_lo = m.d_xyz_lo.as<float4>();
    A.n_nodes = V;
    A.n_elems = m.T;
    const size_t nv = (size_t)kGeoValues * (size_t)std::max<int64_t>(m.T, 1);
    if (o.precision == LFX_PREC_MIXED) {
      A.bad = pb->n_bad > 0 ? pb->d_bad.as<uint8_t>() : nullptr;
      LFX_TRY(pb->geo_hi.alloc(sizeof(float) * nv));
      LFX_TRY(pb->geo_lo.alloc(sizeof(float) * nv));
      LFX_TRY(launch_geometry<dd>(0, A, m.T, nullptr, pb->geo_hi.as<float>(), pb->geo_lo.as<float>()));
    } else {
      LFX_TRY(pb->geo64.alloc(sizeof(double) * nv));
      LFX_TRY(launch_geometry<double>(0, A, m.T, pb->geo64.as<double>(), nullptr, nullptr));
    }
    LFX_CUDA_TRY(cudaStreamSynchronize(0));
  }
  LFX_TRY(pb->d_chunk_color_off.alloc(sizeof(int32_t) * m.chunk_color_off.size()));
  LFX_CUDA_TRY(cudaMemcpy(pb->d_chunk_color_off.p, m.chunk_color_off.data(), sizeof(int32_t) * m.chunk_color_off.size(),
                          cudaMemcpyHostToDevice));
  pb->asm_mode = pb->asm_mode_newton = o.assembly;
  *out = pb.release();
  return LFX_OK;
}

lfx_status lfx_problem_assembly_tuning(const lfx_problem *pb, int32_t *mode, float ms[3]) {
  if (!pb || !mode || !ms) {
    set_error("lfx_problem_assembly_tuning: NULL argument");
    return LFX_ERR_INVALID_ARG;
  }
  lfx_problem *p = const_cast<lfx_problem *>(pb);
  std::lock_guard<std::mutex> lk(p->tune_mu);
  *mode = p->asm_mode;
  for (int i = 0; i < 3; ++i) ms[i] = p->asm_ms[i];
  return LFX_OK;
}

void lfx_problem_destroy(lfx_problem *problem) { delete problem; }

// --------------------------------------------------------------------------------- state
// History levels from the caller's arrays (u [sigma][V][3], p [sigma][V], caller node order):
// copied as they are (a pinned caller buffer is read by DMA directly), permuted and interleaved on
// the device; returns once the caller's buffers may be reused.
static lfx_status upload_history(lfx_state *s, const double *u_hist, const double *p_hist) {
  const Mesh &m = s->pb->mesh->m;
  const int64_t V = m.V;
  const size_t nu = sizeof(double) * 3 * (size_t)V * s->sigma, np = sizeof(double) * (size_t)V * s->sigma;
  if (s->io_u.bytes < nu) LFX_TRY(s->io_u.alloc(nu));
  if (s->io_p.bytes < np) LFX_TRY(s->io_p.alloc(np));
  LFX_CUDA_TRY(cudaMemcpyAsync(s->io_u.p, u_hist, nu, cudaMemcpyHostToDevice, s->stream));
  LFX_CUDA_TRY(cudaMemcpyAsync(s->io_p.p, p_hist, np, cudaMemcpyHostToDevice, s->stream));
  for (int l = 0; l < s->sigma; ++l)
    LFX_TRY(launch_node_scatter(s->stream, V, m.d_node_old.as<int32_t>(), s->io_u.as<double>() + (size_t)l * 3 * V,
                                s->io_p.as<double>() + (size_t)l * V, s->level(l)));
  LFX_CUDA_TRY(cudaStreamSynchronize(s->stream));
  return LFX_OK;
}

extern "C" lfx_status lfx_state_set(lfx_state *s, const double *u_hist, const double *p_hist, double t) {
  clear_error();
  if (!s || !u_hist || !p_hist) {
    set_error("lfx_state_set: NULL argument");
    return LFX_ERR_INVALID_ARG;
  }
  LFX_TRY(upload_history(s, u_hist, p_hist));
  s->t = t;
  s->assembled = false;
  return LFX_OK;
}

lfx_status lfx_state_create(lfx_problem *pb, const double *u_hist, const double *p_hist, double t0,
                            lfx_state **out) {
  clear_error();
  if (!pb || !u_hist || !p_hist || !out) {
    set_error("lfx_state_create: NULL argument");
    return LFX_ERR_INVALID_ARG;
  }
  *out = nullptr;
  std::unique_ptr<lfx_state> s(new (std::nothrow) lfx_state);
  if (!s) return LFX_ERR_OOM;
  const Mesh &m = pb->mesh->m;
  const int64_t V = m.V;
  s->pb = pb;
  s->sigma = pb->bdf_order;
  s->t = t0;
  for (int l = 0; l < s->sigma; ++l) LFX_TRY(s->hist[l].alloc(sizeof(D4) * V));
  LFX_TRY(upload_history(s.get(), u_hist, p_hist));
  LFX_TRY(s->xsol.alloc(sizeof(D4) * V));
  LFX_TRY(s->ubdf.alloc(sizeof(D4) * V));
  LFX_TRY(s->rhs.alloc(sizeof(D4) * V));
  const int64_t nd = (int64_t)pb->dir_node.size();
  LFX_TRY(s->gdir.alloc(sizeof(D4) * std::max<int64_t>(nd, 1)));
  LFX_TRY(s->nodal.alloc(sizeof(double) * 3 * std::max<int64_t>(nd, 1)));
  LFX_CUDA_TRY(cudaMemset(s->nodal.p, 0, s->nodal.bytes));
  LFX_TRY(s->comp_scale.alloc(sizeof(double) * (size_t)m.n_comp));
  const lfx_options &o = pb->opt;
  if (o.precision != LFX_PREC_MIXED) LFX_TRY(s->vals64.alloc(sizeof(double) * 16 * m.nnzb));
  SmootherConfig cfg;
  cfg.f_kind = o.f_smoother;
  cfg.f_steps = o.f_steps;
  cfg.f_omega = o.f_omega;
  cfg.f_ratio = o.f_ratio;
  cfg.s_kind = o.s_smoother;
  cfg.s_steps = o.s_steps;
  cfg.s_omega = o.s_omega;
  cfg.s_ratio = o.s_ratio;
  cfg.n_power = o.n_power;
  s->pc64.time_f = s->pc32.time_f = s->pcbf.time_f = true;   // F-pass timing for the step statistics
  if (o.precision == LFX_PREC_MIXED) {
    LFX_TRY(s->vals32.alloc(sizeof(float) * 16 * m.nnzb));
    LFX_TRY(s->vals_lo.alloc(sizeof(float) * 16 * m.nnzb));
    LFX_TRY(s->rhs_hi.alloc(sizeof(float) * 4 * V));
    LFX_TRY(s->rhs_lo.alloc(sizeof(float) * 4 * V));
    DBuf *f4[6] = {&s->xe_hi, &s->xe_lo, &s->ub_hi, &s->ub_lo, &s->xs_hi, &s->xs_lo};
    for (DBuf *b : f4) LFX_TRY(b->alloc(sizeof(float4) * V));
    if (o.smoother_bf16) {
      LFX_TRY(s->pcbf.init(V, cfg));
      if (o.staged_f && m.ftile_row.size() > 1) s->pcbf.set_tiles(m.d_ftile_row.as<int32_t>(), (int)m.ftile_row.size() - 1);
    } else {
      LFX_TRY(s->pc32.init(V, cfg));
    }
    LFX_TRY(s->gm32.init(V, o.gmres_restart));
    LFX_TRY(s->gmdd.init(V, std::max(1, o.outer_restart)));
    LFX_TRY(s->r32.alloc(sizeof(float) * 4 * V));
    LFX_TRY(s->z32.alloc(sizeof(float) * 4 * V));
  } else {
    LFX_TRY(s->pc64.init(V, cfg));
    LFX_TRY(s->gm64.init(V, o.gmres_restart));
  }
  if (pb->n_r1_tags > 0) {
    if (m.n_comp > 1) {
      set_error("lfx_state_create: resistance conditions are not available on meshes of several pieces");
      return LFX_ERR_INVALID_ARG;
    }
    const Rank1View r1 = pb->rank1();
    if (o.precision == LFX_PREC_MIXED) {
      LFX_TRY(s->gm32.set_rank1(r1));
      LFX_TRY(s->gmdd.set_rank1(r1));
    } else {
      LFX_TRY(s->gm64.set_rank1(r1));
    }
  }
  if (m.n_comp > 1 && o.batch_segmented) {
    // one Arnoldi process per component of a batched mesh
    if (o.precision == LFX_PREC_MIXED) {
      LFX_TRY(s->gm32.set_segments(m.comp_off));
      LFX_TRY(s->gmdd.set_segments(m.comp_off));
    } else {
      LFX_TRY(s->gm64.set_segments(m.comp_off));
    }
  }
  LFX_CUDA_TRY(cudaEventCreate(&s->e0));
  LFX_CUDA_TRY(cudaEventCreate(&s->e1));
  LFX_CUDA_TRY(cudaEventCreate(&s->e2));
  LFX_CUDA_TRY(cudaEventCreate(&s->ea0));
  LFX_CUDA_TRY(cudaEventCreate(&s->ea1));
  *out = s.release();
  return LFX_OK;
}

void lfx_state_destroy(lfx_state *state) { delete state; }

lfx_status lfx_set_stream(lfx_state *s, void *stream) {
  if (!s) {
    set_error("lfx_set_stream: NULL state");
    return LFX_ERR_INVALID_ARG;
  }
  s->stream = (cudaStream_t)stream;
  return LFX_OK;
}

lfx_status lfx_set_dirichlet_nodal(lfx_state *s, int32_t tag, const double *u) {
  if (!s || !u) {
    set_error("lfx_set_dirichlet_nodal: NULL argument");
    return LFX_ERR_INVALID_ARG;
  }
  const lfx_problem *pb = s->pb;
  const Mesh &m = pb->mesh->m;
  int found = -1;
  for (size_t b = 0; b < pb->bcs.size(); ++b)
    if (pb->bcs[b].tag == tag && pb->bcs[b].kind == LFX_BC_NODAL) found = (int)b;
  if (found < 0) {
    set_error("lfx_set_dirichlet_nodal: no NODAL boundary condition on tag %d", tag);
    return LFX_ERR_INVALID_ARG;
  }
  const int64_t nd = (int64_t)pb->dir_node.size();
  std::vector<double> h(3 * nd);
  LFX_CUDA_TRY(cudaMemcpy(h.data(), s->nodal.p, sizeof(double) * 3 * nd, cudaMemcpyDeviceToHost));
  for (int64_t d = 0; d < nd; ++d) {
    if (pb->dir_bc[d] != found) continue;
    const int64_t o = m.node_old[pb->dir_node[d]];
    for (int k = 0; k < 3; ++k) h[3 * d + k] = u[3 * o + k];
  }
  LFX_CUDA_TRY(cudaMemcpy(s->nodal.p, h.data(), sizeof(double) * 3 * nd, cudaMemcpyHostToDevice));
  return LFX_OK;
}

lfx_status lfx_set_pressure_pin(lfx_state *s, double value) {
  if (!s) {
    set_error("lfx_set_pressure_pin: NULL state");
    return LFX_ERR_INVALID_ARG;
  }
  s->pin_value = value;
  return LFX_OK;
}

lfx_status lfx_state_amg_levels(const lfx_state *s, int32_t *n_levels, int64_t *rows, int64_t *nnz,
                                int32_t capacity) {
  if (!s || !n_levels || capacity < 0 || (capacity > 0 && (!rows || !nnz))) {
    set_error("lfx_state_amg_levels: invalid argument");
    return LFX_ERR_INVALID_ARG;
  }
  const lfx_options &o = s->pb->opt;
  const std::vector<int64_t> *r = &s->pc64.lvl_rows, *z = &s->pc64.lvl_nnz;
  if (o.precision == LFX_PREC_MIXED) {
    r = o.smoother_bf16 ? &s->pcbf.lvl_rows : &s->pc32.lvl_rows;
    z = o.smoother_bf16 ? &s->pcbf.lvl_nnz : &s->pc32.lvl_nnz;
  }
  *n_levels = (int32_t)r->size();
  for (int i = 0; i < (int)r->size() && i < capacity; ++i) {
    rows[i] = (*r)[i];
    nnz[i] = (*z)[i];
  }
  return LFX_OK;
}

lfx_status lfx_state_device_bytes(const lfx_state *s, int64_t *bytes) {
  if (!s || !bytes) {
    set_error("lfx_state_device_bytes: NULL argument");
    return LFX_ERR_INVALID_ARG;
  }
  size_t b = s->pb->mesh->m.device_bytes() + s->pb->device_bytes() + s->xsol.bytes + s->ubdf.bytes +
             s->rhs.bytes + s->gdir.bytes + s->nodal.bytes + s->vals64.bytes + s->vals32.bytes +
             s->pc64.device_bytes() + s->pc64.amg_bytes() + s->gm64.device_bytes() +
             s->pc32.device_bytes() + s->pc32.amg_bytes() + s->pcbf.device_bytes() + s->pcbf.amg_bytes() +
             s->gm32.device_bytes() + s->r32.bytes + s->z32.bytes + s->gmdd.device_bytes() + s->vals_lo.bytes +
             s->rhs_hi.bytes + s->rhs_lo.bytes + s->xe_hi.bytes + s->xe_lo.bytes + s->ub_hi.bytes + s->ub_lo.bytes +
             s->xs_hi.bytes + s->xs_lo.bytes;
  for (int l = 0; l < 3; ++l) b += s->hist[l].bytes;
  b += s->io_u.bytes + s->io_p.bytes;
  *bytes = (int64_t)b;
  return LFX_OK;
}

// Assembly of the system for t^{n+1} = t + dt into vals64 / rhs, x0 = extrapolation.  With
// newton, the Jacobian of the fully implicit formulation at the iterate held in xsol and the
// right-hand side J U - R(U) instead (the BDF fields of the step's first assembly are kept).
// newton: the Newton system of the fully implicit step at the iterate in xsol; at_iterate: the
// semi-implicit system with u^EXT, p^EXT taken from the iterate in xsol (its residual A U - b is the
// implicit residual R(U)); otherwise the semi-implicit system of the step (the BDF fields are formed
// and xsol receives the extrapolation).
static lfx_status assemble_system(lfx_state *s, bool apply_bcs, bool newton = false, bool at_iterate = false) {
  lfx_problem *pb = s->pb;
  const Mesh &m = pb->mesh->m;
  cudaStream_t st = s->stream;
  const double t1 = s->t + pb->P.dt;
  const int sg = s->sigma;
  const bool mixed = s->mixed();
  if (newton || at_iterate) {
    if (mixed) LFX_TRY(launch_split_vec(st, m.V, s->xsol.as<double>(), s->xe_hi.as<float4>(), s->xe_lo.as<float4>()));
  } else {
    LFX_TRY(launch_bdf(st, m.V, sg, s->level(0), sg > 1 ? s->level(1) : nullptr, sg > 2 ? s->level(2) : nullptr,
                       pb->beta, pb->gamma, s->xsol.as<D4>(), s->ubdf.as<D4>(), s->xe_hi.as<float4>(),
                       s->xe_lo.as<float4>(), s->ub_hi.as<float4>(), s->ub_lo.as<float4>()));
  }
  // (every block and row written by its first element needs no clearing beforehand)
  if (mixed) {
    if (!m.all_blocks_touched) {
      LFX_CUDA_TRY(cudaMemsetAsync(s->vals32.p, 0, s->vals32.bytes, st));
      LFX_CUDA_TRY(cudaMemsetAsync(s->vals_lo.p, 0, s->vals_lo.bytes, st));
    }
    if (!m.all_nodes_touched) {
      LFX_CUDA_TRY(cudaMemsetAsync(s->rhs_hi.p, 0, s->rhs_hi.bytes, st));
      LFX_CUDA_TRY(cudaMemsetAsync(s->rhs_lo.p, 0, s->rhs_lo.bytes, st));
    }
  } else {
    if (!m.all_blocks_touched) LFX_CUDA_TRY(cudaMemsetAsync(s->vals64.p, 0, s->vals64.bytes, st));
    if (!m.all_nodes_touched) LFX_CUDA_TRY(cudaMemsetAsync(s->rhs.p, 0, s->rhs.bytes, st));
  }
  AssembleArgs A{};
  A.conn = m.d_conn.as<int4>();
  A.slot = m.d_slot.as<int32_t>();
  A.first = m.d_first.as<uint16_t>();
  A.xyz = m.d_xyz.as<D4>();
  A.xext = s->xsol.as<D4>();
  A.ubdf = s->ubdf.as<D4>();
  A.phi_riis = pb->d_phi.as<double>();
  A.bad = nullptr;
  A.rhs = s->rhs.as<double>();
  A.n_nodes = m.V;
  A.xyz_hi = m.d_xyz_hi.as<float4>();
  A.xyz_lo = m.d_xyz_lo.as<float4>();
  A.xext_hi = s->xe_hi.as<float4>();
  A.xext_lo = s->xe_lo.as<float4>();
  A.ubdf_hi = s->ub_hi.as<float4>();
  A.ubdf_lo = s->ub_lo.as<float4>();
  A.vals_lo = s->vals_lo.as<float>();
  A.rhs_hi = s->rhs_hi.as<float>();
  A.rhs_lo = s->rhs_lo.as<float>();
  A.n_elems = m.T;
  A.geo64 = pb->geo64.as<double>();
  A.geo_hi = pb->geo_hi.as<float>();
  A.geo_lo = pb->geo_lo.as<float>();
  if (s->ale) {
    // the configuration x^ + d^{n+1} and the advection velocity u^EXT - u_ALE
    A.xyz = s->xyz.as<D4>();
    A.xyz_hi = s->xyz_hi.as<float4>();
    A.xyz_lo = s->xyz_lo.as<float4>();
    A.geo64 = s->geo64.as<double>();
    A.geo_hi = s->geo_hi.as<float>();
    A.geo_lo = s->geo_lo.as<float>();
    A.uale = s->uale.as<D4>();
  }
  A.elist = m.d_color_elems.as<int32_t>();
  const ChunkArgs CA{m.d_chunk_elem_off.as<int32_t>(), m.d_chunk_pass_off.as<int32_t>(), m.d_pass_code.as<uint16_t>(),
                     m.d_pass_run_off.as<int32_t>(), m.d_pass_ndiag.as<int32_t>(), m.d_run_meta.as<uint16_t>(),
                     m.d_run_block.as<int32_t>(), m.d_run_node.as<int32_t>()};
  const int n_cc = (int)m.chunk_color_off.size() - 1;
  if (mixed) A.bad = pb->n_bad > 0 ? pb->d_bad.as<uint8_t>() : nullptr;   // badly shaped: FP64 geometry
  if (!s->asm_sync.p) {
    LFX_TRY(s->asm_sync.alloc(64));
    LFX_CUDA_TRY(cudaMallocHost(&s->asm_err_host, sizeof(int)));
    *s->asm_err_host = 0;
  }
  unsigned *barrier = s->asm_sync.as<unsigned>();
  int *err = reinterpret_cast<int *>(s->asm_sync.as<char>() + 32);
  // one assembly of the semi-implicit system (or the Newton system) in launch shape `mode`
  auto launch = [&](int mode) -> lfx_status {
    if (mixed) {
      if (mode == LFX_ASM_COLORS)
        return launch_assemble<dd, float>(st, A, pb->P, m.color_off.data(), (int)m.color_off.size() - 1,
                                          s->vals32.as<float>(), newton);
      if (mode == LFX_ASM_CHUNKS)
        return launch_assemble_chunks<dd, float>(st, A, pb->P, CA, m.chunk_color_off.data(), n_cc,
                                                 s->vals32.as<float>(), newton);
      return launch_assemble_persistent<dd, float>(st, A, pb->P, CA, pb->d_chunk_color_off.as<int32_t>(), n_cc,
                                                   s->vals32.as<float>(), barrier, err, s->force_timeout, newton);
    }
    if (mode == LFX_ASM_COLORS)
      return launch_assemble<double, double>(st, A, pb->P, m.color_off.data(), (int)m.color_off.size() - 1,
                                             s->vals64.as<double>(), newton);
    if (mode == LFX_ASM_CHUNKS)
      return launch_assemble_chunks<double, double>(st, A, pb->P, CA, m.chunk_color_off.data(), n_cc,
                                                    s->vals64.as<double>(), newton);
    return launch_assemble_persistent<double, double>(st, A, pb->P, CA, pb->d_chunk_color_off.as<int32_t>(), n_cc,
                                                      s->vals64.as<double>(), barrier, err, s->force_timeout, newton);
  };
  int mode = LFX_ASM_COLORS;
  {
    // the semi-implicit and the Newton systems are tuned apart (their kernels fit the SMs differently)
    std::lock_guard<std::mutex> lk(pb->tune_mu);
    int &tuned = newton ? pb->asm_mode_newton : pb->asm_mode;
    float *tuned_ms = newton ? pb->asm_ms_newton : pb->asm_ms;
    if (tuned == LFX_ASM_AUTO) {
      // autotuner: each launch shape twice (the second timed) on this state's buffers; the fastest
      // becomes the problem's shape (every assembly writes the complete system, so the last one run
      // leaves a valid matrix behind)
      float best = 0.0f;
      int pick = LFX_ASM_COLORS;
      for (int cand = LFX_ASM_COLORS; cand <= LFX_ASM_PERSISTENT; ++cand) {
        LFX_TRY(launch(cand));
        LFX_CUDA_TRY(cudaEventRecord(s->ea0, st));
        LFX_TRY(launch(cand));
        LFX_CUDA_TRY(cudaEventRecord(s->ea1, st));
        LFX_CUDA_TRY(cudaEventSynchronize(s->ea1));
        float ms = 0.0f;
        LFX_CUDA_TRY(cudaEventElapsedTime(&ms, s->ea0, s->ea1));
        tuned_ms[cand - 1] = ms;
        if (cand == LFX_ASM_COLORS || ms < best) {
          best = ms;
          pick = cand;
        }
      }
      tuned = pick;
    }
    mode = tuned;
  }
  if (!newton) s->asm_mode_used = mode;
  LFX_CUDA_TRY(cudaEventRecord(s->ea0, st));
  LFX_TRY(launch(mode));
  LFX_CUDA_TRY(cudaEventRecord(s->ea1, st));
  if (mode == LFX_ASM_PERSISTENT)
    LFX_CUDA_TRY(cudaMemcpyAsync(s->asm_err_host, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  if (pb->n_bf_edges > 0)
    LFX_TRY(launch_backflow(st, pb->n_bf_edges, pb->d_bf_ij.as<int32_t>(), pb->d_bf_an.as<double>(),
                            pb->d_bf_coef.as<double>(), pb->d_bf_slot4.as<int32_t>(), s->xsol.as<D4>(),
                            pb->n_bf_blocks, pb->d_bf_blk.as<int32_t>(), pb->d_bf_acc.as<double>(),
                            mixed ? nullptr : s->vals64.as<double>(), mixed ? s->vals32.as<float>() : nullptr,
                            mixed ? s->vals_lo.as<float>() : nullptr));
  if (mixed) LFX_TRY(launch_dd_combine(st, 4 * m.V, s->rhs_hi.as<float>(), s->rhs_lo.as<float>(), s->rhs.as<double>()));
  if (!newton)
    s->n_asm_launch = mode == LFX_ASM_COLORS ? (int)m.color_off.size() - 1 : (mode == LFX_ASM_CHUNKS ? n_cc : 1);
  // boundary data at t^{n+1}
  DirCoef C;
  memset(&C, 0, sizeof(C));
  const int nb = (int)pb->bcs.size();
  for (int b = 0; b < nb; ++b)
    if (pb->bcs[b].kind == LFX_BC_NEUMANN || pb->bcs[b].kind == LFX_BC_RESISTANCE)
      C.c[b] = time_law(pb->bcs[b].time, t1);
  if (s->ale)
    LFX_TRY(launch_neumann_faces(st, pb->n_neu_faces, pb->d_neu_faces.as<int32_t>(), pb->d_neu_face_bc.as<int32_t>(), C,
                                 s->xyz.as<D4>(), s->rhs.as<double>()));
  else
    LFX_TRY(launch_neumann(st, (int64_t)pb->neu_node.size(), pb->d_neu_node.as<int32_t>(), pb->d_neu_bc.as<int32_t>(),
                           pb->d_neu_vec.as<double>(), C, s->rhs.as<double>()));
  if (!apply_bcs) return LFX_OK;
  memset(&C, 0, sizeof(C));
  const int H = pb->H;
  for (int b = 0; b < nb; ++b) {
    const lfx_bc &bc = pb->bcs[b];
    if (bc.kind == LFX_BC_NODAL) {
      C.c[nb * H + b] = 1.0;
    } else if (bc.kind == LFX_BC_DIRICHLET) {
      if (bc.profile == LFX_PROFILE_WOMERSLEY) {
        const lfx_time_law &L = bc.time;
        const double w = 2.0 * M_PI / L.p[0];
        C.c[b * H + 0] = bc.theta * L.a[0];
        for (int h = 1; h <= L.n_harmonics; ++h) {
          // Re[(a - i b) W e^{i h w t}] = (a cos + b sin) Re W + (b cos - a sin) Im W
          const double cw = std::cos(h * w * t1), sw = std::sin(h * w * t1);
          C.c[b * H + 2 * h - 1] = bc.theta * (L.a[h] * cw + L.b[h] * sw);
          C.c[b * H + 2 * h] = bc.theta * (L.b[h] * cw - L.a[h] * sw);
        }
      } else {
        C.c[b * H + 0] = bc.theta * time_law(bc.time, t1);
      }
    }
  }
  const int64_t nd = (int64_t)pb->dir_node.size();
  LFX_TRY(launch_dirichlet_values(st, nd, H, pb->d_dir_bc.as<int32_t>(), pb->d_S.as<double>(), C,
                                  s->nodal.as<double>(), nb, s->gdir.as<D4>()));
  if (mixed)
    LFX_TRY(launch_apply_dirichlet_dd(st, nd, pb->d_dir_node.as<int32_t>(), s->gdir.as<D4>(), pb->pin_node,
                                      s->pin_value, m.d_rowptr.as<int32_t>(), m.d_diag.as<int32_t>(),
                                      s->vals32.as<float>(), s->vals_lo.as<float>(), s->rhs.as<double>(),
                                      s->xsol.as<double>()));
  else
    LFX_TRY(launch_apply_dirichlet<double>(st, nd, pb->d_dir_node.as<int32_t>(), s->gdir.as<D4>(), pb->pin_node,
                                           s->pin_value, m.d_rowptr.as<int32_t>(), m.d_diag.as<int32_t>(),
                                           s->vals64.as<double>(), s->rhs.as<double>(), s->xsol.as<double>()));
  // (segmented solves test every component against its own ||b_c|| and need no scaling; the
  // Jacobi-scaled smoothers are invariant under it, but a Schur AMG hierarchy built at an earlier
  // step is not: its coarse operators keep that step's scale)
  if (m.n_comp > 1 && pb->opt.batch_normalize && !pb->opt.batch_segmented) {
    if (mixed)
      LFX_TRY(launch_comp_normalize_dd(st, m.V, m.n_comp, m.d_comp_off.as<int32_t>(), s->comp_scale.as<double>(),
                                       m.d_rowptr.as<int32_t>(), s->vals32.as<float>(), s->vals_lo.as<float>(),
                                       s->rhs.as<double>()));
    else
      LFX_TRY(launch_comp_normalize(st, m.V, m.n_comp, m.d_comp_off.as<int32_t>(), s->comp_scale.as<double>(),
                                    m.d_rowptr.as<int32_t>(), s->vals64.as<double>(), s->rhs.as<double>()));
  }
  return LFX_OK;
}

}  // extern "C"

// Device bytes a state of this problem will allocate (mirrors lfx_state_create and the first
// step's lazily built preconditioner data), plus 10 % slack.
int64_t lfx_internal_state_bytes_estimate(const lfx_problem *pb, int64_t *V_out, int *sigma_out) {
  const Mesh &m = pb->mesh->m;
  const lfx_options &o = pb->opt;
  const int64_t V = m.V, nnzb = m.nnzb;
  const int sigma = pb->bdf_order;
  if (V_out) *V_out = V;
  if (sigma_out) *sigma_out = sigma;
  const int64_t v64 = 32 * V, v32 = 16 * V;
  int64_t b = (sigma + 3) * v64 + 64 * (int64_t)pb->dir_node.size() + 8 * m.n_comp;
  b += sigma * v64;                                          // caller-layout staging (history in, solution out)
  b += 128 * nnzb;                                           // FP64 or double-float matrix
  const int64_t amg = o.s_smoother == LFX_SMOOTH_AMG ? 300 * V + 8LL * o.amg_coarse_size * o.amg_coarse_size : 0;
  const int64_t part = 8LL * 152 * 4 * 65 + 8 * (V * 8 / 256 + 64);
  if (o.precision == LFX_PREC_MIXED) {
    b += (o.smoother_bf16 ? 40 * nnzb : 80 * nnzb) + 8 * v32;     // F, G, (D, C) apart; split inputs
    b += 7 * v32 + 4 * V + amg;                               // FP32 aSIMPLE work
    b += (2 * (int64_t)o.gmres_restart + 2) * v32 + part;    // inner GMRES
    b += (2 * (int64_t)std::max(1, o.outer_restart) + 2) * v64 + part;   // outer FGMRES
    b += 2 * v32;
  } else {
    b += 160 * nnzb + 7 * v64 + 8 * V + amg;                 // F, G, (D, C) apart in FP64
    b += (2 * (int64_t)o.gmres_restart + 2) * v64 + part;
  }
  return b + b / 10;
}

extern "C" {

lfx_status lfx_problem_state_bytes(const lfx_problem *pb, int64_t *bytes) {
  if (!pb || !bytes) {
    set_error("lfx_problem_state_bytes: NULL argument");
    return LFX_ERR_INVALID_ARG;
  }
  *bytes = lfx_internal_state_bytes_estimate(pb, nullptr, nullptr);
  return LFX_OK;
}

}  // extern "C"

// The assembled matrix as FP64 values on the host (hi + lo for the double-float matrix).
static lfx_status download_matrix(lfx_state *s, std::vector<double> &h) {
  const Mesh &m = s->pb->mesh->m;
  const size_t n = 16 * (size_t)m.nnzb;
  h.resize(n);
  if (!s->mixed()) {
    LFX_CUDA_TRY(cudaMemcpyAsync(h.data(), s->vals64.p, sizeof(double) * n, cudaMemcpyDeviceToHost, s->stream));
    LFX_CUDA_TRY(cudaStreamSynchronize(s->stream));
    return LFX_OK;
  }
  std::vector<float> hi(n), lo(n);
  LFX_CUDA_TRY(cudaMemcpyAsync(hi.data(), s->vals32.p, sizeof(float) * n, cudaMemcpyDeviceToHost, s->stream));
  LFX_CUDA_TRY(cudaMemcpyAsync(lo.data(), s->vals_lo.p, sizeof(float) * n, cudaMemcpyDeviceToHost, s->stream));
  LFX_CUDA_TRY(cudaStreamSynchronize(s->stream));
  for (size_t i = 0; i < n; ++i) h[i] = (double)hi[i] + (double)lo[i];
  return LFX_OK;
}

// aSIMPLE set-up for the current matrix: the sub-blocks F, G, (D, C) stored apart in the
// smoother's storage type (FP64, FP32 or BF16), diagonals and eigenvalue bounds every step; the
// Schur AMG hierarchy (built from the FP64 matrix) on first use and then every amg_refresh steps.
template <class S, class T>
static lfx_status setup_asimple(lfx_state *s, ASimple<S, T> &pc) {
  lfx_problem *pb = s->pb;
  const lfx_options &o = pb->opt;
  const Mesh &m = pb->mesh->m;
  if (s->mixed())
    LFX_TRY(pc.setup_split(s->stream, s->view<float>(s->vals32), m.nnzb));   // from the high parts
  else
    LFX_TRY(pc.setup_split(s->stream, s->view64(), m.nnzb));
  if (o.s_smoother != LFX_SMOOTH_AMG) return LFX_OK;
  if (pc.amg_ready && !(o.amg_refresh > 0 && s->amg_age >= o.amg_refresh)) {
    ++s->amg_age;
    return LFX_OK;
  }
  std::vector<double> h;
  LFX_TRY(download_matrix(s, h));
  CsrHost S0 = schur_explicit(m.V, m.row_ptr, m.col_idx, m.diag_idx, h.data());
  AmgParams prm;
  prm.coarse_size = o.amg_coarse_size;
  prm.theta = o.amg_theta;
  AmgHost H;
  LFX_TRY(amg_setup_host(std::move(S0), m.row_ptr, m.col_idx, prm, H));
  pc.amg_alpha = o.amg_alpha;
  LFX_TRY(pc.upload_amg(H));
  s->amg_age = 1;
  return LFX_OK;
}

// Arnoldi steps the host reads a Krylov solve's stop flag behind its launches (the FP64 solve and
// the inner solves of the mixed one): one step queued ahead keeps the device busy, and after
// convergence only one step of launches returns at once (two cost 0.18 ms per 1M-tet step)
constexpr int kInnerLag = 1;

static lfx_status prepare_precond(lfx_state *s) {
  const lfx_options &o = s->pb->opt;
  const Mesh &m = s->pb->mesh->m;
  (void)m;
  if (o.precision != LFX_PREC_MIXED) return setup_asimple(s, s->pc64);
  // the inner Krylov solve's FP32 operator is the high part of the double-float matrix
  if (o.smoother_bf16) return setup_asimple(s, s->pcbf);
  return setup_asimple(s, s->pc32);
}

// The configured Krylov solve of the assembled system (rhs -> x, x holds the initial guess).
static lfx_status run_solve(lfx_state *s, double *x, bool x_zero, int *its, int *outer, double *rel) {
  const lfx_options &o = s->pb->opt;
  cudaStream_t st = s->stream;
  const BsrView<double> A = s->view64();
  *outer = 0;
  if (o.precision != LFX_PREC_MIXED) {
    auto pc = [s, A](cudaStream_t q, const double *v, double *z, const KState *ks) {
      return s->pc64.apply(q, A, v, z, ks);
    };
    return s->gm64.solve(st, A, pc, s->rhs.as<double>(), x, o.gmres_rtol, o.gmres_max_iters,
                         o.reorthogonalize != 0, kInnerLag, x_zero, its, rel);
  }
  // outer flexible GMRES with FP64 vectors on the double-float operator; each preconditioner
  // application is an FP32 GMRES solve (to inner_rtol) with the FP32/BF16 aSIMPLE
  const int64_t n = 4 * s->pb->mesh->m.V;
  const BsrView<float> A32 = s->view<float>(s->vals32);
  s->inner_total = 0;
  const bool adaptive = o.inner_adaptive != 0;
  // single systems: the inner solves run without host round trips (tolerance from the outer's
  // status on the device, step counts read back after the outer solve)
  const bool async_inner = !s->gm32.segmented() && o.inner_max_iters <= s->gm32.restart;
  if (async_inner && s->inner_cap < o.outer_max_iters + 2) {
    if (s->inner_its) cudaFreeHost(s->inner_its);
    s->inner_its = nullptr;
    s->inner_cap = 0;
    LFX_CUDA_TRY(cudaMallocHost(&s->inner_its, sizeof(int) * (size_t)(o.outer_max_iters + 2)));
    s->inner_cap = o.outer_max_iters + 2;
  }
  s->n_inner = 0;
  auto inner = [s, A32, n, &o, adaptive, async_inner](cudaStream_t q, const double *v, double *z,
                                                      const KState *ks) -> lfx_status {
    LFX_TRY((launch_convert<double, float>(q, v, s->r32.as<float>(), n, ks)));
    if (async_inner) {
      int *slot = s->inner_its + std::min(s->n_inner, s->inner_cap - 1);
      *slot = 0;
      ++s->n_inner;
      lfx_status rc;
      if (o.smoother_bf16) {
        const BsrView<__nv_bfloat16> Ab = s->view<__nv_bfloat16>(s->nopat);
        auto pc = [s, Ab](cudaStream_t qq, const float *vv, float *zz, const KState *kk) {
          return s->pcbf.apply(qq, Ab, vv, zz, kk);
        };
        rc = s->gm32.solve_inner(q, A32, pc, s->r32.as<float>(), s->z32.as<float>(), o.inner_rtol,
                                 adaptive ? ks : nullptr, o.inner_rtol, 0.1, o.inner_max_iters,
                                 o.reorthogonalize == 2, kInnerLag, slot);
      } else {
        auto pc = [s, A32](cudaStream_t qq, const float *vv, float *zz, const KState *kk) {
          return s->pc32.apply(qq, A32, vv, zz, kk);
        };
        rc = s->gm32.solve_inner(q, A32, pc, s->r32.as<float>(), s->z32.as<float>(), o.inner_rtol,
                                 adaptive ? ks : nullptr, o.inner_rtol, 0.1, o.inner_max_iters,
                                 o.reorthogonalize == 2, kInnerLag, slot);
      }
      LFX_TRY(rc);
      return launch_convert<float, double>(q, s->z32.as<float>(), z, n, ks);
    }
    int it = 0;
    double r = 0.0;
    lfx_status rc;
    double eta = o.inner_rtol;
    if (adaptive) LFX_TRY(s->gmdd.inner_tolerance(q, o.inner_rtol, 0.1, &eta));
    if (o.smoother_bf16) {
      const BsrView<__nv_bfloat16> Ab = s->view<__nv_bfloat16>(s->nopat);
      auto pc = [s, Ab](cudaStream_t qq, const float *vv, float *zz, const KState *kk) {
        return s->pcbf.apply(qq, Ab, vv, zz, kk);
      };
      rc = s->gm32.solve(q, A32, pc, s->r32.as<float>(), s->z32.as<float>(), eta, o.inner_max_iters,
                         o.reorthogonalize == 2, kInnerLag, true, &it, &r);
    } else {
      auto pc = [s, A32](cudaStream_t qq, const float *vv, float *zz, const KState *kk) {
        return s->pc32.apply(qq, A32, vv, zz, kk);
      };
      rc = s->gm32.solve(q, A32, pc, s->r32.as<float>(), s->z32.as<float>(), eta, o.inner_max_iters,
                         o.reorthogonalize == 2, kInnerLag, true, &it, &r);
    }
    s->inner_total += it;
    if (rc != LFX_OK && rc != LFX_ERR_NOT_CONVERGED) return rc;
    clear_error();
    return launch_convert<float, double>(q, s->z32.as<float>(), z, n, ks);
  };
  lfx_status rc = s->gmdd.solve(st, s->view_dd(), inner, s->rhs.as<double>(), x, o.gmres_rtol, o.outer_max_iters,
                                o.reorthogonalize != 0, 0, x_zero, outer, rel);
  if (async_inner) {
    // the outer solve ended on a stream synchronisation, after every inner count was copied
    for (int i = 0; i < std::min(s->n_inner, s->inner_cap); ++i) s->inner_total += s->inner_its[i];
  }
  *its = s->inner_total;
  return rc;
}

// ALE before a step: the lifting of the prescribed displacements (CG from d^n), the moved
// coordinates x^ + d^{n+1} and their element geometry, and u_ALE (Section 2.3).
static lfx_status ale_prepare(lfx_state *s) {
  lfx_problem *pb = s->pb;
  const Mesh &m = pb->mesh->m;
  cudaStream_t st = s->stream;
  const int64_t V = m.V;
  if (!s->have_bnd) {
    set_error("lfx_step: a moving-mesh state needs lfx_set_boundary_displacement before every step");
    return LFX_ERR_INVALID_ARG;
  }
  LFX_CUDA_TRY(cudaMemcpyAsync(s->dnew.p, s->dlevel(0), sizeof(D4) * (size_t)V, cudaMemcpyDeviceToDevice, st));
  const LiftingView L{V, m.d_rowptr.as<int32_t>(), m.d_col.as<int32_t>(), s->lapK.as<double>(), s->lapDinv.as<double>(),
                      s->lapFixed.as<uint8_t>(), s->lapR.as<D4>(), s->lapZ.as<D4>(), s->lapP.as<D4>(),
                      s->lapAp.as<D4>(), s->lapPart.as<double>(), s->lapCg.p};
  LFX_TRY(lifting_solve(st, L, s->n_bnd, s->bnd_node.as<int32_t>(), s->bnd_val.as<D4>(), s->dnew.as<D4>(), 1e-12,
                        20000, &s->lifting_iters));
  const bool mixed = s->mixed();
  LFX_TRY(launch_move_nodes(st, V, m.d_xyz.as<D4>(), s->dnew.as<D4>(), s->xyz.as<D4>(),
                            mixed ? s->xyz_hi.as<float4>() : nullptr, mixed ? s->xyz_lo.as<float4>() : nullptr));
  AssembleArgs G{};
  G.conn = m.d_conn.as<int4>();
  G.xyz = s->xyz.as<D4>();
  G.xyz_hi = s->xyz_hi.as<float4>();
  G.xyz_lo = s->xyz_lo.as<float4>();
  G.n_nodes = V;
  G.n_elems = m.T;
  if (mixed) {
    G.bad = pb->n_bad > 0 ? pb->d_bad.as<uint8_t>() : nullptr;
    LFX_TRY(launch_geometry<dd>(st, G, m.T, nullptr, s->geo_hi.as<float>(), s->geo_lo.as<float>()));
  } else {
    LFX_TRY(launch_geometry<double>(st, G, m.T, s->geo64.as<double>(), nullptr, nullptr));
  }
  const int sg = s->sigma;
  LFX_TRY(launch_mesh_velocity(st, V, sg, s->dnew.as<D4>(), s->dlevel(0), sg > 1 ? s->dlevel(1) : nullptr,
                               sg > 2 ? s->dlevel(2) : nullptr, pb->P.alpha, pb->beta, pb->P.dt, s->uale.as<D4>()));
  return LFX_OK;
}

// ||v|| (n values) on the device, read back (synchronises the stream)
static lfx_status device_norm(lfx_state *s, const double *v, int64_t n, double *out) {
  const int64_t V = s->pb->mesh->m.V;
  const size_t cap = sizeof(double) * (size_t)norm_partials_capacity(V);
  if (s->npart.bytes < cap) LFX_TRY(s->npart.alloc(cap));
  int ng = 0;
  LFX_TRY(launch_norm_partials(s->stream, v, n, s->npart.as<double>(), &ng));
  std::vector<double> h(ng);
  LFX_CUDA_TRY(cudaMemcpyAsync(h.data(), s->npart.p, sizeof(double) * ng, cudaMemcpyDeviceToHost, s->stream));
  LFX_CUDA_TRY(cudaStreamSynchronize(s->stream));
  double a = 0.0;
  for (double x : h) a += x;
  *out = std::sqrt(a);
  return LFX_OK;
}

// ||rhs - J U|| for the assembled Newton system and the iterate in xsol (read back)
static lfx_status newton_residual_norm(lfx_state *s, double *out) {
  const int64_t V = s->pb->mesh->m.V;
  if (s->fres.bytes < sizeof(D4) * (size_t)V) LFX_TRY(s->fres.alloc(sizeof(D4) * (size_t)V));
  const size_t cap = sizeof(double) * (size_t)norm_partials_capacity(V);
  if (s->npart.bytes < cap) LFX_TRY(s->npart.alloc(cap));
  int ng = 0;
  if (s->mixed())
    LFX_TRY((launch_spmv<DDMat, double>(s->stream, s->view_dd(), s->xsol.as<double>(), s->rhs.as<double>(),
                                        s->fres.as<double>(), 1, s->npart.as<double>(), &ng)));
  else
    LFX_TRY((launch_spmv<double, double>(s->stream, s->view64(), s->xsol.as<double>(), s->rhs.as<double>(),
                                         s->fres.as<double>(), 1, s->npart.as<double>(), &ng)));
  std::vector<double> h(ng);
  LFX_CUDA_TRY(cudaMemcpyAsync(h.data(), s->npart.p, sizeof(double) * ng, cudaMemcpyDeviceToHost, s->stream));
  LFX_CUDA_TRY(cudaStreamSynchronize(s->stream));
  double a = 0.0;
  for (double x : h) a += x;
  *out = std::sqrt(a);
  return LFX_OK;
}

// Newton iterations of the fully implicit formulation (Section 2.4) from the semi-implicit solution
// in xsol: stop once ||R(U_k)|| <= newton_rtol * scale, else assemble J(U_k) and b + X U_k and solve
// J U_{k+1} = b + X U_k from U_k.
static lfx_status newton_loop(lfx_state *s, double scale, int *n_newton, int *its, int *outer, double *rel,
                              float *ms_asm) {
  const lfx_options &o = s->pb->opt;
  s->newton_res.clear();
  *n_newton = 0;
  *ms_asm = 0.0f;
  lfx_status status = LFX_OK;
  for (int k = 0;; ++k) {
    // R(U_k) = A(U_k) U_k - b(U_k) from the semi-implicit system at the iterate (the chunked
    // launches); the Newton system is assembled only when an update follows
    LFX_TRY(assemble_system(s, true, false, true));
    double fn = 0.0;
    LFX_TRY(newton_residual_norm(s, &fn));
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, s->ea0, s->ea1) == cudaSuccess) *ms_asm += ms;
    s->newton_res.push_back(scale > 0.0 ? fn / scale : fn);
    if (!std::isfinite(fn)) {
      set_error("Newton: non-finite residual at iteration %d", k);
      return LFX_ERR_NONFINITE;
    }
    if (fn <= o.newton_rtol * scale) break;
    if (k >= o.newton_max_iters) {
      set_error("Newton: not converged after %d iterations (relative residual %.3e)", k, fn / scale);
      status = LFX_ERR_NOT_CONVERGED;
      break;
    }
    LFX_TRY(assemble_system(s, true, true));
    LFX_TRY(prepare_precond(s));
    int it = 0, ou = 0;
    double r = 0.0;
    lfx_status rc = run_solve(s, s->xsol.as<double>(), false, &it, &ou, &r);
    if (rc != LFX_OK && rc != LFX_ERR_NOT_CONVERGED) return rc;
    // the Newton assembly's time (its events are reused by the next assembly)
    if (cudaEventSynchronize(s->ea1) == cudaSuccess && cudaEventElapsedTime(&ms, s->ea0, s->ea1) == cudaSuccess)
      *ms_asm += ms;
    *its += it;
    *outer += ou;
    *rel = r;
    ++*n_newton;
  }
  return status;
}

extern "C" {

lfx_status lfx_state_newton_residuals(const lfx_state *s, double *res, int32_t capacity, int32_t *n) {
  if (!s || !n || capacity < 0 || (capacity > 0 && !res)) {
    set_error("lfx_state_newton_residuals: invalid argument");
    return LFX_ERR_INVALID_ARG;
  }
  *n = (int32_t)s->newton_res.size();
  for (int32_t k = 0; k < *n && k < capacity; ++k) res[k] = s->newton_res[k];
  return LFX_OK;
}

lfx_status lfx_state_set_displacement(lfx_state *s, const double *d_hist) {
  clear_error();
  if (!s || !d_hist) {
    set_error("lfx_state_set_displacement: NULL argument");
    return LFX_ERR_INVALID_ARG;
  }
  lfx_problem *pb = s->pb;
  const Mesh &m = pb->mesh->m;
  for (size_t b = 0; b < pb->bcs.size(); ++b) {
    const lfx_bc &bc = pb->bcs[b];
    if (bc.kind == LFX_BC_DIRICHLET || bc.kind == LFX_BC_RESISTANCE || (bc.kind == LFX_BC_NEUMANN && bc.beta > 0.0)) {
      set_error("lfx_state_set_displacement: on a moving mesh the boundary conditions must be NOSLIP, NODAL or "
                "NEUMANN without backflow stabilisation (boundary condition %d)", (int)b);
      return LFX_ERR_INVALID_ARG;
    }
  }
  if (m.n_comp > 1) {
    set_error("lfx_state_set_displacement: moving meshes of several pieces are not supported");
    return LFX_ERR_INVALID_ARG;
  }
  const int64_t V = m.V;
  cudaStream_t st = s->stream;
  if (!s->ale) {
    const size_t v4 = sizeof(D4) * (size_t)V;
    for (int l = 0; l < s->sigma; ++l) LFX_TRY(s->dhist[l].alloc(v4));
    DBuf *b4[] = {&s->dnew, &s->uale, &s->xyz, &s->lapR, &s->lapZ, &s->lapP, &s->lapAp};
    for (DBuf *b : b4) LFX_TRY(b->alloc(v4));
    const size_t nv = (size_t)kGeoValues * (size_t)std::max<int64_t>(m.T, 1);
    if (s->mixed()) {
      LFX_TRY(s->xyz_hi.alloc(sizeof(float4) * (size_t)V));
      LFX_TRY(s->xyz_lo.alloc(sizeof(float4) * (size_t)V));
      LFX_TRY(s->geo_hi.alloc(sizeof(float) * nv));
      LFX_TRY(s->geo_lo.alloc(sizeof(float) * nv));
    } else {
      LFX_TRY(s->geo64.alloc(sizeof(double) * nv));
    }
    LFX_TRY(s->lapK.alloc(sizeof(double) * (size_t)m.nnzb));
    LFX_TRY(s->lapDinv.alloc(sizeof(double) * (size_t)V));
    LFX_TRY(s->lapFixed.alloc((size_t)V));
    LFX_TRY(s->lapPart.alloc(sizeof(double) * (size_t)lifting_part_entries(V)));
    LFX_TRY(s->lapCg.alloc(lifting_cg_state_bytes()));
    LFX_TRY(launch_lifting_matrix(st, m.T, V, m.nnzb, m.d_slot.as<int32_t>(), m.d_diag.as<int32_t>(),
                                  pb->geo64.as<double>(), pb->geo_hi.as<float>(), pb->geo_lo.as<float>(),
                                  s->lapK.as<double>(), s->lapDinv.as<double>()));
  }
  // the levels in the caller's layout [sigma][V][3], scattered to the internal order (w = 0)
  const size_t nu = sizeof(double) * 3 * (size_t)V * s->sigma;
  if (s->io_u.bytes < nu) LFX_TRY(s->io_u.alloc(nu));
  if (s->io_p.bytes < sizeof(double) * (size_t)V) LFX_TRY(s->io_p.alloc(sizeof(double) * (size_t)V));
  LFX_CUDA_TRY(cudaMemcpyAsync(s->io_u.p, d_hist, nu, cudaMemcpyHostToDevice, st));
  LFX_CUDA_TRY(cudaMemsetAsync(s->io_p.p, 0, sizeof(double) * (size_t)V, st));
  s->dhead = 0;
  for (int l = 0; l < s->sigma; ++l)
    LFX_TRY(launch_node_scatter(st, V, m.d_node_old.as<int32_t>(), s->io_u.as<double>() + (size_t)l * 3 * V,
                                s->io_p.as<double>(), s->dhist[l].as<D4>()));
  LFX_CUDA_TRY(cudaStreamSynchronize(st));
  s->ale = true;
  s->have_bnd = false;
  s->assembled = false;
  return LFX_OK;
}

lfx_status lfx_set_boundary_displacement(lfx_state *s, int64_t n, const int32_t *nodes, const double *d) {
  clear_error();
  if (!s || n < 0 || (n > 0 && (!nodes || !d))) {
    set_error("lfx_set_boundary_displacement: invalid argument");
    return LFX_ERR_INVALID_ARG;
  }
  if (!s->ale) {
    set_error("lfx_set_boundary_displacement: call lfx_state_set_displacement first");
    return LFX_ERR_INVALID_ARG;
  }
  const Mesh &m = s->pb->mesh->m;
  std::vector<int32_t> in((size_t)std::max<int64_t>(n, 1));
  std::vector<D4> val((size_t)std::max<int64_t>(n, 1));
  for (int64_t k = 0; k < n; ++k) {
    if (nodes[k] < 0 || nodes[k] >= m.V) {
      set_error("lfx_set_boundary_displacement: node %d out of range", nodes[k]);
      return LFX_ERR_INVALID_ARG;
    }
    in[k] = m.node_new[nodes[k]];
    val[k] = D4{d[3 * k], d[3 * k + 1], d[3 * k + 2], 0.0};
  }
  if (s->bnd_node.bytes < sizeof(int32_t) * in.size()) LFX_TRY(s->bnd_node.alloc(sizeof(int32_t) * in.size()));
  if (s->bnd_val.bytes < sizeof(D4) * val.size()) LFX_TRY(s->bnd_val.alloc(sizeof(D4) * val.size()));
  LFX_CUDA_TRY(cudaMemcpyAsync(s->bnd_node.p, in.data(), sizeof(int32_t) * in.size(), cudaMemcpyHostToDevice, s->stream));
  LFX_CUDA_TRY(cudaMemcpyAsync(s->bnd_val.p, val.data(), sizeof(D4) * val.size(), cudaMemcpyHostToDevice, s->stream));
  LFX_CUDA_TRY(cudaStreamSynchronize(s->stream));
  s->n_bnd = n;
  s->have_bnd = true;
  return LFX_OK;
}

lfx_status lfx_state_get_displacement(const lfx_state *s, double *d, int32_t *lifting_iterations) {
  clear_error();
  if (!s || !d) {
    set_error("lfx_state_get_displacement: NULL argument");
    return LFX_ERR_INVALID_ARG;
  }
  if (!s->ale) {
    set_error("lfx_state_get_displacement: not a moving-mesh state");
    return LFX_ERR_INVALID_ARG;
  }
  const Mesh &m = s->pb->mesh->m;
  const int64_t V = m.V;
  if (s->io_u.bytes < sizeof(double) * 3 * (size_t)V) LFX_TRY(s->io_u.alloc(sizeof(double) * 3 * (size_t)V));
  if (s->io_p.bytes < sizeof(double) * (size_t)V) LFX_TRY(s->io_p.alloc(sizeof(double) * (size_t)V));
  lfx_state *sm = const_cast<lfx_state *>(s);
  LFX_TRY(launch_node_gather(s->stream, V, m.d_node_old.as<int32_t>(), sm->dlevel(0), s->io_u.as<double>(),
                             s->io_p.as<double>()));
  LFX_CUDA_TRY(cudaMemcpyAsync(d, s->io_u.p, sizeof(double) * 3 * (size_t)V, cudaMemcpyDeviceToHost, s->stream));
  LFX_CUDA_TRY(cudaStreamSynchronize(s->stream));
  if (lifting_iterations) *lifting_iterations = s->lifting_iters;
  return LFX_OK;
}

lfx_status lfx_step(lfx_state *s, lfx_step_stats *stats) {
  clear_error();
  if (!s) {
    set_error("lfx_step: NULL state");
    return LFX_ERR_INVALID_ARG;
  }
  lfx_problem *pb = s->pb;
  const lfx_options &o = pb->opt;
  cudaStream_t st = s->stream;
  LFX_CUDA_TRY(cudaEventRecord(s->e0, st));
  if (s->ale) LFX_TRY(ale_prepare(s));
  LFX_TRY(assemble_system(s, true));
  LFX_CUDA_TRY(cudaEventRecord(s->e1, st));
  double scale = 0.0;
  if (o.implicit) LFX_TRY(device_norm(s, s->rhs.as<double>(), 4 * pb->mesh->m.V, &scale));
  LFX_TRY(prepare_precond(s));
  int its = 0, outer = 0;
  double rel = 0.0;
  s->gm64.n_tev = s->gm64.n_spmv_calls = 0;
  s->gm32.n_tev = s->gm32.n_spmv_calls = 0;
  s->gmdd.n_tev = s->gmdd.n_spmv_calls = 0;
  s->pc64.n_fev = 0;
  s->pc32.n_fev = 0;
  s->pcbf.n_fev = 0;
  lfx_status rc = run_solve(s, s->xsol.as<double>(), false, &its, &outer, &rel);
  if (rc != LFX_OK && rc != LFX_ERR_NOT_CONVERGED) return rc;
  int n_newton = 0;
  float ms_newton = 0.0f, ms_asm_semi = 0.0f;
  if (o.implicit) {
    LFX_CUDA_TRY(cudaEventSynchronize(s->ea1));
    cudaEventElapsedTime(&ms_asm_semi, s->ea0, s->ea1);
    lfx_status rn = newton_loop(s, scale, &n_newton, &its, &outer, &rel, &ms_newton);
    if (rn != LFX_OK && rn != LFX_ERR_NOT_CONVERGED) return rn;
    if (rn == LFX_ERR_NOT_CONVERGED) rc = rn;
  } else {
    s->newton_res.clear();
  }
  if (s->mixed() && o.smoother_bf16) LFX_TRY(s->pcbf.queue_bulk_check(st));
  LFX_CUDA_TRY(cudaEventRecord(s->e2, st));
  LFX_CUDA_TRY(cudaEventSynchronize(s->e2));
  s->assembled = false;
  // a bounded wait that gave up leaves the state as it was: the history is not shifted, and a
  // repeated step assembles anew from it (the extrapolation is rewritten at every assembly)
  if (s->asm_err_host && *s->asm_err_host) {
    *s->asm_err_host = 0;
    set_error("lfx_step: a grid-wide wait of the persistent assembly gave up; the state was not advanced");
    return LFX_ERR_TIMEOUT;
  }
  if (s->pcbf.bulk_failed()) {
    set_error("lfx_step: a wait for a staged tile of the velocity smoothing pass gave up; the state was not "
              "advanced");
    return LFX_ERR_TIMEOUT;
  }
  // history shift: the solution becomes level 0 (and d^{n+1} the displacement's level 0)
  const int oldest = (s->head + s->sigma - 1) % s->sigma;
  std::swap(s->hist[oldest].p, s->xsol.p);
  std::swap(s->hist[oldest].bytes, s->xsol.bytes);
  s->head = oldest;
  if (s->ale) {
    const int dold = (s->dhead + s->sigma - 1) % s->sigma;
    std::swap(s->dhist[dold], s->dnew);
    s->dhead = dold;
    s->have_bnd = false;
  }
  s->t += pb->P.dt;
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->iterations = its;
    stats->outer_iterations = outer;
    stats->rel_residual = rel;
    stats->t = s->t;
    cudaEventElapsedTime(&stats->ms_assembly, s->e0, s->e1);
    cudaEventElapsedTime(&stats->ms_solve, s->e1, s->e2);
    cudaEventElapsedTime(&stats->ms_total, s->e0, s->e2);
    if (o.implicit) stats->ms_assembly_kernels = ms_asm_semi;
    else cudaEventElapsedTime(&stats->ms_assembly_kernels, s->ea0, s->ea1);
    stats->n_assembly_launches = s->n_asm_launch;
    stats->newton_iterations = n_newton;
    stats->ms_newton_assembly = ms_newton;
    stats->assembly_mode = s->asm_mode_used;
    if (o.precision == LFX_PREC_MIXED) {
      if (o.smoother_bf16) s->pcbf.read_f_timing(&stats->ms_fpass_median, &stats->n_fpass);
      else s->pc32.read_f_timing(&stats->ms_fpass_median, &stats->n_fpass);
      s->gm32.read_spmv_timing(&stats->ms_spmv, &stats->n_spmv);
      int dummy = 0;
      float d2 = 0.0f;
      s->gmdd.read_spmv_timing(&d2, &dummy);
    } else {
      s->pc64.read_f_timing(&stats->ms_fpass_median, &stats->n_fpass);
      s->gm64.read_spmv_timing(&stats->ms_spmv, &stats->n_spmv);
    }
    stats->converged = rc == LFX_OK;
  }
  return rc;
}

lfx_status lfx_state_get(const lfx_state *s, double *u, double *p) {
  if (!s || !u || !p) {
    set_error("lfx_state_get: NULL argument");
    return LFX_ERR_INVALID_ARG;
  }
  // permuted to the caller's layout on the device, then copied straight into the caller's arrays
  const Mesh &m = s->pb->mesh->m;
  const int64_t V = m.V;
  if (s->io_u.bytes < sizeof(double) * 3 * (size_t)V) LFX_TRY(s->io_u.alloc(sizeof(double) * 3 * (size_t)V));
  if (s->io_p.bytes < sizeof(double) * (size_t)V) LFX_TRY(s->io_p.alloc(sizeof(double) * (size_t)V));
  LFX_TRY(launch_node_gather(s->stream, V, m.d_node_old.as<int32_t>(), s->hist[s->head].as<D4>(),
                             s->io_u.as<double>(), s->io_p.as<double>()));
  LFX_CUDA_TRY(cudaMemcpyAsync(u, s->io_u.p, sizeof(double) * 3 * (size_t)V, cudaMemcpyDeviceToHost, s->stream));
  LFX_CUDA_TRY(cudaMemcpyAsync(p, s->io_p.p, sizeof(double) * (size_t)V, cudaMemcpyDeviceToHost, s->stream));
  LFX_CUDA_TRY(cudaStreamSynchronize(s->stream));
  return LFX_OK;
}

// ------------------------------------------------------------------------------- debug API
static lfx_status vec_to_device(const Mesh &m, const double *x /*[V][4] caller*/, double *dst, cudaStream_t st) {
  std::vector<D4> h(m.V);
  for (int64_t i = 0; i < m.V; ++i) {
    const int64_t o = m.node_old[i];
    h[i] = D4{x[4 * o], x[4 * o + 1], x[4 * o + 2], x[4 * o + 3]};
  }
  LFX_CUDA_TRY(cudaMemcpyAsync(dst, h.data(), sizeof(D4) * m.V, cudaMemcpyHostToDevice, st));
  LFX_CUDA_TRY(cudaStreamSynchronize(st));
  return LFX_OK;
}
static lfx_status vec_to_host(const Mesh &m, const double *src, double *x, cudaStream_t st) {
  std::vector<D4> h(m.V);
  LFX_CUDA_TRY(cudaMemcpyAsync(h.data(), src, sizeof(D4) * m.V, cudaMemcpyDeviceToHost, st));
  LFX_CUDA_TRY(cudaStreamSynchronize(st));
  for (int64_t i = 0; i < m.V; ++i) {
    const int64_t o = m.node_old[i];
    x[4 * o] = h[i].x;
    x[4 * o + 1] = h[i].y;
    x[4 * o + 2] = h[i].z;
    x[4 * o + 3] = h[i].w;
  }
  return LFX_OK;
}

lfx_status lfx_debug_assemble(lfx_state *s, int32_t apply_bcs, double *blocks, double *rhs) {
  clear_error();
  if (!s || !blocks || !rhs) {
    set_error("lfx_debug_assemble: NULL argument");
    return LFX_ERR_INVALID_ARG;
  }
  const Mesh &m = s->pb->mesh->m;
  LFX_TRY(assemble_system(s, apply_bcs != 0));
  s->assembled = true;
  std::vector<double> v;
  LFX_TRY(download_matrix(s, v));
  LFX_TRY(vec_to_host(m, s->rhs.as<double>(), rhs, s->stream));
  std::vector<int64_t> rp, ib;
  std::vector<int32_t> ci;
  user_pattern(m, rp, ci, ib);
  for (int64_t q = 0; q < m.nnzb; ++q) memcpy(blocks + 16 * q, v.data() + 16 * ib[q], 16 * sizeof(double));
  return LFX_OK;
}

lfx_status lfx_debug_assemble_newton(lfx_state *s, const double *U, double *blocks, double *rhs) {
  clear_error();
  if (!s || !U || !blocks || !rhs) {
    set_error("lfx_debug_assemble_newton: NULL argument");
    return LFX_ERR_INVALID_ARG;
  }
  const Mesh &m = s->pb->mesh->m;
  LFX_TRY(assemble_system(s, false));          // the step's BDF fields (u^BDF)
  LFX_TRY(vec_to_device(m, U, s->xsol.as<double>(), s->stream));
  LFX_TRY(assemble_system(s, false, true));
  s->assembled = false;
  std::vector<double> v;
  LFX_TRY(download_matrix(s, v));
  LFX_TRY(vec_to_host(m, s->rhs.as<double>(), rhs, s->stream));
  std::vector<int64_t> rp, ib;
  std::vector<int32_t> ci;
  user_pattern(m, rp, ci, ib);
  for (int64_t q = 0; q < m.nnzb; ++q) memcpy(blocks + 16 * q, v.data() + 16 * ib[q], 16 * sizeof(double));
  return LFX_OK;
}

lfx_status lfx_debug_persistent_timeout(lfx_state *s) {
  clear_error();
  if (!s) {
    set_error("lfx_debug_persistent_timeout: NULL state");
    return LFX_ERR_INVALID_ARG;
  }
  lfx_problem *pb = s->pb;
  int mode = 0;
  {
    std::lock_guard<std::mutex> lk(pb->tune_mu);
    mode = pb->asm_mode;
  }
  if (mode != LFX_ASM_PERSISTENT) {
    set_error("lfx_debug_persistent_timeout: the problem's assembly is not the persistent launch");
    return LFX_ERR_INVALID_ARG;
  }
  s->force_timeout = true;
  lfx_status rc = assemble_system(s, true);
  s->force_timeout = false;
  LFX_TRY(rc);
  LFX_CUDA_TRY(cudaStreamSynchronize(s->stream));
  s->assembled = false;
  if (s->asm_err_host && *s->asm_err_host) {
    *s->asm_err_host = 0;
    set_error("persistent assembly: a grid-wide wait gave up");
    return LFX_ERR_TIMEOUT;
  }
  return LFX_OK;
}

lfx_status lfx_debug_staged_timeout(lfx_state *s) {
  clear_error();
  if (!s || !s->mixed() || !s->pb->opt.smoother_bf16 || s->pcbf.n_ftile <= 0) {
    set_error("lfx_debug_staged_timeout: needs a mixed-precision state with the staged BF16 smoothing pass");
    return LFX_ERR_INVALID_ARG;
  }
  cudaStream_t st = s->stream;
  LFX_TRY(assemble_system(s, true));
  LFX_TRY(prepare_precond(s));
  const BsrView<__nv_bfloat16> Ab = s->view<__nv_bfloat16>(s->nopat);
  LFX_CUDA_TRY(cudaMemsetAsync(s->r32.p, 0, s->r32.bytes, st));
  s->pcbf.force_bulk_timeout = true;
  lfx_status rc = s->pcbf.apply(st, Ab, s->r32.as<float>(), s->z32.as<float>(), nullptr);
  s->pcbf.force_bulk_timeout = false;
  LFX_TRY(rc);
  LFX_TRY(s->pcbf.queue_bulk_check(st));
  LFX_CUDA_TRY(cudaStreamSynchronize(st));
  s->assembled = false;
  if (s->pcbf.bulk_failed()) {
    set_error("staged velocity smoothing pass: a wait for a tile gave up");
    return LFX_ERR_TIMEOUT;
  }
  return LFX_OK;
}

lfx_status lfx_debug_spmv(lfx_state *s, const double *x, double *y) {
  clear_error();
  if (!s || !x || !y || !s->assembled) {
    set_error("lfx_debug_spmv: NULL argument or no assembled matrix");
    return LFX_ERR_INVALID_ARG;
  }
  const Mesh &m = s->pb->mesh->m;
  DBuf dx, dy;
  LFX_TRY(dx.alloc(sizeof(D4) * m.V));
  LFX_TRY(dy.alloc(sizeof(D4) * m.V));
  LFX_TRY(vec_to_device(m, x, dx.as<double>(), s->stream));
  if (s->mixed())
    LFX_TRY((launch_spmv<DDMat, double>(s->stream, s->view_dd(), dx.as<double>(), nullptr, dy.as<double>(), 0,
                                        nullptr, nullptr)));
  else
    LFX_TRY((launch_spmv<double, double>(s->stream, s->view64(), dx.as<double>(), nullptr, dy.as<double>(), 0,
                                         nullptr, nullptr)));
  return vec_to_host(m, dy.as<double>(), y, s->stream);
}

lfx_status lfx_debug_precond(lfx_state *s, const double *r, double *z, double *lam_f, double *lam_s) {
  clear_error();
  if (!s || !r || !z || !s->assembled) {
    set_error("lfx_debug_precond: NULL argument or no assembled matrix");
    return LFX_ERR_INVALID_ARG;
  }
  const Mesh &m = s->pb->mesh->m;
  DBuf dr, dz;
  LFX_TRY(dr.alloc(sizeof(D4) * m.V));
  LFX_TRY(dz.alloc(sizeof(D4) * m.V));
  LFX_TRY(vec_to_device(m, r, dr.as<double>(), s->stream));
  if (s->pb->opt.precision != LFX_PREC_FP64) {
    set_error("lfx_debug_precond: available for the FP64 path only");
    return LFX_ERR_INVALID_ARG;
  }
  const BsrView<double> A = s->view64();
  LFX_TRY(prepare_precond(s));
  LFX_TRY(s->pc64.apply(s->stream, A, dr.as<double>(), dz.as<double>(), nullptr));
  LFX_TRY(vec_to_host(m, dz.as<double>(), z, s->stream));
  return s->pc64.lambdas(lam_f, lam_s);
}

lfx_status lfx_debug_amg_level(lfx_state *s, int32_t level, int64_t sizes[4], int32_t *a_rp, int32_t *a_ci,
                               double *a_v, int32_t *p_rp, int32_t *p_ci, double *p_v, double *lam) {
  clear_error();
  if (!s || !sizes || s->mixed() || !s->pc64.amg_ready || level < 0 || level >= (int)s->pc64.amg.size()) {
    set_error("lfx_debug_amg_level: needs the FP64 path with a built Schur AMG hierarchy and a level in range");
    return LFX_ERR_INVALID_ARG;
  }
  const AmgDevLevel &D = s->pc64.amg[level];
  const bool has_a = level >= 1 && D.rp.p != nullptr, has_p = D.Prp.p != nullptr;
  const int64_t nnz_a = has_a ? (int64_t)(D.v.bytes / sizeof(double)) : 0;
  const int64_t nnz_p = has_p ? (int64_t)(D.Pv.bytes / sizeof(double)) : 0;
  sizes[0] = D.n;
  sizes[1] = nnz_a;
  sizes[2] = has_p ? D.nnext : 0;
  sizes[3] = nnz_p;
  if (lam) *lam = D.lam;
  auto get = [&](void *dst, const DBuf &src, size_t bytes) -> lfx_status {
    if (dst && bytes) LFX_CUDA_TRY(cudaMemcpy(dst, src.p, bytes, cudaMemcpyDeviceToHost));
    return LFX_OK;
  };
  if (has_a) {
    LFX_TRY(get(a_rp, D.rp, sizeof(int32_t) * (size_t)(D.n + 1)));
    LFX_TRY(get(a_ci, D.ci, sizeof(int32_t) * (size_t)nnz_a));
    LFX_TRY(get(a_v, D.v, sizeof(double) * (size_t)nnz_a));
  }
  if (has_p) {
    LFX_TRY(get(p_rp, D.Prp, sizeof(int32_t) * (size_t)(D.n + 1)));
    LFX_TRY(get(p_ci, D.Pci, sizeof(int32_t) * (size_t)nnz_p));
    LFX_TRY(get(p_v, D.Pv, sizeof(double) * (size_t)nnz_p));
  }
  return LFX_OK;
}

lfx_status lfx_debug_amg_host(int64_t n, const int32_t *row_ptr, const int32_t *col_idx, const int32_t *diag_idx,
                              const double *blocks, const lfx_options *opt, int32_t level, int64_t sizes[5],
                              int32_t *a_rp, int32_t *a_ci, double *a_v, int32_t *p_rp, int32_t *p_ci, double *p_v,
                              double *lam, double *coarse_inv) {
  clear_error();
  if (n < 1 || n >= INT32_MAX || !row_ptr || !col_idx || !diag_idx || !blocks || !sizes || level < 0 ||
      row_ptr[0] != 0) {
    set_error("lfx_debug_amg_host: invalid argument");
    return LFX_ERR_INVALID_ARG;
  }
  for (int64_t i = 0; i < n; ++i)
    if (row_ptr[i + 1] < row_ptr[i]) {
      set_error("lfx_debug_amg_host: row_ptr decreases at row %lld", (long long)i);
      return LFX_ERR_INVALID_ARG;
    }
  const int64_t nnz = row_ptr[n];
  for (int64_t k = 0; k < nnz; ++k)
    if (col_idx[k] < 0 || col_idx[k] >= n) {
      set_error("lfx_debug_amg_host: column index out of range at %lld", (long long)k);
      return LFX_ERR_INVALID_ARG;
    }
  for (int64_t i = 0; i < n; ++i)
    if (diag_idx[i] < row_ptr[i] || diag_idx[i] >= row_ptr[i + 1] || col_idx[diag_idx[i]] != i) {
      set_error("lfx_debug_amg_host: diag_idx[%lld] is not the position of block (i, i)", (long long)i);
      return LFX_ERR_INVALID_ARG;
    }
  lfx_options o;
  if (opt) o = *opt;
  else lfx_options_default(&o);
  if (o.amg_coarse_size < 1 || !(o.amg_theta >= 0.0)) {
    set_error("lfx_debug_amg_host: amg_coarse_size >= 1 and amg_theta >= 0 needed");
    return LFX_ERR_INVALID_ARG;
  }
  const std::vector<int32_t> rp(row_ptr, row_ptr + n + 1), ci(col_idx, col_idx + nnz), dg(diag_idx, diag_idx + n);
  CsrHost S0 = schur_explicit(n, rp, ci, dg, blocks);
  AmgParams prm;
  prm.coarse_size = o.amg_coarse_size;
  prm.theta = o.amg_theta;
  AmgHost H;
  LFX_TRY(amg_setup_host(std::move(S0), rp, ci, prm, H));
  const int levels = (int)H.A.size();
  if (level >= levels) {
    set_error("lfx_debug_amg_host: level %d beyond the last of %d", level, levels);
    return LFX_ERR_INVALID_ARG;
  }
  const CsrHost &A = H.A[level];
  const bool has_p = level + 1 < levels;
  sizes[0] = levels;
  sizes[1] = A.n;
  sizes[2] = (int64_t)A.v.size();
  sizes[3] = has_p ? H.P[level].m : 0;
  sizes[4] = has_p ? (int64_t)H.P[level].v.size() : 0;
  if (a_rp) std::copy(A.rp.begin(), A.rp.end(), a_rp);
  if (a_ci) std::copy(A.ci.begin(), A.ci.end(), a_ci);
  if (a_v) std::copy(A.v.begin(), A.v.end(), a_v);
  if (has_p) {
    const CsrHost &P = H.P[level];
    if (p_rp) std::copy(P.rp.begin(), P.rp.end(), p_rp);
    if (p_ci) std::copy(P.ci.begin(), P.ci.end(), p_ci);
    if (p_v) std::copy(P.v.begin(), P.v.end(), p_v);
  }
  if (lam) *lam = has_p ? H.lam[level] : 0.0;
  if (!has_p && coarse_inv) std::copy(H.coarse_inv.begin(), H.coarse_inv.end(), coarse_inv);
  return LFX_OK;
}

lfx_status lfx_debug_amg_vcycle(lfx_state *s, const double *b1, double *x1) {
  clear_error();
  if (!s || !b1 || !x1 || s->mixed() || !s->pc64.amg_ready || s->pc64.amg.size() < 3) {
    set_error("lfx_debug_amg_vcycle: needs the FP64 path with a built Schur AMG hierarchy of >= 3 levels");
    return LFX_ERR_INVALID_ARG;
  }
  ASimple<double, double> &pc = s->pc64;
  AmgDevLevel &L1 = pc.amg[1];
  LFX_CUDA_TRY(cudaMemcpyAsync(L1.b.p, b1, sizeof(double) * (size_t)L1.n, cudaMemcpyHostToDevice, s->stream));
  LFX_TRY(pc.coarse_cycle(s->stream, nullptr));
  LFX_CUDA_TRY(cudaMemcpyAsync(x1, pc.coarse_x(), sizeof(double) * (size_t)L1.n, cudaMemcpyDeviceToHost, s->stream));
  LFX_CUDA_TRY(cudaStreamSynchronize(s->stream));
  return LFX_OK;
}

lfx_status lfx_debug_solve(lfx_state *s, double *x, lfx_step_stats *stats) {
  clear_error();
  if (!s || !x || !s->assembled) {
    set_error("lfx_debug_solve: NULL argument or no assembled matrix");
    return LFX_ERR_INVALID_ARG;
  }
  const Mesh &m = s->pb->mesh->m;
  const lfx_options &o = s->pb->opt;
  DBuf dx;
  LFX_TRY(dx.alloc(sizeof(D4) * m.V));
  LFX_CUDA_TRY(cudaMemsetAsync(dx.p, 0, dx.bytes, s->stream));
  (void)o;
  LFX_TRY(prepare_precond(s));
  s->gm64.n_tev = 0;
  s->gm32.n_tev = 0;
  s->gmdd.n_tev = 0;
  int its = 0, outer = 0;
  double rel = 0;
  lfx_status rc = run_solve(s, dx.as<double>(), true, &its, &outer, &rel);
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->iterations = its;
    stats->outer_iterations = outer;
    stats->rel_residual = rel;
    stats->converged = rc == LFX_OK;
  }
  LFX_TRY(vec_to_host(m, dx.as<double>(), x, s->stream));
  return rc;
}

}  // extern "C"
