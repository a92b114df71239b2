// Kernel launchers shared across the CUDA translation units of liblfx.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dd.h"
#include "lfx_internal.h"

namespace lfx {

// 32-byte node records (x, y, z, w) and their FP32 counterpart
struct alignas(32) D4 {
  double x, y, z, w;
};
struct alignas(16) F4 {
  float x, y, z, w;
};

// ------------------------------------------------------------------ assembly
struct AssembleArgs {
  const int4 *conn;          // [T] internal numbering, colour-sorted
  const int32_t *slot;       // [T][16]
  const uint16_t *first;     // [T] bit 4a+b: this element writes block (a, b) first (null: add everywhere)
  const D4 *xyz;        // [V] (x, y, z, 0)
  const D4 *xext;       // [V] (u^EXT, p^EXT)
  const D4 *ubdf;       // [V] (u^BDF, 0)
  const double *phi_riis;    // [n_riis][V]
  const uint8_t *bad;        // [T] FP64 geometry flag (mixed assembly), may be null
  double *rhs;               // [V][4]
  int64_t n_nodes;
  int64_t n_elems;
  // double-float assembly only: inputs split into FP32 high and low parts (x = hi + lo), the
  // matrix accumulated as high parts (the vals argument) plus low parts, the rhs likewise
  const float4 *xyz_hi, *xyz_lo;
  const float4 *xext_hi, *xext_lo;
  const float4 *ubdf_hi, *ubdf_lo;
  float *vals_lo;            // [nnzb][16]
  float *rhs_hi, *rhs_lo;    // [V][4]
  // per-element geometry computed once (the mesh does not move): kGeoValues values per element,
  // structure of arrays [kGeoValues][T] (grad phi 12, G 9, 1/(g.g), |K|/4, G:G); FP64 kernel: geo64;
  // double-float kernel: geo_hi + geo_lo.  Null: the kernel computes the geometry itself.
  const double *geo64;
  const float *geo_hi, *geo_lo;
  // moving mesh: u_ALE at the nodes (the advection velocity is u* = u^EXT - u_ALE); null: fixed mesh
  const D4 *uale;
  // per-colour kernel: the elements of the colour ranges (internal ids); null: the ranges are ids
  const int32_t *elist;
};
// chunk tables of the chunked assembly (device copies of the Mesh vectors of the same names)
struct ChunkArgs {
  const int32_t *elem_off, *pass_off;
  const uint16_t *code;
  const int32_t *run_off, *ndiag;
  const uint16_t *meta;
  const int32_t *block, *node;
};
constexpr int kGeoValues = 24;

// Fills the geometry cache of the arithmetic type R (double: out64 [kGeoValues][T]; dd: out_hi,
// out_lo) for the T elements of A.conn.
template <class R>
lfx_status launch_geometry(cudaStream_t st, const AssembleArgs &A, int64_t T, double *out64, float *out_hi,
                           float *out_lo);

constexpr int kMaxDirCoef = 1024;   // n_bcs x (H + 1) boundary terms (an 8 KB kernel parameter)
struct DirCoef {
  double c[kMaxDirCoef];
};

// u^EXT / p^EXT and u^BDF at every node (Eq. bdf); when xe_hi is non-null also their
// double-float splits (hi + lo) for the double-float assembly.
lfx_status launch_bdf(cudaStream_t st, int64_t V, int order, const D4 *h0, const D4 *h1,
                      const D4 *h2, const double beta[3], const double gamma[3],
                      D4 *xext, D4 *ubdf, float4 *xe_hi = nullptr, float4 *xe_lo = nullptr,
                      float4 *ub_hi = nullptr, float4 *ub_lo = nullptr);
// rhs[i] = hi[i] + lo[i] (double-float right-hand side to FP64)
lfx_status launch_dd_combine(cudaStream_t st, int64_t n, const float *hi, const float *lo, double *out);
// Dirichlet row replacement and per-component row scaling on a double-float matrix (hi, lo)
lfx_status launch_apply_dirichlet_dd(cudaStream_t st, int64_t nd, const int32_t *dnode, const D4 *g,
                                     int32_t pin_node, double pin_value, const int32_t *rowptr,
                                     const int32_t *diag, float *hi, float *lo, double *rhs, double *x0);
lfx_status launch_comp_normalize_dd(cudaStream_t st, int64_t V, int n_comp, const int32_t *comp_off,
                                    double *scale, const int32_t *rowptr, float *hi, float *lo, double *rhs);
// Node fields between the caller's layout (u [V][3], p [V], caller node order) and the internal
// interleaved D4 [V] in internal order (node_old[i] = caller index of internal node i)
lfx_status launch_node_scatter(cudaStream_t st, int64_t V, const int32_t *node_old, const double *u, const double *p,
                               D4 *dst);
lfx_status launch_node_gather(cudaStream_t st, int64_t V, const int32_t *node_old, const D4 *src, double *u, double *p);
// Inertial backflow stabilisation (Section 2.2.2): for each face edge (i, j), at its midpoint
// c = -coef min(u^EXT . a, 0) / 3 (a = A_f n_f, weight A_f/3), times phi_a phi_b = 1/4, added to
// the velocity diagonal of blocks (i,i), (i,j), (j,i), (j,j) through FP64 accumulators; then into
// the FP64 matrix (vals64) or the double-float one (hi, lo).
lfx_status launch_backflow(cudaStream_t st, int64_t n_edges, const int32_t *ij, const double *an, const double *coef,
                           const int32_t *slot4, const D4 *xext, int64_t n_blocks, const int32_t *blk, double *acc,
                           double *vals64, float *hi, float *lo);
// newton: the Jacobian of the fully implicit formulation at the iterate held in A.xext (the
// semi-implicit system assembled there plus the Newton terms) and the right-hand side J U - R(U)
template <class R, class S>
lfx_status launch_assemble(cudaStream_t st, const AssembleArgs &A, const PhysParams &P,
                           const int32_t *color_off, int n_colors, S *vals, bool newton = false);
// the semi-implicit system (newton: the Newton system at the iterate) by chunks in ONE cooperative
// launch over every chunk colour, the colours separated by bounded grid-wide waits; *err (device)
// is set to 1 if a wait gave up.  d_chunk_color_off: device copy of the colour offsets; barrier: a
// device counter (zeroed here).  force_timeout (tests): the first wait's target is one more than
// the grid, its poll limit 4096, so that it runs out and every CTA returns with *err set.
template <class R, class S>
lfx_status launch_assemble_persistent(cudaStream_t st, const AssembleArgs &A, const PhysParams &P, const ChunkArgs &C,
                                      const int32_t *d_chunk_color_off, int n_colors, S *vals, unsigned *barrier,
                                      int *err, bool force_timeout = false, bool newton = false);
// the semi-implicit system (newton: the Newton system) by chunks, one launch per chunk colour
template <class R, class S>
lfx_status launch_assemble_chunks(cudaStream_t st, const AssembleArgs &A, const PhysParams &P, const ChunkArgs &C,
                                  const int32_t *chunk_color_off, int n_colors, S *vals, bool newton = false);
lfx_status launch_dirichlet_values(cudaStream_t st, int64_t nd, int H, const int32_t *bc_of,
                                   const double *S, const DirCoef &C, const double *N, int nb, D4 *g);
lfx_status launch_neumann(cudaStream_t st, int64_t n, const int32_t *node, const int32_t *bc_of,
                          const double *vec, const DirCoef &C, double *rhs);
template <class S>
lfx_status launch_apply_dirichlet(cudaStream_t st, int64_t nd, const int32_t *dnode, const D4 *g,
                                  int32_t pin_node, double pin_value, const int32_t *rowptr,
                                  const int32_t *diag, S *vals, double *rhs, double *x0);

// Batched independent meshes: each connected component's rows (matrix and rhs) scaled by
// 1/||rhs_component|| so that one Krylov solve meets every component's own tolerance.
lfx_status launch_comp_normalize(cudaStream_t st, int64_t V, int n_comp, const int32_t *comp_off, double *scale,
                                 const int32_t *rowptr, double *vals, double *rhs);

// ------------------------------------------------------------------ block-CSR views
template <class S>
struct BsrView {
  int64_t V;                 // block rows
  const int32_t *rowptr;     // [V+1]
  const int32_t *col;        // [nnzb]
  const int32_t *diag;       // [V]
  const int32_t *trans;      // [nnzb]
  const S *vals;             // [nnzb][16]
};

// A double-float matrix: every value is hi + lo with FP32 parts (the FP32 matrix of the inner
// solve is its high part).  Products with FP64 vectors first split the operand into FP32 high
// and low parts in the scratch arrays xs_hi, xs_lo.
struct DDMat {};
template <>
struct BsrView<DDMat> {
  int64_t V;
  const int32_t *rowptr, *col, *diag, *trans;
  const float *hi, *lo;      // [nnzb][16]
  float4 *xs_hi, *xs_lo;     // [V] operand scratch
};

// y = A x  (mode 0)  or  y = b - A x  (mode 1); vectors [V][4] of type T.  Optionally writes
// per-CTA partial sums of y.y into part (deterministic two-stage norm).
template <class S, class T>
lfx_status launch_spmv(cudaStream_t st, const BsrView<S> &A, const T *x, const T *b, T *y,
                       int mode, double *part, int *n_part);
template <>
lfx_status launch_spmv<DDMat, double>(cudaStream_t st, const BsrView<DDMat> &A, const double *x, const double *b,
                                      double *y, int mode, double *part, int *n_part);

// ------------------------------------------------------------------ moving domains (ale.cu)
// The lifting problem (Eq. lifting): the P1 Laplacian K of the reference mesh over the block pattern
// (one FP64 value per block) and its work arrays for conjugate gradients with Jacobi scaling.
struct LiftingView {
  int64_t V;
  const int32_t *rowptr, *col;
  const double *K, *dinv;
  uint8_t *fixed;          // [V] 1 where the displacement is prescribed
  D4 *r, *z, *p, *Ap;      // [V]
  double *part;            // lifting_part_entries(V)
  void *cg_state;          // lifting_cg_state_bytes()
};
lfx_status launch_lifting_matrix(cudaStream_t st, int64_t T, int64_t V, int64_t nnzb, const int32_t *slot,
                                 const int32_t *diag, const double *geo64, const float *geo_hi, const float *geo_lo,
                                 double *K, double *dinv);
// d = harmonic extension: d = fixed_val at fixed_node, K d = 0 on the other nodes (zero normal
// flux on the free boundary), from the initial guess in d; stops at ||r||_{D^-1} <= rtol of the
// initial residual for each component (synchronises st every 16 iterations).
lfx_status lifting_solve(cudaStream_t st, const LiftingView &L, int64_t n_fixed, const int32_t *fixed_node,
                         const D4 *fixed_val, D4 *d, double rtol, int max_iters, int *iters_out);
size_t lifting_cg_state_bytes();
int lifting_part_entries(int64_t V);
// x = ref + d, and its double-float split when hi is non-null
lfx_status launch_move_nodes(cudaStream_t st, int64_t V, const D4 *ref, const D4 *d, D4 *x, float4 *hi, float4 *lo);
// u_ALE = (alpha d^{n+1} - sum_j beta_j d^{n-j}) / dt (Section 2.3)
lfx_status launch_mesh_velocity(cudaStream_t st, int64_t V, int order, const D4 *dn1, const D4 *d0, const D4 *d1,
                                const D4 *d2, double alpha, const double beta[3], double dt, D4 *u);
// Neumann loads -(h n, v) of the listed faces (internal numbering, h = C.c[face_bc]) at coordinates x
lfx_status launch_neumann_faces(cudaStream_t st, int64_t nf, const int32_t *faces, const int32_t *face_bc,
                                const DirCoef &C, const D4 *x, double *rhs);

// Per-CTA partial sums of v.v (n values) into part[*n_part]; part needs
// norm_partials_capacity(V) entries for vectors of up to 4 V values or a residual SpMV of V rows.
lfx_status launch_norm_partials(cudaStream_t st, const double *v, int64_t n, double *part, int *n_part);
int norm_partials_capacity(int64_t V);
// x [V][4] FP64 split into FP32 high and low parts (x = hi + lo)
lfx_status launch_split_vec(cudaStream_t st, int64_t V, const double *x, float4 *hi, float4 *lo);

}  // namespace lfx
