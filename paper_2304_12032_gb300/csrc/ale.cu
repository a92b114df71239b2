// Moving domains (arbitrary Lagrangian-Eulerian form, Sections 2.1-2.4): the lifting problem of
// Eq. (lifting) (harmonic extension of a boundary displacement into the domain, P1 Laplacian on the
// reference mesh, solved by conjugate gradients on the device), the moved node coordinates
// x = x^ + d, the mesh velocity u_ALE as the BDF derivative of d (Section 2.3), and the Neumann
// loads on the moved boundary faces.
//
// Layout: displacements and velocities are D4 [V] records (x, y, z, unused) in the internal node
// numbering; the Laplacian is stored as one FP64 value per block of the 4x4 block pattern (the node
// graph), so the element -> block slot map of the assembly serves it unchanged.
#include <cuda_runtime.h>

#include "dd.h"
#include "kernels.h"
#include "lfx_internal.h"
#include "pdl.h"

namespace lfx {

namespace {

constexpr int kThr = 256;

inline int grid_of(int64_t n) {
  int64_t g = (n + kThr - 1) / kThr;
  if (g > 152 * 16) g = 152 * 16;
  return (int)(g < 1 ? 1 : g);
}

// K_ab += |K| grad phi_a . grad phi_b for the 16 node pairs of every element (FP64 atomics: the
// matrix is built once per state).  Geometry from the reference mesh's cache (FP64, or the
// double-float pair hi + lo).
__global__ void lifting_matrix_kernel(int64_t T, const int32_t *slot, const double *geo64, const float *geo_hi,
                                      const float *geo_lo, double *K) {
  pdl_entry();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < T; e += (int64_t)gridDim.x * blockDim.x) {
    double g[12], w;
#pragma unroll
    for (int k = 0; k < 12; ++k) g[k] = geo64 ? geo64[k * T + e] : (double)geo_hi[k * T + e] + (double)geo_lo[k * T + e];
    w = geo64 ? geo64[22 * T + e] : (double)geo_hi[22 * T + e] + (double)geo_lo[22 * T + e];
    const double vol = 4.0 * w;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const double v = vol * (g[3 * a] * g[3 * b] + g[3 * a + 1] * g[3 * b + 1] + g[3 * a + 2] * g[3 * b + 2]);
        atomicAdd(K + slot[e * 16 + 4 * a + b], v);
      }
  }
}

__global__ void diag_inverse_kernel(int64_t V, const int32_t *diag, const double *K, double *dinv) {
  pdl_entry();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < V; i += (int64_t)gridDim.x * blockDim.x) {
    const double d = K[diag[i]];
    dinv[i] = d != 0.0 ? 1.0 / d : 0.0;
  }
}

// block-wide sums of three values into part[3 * blockIdx.x + c]
__device__ __forceinline__ void cta_sum3(double a0, double a1, double a2, double *part) {
  __shared__ double red[3][kThr / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a0 += __shfl_xor_sync(0xffffffffu, a0, o);
    a1 += __shfl_xor_sync(0xffffffffu, a1, o);
    a2 += __shfl_xor_sync(0xffffffffu, a2, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    red[0][w] = a0;
    red[1][w] = a1;
    red[2][w] = a2;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[threadIdx.x][k];
    part[3 * blockIdx.x + threadIdx.x] = s;
  }
}

// CG state of the three components (lifting)
struct CgState {
  double rz[3], rz0[3], alpha[3], beta[3];
  int iters, converged;
};

// y = P K P x (P zeroes the fixed nodes), and partial sums of x . y per component
__global__ void lap_apply_kernel(int64_t V, const int32_t *rowptr, const int32_t *col, const double *K,
                                 const uint8_t *fixed, const D4 *x, D4 *y, double *part, const CgState *cs) {
  pdl_entry();
  if (cs && cs->converged) return;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < V; i += (int64_t)gridDim.x * blockDim.x) {
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    if (!fixed[i]) {
      for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
        const int32_t j = col[k];
        if (fixed[j]) continue;
        const double kv = K[k];
        const D4 xj = x[j];
        a0 += kv * xj.x;
        a1 += kv * xj.y;
        a2 += kv * xj.z;
      }
      const D4 xi = x[i];
      s0 += xi.x * a0;
      s1 += xi.y * a1;
      s2 += xi.z * a2;
    }
    y[i] = D4{a0, a1, a2, 0.0};
  }
  if (part) cta_sum3(s0, s1, s2, part);
}

// r = -(K d) on the free nodes (d holds the fixed values and the initial guess), 0 on fixed ones
__global__ void lap_residual_kernel(int64_t V, const int32_t *rowptr, const int32_t *col, const double *K,
                                    const uint8_t *fixed, const D4 *d, D4 *r) {
  pdl_entry();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < V; i += (int64_t)gridDim.x * blockDim.x) {
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    if (!fixed[i]) {
      for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
        const D4 dj = d[col[k]];
        a0 -= K[k] * dj.x;
        a1 -= K[k] * dj.y;
        a2 -= K[k] * dj.z;
      }
    }
    r[i] = D4{a0, a1, a2, 0.0};
  }
}

// z = D^-1 r, p = z (start), partial sums of r . z
__global__ void cg_start_kernel(int64_t V, const double *dinv, const uint8_t *fixed, const D4 *r, D4 *z, D4 *p,
                                double *part) {
  pdl_entry();
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < V; i += (int64_t)gridDim.x * blockDim.x) {
    const double di = fixed[i] ? 0.0 : dinv[i];
    const D4 ri = r[i];
    const D4 zi{di * ri.x, di * ri.y, di * ri.z, 0.0};
    z[i] = zi;
    p[i] = zi;
    s0 += ri.x * zi.x;
    s1 += ri.y * zi.y;
    s2 += ri.z * zi.z;
  }
  cta_sum3(s0, s1, s2, part);
}

// one thread: sums the partials; mode 0: rz = rz0 = sum; mode 1: alpha = rz / sum (p.Ap);
// mode 2: beta = sum / rz, rz = sum, convergence test sum <= tol2 * rz0 for every component
__global__ void cg_scalar_kernel(const double *part, int ng, CgState *cs, int mode, double tol2, int max_iters) {
  pdl_entry();
  if (threadIdx.x != 0 || (mode != 0 && cs->converged)) return;
  double s[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k < ng; ++k)
    for (int c = 0; c < 3; ++c) s[c] += part[3 * k + c];
  if (mode == 0) {
    for (int c = 0; c < 3; ++c) cs->rz[c] = cs->rz0[c] = s[c];
    cs->iters = 0;
    cs->converged = (s[0] <= 0.0 && s[1] <= 0.0 && s[2] <= 0.0) ? 1 : 0;
  } else if (mode == 1) {
    for (int c = 0; c < 3; ++c) cs->alpha[c] = s[c] > 0.0 ? cs->rz[c] / s[c] : 0.0;
  } else {
    bool done = true;
    for (int c = 0; c < 3; ++c) {
      cs->beta[c] = cs->rz[c] > 0.0 ? s[c] / cs->rz[c] : 0.0;
      cs->rz[c] = s[c];
      if (s[c] > tol2 * cs->rz0[c]) done = false;
    }
    cs->iters += 1;
    if (done || cs->iters >= max_iters) cs->converged = done ? 1 : 2;
  }
}

// x += alpha p, r -= alpha Ap, z = D^-1 r, partial sums of r . z
__global__ void cg_update_kernel(int64_t V, const double *dinv, const uint8_t *fixed, const D4 *p, const D4 *Ap,
                                 D4 *x, D4 *r, D4 *z, double *part, const CgState *cs) {
  pdl_entry();
  if (cs->converged) return;
  const double a0 = cs->alpha[0], a1 = cs->alpha[1], a2 = cs->alpha[2];
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < V; i += (int64_t)gridDim.x * blockDim.x) {
    if (fixed[i]) continue;
    const D4 pi = p[i], qi = Ap[i];
    D4 xi = x[i], ri = r[i];
    xi.x += a0 * pi.x;
    xi.y += a1 * pi.y;
    xi.z += a2 * pi.z;
    ri.x -= a0 * qi.x;
    ri.y -= a1 * qi.y;
    ri.z -= a2 * qi.z;
    x[i] = xi;
    r[i] = ri;
    const double di = dinv[i];
    const D4 zi{di * ri.x, di * ri.y, di * ri.z, 0.0};
    z[i] = zi;
    s0 += ri.x * zi.x;
    s1 += ri.y * zi.y;
    s2 += ri.z * zi.z;
  }
  cta_sum3(s0, s1, s2, part);
}

// p = z + beta p
__global__ void cg_direction_kernel(int64_t V, const D4 *z, D4 *p, const CgState *cs) {
  pdl_entry();
  if (cs->converged) return;
  const double b0 = cs->beta[0], b1 = cs->beta[1], b2 = cs->beta[2];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < V; i += (int64_t)gridDim.x * blockDim.x) {
    const D4 zi = z[i];
    D4 pi = p[i];
    pi.x = zi.x + b0 * pi.x;
    pi.y = zi.y + b1 * pi.y;
    pi.z = zi.z + b2 * pi.z;
    p[i] = pi;
  }
}

// d at the listed nodes (fixed) = the given values; fixed flags set
__global__ void set_fixed_kernel(int64_t n, const int32_t *node, const D4 *val, D4 *d, uint8_t *fixed) {
  pdl_entry();
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t i = node[k];
    d[i] = val[k];
    fixed[i] = 1;
  }
}

// x = x^ + d (w = 0) and its double-float split
__global__ void move_nodes_kernel(int64_t V, const D4 *ref, const D4 *d, D4 *x, float4 *hi, float4 *lo) {
  pdl_entry();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < V; i += (int64_t)gridDim.x * blockDim.x) {
    const D4 a = ref[i], b = d[i];
    const D4 c{a.x + b.x, a.y + b.y, a.z + b.z, 0.0};
    x[i] = c;
    if (hi) {
      const dd p(c.x), q(c.y), r(c.z);
      hi[i] = make_float4(p.hi, q.hi, r.hi, 0.0f);
      lo[i] = make_float4(p.lo, q.lo, r.lo, 0.0f);
    }
  }
}

// u_ALE = (alpha d^{n+1} - sum_j beta_j d^{n-j}) / dt
__global__ void mesh_velocity_kernel(int64_t V, int order, const D4 *dn1, const D4 *d0, const D4 *d1, const D4 *d2,
                                     double alpha, double b0, double b1, double b2, double inv_dt, D4 *u) {
  pdl_entry();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < V; i += (int64_t)gridDim.x * blockDim.x) {
    const D4 a = dn1[i], c0 = d0[i];
    double x = alpha * a.x - b0 * c0.x, y = alpha * a.y - b0 * c0.y, z = alpha * a.z - b0 * c0.z;
    if (order >= 2) {
      const D4 c1 = d1[i];
      x -= b1 * c1.x;
      y -= b1 * c1.y;
      z -= b1 * c1.z;
    }
    if (order >= 3) {
      const D4 c2 = d2[i];
      x -= b2 * c2.x;
      y -= b2 * c2.y;
      z -= b2 * c2.z;
    }
    u[i] = D4{x * inv_dt, y * inv_dt, z * inv_dt, 0.0};
  }
}

// -(h n, v) on the faces of Neumann tags at the moved coordinates: each vertex gets A_f n_f / 3
__global__ void neumann_faces_kernel(int64_t nf, const int32_t *faces, const int32_t *face_bc, DirCoef C,
                                     const D4 *x, double *rhs) {
  pdl_entry();
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf; f += (int64_t)gridDim.x * blockDim.x) {
    const double h = C.c[face_bc[f]];
    if (h == 0.0) continue;
    const int32_t i0 = faces[3 * f], i1 = faces[3 * f + 1], i2 = faces[3 * f + 2];
    const D4 a = x[i0], b = x[i1], c = x[i2];
    const double u0 = b.x - a.x, u1 = b.y - a.y, u2 = b.z - a.z;
    const double v0 = c.x - a.x, v1 = c.y - a.y, v2 = c.z - a.z;
    const double s = -h * 0.5 / 3.0;
    const double an[3] = {s * (u1 * v2 - u2 * v1), s * (u2 * v0 - u0 * v2), s * (u0 * v1 - u1 * v0)};
    const int32_t vv[3] = {i0, i1, i2};
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
      for (int k = 0; k < 3; ++k) atomicAdd(rhs + 4 * (int64_t)vv[q] + k, an[k]);
  }
}

}  // namespace

lfx_status launch_lifting_matrix(cudaStream_t st, int64_t T, int64_t V, int64_t nnzb, const int32_t *slot,
                                 const int32_t *diag, const double *geo64, const float *geo_hi, const float *geo_lo,
                                 double *K, double *dinv) {
  LFX_CUDA_TRY(cudaMemsetAsync(K, 0, sizeof(double) * (size_t)nnzb, st));
  pdl_launch(lifting_matrix_kernel, grid_of(T), kThr, 0, st, T, slot, geo64, geo_hi, geo_lo, K);
  pdl_launch(diag_inverse_kernel, grid_of(V), kThr, 0, st, V, diag, (const double *)K, dinv);
  note_launches(2);
  LFX_CUDA_TRY(cudaGetLastError());
  return LFX_OK;
}

lfx_status lifting_solve(cudaStream_t st, const LiftingView &L, int64_t n_fixed, const int32_t *fixed_node,
                         const D4 *fixed_val, D4 *d, double rtol, int max_iters, int *iters_out) {
  const int64_t V = L.V;
  const int g = grid_of(V);
  CgState *cs = reinterpret_cast<CgState *>(L.cg_state);
  LFX_CUDA_TRY(cudaMemsetAsync(L.fixed, 0, (size_t)V, st));
  if (n_fixed > 0) pdl_launch(set_fixed_kernel, grid_of(n_fixed), kThr, 0, st, n_fixed, fixed_node, fixed_val, d, L.fixed);
  pdl_launch(lap_residual_kernel, g, kThr, 0, st, V, L.rowptr, L.col, L.K, (const uint8_t *)L.fixed, (const D4 *)d, L.r);
  pdl_launch(cg_start_kernel, g, kThr, 0, st, V, L.dinv, (const uint8_t *)L.fixed, (const D4 *)L.r, L.z, L.p, L.part);
  pdl_launch(cg_scalar_kernel, 1, 32, 0, st, (const double *)L.part, g, cs, 0, rtol * rtol, max_iters);
  note_launches(4 + (n_fixed > 0));
  // iterations queued in batches; the host reads the convergence word between batches
  CgState h{};
  const int batch = 16;
  for (int it = 0; it < max_iters; it += batch) {
    for (int k = 0; k < batch; ++k) {
      pdl_launch(lap_apply_kernel, g, kThr, 0, st, V, L.rowptr, L.col, L.K, (const uint8_t *)L.fixed, (const D4 *)L.p,
                 L.Ap, L.part, (const CgState *)cs);
      pdl_launch(cg_scalar_kernel, 1, 32, 0, st, (const double *)L.part, g, cs, 1, rtol * rtol, max_iters);
      pdl_launch(cg_update_kernel, g, kThr, 0, st, V, L.dinv, (const uint8_t *)L.fixed, (const D4 *)L.p,
                 (const D4 *)L.Ap, d, L.r, L.z, L.part, (const CgState *)cs);
      pdl_launch(cg_scalar_kernel, 1, 32, 0, st, (const double *)L.part, g, cs, 2, rtol * rtol, max_iters);
      pdl_launch(cg_direction_kernel, g, kThr, 0, st, V, (const D4 *)L.z, L.p, (const CgState *)cs);
    }
    note_launches(5 * batch);
    LFX_CUDA_TRY(cudaMemcpyAsync(&h, cs, sizeof(CgState), cudaMemcpyDeviceToHost, st));
    LFX_CUDA_TRY(cudaStreamSynchronize(st));
    if (h.converged) break;
  }
  LFX_CUDA_TRY(cudaGetLastError());
  if (iters_out) *iters_out = h.iters;
  if (h.converged != 1) {
    set_error("lifting: conjugate gradients did not converge in %d iterations", h.iters);
    return LFX_ERR_NOT_CONVERGED;
  }
  return LFX_OK;
}

size_t lifting_cg_state_bytes() { return sizeof(CgState); }
int lifting_part_entries(int64_t V) { return 3 * grid_of(V) + 8; }

lfx_status launch_move_nodes(cudaStream_t st, int64_t V, const D4 *ref, const D4 *d, D4 *x, float4 *hi, float4 *lo) {
  pdl_launch(move_nodes_kernel, grid_of(V), kThr, 0, st, V, ref, d, x, hi, lo);
  note_launches(1);
  LFX_CUDA_TRY(cudaGetLastError());
  return LFX_OK;
}

lfx_status launch_mesh_velocity(cudaStream_t st, int64_t V, int order, const D4 *dn1, const D4 *d0, const D4 *d1,
                                const D4 *d2, double alpha, const double beta[3], double dt, D4 *u) {
  pdl_launch(mesh_velocity_kernel, grid_of(V), kThr, 0, st, V, order, dn1, d0, d1, d2, alpha, beta[0], beta[1],
             beta[2], 1.0 / dt, u);
  note_launches(1);
  LFX_CUDA_TRY(cudaGetLastError());
  return LFX_OK;
}

lfx_status launch_neumann_faces(cudaStream_t st, int64_t nf, const int32_t *faces, const int32_t *face_bc,
                                const DirCoef &C, const D4 *x, double *rhs) {
  if (nf == 0) return LFX_OK;
  pdl_launch(neumann_faces_kernel, grid_of(nf), kThr, 0, st, nf, faces, face_bc, C, x, rhs);
  note_launches(1);
  LFX_CUDA_TRY(cudaGetLastError());
  return LFX_OK;
}

}  // namespace lfx
