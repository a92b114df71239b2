// Linear algebra of Section 2.4: block-CSR matrix-vector products, the aSIMPLE preconditioner
// [deparis2014parallel] with Jacobi / Chebyshev smoothing of the velocity block F and of the
// Schur approximation S = C - D diag(F)^-1 G, and restarted right-preconditioned (flexible)
// GMRES with classical Gram-Schmidt (optionally twice), Givens rotations and a device-resident
// convergence flag.
//
// Vectors are [V][4] (u_x, u_y, u_z, p per node).  Every reduction is two-stage (per-CTA
// partials, then one CTA sums them in a fixed order), so results are bitwise reproducible.
// Every kernel of an Arnoldi step reads the solver's status word first and returns at once if
// the cycle is already finished, so the host may queue a few steps ahead of the convergence test.
#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <cstddef>
#include <cstring>
#include <type_traits>

#include "amg.h"
#include "dd.h"
#include "kernels.h"
#include "pdl.h"
#include "solver.h"

namespace lfx {

namespace {

constexpr int kThreads = 256;
#ifndef LFX_ROW_GROUP
#define LFX_ROW_GROUP 4
#endif
constexpr int kRowGroup = LFX_ROW_GROUP;   // lanes per block row in the row kernels
// blocks in flight per lane in the row kernels (full 4x4 blocks / sub-blocks)
#ifndef LFX_U_FULL
#define LFX_U_FULL 2
#endif
#ifndef LFX_U_F
#define LFX_U_F 2
#endif
#ifndef LFX_U_GDC
#define LFX_U_GDC 2
#endif

template <class T> struct Vec4T;
template <> struct Vec4T<double> { using type = D4; };
template <> struct Vec4T<float> { using type = F4; };

// Arithmetic type of the vector kernels: FP32 vectors (the inner solve) are combined in FP32 and
// only per-thread partial sums are widened to FP64 for the cross-thread reduction; FP64 vectors
// stay FP64 throughout.  (FP64 instructions issue at 1/61 of the FP32 rate on this part, so an
// FP64 accumulator would make the FP32 Krylov kernels arithmetic-bound.)
template <class T, class X = T> struct AccT { using type = double; };
template <> struct AccT<float, float> { using type = float; };

template <class T>
__device__ __forceinline__ typename Vec4T<T>::type ld4(const T *p, int64_t i) {
  return reinterpret_cast<const typename Vec4T<T>::type *>(p)[i];
}
template <class T>
__device__ __forceinline__ void st4(T *p, int64_t i, const typename Vec4T<T>::type &v) {
  reinterpret_cast<typename Vec4T<T>::type *>(p)[i] = v;
}

// Two packed BF16 values to FP32 (exact: a BF16 value is the top half of its FP32 value).  Bit
// operations on the integer pipe; the conversion instruction would take FP64-pipe issue slots.
__device__ __forceinline__ void bf16x2_to_f32(uint32_t w, float &lo, float &hi) {
  lo = __uint_as_float(w << 16);
  hi = __uint_as_float(w & 0xffff0000u);
}

template <class S, class A>
__device__ __forceinline__ void ld_block(const S *vals, int64_t k, A b[16]);
template <>
__device__ __forceinline__ void ld_block<double, double>(const double *vals, int64_t k, double b[16]) {
  const double2 *p = reinterpret_cast<const double2 *>(vals + 16 * k);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    double2 v = __ldg(p + i);
    b[2 * i] = v.x;
    b[2 * i + 1] = v.y;
  }
}
template <>
__device__ __forceinline__ void ld_block<float, float>(const float *vals, int64_t k, float b[16]) {
  const float4 *p = reinterpret_cast<const float4 *>(vals + 16 * k);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float4 v = __ldg(p + i);
    b[4 * i] = v.x;
    b[4 * i + 1] = v.y;
    b[4 * i + 2] = v.z;
    b[4 * i + 3] = v.w;
  }
}
template <>
__device__ __forceinline__ void ld_block<__nv_bfloat16, float>(const __nv_bfloat16 *vals, int64_t k, float b[16]) {
  const uint4 *p = reinterpret_cast<const uint4 *>(vals + 16 * k);
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    uint4 v = __ldg(p + i);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) bf16x2_to_f32(w[q], b[8 * i + 2 * q], b[8 * i + 2 * q + 1]);
  }
}
template <>
__device__ __forceinline__ void ld_block<float, double>(const float *vals, int64_t k, double b[16]) {
  const float4 *p = reinterpret_cast<const float4 *>(vals + 16 * k);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float4 v = __ldg(p + i);
    b[4 * i] = v.x;
    b[4 * i + 1] = v.y;
    b[4 * i + 2] = v.z;
    b[4 * i + 3] = v.w;
  }
}

template <class A>
__device__ __forceinline__ A group_sum(A v) {
#pragma unroll
  for (int o = kRowGroup / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// The blocks k0 + lane, k0 + lane + G, ... (< k1) of one block row, U per lane at a time: for a
// batch, load(u, k) issues the matrix and index loads of every valid slot, then gather(u) the
// dependent vector loads, then use(u) consumes them, so that U blocks' loads of each lane are in
// flight together instead of one dependent pair after another.
template <int U, class Load, class Gather, class Use>
__device__ __forceinline__ void row_blocks(int32_t k0, int32_t k1, int lane, Load load, Gather gather, Use use) {
  for (int32_t kb = k0 + lane; kb < k1; kb += U * kRowGroup) {
    bool ok[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      ok[u] = kb + u * kRowGroup < k1;
      if (ok[u]) load(u, kb + u * kRowGroup);
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (ok[u]) gather(u);
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (ok[u]) use(u);
  }
}

// CTA-wide sum of one double per thread; result valid in thread 0.
__device__ __forceinline__ double cta_sum(double v) {
  __shared__ double red[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  return s;
}

// CTA-wide sum with the warp stage in the value's own type (FP32 values are widened to FP64 only
// per warp); result valid in thread 0.
template <class A>
__device__ __forceinline__ double cta_sum_t(A v) {
  __shared__ double red[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = (double)v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  return s;
}

// CTA-wide max of one double per thread; result valid in thread 0.
__device__ __forceinline__ double cta_max(double v) {
  __shared__ double red[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s = fmax(s, red[i]);
  return s;
}

// a smoothing coefficient in the arithmetic type T (the FP32 kernels read the FP32 copy)
template <class T>
__device__ __forceinline__ T coef_t(const double &d, const float &) {
  return (T)d;
}
template <>
__device__ __forceinline__ float coef_t<float>(const double &, const float &f) {
  return f;
}

__device__ __forceinline__ bool finished(const KState *st) {
  return st != nullptr && *(volatile const int *)&st->done != 0;
}

// ------------------------------------------------------------------------------------------
// y = A x (mode 0) or y = b - A x (mode 1); optional partial sums of y.y per CTA
// ------------------------------------------------------------------------------------------
template <class S, class T>
__global__ void __launch_bounds__(kThreads) spmv_kernel(BsrView<S> A, const T *__restrict__ x,
                                                        const T *__restrict__ b, T *__restrict__ y,
                                                        int mode, double *part, const KState *st) {
  pdl_entry();
  if (finished(st)) return;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kRowGroup;
  const int lane = threadIdx.x % kRowGroup;
  T acc[4] = {T(0), T(0), T(0), T(0)};
  if (row < A.V) {
    constexpr int U = LFX_U_FULL;
    T blk[U][16];
    int32_t c[U];
    typename Vec4T<T>::type xv[U];
    row_blocks<U>(
        A.rowptr[row], A.rowptr[row + 1], lane,
        [&](int u, int32_t k) {
          ld_block<S, T>(A.vals, k, blk[u]);
          c[u] = __ldg(A.col + k);
        },
        [&](int u) { xv[u] = ld4(x, c[u]); },
        [&](int u) {
#pragma unroll
          for (int i = 0; i < 4; ++i)
            acc[i] += blk[u][4 * i] * xv[u].x + blk[u][4 * i + 1] * xv[u].y + blk[u][4 * i + 2] * xv[u].z +
                      blk[u][4 * i + 3] * xv[u].w;
        });
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) acc[i] = group_sum(acc[i]);
  typename AccT<T>::type nrm = 0;
  if (row < A.V && lane == 0) {
    typename Vec4T<T>::type o;
    if (mode == 1) {
      const auto bv = ld4(b, row);
      o.x = bv.x - acc[0]; o.y = bv.y - acc[1]; o.z = bv.z - acc[2]; o.w = bv.w - acc[3];
    } else {
      o.x = acc[0]; o.y = acc[1]; o.z = acc[2]; o.w = acc[3];
    }
    st4(y, row, o);
    nrm = o.x * o.x + o.y * o.y + o.z * o.z + o.w * o.w;
  }
  if (part) {
    double s = cta_sum_t(nrm);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
  }
}

// ---- double-float operator with FP64 vectors.  The operand is split into FP32 high and low
// parts first; every block row then accumulates compensated (Ogita, Rump and Oishi's Dot2:
// products made exact by two_prod, sums by two_sum, the rounding errors gathered in an FP32
// correction), so the product carries about 48 significant bits while running on the FP32 pipes.
__global__ void split_vec_kernel(int64_t V, const double *x, float4 *hi, float4 *lo, const KState *st) {
  pdl_entry();
  if (finished(st)) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < V; i += (int64_t)gridDim.x * blockDim.x) {
    const D4 v = reinterpret_cast<const D4 *>(x)[i];
    const dd a(v.x), b(v.y), c(v.z), d(v.w);
    hi[i] = make_float4(a.hi, b.hi, c.hi, d.hi);
    lo[i] = make_float4(a.lo, b.lo, c.lo, d.lo);
  }
}

__global__ void __launch_bounds__(kThreads) spmv_dd_kernel(BsrView<DDMat> A, const double *__restrict__ b,
                                                           double *__restrict__ y, int mode, double *part,
                                                           const KState *st) {
  pdl_entry();
  if (finished(st)) return;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kRowGroup;
  const int lane = threadIdx.x % kRowGroup;
  float s[4] = {0.f, 0.f, 0.f, 0.f}, c[4] = {0.f, 0.f, 0.f, 0.f};
  if (row < A.V) {
    const int32_t k1 = A.rowptr[row + 1];
#pragma unroll 2
    for (int32_t k = A.rowptr[row] + lane; k < k1; k += kRowGroup) {
      float h[16], l[16];
      ld_block<float, float>(A.hi, k, h);
      ld_block<float, float>(A.lo, k, l);
      const int32_t col = __ldg(A.col + k);
      const float4 xh4 = A.xs_hi[col], xl4 = A.xs_lo[col];
      const float xh[4] = {xh4.x, xh4.y, xh4.z, xh4.w}, xl[4] = {xl4.x, xl4.y, xl4.z, xl4.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const dd p = two_prod(h[4 * i + j], xh[j]);
          float e = f_fma(h[4 * i + j], xl[j], p.lo);
          e = f_fma(l[4 * i + j], xh[j], e);
          const dd t = two_sum(s[i], p.hi);
          s[i] = t.hi;
          c[i] = f_add(c[i], f_add(t.lo, e));
        }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int o = kRowGroup / 2; o > 0; o >>= 1) {
      const float os = __shfl_xor_sync(0xffffffffu, s[i], o), oc = __shfl_xor_sync(0xffffffffu, c[i], o);
      const dd t = two_sum(s[i], os);
      s[i] = t.hi;
      c[i] = f_add(c[i], f_add(oc, t.lo));
    }
  double nrm = 0.0;
  if (row < A.V && lane == 0) {
    D4 o;
    double r[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) r[i] = (double)s[i] + (double)c[i];
    if (mode == 1) {
      const D4 bv = reinterpret_cast<const D4 *>(b)[row];
      o = D4{bv.x - r[0], bv.y - r[1], bv.z - r[2], bv.w - r[3]};
    } else {
      o = D4{r[0], r[1], r[2], r[3]};
    }
    reinterpret_cast<D4 *>(y)[row] = o;
    nrm = o.x * o.x + o.y * o.y + o.z * o.z + o.w * o.w;
  }
  if (part) {
    double sum = cta_sum(nrm);
    if (threadIdx.x == 0) part[blockIdx.x] = sum;
  }
}

// sum of part[0..n) -> *out (sqrt if root == 1, max instead of sum if root == 2); one CTA
__global__ void reduce_kernel(const double *part, int n, double *out, int root) {
  pdl_entry();
  double s = 0.0;
  if (root == 2) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) s = fmax(s, part[i]);
    s = cta_max(s);
    if (threadIdx.x == 0) *out = s;
    return;
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
  s = cta_sum(s);
  if (threadIdx.x == 0) *out = root ? sqrt(s) : s;
}

// ---- access to the aSIMPLE sub-blocks of block k, in the arithmetic type T:
//   F (3x3, row-major, 9 values), G (velocity rows x pressure column, 3), D (pressure row x
//   velocity columns) with C appended (4).  Two storages: the full 4x4 blocks (BsrView) and the
//   blocks stored apart (SplitView), where every pass over the matrix reads only the sub-block
//   it needs.
template <class S>
struct SplitView {
  int64_t V;
  const int32_t *rowptr, *col, *diag, *trans;
  const S *F;    // [nnzb][12]: F00 F01 F02 F10 F11 F12 F20 F21 F22 0 0 0
  const S *G;    // [nnzb][4]:  G0 G1 G2 0
  const S *DC;   // [nnzb][4]:  D0 D1 D2 C
};

// N consecutive values (N a multiple of 4) from an aligned record
template <int N>
__device__ __forceinline__ void ld_rec(const double *p, double *o) {
#pragma unroll
  for (int i = 0; i < N / 2; ++i) {
    const double2 v = __ldg(reinterpret_cast<const double2 *>(p) + i);
    o[2 * i] = v.x;
    o[2 * i + 1] = v.y;
  }
}
template <int N>
__device__ __forceinline__ void ld_rec(const float *p, float *o) {
#pragma unroll
  for (int i = 0; i < N / 4; ++i) {
    const float4 v = __ldg(reinterpret_cast<const float4 *>(p) + i);
    o[4 * i] = v.x;
    o[4 * i + 1] = v.y;
    o[4 * i + 2] = v.z;
    o[4 * i + 3] = v.w;
  }
}
template <int N>
__device__ __forceinline__ void ld_rec(const __nv_bfloat16 *p, float *o) {
#pragma unroll
  for (int i = 0; i < N / 4; ++i) {
    const uint2 v = __ldg(reinterpret_cast<const uint2 *>(p) + i);
    bf16x2_to_f32(v.x, o[4 * i], o[4 * i + 1]);
    bf16x2_to_f32(v.y, o[4 * i + 2], o[4 * i + 3]);
  }
}

template <class S, class T>
__device__ __forceinline__ void ld_F(const BsrView<S> &A, int64_t k, T f[9]) {
  T b[16];
  ld_block<S, T>(A.vals, k, b);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) f[3 * i + j] = b[4 * i + j];
}
template <class S, class T>
__device__ __forceinline__ void ld_G(const BsrView<S> &A, int64_t k, T g[4]) {
  const S *blk = A.vals + 16 * k;
  g[0] = (T)blk[3];
  g[1] = (T)blk[7];
  g[2] = (T)blk[11];
  g[3] = T(0);
}
template <class S, class T>
__device__ __forceinline__ void ld_DC(const BsrView<S> &A, int64_t k, T dc[4]) {
  const S *blk = A.vals + 16 * k + 12;
  dc[0] = (T)blk[0];
  dc[1] = (T)blk[1];
  dc[2] = (T)blk[2];
  dc[3] = (T)blk[3];
}
template <class S, class T>
__device__ __forceinline__ void ld_F(const SplitView<S> &A, int64_t k, T f[9]) {
  T b[12];
  ld_rec<12>(A.F + 12 * k, b);
#pragma unroll
  for (int i = 0; i < 9; ++i) f[i] = b[i];
}
template <class S, class T>
__device__ __forceinline__ void ld_G(const SplitView<S> &A, int64_t k, T g[4]) {
  ld_rec<4>(A.G + 4 * k, g);
}
template <class S, class T>
__device__ __forceinline__ void ld_DC(const SplitView<S> &A, int64_t k, T dc[4]) {
  ld_rec<4>(A.DC + 4 * k, dc);
}

// Blocks stored apart (in the preconditioner's storage type S) from the FP64 or FP32 4x4 blocks.
// Record slots 9..11 of an F sub-block: zero, except in BF16 storage, where slots 9 and 10 carry the
// block's column index (low and high 16 bits) for the staged pass, which reads records only.
template <class S>
__device__ __forceinline__ void put_f_tail(S *rec, int32_t) {
  rec[9] = rec[10] = rec[11] = (S)0.0;
}
template <>
__device__ __forceinline__ void put_f_tail<__nv_bfloat16>(__nv_bfloat16 *rec, int32_t c) {
  rec[9] = __ushort_as_bfloat16((unsigned short)((uint32_t)c & 0xffffu));
  rec[10] = __ushort_as_bfloat16((unsigned short)((uint32_t)c >> 16));
  rec[11] = __ushort_as_bfloat16(0);
}

template <class S, class Src>
__global__ void split_kernel(int64_t nnzb, const Src *__restrict__ vals, const int32_t *__restrict__ col, S *F, S *G,
                             S *DC) {
  pdl_entry();
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnzb; k += (int64_t)gridDim.x * blockDim.x) {
    Src b[16];
    ld_block<Src, Src>(vals, k, b);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) F[12 * k + 3 * i + j] = (S)b[4 * i + j];
    put_f_tail<S>(F + 12 * k, col[k]);
    G[4 * k] = (S)b[3];
    G[4 * k + 1] = (S)b[7];
    G[4 * k + 2] = (S)b[11];
    G[4 * k + 3] = (S)0.0;
#pragma unroll
    for (int i = 0; i < 4; ++i) DC[4 * k + i] = (S)b[12 + i];
  }
}

// Gershgorin bounds for the Chebyshev intervals (every eigenvalue lies in a Gershgorin disc):
//   mode 0: per row max_i |dinvF_i| sum_{k,j<3} |F_k[i][j]|                    -> part (max)
//   mode 1: gs.xyz = sum_k |G_k[i][3]| (absolute row sums of G)                 -> gs
//   mode 2: |dinvS| (sum_k |C_k| + sum_{k,j} |D_k[3][j]| |dinvF_col,j| gs_col,j) -> part (max)
template <class View, class T>
__global__ void __launch_bounds__(kThreads) bound_kernel(View A, const T *dinvF, const T *dinvS, T *gs,
                                                         double *part, int mode) {
  pdl_entry();
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kRowGroup;
  const int lane = threadIdx.x % kRowGroup;
  using Acc = typename AccT<T>::type;
  Acc a0 = Acc(0), a1 = Acc(0), a2 = Acc(0);
  if (row < A.V) {
    const int32_t kend = A.rowptr[row + 1];
#pragma unroll 4
    for (int32_t kb = A.rowptr[row] + lane; kb < kend; kb += kRowGroup) {
      if (mode == 0) {
        T f[9];
        ld_F(A, kb, f);
        a0 += fabs((Acc)f[0]) + fabs((Acc)f[1]) + fabs((Acc)f[2]);
        a1 += fabs((Acc)f[3]) + fabs((Acc)f[4]) + fabs((Acc)f[5]);
        a2 += fabs((Acc)f[6]) + fabs((Acc)f[7]) + fabs((Acc)f[8]);
      } else if (mode == 1) {
        T g[4];
        ld_G(A, kb, g);
        a0 += fabs((Acc)g[0]);
        a1 += fabs((Acc)g[1]);
        a2 += fabs((Acc)g[2]);
      } else {
        T dc[4];
        ld_DC(A, kb, dc);
        const auto df = ld4(dinvF, __ldg(A.col + kb));
        const auto g = ld4(gs, __ldg(A.col + kb));
        a0 += fabs((Acc)dc[3]) + fabs((Acc)dc[0]) * fabs((Acc)df.x) * (Acc)g.x +
              fabs((Acc)dc[1]) * fabs((Acc)df.y) * (Acc)g.y + fabs((Acc)dc[2]) * fabs((Acc)df.z) * (Acc)g.z;
      }
    }
  }
  a0 = group_sum(a0);
  a1 = group_sum(a1);
  a2 = group_sum(a2);
  double val = 0.0;
  if (row < A.V && lane == 0) {
    if (mode == 0) {
      const auto df = ld4(dinvF, row);
      val = (double)fmax(fabs((Acc)df.x) * a0, fmax(fabs((Acc)df.y) * a1, fabs((Acc)df.z) * a2));
    } else if (mode == 1) {
      auto o = ld4(gs, row);
      o.x = (T)a0;
      o.y = (T)a1;
      o.z = (T)a2;
      st4(gs, row, o);
    } else {
      val = (double)(fabs((Acc)dinvS[row]) * a0);
    }
  }
  if (mode != 1) {
    double m = cta_max(val);
    if (threadIdx.x == 0) part[blockIdx.x] = m;
  }
}

// ------------------------------------------------------------------------------------------
// aSIMPLE building blocks on the 4x4 blocks (row-major: [i][j], i test comp, j trial comp)
//   F = [0..2][0..2], G = [0..2][3], D = [3][0..2], C = [3][3]
// ------------------------------------------------------------------------------------------
template <class View, class T>
__global__ void diag_f_kernel(View A, T *dinvF) {
  pdl_entry();
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < A.V; r += (int64_t)gridDim.x * blockDim.x) {
    T f[9];
    ld_F(A, A.diag[r], f);
    typename Vec4T<T>::type o;
    o.x = T(1) / f[0];
    o.y = T(1) / f[4];
    o.z = T(1) / f[8];
    o.w = T(0);
    st4(dinvF, r, o);
  }
}

// diag(S)_a = C_aa - sum_{b,j} D_{a,(b,j)} G_{(b,j),a} / F_{(b,j),(b,j)}
template <class View, class T>
__global__ void diag_s_kernel(View A, const T *dinvF, T *dinvS) {
  pdl_entry();
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kRowGroup;
  const int lane = threadIdx.x % kRowGroup;
  T acc = T(0);
  if (row < A.V) {
    const int32_t kend = A.rowptr[row + 1];
#pragma unroll 4
    for (int32_t k = A.rowptr[row] + lane; k < kend; k += kRowGroup) {
      T dc[4], g[4];
      ld_DC(A, k, dc);             // block (a, b)
      ld_G(A, A.trans[k], g);      // block (b, a)
      const auto df = ld4(dinvF, __ldg(A.col + k));
      acc += dc[0] * g[0] * df.x + dc[1] * g[1] * df.y + dc[2] * g[2] * df.z;
    }
  }
  acc = group_sum(acc);
  if (row < A.V && lane == 0) {
    T dcd[4];
    ld_DC(A, A.diag[row], dcd);
    const T c = dcd[3];
    const T dd = c - acc;
    dinvS[row] = dd != T(0) ? T(1) / dd : T(0);   // a vanishing diagonal leaves the unknown unsmoothed
  }
}

// Velocity smoothing step on F.  mode 0 (power): y = dinvF (F v), partial |y|^2.
// mode 1 (Chebyshev/Jacobi step k): y = F d_old; r -= dinvF y; d_new = c1 d_old + c2 r; x += d_new.
// kFirst: step 1 fused with the start of the smoothing (f_init_kernel): d_old = init dinvF b0 and
// r = dinvF b0 are formed on the fly from b0 by the same operations, so d_old is never stored.
template <class View, class T, bool kFirst = false>
__global__ void __launch_bounds__(kThreads) f_step_kernel(View A, const T *dinvF, const T *d_old,
                                                          T *d_new, T *r, T *x, const SmoothCoef *cf,
                                                          int k, int mode, double *part, const KState *st,
                                                          const T *b0) {
  pdl_entry();
  if (finished(st)) return;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kRowGroup;
  const int lane = threadIdx.x % kRowGroup;
  T acc[3] = {T(0), T(0), T(0)};
  // the row's own vector entries, loaded before the row's blocks so that their latency overlaps
  // the block loads and gathers
  const bool owner = row < A.V && lane == 0;
  typename Vec4T<T>::type df{}, rr{}, xx{}, dold{}, dn{}, bv{};
  if (owner) {
    df = ld4(dinvF, row);
    if (mode == 0) {
      dn = ld4(d_new, row);
    } else {
      rr = ld4(r, row);
      xx = ld4(x, row);
      dn = ld4(d_new, row);
      if constexpr (kFirst) bv = ld4(b0, row);
      else dold = ld4(d_old, row);
    }
  }
  if (row < A.V) {
    // two blocks per lane in flight; one in the first pass, whose two gathers per block (b0 and
    // diag(F)^-1) would otherwise take it to 66 registers and 3 CTAs per SM
    constexpr int U = kFirst ? 1 : LFX_U_F;
    T f[U][9];
    int32_t c[U];
    typename Vec4T<T>::type dv[U];
    row_blocks<U>(
        A.rowptr[row], A.rowptr[row + 1], lane,
        [&](int u, int32_t k) {
          ld_F(A, k, f[u]);
          c[u] = __ldg(A.col + k);
        },
        [&](int u) {
          if constexpr (kFirst) {
            const T s0 = coef_t<T>(cf->f_init, cf->f_initf);
            const auto dfc = ld4(dinvF, c[u]);
            const auto bc = ld4(b0, c[u]);
            dv[u].x = s0 * (dfc.x * bc.x);
            dv[u].y = s0 * (dfc.y * bc.y);
            dv[u].z = s0 * (dfc.z * bc.z);
          } else {
            dv[u] = ld4(d_old, c[u]);
          }
        },
        [&](int u) {
#pragma unroll
          for (int i = 0; i < 3; ++i) acc[i] += f[u][3 * i] * dv[u].x + f[u][3 * i + 1] * dv[u].y + f[u][3 * i + 2] * dv[u].z;
        });
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) acc[i] = group_sum(acc[i]);
  double nrm = 0.0;
  if (owner) {
    if (mode == 0) {
      auto o = dn;
      o.x = df.x * acc[0]; o.y = df.y * acc[1]; o.z = df.z * acc[2];
      st4(d_new, row, o);
      nrm = (double)o.x * o.x + (double)o.y * o.y + (double)o.z * o.z;
    } else {
      const T c1 = coef_t<T>(cf->f_c1[k], cf->f_c1f[k]), c2 = coef_t<T>(cf->f_c2[k], cf->f_c2f[k]);
      if constexpr (kFirst) {
        const T s0 = coef_t<T>(cf->f_init, cf->f_initf);
        rr.x = df.x * bv.x; rr.y = df.y * bv.y; rr.z = df.z * bv.z;
        dold.x = s0 * rr.x; dold.y = s0 * rr.y; dold.z = s0 * rr.z;
        xx.x = dold.x; xx.y = dold.y; xx.z = dold.z;
      }
      rr.x -= df.x * acc[0]; rr.y -= df.y * acc[1]; rr.z -= df.z * acc[2];
      dn.x = c1 * dold.x + c2 * rr.x; dn.y = c1 * dold.y + c2 * rr.y; dn.z = c1 * dold.z + c2 * rr.z;
      xx.x += dn.x; xx.y += dn.y; xx.z += dn.z;
      st4(r, row, rr);
      st4(d_new, row, dn);
      st4(x, row, xx);
    }
  }
  if (part) {
    double s = cta_sum(nrm);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
  }
}

// ------------------------------------------------------------------------------------------
// Staged velocity smoothing pass (BF16 sub-blocks).  The plain pass above waits, per lane, on a
// chain of small dependent loads (row pointer -> 24-byte record and column -> gathered iterate),
// which leaves HBM idle between them.  Here a persistent CTA walks row tiles (the mesh's table:
// at most kFTileRows rows and kFTileBlocks blocks each); one thread stages a whole tile's F records
// (the column index rides in each record's padding) into shared memory with one bulk asynchronous
// copy completing on an mbarrier, double-buffered, so that the next tile streams in while this one
// is processed.  Each lane then takes its row's blocks in the plain pass's order (the results are
// the same bit for bit).  Every wait is bounded (polls tries; a test passes 0): a wait that runs
// out sets *err, and the CTA waits (bounded again) for its copies in flight before it returns.
// ------------------------------------------------------------------------------------------
constexpr int kFTileThreads = kFTileRows * kRowGroup;
constexpr int64_t kFRec = 24;   // bytes of one BF16 F record (12 values)
constexpr uint32_t kFStageBytes = (uint32_t)(((kFTileBlocks * kFRec + 32) + 127) / 128 * 128);
constexpr size_t kFStagedSmem = 128 + 2 * (size_t)kFStageBytes;
constexpr uint32_t kFWaitPolls = 1u << 22;   // about 0.3 s of polls (32 ns sleeps) per wait

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
// bytes (a multiple of 16) from global src (16-byte aligned) to shared dst (16-byte aligned),
// completing on bar
__device__ __forceinline__ void bulk_to_smem(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint32_t polls) {
  for (uint32_t i = 0; i < polls; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    __nanosleep(32);
  }
  return false;
}

template <bool kFirst>
__global__ void __launch_bounds__(kFTileThreads) f_step_staged_kernel(
    SplitView<__nv_bfloat16> A, const int32_t *__restrict__ tile_row, int n_tiles, const float *dinvF,
    const float *d_old, float *d_new, float *r, float *x, const SmoothCoef *cf, int k, const KState *st,
    const float *b0, int *err, uint32_t polls) {
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
  unsigned char *stage0 = smem + 128;
  pdl_entry();
  if (finished(st)) return;
  const unsigned char *recs = reinterpret_cast<const unsigned char *>(A.F);
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init_fence();
  }
  __syncthreads();
  // thread 0: the records of tile t (whole 16-byte units around them) into buffer b
  auto issue = [&](int t, int b) {
    const int64_t k0 = A.rowptr[tile_row[t]], k1 = A.rowptr[tile_row[t + 1]];
    const int64_t a0 = (kFRec * k0) & ~(int64_t)15, a1 = (kFRec * k1 + 15) & ~(int64_t)15;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // the buffer's earlier reads before the copy
    mbar_expect_tx(&bar[b], (uint32_t)(a1 - a0));
    bulk_to_smem(stage0 + (size_t)b * kFStageBytes, recs + a0, (uint32_t)(a1 - a0), &bar[b]);
  };
  constexpr int U = 4;   // a row's blocks per lane gathered together (most rows: all of them)
  const float c1 = cf->f_c1f[k], c2 = cf->f_c2f[k], s0 = cf->f_initf;
  const int lane = threadIdx.x % kRowGroup;
  int j = 0, t = blockIdx.x;
  bool ok = true;
  if (threadIdx.x == 0 && t < n_tiles) issue(t, 0);
  for (; t < n_tiles; t += gridDim.x, ++j) {
    const int b = j & 1;
    // the row's own data first: its latency overlaps the wait for the staged records
    const int32_t r0 = tile_row[t], r1 = tile_row[t + 1];
    const int32_t row = r0 + (int32_t)(threadIdx.x / kRowGroup);
    const bool has = row < r1, owner = has && lane == 0;
    const int32_t kt = A.rowptr[r0];
    int32_t kb = 0, ke = 0;
    if (has) {
      kb = A.rowptr[row];
      ke = A.rowptr[row + 1];
    }
    F4 df{}, rr{}, xx{}, dn{}, dold{}, bv{};
    if (owner) {
      df = ld4(dinvF, row);
      rr = ld4(r, row);
      xx = ld4(x, row);
      dn = ld4(d_new, row);
      if constexpr (kFirst) bv = ld4(b0, row);
      else dold = ld4(d_old, row);
    }
    const bool got = mbar_wait_bounded(&bar[b], (uint32_t)(j >> 1) & 1u, polls);
    if (__syncthreads_or(!got)) {
      ok = false;
      break;
    }
    // past this barrier every thread is done with the previous tile: its buffer takes the next one
    if (threadIdx.x == 0 && t + (int)gridDim.x < n_tiles) issue(t + gridDim.x, b ^ 1);
    // record kk of the tile sits at rec + kFRec (kk - kt) (8-byte aligned)
    const unsigned char *rec = stage0 + (size_t)b * kFStageBytes + ((kFRec * kt) & 15);
    float acc[3] = {0.0f, 0.0f, 0.0f};
    for (int32_t kk = kb + lane; kk < ke; kk += U * kRowGroup) {
      uint2 w[U][3];
      F4 dv[U];
      bool v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        v[u] = kk + u * kRowGroup < ke;
        if (v[u]) {
          const uint2 *p = reinterpret_cast<const uint2 *>(rec + kFRec * (kk + u * kRowGroup - kt));
          w[u][0] = p[0];
          w[u][1] = p[1];
          w[u][2] = p[2];
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (!v[u]) continue;
        const int32_t c = (int32_t)((w[u][2].x >> 16) | (w[u][2].y << 16));
        if constexpr (kFirst) {
          const F4 dfc = ld4(dinvF, c), bc = ld4(b0, c);
          dv[u].x = s0 * (dfc.x * bc.x);
          dv[u].y = s0 * (dfc.y * bc.y);
          dv[u].z = s0 * (dfc.z * bc.z);
        } else {
          dv[u] = ld4(d_old, c);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (!v[u]) continue;
        float f[10];
        bf16x2_to_f32(w[u][0].x, f[0], f[1]);
        bf16x2_to_f32(w[u][0].y, f[2], f[3]);
        bf16x2_to_f32(w[u][1].x, f[4], f[5]);
        bf16x2_to_f32(w[u][1].y, f[6], f[7]);
        bf16x2_to_f32(w[u][2].x, f[8], f[9]);
#pragma unroll
        for (int i = 0; i < 3; ++i) acc[i] += f[3 * i] * dv[u].x + f[3 * i + 1] * dv[u].y + f[3 * i + 2] * dv[u].z;
      }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) acc[i] = group_sum(acc[i]);
    if (owner) {
      if constexpr (kFirst) {
        rr.x = df.x * bv.x; rr.y = df.y * bv.y; rr.z = df.z * bv.z;
        dold.x = s0 * rr.x; dold.y = s0 * rr.y; dold.z = s0 * rr.z;
        xx.x = dold.x; xx.y = dold.y; xx.z = dold.z;
      }
      rr.x -= df.x * acc[0]; rr.y -= df.y * acc[1]; rr.z -= df.z * acc[2];
      dn.x = c1 * dold.x + c2 * rr.x; dn.y = c1 * dold.y + c2 * rr.y; dn.z = c1 * dold.z + c2 * rr.z;
      xx.x += dn.x; xx.y += dn.y; xx.z += dn.z;
      st4(r, row, rr);
      st4(d_new, row, dn);
      st4(x, row, xx);
    }
  }
  if (!ok && threadIdx.x == 0) {
    atomicExch(err, 1);
    // the copy still in flight into this CTA's buffers: tile t's (the next one is issued only
    // after the wait for tile t)
    mbar_wait_bounded(&bar[j & 1], (uint32_t)(j >> 1) & 1u, kFWaitPolls);
  }
}

// w.xyz = dinvF (G p) with p = in.w   (velocity rows, pressure column)
template <class View, class T>
__global__ void __launch_bounds__(kThreads) g_scaled_kernel(View A, const T *dinvF, const T *in,
                                                            T *w, const KState *st) {
  pdl_entry();
  if (finished(st)) return;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kRowGroup;
  const int lane = threadIdx.x % kRowGroup;
  T acc[3] = {T(0), T(0), T(0)};
  if (row < A.V) {
    constexpr int U = LFX_U_GDC;
    T g[U][4], p[U];
    int32_t c[U];
    row_blocks<U>(
        A.rowptr[row], A.rowptr[row + 1], lane,
        [&](int u, int32_t k) {
          ld_G(A, k, g[u]);
          c[u] = __ldg(A.col + k);
        },
        [&](int u) { p[u] = in[4 * (int64_t)c[u] + 3]; },
        [&](int u) {
          acc[0] += g[u][0] * p[u];
          acc[1] += g[u][1] * p[u];
          acc[2] += g[u][2] * p[u];
        });
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) acc[i] = group_sum(acc[i]);
  if (row < A.V && lane == 0) {
    const auto df = ld4(dinvF, row);
    auto o = ld4(w, row);
    o.x = df.x * acc[0]; o.y = df.y * acc[1]; o.z = df.z * acc[2];
    st4(w, row, o);
  }
}

// Pressure smoothing step on S = C - D diag(F)^-1 G, with w.xyz = diag(F)^-1 G d_old.w given.
// mode 0 (power): y.w = dinvS (C v - D w), partial |y|^2.  mode 1: Chebyshev/Jacobi step.
template <class View, class T>
__global__ void __launch_bounds__(kThreads) s_step_kernel(View A, const T *dinvS, const T *d_old,
                                                          const T *w, T *d_new, T *r, T *x,
                                                          const SmoothCoef *cf, int k, int mode,
                                                          double *part, const KState *st) {
  pdl_entry();
  if (finished(st)) return;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kRowGroup;
  const int lane = threadIdx.x % kRowGroup;
  T acc = T(0);
  if (row < A.V) {
    constexpr int U = LFX_U_GDC;
    T dc[U][4], p[U];
    int32_t c[U];
    typename Vec4T<T>::type wv[U];
    row_blocks<U>(
        A.rowptr[row], A.rowptr[row + 1], lane,
        [&](int u, int32_t k) {
          ld_DC(A, k, dc[u]);
          c[u] = __ldg(A.col + k);
        },
        [&](int u) {
          p[u] = d_old[4 * (int64_t)c[u] + 3];
          wv[u] = ld4(w, c[u]);
        },
        [&](int u) { acc += dc[u][3] * p[u] - (dc[u][0] * wv[u].x + dc[u][1] * wv[u].y + dc[u][2] * wv[u].z); });
  }
  acc = group_sum(acc);
  double nrm = 0.0;
  if (row < A.V && lane == 0) {
    const T ds = dinvS[row];
    if (mode == 0) {
      auto o = ld4(d_new, row);
      o.w = ds * acc;
      st4(d_new, row, o);
      nrm = (double)o.w * o.w;
    } else {
      const T c1 = coef_t<T>(cf->s_c1[k], cf->s_c1f[k]), c2 = coef_t<T>(cf->s_c2[k], cf->s_c2f[k]);
      auto rr = ld4(r, row);
      const T dold = ld4(d_old, row).w;
      auto dn = ld4(d_new, row);
      auto xx = ld4(x, row);
      rr.w -= ds * acc;
      dn.w = c1 * dold + c2 * rr.w;
      xx.w += dn.w;
      st4(r, row, rr);
      st4(d_new, row, dn);
      st4(x, row, xx);
    }
  }
  if (part) {
    double s = cta_sum(nrm);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
  }
}

// Start of the velocity smoothing: r.xyz = dinvF b.xyz, d.xyz = init r.xyz, x.xyz = d.xyz
template <class T>
__global__ void f_init_kernel(int64_t V, const T *dinvF, const T *b, T *r, T *d, T *x,
                              const SmoothCoef *cf, const KState *st) {
  pdl_entry();
  if (finished(st)) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < V; i += (int64_t)gridDim.x * blockDim.x) {
    const T s = coef_t<T>(cf->f_init, cf->f_initf);
    const auto df = ld4(dinvF, i);
    const auto bv = ld4(b, i);
    auto rr = ld4(r, i);
    auto dd = ld4(d, i);
    auto xx = ld4(x, i);
    rr.x = df.x * bv.x; rr.y = df.y * bv.y; rr.z = df.z * bv.z;
    dd.x = s * rr.x; dd.y = s * rr.y; dd.z = s * rr.z;
    xx.x = dd.x; xx.y = dd.y; xx.z = dd.z;
    st4(r, i, rr);
    st4(d, i, dd);
    st4(x, i, xx);
  }
}

// t = b.w - D x.xyz, then start of the pressure smoothing: r.w = dinvS t, d.w = init r.w, x.w = d.w
template <class View, class T>
__global__ void __launch_bounds__(kThreads) d_init_kernel(View A, const T *dinvS, const T *b,
                                                          T *r, T *d, T *x, const SmoothCoef *cf,
                                                          const KState *st, T *bs) {
  pdl_entry();
  if (finished(st)) return;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kRowGroup;
  const int lane = threadIdx.x % kRowGroup;
  T acc = T(0);
  if (row < A.V) {
    constexpr int U = LFX_U_GDC;
    T dc[U][4];
    int32_t c[U];
    typename Vec4T<T>::type xv[U];
    row_blocks<U>(
        A.rowptr[row], A.rowptr[row + 1], lane,
        [&](int u, int32_t k) {
          ld_DC(A, k, dc[u]);
          c[u] = __ldg(A.col + k);
        },
        [&](int u) { xv[u] = ld4(x, c[u]); },
        [&](int u) { acc += dc[u][0] * xv[u].x + dc[u][1] * xv[u].y + dc[u][2] * xv[u].z; });
  }
  acc = group_sum(acc);
  if (row < A.V && lane == 0) {
    const T t = ld4(b, row).w - acc;
    if (bs) {
      auto o = ld4(bs, row);
      o.w = t;
      st4(bs, row, o);
    }
    auto rr = ld4(r, row);
    auto dd = ld4(d, row);
    rr.w = dinvS[row] * t;
    dd.w = coef_t<T>(cf->s_init, cf->s_initf) * rr.w;
    st4(r, row, rr);
    st4(d, row, dd);
    x[4 * row + 3] = dd.w;   // only the pressure component: the velocity part is read at neighbours
  }
}

// z.xyz = x.xyz - dinvF (G x.w), z.w = x.w
// kAddW: the iterate's pressure is read as x.w + dw.w (the pending update x.w += d.w of the
// Schur post-smoothing, left to this pass)
template <class View, class T, bool kAddW = false>
__global__ void __launch_bounds__(kThreads) final_kernel(View A, const T *dinvF, const T *x, T *z,
                                                         const KState *st, const T *dw) {
  pdl_entry();
  if (finished(st)) return;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kRowGroup;
  const int lane = threadIdx.x % kRowGroup;
  T acc[3] = {T(0), T(0), T(0)};
  if (row < A.V) {
    constexpr int U = LFX_U_GDC;
    T g[U][4], p[U];
    int32_t c[U];
    row_blocks<U>(
        A.rowptr[row], A.rowptr[row + 1], lane,
        [&](int u, int32_t k) {
          ld_G(A, k, g[u]);
          c[u] = __ldg(A.col + k);
        },
        [&](int u) {
          p[u] = x[4 * (int64_t)c[u] + 3];
          if constexpr (kAddW) p[u] += dw[4 * (int64_t)c[u] + 3];
        },
        [&](int u) {
          acc[0] += g[u][0] * p[u];
          acc[1] += g[u][1] * p[u];
          acc[2] += g[u][2] * p[u];
        });
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) acc[i] = group_sum(acc[i]);
  if (row < A.V && lane == 0) {
    const auto df = ld4(dinvF, row);
    auto xx = ld4(x, row);
    if constexpr (kAddW) xx.w += ld4(dw, row).w;
    typename Vec4T<T>::type o;
    o.x = xx.x - df.x * acc[0];
    o.y = xx.y - df.y * acc[1];
    o.z = xx.z - df.z * acc[2];
    o.w = xx.w;
    st4(z, row, o);
  }
}


// Level-0 Schur residual with w.xyz = diag(F)^-1 G x.w given:
//   mode 0: out[row] = bs.w - (C x.w - D w)                       (for restriction)
//   mode 1: r.w = dinvS (bs.w - (C x.w - D w)); d.w = init r.w     (post-smoothing start; the
//           iterate is read at the neighbours here, so x.w += d.w is a separate kernel)
template <class View, class T>
__global__ void __launch_bounds__(kThreads) s_resid_kernel(View A, const T *dinvS, T *x, const T *w,
                                                           const T *bs, T *out, T *r, T *d,
                                                           const SmoothCoef *cf, int mode, const KState *st) {
  pdl_entry();
  if (finished(st)) return;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kRowGroup;
  const int lane = threadIdx.x % kRowGroup;
  T acc = T(0);
  if (row < A.V) {
    constexpr int U = LFX_U_GDC;
    T dc[U][4], p[U];
    int32_t c[U];
    typename Vec4T<T>::type wv[U];
    row_blocks<U>(
        A.rowptr[row], A.rowptr[row + 1], lane,
        [&](int u, int32_t k) {
          ld_DC(A, k, dc[u]);
          c[u] = __ldg(A.col + k);
        },
        [&](int u) {
          p[u] = x[4 * (int64_t)c[u] + 3];
          wv[u] = ld4(w, c[u]);
        },
        [&](int u) { acc += dc[u][3] * p[u] - (dc[u][0] * wv[u].x + dc[u][1] * wv[u].y + dc[u][2] * wv[u].z); });
  }
  acc = group_sum(acc);
  if (row < A.V && lane == 0) {
    const T res = ld4(bs, row).w - acc;
    if (mode == 0) {
      out[row] = res;
    } else {
      auto rr = ld4(r, row);
      auto dd = ld4(d, row);
      rr.w = dinvS[row] * res;
      dd.w = coef_t<T>(cf->s_init, cf->s_initf) * rr.w;
      st4(r, row, rr);
      st4(d, row, dd);
    }
  }
}

// x.w += d.w (elementwise)
template <class T>
__global__ void add_w_kernel(int64_t V, const T *d, T *x, const KState *st) {
  pdl_entry();
  if (finished(st)) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < V; i += (int64_t)gridDim.x * blockDim.x) {
    auto xx = ld4(x, i);
    xx.w += ld4(d, i).w;
    st4(x, i, xx);
  }
}

// ---- explicit CSR levels of the Schur AMG (scalar unknowns).  Values are stored in the
// preconditioner's vector type T (FP32 for the mixed-precision inner solve, FP64 otherwise).
template <class VT>
struct CsrV {
  int64_t n;
  const int32_t *rp, *ci;
  const VT *v;
};

// sum_k v[k] x[ci[k]*is + io] over the row, G lanes per row (lane = position in the group),
// four nonzeros per lane in flight; the group's total is returned in every lane of the group.
// Lanes with valid == false add nothing but take part in the shuffles.
template <int G, class T>
__device__ __forceinline__ typename AccT<T>::type csr_row_dot(const int32_t *__restrict__ rp,
                                                              const int32_t *__restrict__ ci,
                                                              const T *__restrict__ v, const T *x, int is, int io,
                                                              int64_t row, int lane, bool valid) {
  using A = typename AccT<T>::type;
  A s = A(0);
  if (valid) {
    const int32_t k1 = __ldg(rp + row + 1);
    int32_t k = __ldg(rp + row) + lane;
    for (; k + 3 * G < k1; k += 4 * G) {
      int32_t c[4];
      T w[4], xv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        c[u] = __ldg(ci + k + u * G);
        w[u] = __ldg(v + k + u * G);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) xv[u] = x[(int64_t)c[u] * is + io];
#pragma unroll
      for (int u = 0; u < 4; ++u) s += (A)w[u] * (A)xv[u];
    }
    for (; k < k1; k += G) s += (A)__ldg(v + k) * (A)x[(int64_t)__ldg(ci + k) * is + io];
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// out[i*os + oo] = (acc ? out : 0) + alpha * sum_j M_ij in[j*is + io]
template <class T, int G>
__global__ void __launch_bounds__(kThreads) csr_spmv_kernel(CsrV<T> M, const T *in, int is, int io, T *out, int os,
                                                            int oo, typename AccT<T>::type alpha, int acc,
                                                            const KState *st) {
  pdl_entry();
  if (finished(st)) return;
  using A = typename AccT<T>::type;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int lane = threadIdx.x % G;
  const A s = csr_row_dot<G>(M.rp, M.ci, M.v, in, is, io, row, lane, row < M.n);
  if (row < M.n && lane == 0) {
    T *p = out + row * os + oo;
    *p = (T)((acc ? (A)*p : A(0)) + (A)alpha * s);
  }
}

// r = b - A x  (G lanes per row)
template <class T, int G>
__global__ void __launch_bounds__(kThreads) csr_resid_kernel(CsrV<T> M, const T *x, const T *b, T *out,
                                                             const KState *st) {
  pdl_entry();
  if (finished(st)) return;
  using A = typename AccT<T>::type;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int lane = threadIdx.x % G;
  const A s = csr_row_dot<G>(M.rp, M.ci, M.v, x, 1, 0, row, lane, row < M.n);
  if (row < M.n && lane == 0) out[row] = (T)((A)b[row] - s);
}

// Chebyshev start on a CSR level: r = dinv rhs; d = init r; x = (add ? x : 0) + d
template <class T>
__global__ void csr_cheb_init_kernel(int64_t n, const T *dinv, const T *rhs, T *r, T *d, T *x,
                                     typename AccT<T>::type init, int add,
                                     const KState *st) {
  pdl_entry();
  if (finished(st)) return;
  using A = typename AccT<T>::type;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const A rv = (A)dinv[i] * (A)rhs[i];
    const A dv = (A)init * rv;
    r[i] = (T)rv;
    d[i] = (T)dv;
    x[i] = (T)((add ? (A)x[i] : A(0)) + dv);
  }
}

// Chebyshev step on a CSR level: y = A d_old; r -= dinv y; d_new = c1 d_old + c2 r; x += d_new
template <class T, int G>
__global__ void __launch_bounds__(kThreads) csr_cheb_step_kernel(CsrV<T> M, const T *dinv, const T *d_old, T *d_new,
                                                                 T *r, T *x, typename AccT<T>::type c1,
                                                                 typename AccT<T>::type c2, const KState *st) {
  pdl_entry();
  if (finished(st)) return;
  using A = typename AccT<T>::type;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int lane = threadIdx.x % G;
  const A s = csr_row_dot<G>(M.rp, M.ci, M.v, d_old, 1, 0, row, lane, row < M.n);
  if (row < M.n && lane == 0) {
    const A rv = (A)r[row] - (A)dinv[row] * s;
    const A dv = (A)c1 * (A)d_old[row] + (A)c2 * rv;
    r[row] = (T)rv;
    d_new[row] = (T)dv;
    x[row] = (T)((A)x[row] + dv);
  }
}

// sum_k Minv[row][k] b[k*is+io] over one warp (eight columns per lane in flight)
template <class T>
__device__ __forceinline__ typename AccT<T>::type dense_row_dot(int64_t n, const T *__restrict__ Minv, const T *b,
                                                                int is, int io, int64_t row, int lane, bool valid) {
  using A = typename AccT<T>::type;
  A s = A(0);
  if (valid) {
    const T *m = Minv + row * n;
    int64_t k = lane;
    for (; k + 7 * 32 < n; k += 8 * 32) {
      T w[8], xv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        w[u] = __ldg(m + k + u * 32);
        xv[u] = b[(k + u * 32) * is + io];
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) s += (A)w[u] * (A)xv[u];
    }
    for (; k < n; k += 32) s += (A)__ldg(m + k) * (A)b[k * is + io];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// x[i*os+oo] = sum_k Minv[i][k] b[k*is+io]  (dense, n x n, row-major)
template <class T>
__global__ void __launch_bounds__(kThreads) dense_mv_kernel(int64_t n, const T *Minv, const T *b, int is, int io,
                                                            T *x, int os, int oo, const KState *st) {
  pdl_entry();
  if (finished(st)) return;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x % 32;
  const auto s = dense_row_dot(n, Minv, b, is, io, row, lane, row < n);
  if (row < n && lane == 0) x[row * os + oo] = (T)s;
}


// ---- the coarse part of the Schur AMG V-cycle (levels 1..L-1) in ONE cooperative launch:
// every phase is a grid-strided loop (a warp per matrix row), phases are separated by grid-wide
// barriers.  Replaces ~20 tiny launches per V-cycle whose cost is mostly launch latency.
template <class T>
struct CoarseLevel {
  int64_t n, nnext;
  const int32_t *rp, *ci;
  const T *v, *dinv;
  const int32_t *Prp, *Pci;
  const T *Pv;
  const int32_t *Rrp, *Rci;
  const T *Rv;
  T *x, *b, *r, *d0, *d1, *rr;
  T *xo;   // where the level's final iterate is left (d1 when one smoothing step is fused, else x)
  typename AccT<T>::type init, c1[kMaxSmooth], c2[kMaxSmooth];   // (converted on the host)
};
constexpr int kMaxCoarse = 8;
template <class T>
struct CoarseArgs {
  int L;            // levels in amg[] (level 0 is matrix-free and not part of this launch)
  int s_steps;
  typename AccT<T>::type alpha;
  const T *coarse_inv;
  int64_t nc;
  CoarseLevel<T> lv[kMaxCoarse];
};

template <class T>
__global__ void __launch_bounds__(kThreads) amg_coarse_kernel(const CoarseArgs<T> *__restrict__ args, const KState *st) {
  if (finished(st)) return;
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  using Ac = typename AccT<T>::type;
  const CoarseArgs<T> &A = *args;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  const int64_t gwarp = tid >> 5, nwarps = nthreads >> 5;
  const int lane = threadIdx.x & 31;
  // warp-per-row loops: every lane of a warp runs the same trip count, so the shuffles inside
  // the row dots always see the full warp
  auto rows_of = [&](int64_t n) { return (n + nwarps - 1) / nwarps; };
  auto cheb_init = [&](const CoarseLevel<T> &D, const T *rhs, int add) {
    for (int64_t i = tid; i < D.n; i += nthreads) {
      const Ac rv = (Ac)D.dinv[i] * (Ac)rhs[i];
      const Ac dv = (Ac)D.init * rv;
      D.r[i] = (T)rv;
      D.d0[i] = (T)dv;
      D.x[i] = (T)((add ? (Ac)D.x[i] : Ac(0)) + dv);
    }
  };
  auto cheb_steps = [&](const CoarseLevel<T> &D) {
    for (int k = 1; k < A.s_steps; ++k) {
      const T *dold = (k & 1) ? D.d0 : D.d1;
      T *dnew = (k & 1) ? D.d1 : D.d0;
      for (int64_t it = 0, row = gwarp; it < rows_of(D.n); ++it, row += nwarps) {
        const Ac s = csr_row_dot<32>(D.rp, D.ci, D.v, dold, 1, 0, row, lane, row < D.n);
        if (row < D.n && lane == 0) {
          const Ac rv = (Ac)D.r[row] - (Ac)D.dinv[row] * s;
          const Ac dv = (Ac)D.c1[k] * (Ac)dold[row] + (Ac)D.c2[k] * rv;
          D.r[row] = (T)rv;
          dnew[row] = (T)dv;
          D.x[row] = (T)((Ac)D.x[row] + dv);
        }
      }
      grid.sync();
    }
  };
  auto resid = [&](const CoarseLevel<T> &D) {
    for (int64_t it = 0, row = gwarp; it < rows_of(D.n); ++it, row += nwarps) {
      const Ac s = csr_row_dot<32>(D.rp, D.ci, D.v, D.x, 1, 0, row, lane, row < D.n);
      if (row < D.n && lane == 0) D.rr[row] = (T)((Ac)D.b[row] - s);
    }
  };
  const bool one = A.s_steps == 1;
  // down-sweep
  for (int l = 1; l < A.L - 1; ++l) {
    const CoarseLevel<T> &D = A.lv[l];
    if (one) {
      // x = init dinv b and rr = b - A x in one pass (x of a neighbour is formed from its b)
      for (int64_t it = 0, row = gwarp; it < rows_of(D.n); ++it, row += nwarps) {
        Ac s = Ac(0);
        const bool valid = row < D.n;
        if (valid) {
          const int32_t k1 = __ldg(D.rp + row + 1);
          for (int32_t k = __ldg(D.rp + row) + lane; k < k1; k += 32) {
            const int32_t c = __ldg(D.ci + k);
            s += (Ac)__ldg(D.v + k) * ((Ac)__ldg(D.dinv + c) * (Ac)D.b[c]);
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (valid && lane == 0) {
          const Ac bi = (Ac)D.b[row];
          D.x[row] = (T)((Ac)D.init * (Ac)D.dinv[row] * bi);
          D.rr[row] = (T)(bi - (Ac)D.init * s);
        }
      }
    } else {
      cheb_init(D, D.b, 0);
      grid.sync();
      cheb_steps(D);
      resid(D);
    }
    grid.sync();
    const CoarseLevel<T> &C = A.lv[l + 1];
    for (int64_t it = 0, row = gwarp; it < rows_of(D.nnext); ++it, row += nwarps) {
      const Ac s = csr_row_dot<32>(D.Rrp, D.Rci, D.Rv, D.rr, 1, 0, row, lane, row < D.nnext);
      if (row < D.nnext && lane == 0) C.b[row] = (T)s;
    }
    grid.sync();
  }
  // coarsest: dense inverse
  {
    const CoarseLevel<T> &C = A.lv[A.L - 1];
    for (int64_t it = 0, row = gwarp; it < rows_of(A.nc); ++it, row += nwarps) {
      const Ac s = dense_row_dot(A.nc, A.coarse_inv, C.b, 1, 0, row, lane, row < A.nc);
      if (row < A.nc && lane == 0) C.x[row] = (T)s;
    }
    grid.sync();
  }
  // up-sweep
  for (int l = A.L - 2; l >= 1; --l) {
    const CoarseLevel<T> &D = A.lv[l];
    const CoarseLevel<T> &C = A.lv[l + 1];
    const T *xc = (l + 1 == A.L - 1) ? C.x : C.xo;
    for (int64_t it = 0, row = gwarp; it < rows_of(D.n); ++it, row += nwarps) {
      const Ac s = csr_row_dot<32>(D.Prp, D.Pci, D.Pv, xc, 1, 0, row, lane, row < D.n);
      if (row < D.n && lane == 0) D.x[row] = (T)((Ac)D.x[row] + (Ac)A.alpha * s);
    }
    grid.sync();
    if (one) {
      // rr = b - A x and the smoothing step x_o = x + init dinv rr in one pass (into d1, since
      // other rows still read x)
      for (int64_t it = 0, row = gwarp; it < rows_of(D.n); ++it, row += nwarps) {
        const Ac s = csr_row_dot<32>(D.rp, D.ci, D.v, D.x, 1, 0, row, lane, row < D.n);
        if (row < D.n && lane == 0)
          D.xo[row] = (T)((Ac)D.x[row] + (Ac)D.init * (Ac)D.dinv[row] * ((Ac)D.b[row] - s));
      }
      if (l > 1) grid.sync();
    } else {
      resid(D);
      grid.sync();
      cheb_init(D, D.rr, 1);
      grid.sync();
      cheb_steps(D);
    }
  }
}

// power iteration helpers: v = (1/sqrt(n)) on the selected components; v = y / lambda
template <class T>
__global__ void fill_kernel(int64_t V, T *v, int comp_mask, double val) {
  pdl_entry();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < V; i += (int64_t)gridDim.x * blockDim.x) {
    auto o = ld4(v, i);
    if (comp_mask & 1) o.x = (T)val;
    if (comp_mask & 2) o.y = (T)val;
    if (comp_mask & 4) o.z = (T)val;
    if (comp_mask & 8) o.w = (T)val;
    st4(v, i, o);
  }
}
template <class T>
__global__ void div_kernel(int64_t V, const T *y, T *v, int comp_mask, const double *lam) {
  pdl_entry();
  const double il = 1.0 / *lam;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < V; i += (int64_t)gridDim.x * blockDim.x) {
    const auto a = ld4(y, i);
    auto o = ld4(v, i);
    if (comp_mask & 1) o.x = (T)((double)a.x * il);
    if (comp_mask & 2) o.y = (T)((double)a.y * il);
    if (comp_mask & 4) o.z = (T)((double)a.z * il);
    if (comp_mask & 8) o.w = (T)((double)a.w * il);
    st4(v, i, o);
  }
}

// Chebyshev coefficients (Saad, Chebyshev acceleration) from lambda_max estimates, or the
// constant Jacobi ones.
__global__ void coef_kernel(SmoothCoef *cf, int f_kind, int f_steps, double f_omega, double f_ratio,
                            int s_kind, int s_steps, double s_omega, double s_ratio, double safety) {
  pdl_entry();
  if (threadIdx.x != 0) return;
  for (int which = 0; which < 2; ++which) {
    const int kind = which ? s_kind : f_kind;
    const int steps = which ? s_steps : f_steps;
    const double omega = which ? s_omega : f_omega, ratio = which ? s_ratio : f_ratio;
    double *c1 = which ? cf->s_c1 : cf->f_c1;
    double *c2 = which ? cf->s_c2 : cf->f_c2;
    double init;
    if (kind == LFX_SMOOTH_JACOBI) {
      init = omega;
      for (int k = 0; k < steps; ++k) {
        c1[k] = 0.0;
        c2[k] = omega;
      }
    } else {
      const double lmax = safety * (which ? cf->lam_s : cf->lam_f);
      const double lmin = lmax / ratio;
      const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin);
      const double sigma1 = theta / delta;
      double rho = 1.0 / sigma1;
      init = 1.0 / theta;
      c1[0] = 0.0;
      c2[0] = 0.0;
      for (int k = 1; k < steps; ++k) {
        const double rn = 1.0 / (2.0 * sigma1 - rho);
        c1[k] = rn * rho;
        c2[k] = 2.0 * rn / delta;
        rho = rn;
      }
    }
    if (which) cf->s_init = init;
    else cf->f_init = init;
    float *c1f = which ? cf->s_c1f : cf->f_c1f;
    float *c2f = which ? cf->s_c2f : cf->f_c2f;
    for (int k = 0; k < kMaxSmooth; ++k) {
      c1f[k] = (float)c1[k];
      c2f[k] = (float)c2[k];
    }
    if (which) cf->s_initf = (float)init;
    else cf->f_initf = (float)init;
  }
}

// ------------------------------------------------------------------------------------------
// Krylov kernels
// ------------------------------------------------------------------------------------------
// part[i][blk] = this CTA's share of w . v_i, i < nvec.  Vectors are read four values at a time
// in a grid-strided (coalesced) order; eight basis vectors per pass over w.
template <class T>
__global__ void __launch_bounds__(kThreads) mdot_kernel(const T *Vb, int64_t ld, int nvec, const T *w,
                                                        int64_t n, double *part, int ldp,
                                                        const KState *st) {
  pdl_entry();
  if (finished(st)) return;
  using V4 = typename Vec4T<T>::type;
  __shared__ double red[8][kThreads / 32];
  const int64_t n4 = n >> 2, ld4 = ld >> 2;
  const V4 *w4 = reinterpret_cast<const V4 *>(w);
  const V4 *b4 = reinterpret_cast<const V4 *>(Vb);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  using A = typename AccT<T>::type;
  // blockIdx.y selects a group of eight basis vectors, so every group is read concurrently
  const int v0 = 8 * blockIdx.y;
  if (v0 >= nvec) return;
  A acc[8] = {A(0), A(0), A(0), A(0), A(0), A(0), A(0), A(0)};
  const int nv = min(8, nvec - v0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
    const V4 wv = w4[i];
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (k < nv) {
        const V4 b = b4[(int64_t)(v0 + k) * ld4 + i];
        acc[k] += (A)wv.x * (A)b.x + (A)wv.y * (A)b.y + (A)wv.z * (A)b.z + (A)wv.w * (A)b.w;
      }
  }
  // warp sums in the accumulator type (FP64 adds on every lane would bound the FP32 kernel)
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    A a = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) red[k][warp] = (double)a;
  }
  __syncthreads();
  if ((int)threadIdx.x < nv) {
    double s = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[threadIdx.x][q];
    part[(int64_t)(v0 + threadIdx.x) * ldp + blockIdx.x] = s;   // [vector][block]
  }
}

// h[i] = sum_blk part[i][blk]; hcol[i] (+)= h[i]; hwork[i] = h[i].  One warp per vector i.
__global__ void mdot_finalize_kernel(const double *part, int nblk, int ldp, int nvec, KState *st,
                                     int accumulate) {
  pdl_entry();
  if (finished(st)) return;
  const int i = blockIdx.x;
  if (i >= nvec) return;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += 32) s += part[(int64_t)i * ldp + b];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (threadIdx.x == 0) {
    st->hwork[i] = s;
    st->hcol[i] = accumulate ? st->hcol[i] + s : s;
  }
}

// w -= sum_i hwork[i] v_i ; partial |w|^2 (four values per load, grid-strided)
template <class T>
__global__ void __launch_bounds__(kThreads) maxpy_kernel(const T *Vb, int64_t ld, int nvec, T *w,
                                                         int64_t n, double *part, KState *st) {
  pdl_entry();
  if (finished(st)) return;
  using V4 = typename Vec4T<T>::type;
  using A = typename AccT<T>::type;
  __shared__ A h[kMaxRestart + 1];
  for (int i = threadIdx.x; i < nvec; i += blockDim.x) h[i] = (A)st->hwork[i];
  __syncthreads();
  const int64_t n4 = n >> 2, ld4 = ld >> 2;
  V4 *w4 = reinterpret_cast<V4 *>(w);
  const V4 *b4 = reinterpret_cast<const V4 *>(Vb);
  A nrm_t = A(0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
    const V4 wv = w4[i];
    A a0 = (A)wv.x, a1 = (A)wv.y, a2 = (A)wv.z, a3 = (A)wv.w;
#pragma unroll 4
    for (int k = 0; k < nvec; ++k) {
      const V4 b = b4[(int64_t)k * ld4 + i];
      const A hk = h[k];
      a0 -= hk * (A)b.x;
      a1 -= hk * (A)b.y;
      a2 -= hk * (A)b.z;
      a3 -= hk * (A)b.w;
    }
    V4 o;
    o.x = (T)a0;
    o.y = (T)a1;
    o.z = (T)a2;
    o.w = (T)a3;
    w4[i] = o;
    nrm_t += a0 * a0 + a1 * a1 + a2 * a2 + a3 * a3;
  }
  double s = cta_sum_t(nrm_t);
  if (threadIdx.x == 0 && part) part[blockIdx.x] = s;
}

// Arnoldi column j: h_{j+1,j} = ||w||, Givens rotations, residual estimate, stopping test.
__global__ void givens_kernel(const double *part, int nblk, KState *st, int j, int m, int maxit) {
  pdl_entry();
  if (finished(st)) return;
  // the new Hessenberg column and the earlier rotations, staged in shared memory by every thread:
  // the rotations then run on one thread from shared memory rather than through global memory
  __shared__ double h[kMaxRestart + 2], cs[kMaxRestart], sn_[kMaxRestart];
  for (int i = threadIdx.x; i <= j; i += blockDim.x) h[i] = st->hcol[i];
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    cs[i] = st->cs[i];
    sn_[i] = st->sn[i];
  }
  double s = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) s += part[i];
  s = cta_sum(s);
  __syncthreads();
  double *H = st->H + (int64_t)j * (kMaxRestart + 1);
  const double hn = sqrt(s);
  if (threadIdx.x == 0) {
    h[j + 1] = hn;
    for (int i = 0; i < j; ++i) {
      const double t = cs[i] * h[i] + sn_[i] * h[i + 1];
      h[i + 1] = -sn_[i] * h[i] + cs[i] * h[i + 1];
      h[i] = t;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < j; i += blockDim.x) H[i] = h[i];
  if (threadIdx.x != 0) return;
  const double den = hypot(h[j], h[j + 1]);
  double c = 1.0, sn = 0.0;
  if (den > 0.0) {
    c = h[j] / den;
    sn = h[j + 1] / den;
  }
  st->cs[j] = c;
  st->sn[j] = sn;
  H[j] = den;
  H[j + 1] = 0.0;
  st->g[j + 1] = -sn * st->g[j];
  st->g[j] = c * st->g[j];
  const double res = fabs(st->g[j + 1]);
  st->j = j + 1;
  st->total += 1;
  st->res = res;
  st->scale = hn > 0.0 ? 1.0 / hn : 0.0;
  if (!isfinite(res) || !isfinite(hn)) {
    st->flag = 2;
    st->done = 1;
  } else if (res <= st->tol_abs || hn == 0.0) {
    st->flag = 1;
    st->done = 1;
  } else if (j + 1 >= m || st->total >= maxit) {
    st->done = 1;
  }
}

template <class A, class B>
__global__ void convert_kernel(const A *src, B *dst, int64_t n, const KState *st) {
  pdl_entry();
  if (finished(st)) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (B)src[i];
}
template <>
__global__ void convert_kernel<double, __nv_bfloat16>(const double *src, __nv_bfloat16 *dst, int64_t n,
                                                      const KState *st) {
  pdl_entry();
  if (finished(st)) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = __double2bfloat16(src[i]);
}

template <class T>
__global__ void norm_kernel(const T *v, int64_t n, double *part) {
  pdl_entry();
  using A = typename AccT<T>::type;
  A a = A(0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a += (A)v[i] * (A)v[i];
  double s = cta_sum_t(a);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

template <class T>
__global__ void scale_kernel(const T *w, T *v, int64_t n, const double *sc, const KState *st) {
  pdl_entry();
  if (finished(st)) return;
  using A = typename AccT<T>::type;
  const A s = (A)*sc;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = (T)((A)w[i] * s);
}
// variant used at the start of a cycle (no early exit): v0 = r / beta
template <class T>
__global__ void scale_beta_kernel(const T *w, T *v, int64_t n, const KState *st) {
  pdl_entry();
  using A = typename AccT<T>::type;
  const double b = st->beta;
  const A s = (A)(b > 0.0 ? 1.0 / b : 0.0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = (T)((A)w[i] * s);
}

// start of a cycle: beta = ||r||, g = (beta, 0, ...), j = 0, done if beta <= tol
__global__ void cycle_start_kernel(const double *part, int nblk, KState *st) {
  pdl_entry();
  double s = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) s += part[i];
  s = cta_sum(s);
  if (threadIdx.x != 0) return;
  const double beta = sqrt(s);
  st->beta = beta;
  st->g[0] = beta;
  st->j = 0;
  st->res = beta;
  st->flag = 0;
  st->done = 0;
  if (!isfinite(beta)) {
    st->flag = 2;
    st->done = 1;
  } else if (beta <= st->tol_abs) {
    st->flag = 1;
    st->done = 1;
  }
}

// Start of a solve: ||b|| from the partial sums, the tolerance rtol ||b||, the step count.
__global__ void solve_start_kernel(const double *part, int nblk, KState *st, double rtol) {
  pdl_entry();
  double s = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) s += part[i];
  s = cta_sum(s);
  if (threadIdx.x != 0) return;
  const double bnorm = sqrt(s);
  st->bnorm = bnorm;
  st->tol_abs = rtol * bnorm;
  st->total = 0;
}

// x = 0 when *bnorm == 0 (the solution of A x = 0)
template <class T>
__global__ void zero_if_b_zero_kernel(T *x, int64_t n, const double *bnorm) {
  pdl_entry();
  if (*bnorm != 0.0) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = T(0);
}

// Start of an inner solve from x = 0 (r = b): ||b|| from the partial sums, the tolerance
// eta ||b|| (eta = rtol, or from the outer flexible solve's status: 1/2 sqrt(tol / r) at its
// cycle's first step, 1/2 tol / r after, within [lo, hi]), beta = ||b||, g = (beta, 0, ...).
__global__ void inner_start_kernel(const double *part, int nblk, KState *st, const KState *outer, double rtol,
                                   double lo, double hi) {
  pdl_entry();
  double s = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) s += part[i];
  s = cta_sum(s);
  if (threadIdx.x != 0) return;
  const double beta = sqrt(s);
  double eta = rtol;
  if (outer != nullptr) {
    eta = hi;
    const double r = outer->res, tol = outer->tol_abs;
    if (r > 0.0 && tol > 0.0 && isfinite(r)) {
      const double need = tol / r;
      eta = fmin(hi, 0.5 * (outer->j == 0 ? sqrt(need) : need));
    }
    eta = fmax(lo, eta);
  }
  st->bnorm = beta;
  st->tol_abs = eta * beta;
  st->total = 0;
  st->beta = beta;
  st->g[0] = beta;
  st->j = 0;
  st->res = beta;
  st->flag = 0;
  st->done = 0;
  if (!isfinite(beta)) {
    st->flag = 2;
    st->done = 1;
  } else if (beta <= st->tol_abs) {   // b = 0: x = 0 is the solution
    st->flag = 1;
    st->done = 1;
  }
}

// y = H(0:j,0:j)^-1 g(0:j) by back substitution (j = completed steps of this cycle)
// y = R^-1 g for the j x j upper-triangular R of the rotated Hessenberg matrix (column k of R is
// H[k][0..k]): one warp; R and g staged in shared memory, each back-substitution row's sum over the
// solved unknowns split over the lanes
__global__ void trisolve_kernel(KState *st) {
  pdl_entry();
  __shared__ double R[kMaxRestart][kMaxRestart + 1];
  __shared__ double y[kMaxRestart], g[kMaxRestart];
  const int j = st->j;
  const int lane = threadIdx.x & 31;
  for (int idx = threadIdx.x; idx < j * j; idx += blockDim.x) {
    const int k = idx / j, i = idx % j;
    if (i <= k) R[k][i] = st->H[(int64_t)k * (kMaxRestart + 1) + i];
  }
  for (int i = threadIdx.x; i < j; i += blockDim.x) g[i] = st->g[i];
  __syncthreads();
  if (threadIdx.x < 32) {
    for (int i = j - 1; i >= 0; --i) {
      double part = 0.0;
      for (int k = i + 1 + lane; k < j; k += 32) part += R[k][i] * y[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
      if (lane == 0) {
        const double d = R[i][i];
        y[i] = d != 0.0 ? (g[i] - part) / d : 0.0;   // d = 0 only after a breakdown (w = 0)
      }
      __syncwarp();
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < j; i += blockDim.x) st->y[i] = y[i];
}

// x += sum_{i<j} y_i z_i
template <class T, class X>
__global__ void update_x_kernel(const T *Zb, int64_t ld, X *x, int64_t n, const KState *st) {
  pdl_entry();
  using A = typename AccT<T, X>::type;
  __shared__ A y[kMaxRestart];
  const int j = st->j;
  for (int i = threadIdx.x; i < j; i += blockDim.x) y[i] = (A)st->y[i];
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    A a = (A)x[i];
#pragma unroll 4
    for (int k = 0; k < j; ++k) a += y[k] * (A)Zb[(int64_t)k * ld + i];
    x[i] = (X)a;
  }
}

// ------------------------------------------------------------------------------------------
// Segmented Krylov kernels.  A batch of independent problems (the connected components of a
// batched mesh: contiguous node ranges, a block-diagonal matrix) runs one Arnoldi process per
// component in lockstep: every component has its own Hessenberg matrix, rotations, tolerance
// and convergence test, exactly as if it were solved alone.  Reductions run over "tasks",
// node ranges of at most kSegNodes nodes inside one component, one CTA each; a component that
// has converged carries zero basis vectors until the shared status word ks0 (read by every
// kernel for early exit, preconditioner included) says that all components have finished.
// ------------------------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(kThreads) seg_norm_kernel(const T *v, SegTasks tk, double *pn, const KState *st) {
  pdl_entry();
  if (finished(st)) return;
  using V4 = typename Vec4T<T>::type;
  using A = typename AccT<T>::type;
  const int t = blockIdx.x;
  const V4 *v4 = reinterpret_cast<const V4 *>(v);
  A a = A(0);
  for (int64_t i = tk.lo[t] + threadIdx.x; i < tk.hi[t]; i += blockDim.x) {
    const V4 q = v4[i];
    a += (A)q.x * (A)q.x + (A)q.y * (A)q.y + (A)q.z * (A)q.z + (A)q.w * (A)q.w;
  }
  const double s = cta_sum_t(a);
  if (threadIdx.x == 0) pn[t] = s;
}

__device__ __forceinline__ double seg_sum(const double *pn, const SegTasks &tk, int c) {
  double s = 0.0;
  for (int t = tk.task_off[c]; t < tk.task_off[c + 1]; ++t) s += pn[t];
  return s;
}

// ||b_c|| and tol_c = rtol ||b_c|| per component; ks0 gets ||b|| over all components
__global__ void seg_bnorm_kernel(const double *pn, SegTasks tk, KState *kseg, KState *ks0, double rtol) {
  pdl_entry();
  __shared__ double tot[kThreads];
  double mine = 0.0;
  for (int c = threadIdx.x; c < tk.n_seg; c += blockDim.x) {
    const double s = seg_sum(pn, tk, c);
    mine += s;
    kseg[c].bnorm = sqrt(s);
    kseg[c].tol_abs = rtol * sqrt(s);
    kseg[c].total = 0;
  }
  tot[threadIdx.x] = mine;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < (int)blockDim.x; ++i) s += tot[i];
    ks0->bnorm = sqrt(s);
    ks0->tol_abs = rtol * sqrt(s);
    ks0->total = 0;
    ks0->done = 0;
    ks0->flag = 0;
  }
}

// x_c = 0 for components with b_c = 0 (their solution), so that they start converged
template <class X>
__global__ void __launch_bounds__(kThreads) seg_zero_x_kernel(X *x, SegTasks tk, const KState *kseg) {
  pdl_entry();
  const int t = blockIdx.x;
  if (kseg[tk.seg[t]].bnorm != 0.0) return;
  for (int64_t e = 4 * tk.lo[t] + threadIdx.x; e < 4 * tk.hi[t]; e += blockDim.x) x[e] = X(0);
}

// start of a cycle: beta_c = ||r_c||, g_c = (beta_c, 0, ...), j_c = 0, done_c if beta_c <= tol_c
__global__ void seg_cycle_start_kernel(const double *pn, SegTasks tk, KState *kseg, KState *ks0) {
  pdl_entry();
  __shared__ int all_done, any_bad;
  if (threadIdx.x == 0) {
    all_done = 1;
    any_bad = 0;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < tk.n_seg; c += blockDim.x) {
    KState &k = kseg[c];
    const double beta = sqrt(seg_sum(pn, tk, c));
    k.beta = beta;
    k.g[0] = beta;
    k.j = 0;
    k.res = beta;
    k.flag = 0;
    k.done = 0;
    k.scale = 0.0;
    if (!isfinite(beta)) {
      k.flag = 2;
      k.done = 1;
      atomicExch(&any_bad, 1);
    } else if (beta <= k.tol_abs) {
      k.flag = 1;
      k.done = 1;
    }
    if (!k.done) atomicExch(&all_done, 0);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    ks0->j = 0;
    ks0->flag = any_bad ? 2 : (all_done ? 1 : 0);
    ks0->done = (all_done || any_bad) ? 1 : 0;
  }
}

// v = r / beta_c over each task's nodes (zero for components that start converged)
template <class T>
__global__ void __launch_bounds__(kThreads) seg_scale_beta_kernel(const T *w, T *v, SegTasks tk, const KState *kseg) {
  pdl_entry();
  using V4 = typename Vec4T<T>::type;
  using A = typename AccT<T>::type;
  const int t = blockIdx.x;
  const KState &k = kseg[tk.seg[t]];
  const A s = (A)((k.done || !(k.beta > 0.0)) ? 0.0 : 1.0 / k.beta);
  const V4 *w4 = reinterpret_cast<const V4 *>(w);
  V4 *v4 = reinterpret_cast<V4 *>(v);
  for (int64_t i = tk.lo[t] + threadIdx.x; i < tk.hi[t]; i += blockDim.x) {
    const V4 q = w4[i];
    V4 o;
    o.x = (T)((A)q.x * s);
    o.y = (T)((A)q.y * s);
    o.z = (T)((A)q.z * s);
    o.w = (T)((A)q.w * s);
    v4[i] = o;
  }
}

// part[i][task] = the task's share of w . v_i, i < nvec; blockIdx.y selects eight vectors
template <class T>
__global__ void __launch_bounds__(kThreads) seg_mdot_kernel(const T *Vb, int64_t ld, int nvec, const T *w,
                                                            double *part, SegTasks tk, const KState *st) {
  pdl_entry();
  if (finished(st)) return;
  using V4 = typename Vec4T<T>::type;
  using A = typename AccT<T>::type;
  __shared__ double red[8][kThreads / 32];
  const int t = blockIdx.x, v0 = 8 * blockIdx.y;
  if (v0 >= nvec) return;
  const int nv = min(8, nvec - v0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t ld4 = ld >> 2;
  const V4 *w4 = reinterpret_cast<const V4 *>(w);
  const V4 *b4 = reinterpret_cast<const V4 *>(Vb);
  A acc[8] = {A(0), A(0), A(0), A(0), A(0), A(0), A(0), A(0)};
  for (int64_t i = tk.lo[t] + threadIdx.x; i < tk.hi[t]; i += blockDim.x) {
    const V4 wv = w4[i];
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (k < nv) {
        const V4 b = b4[(int64_t)(v0 + k) * ld4 + i];
        acc[k] += (A)wv.x * (A)b.x + (A)wv.y * (A)b.y + (A)wv.z * (A)b.z + (A)wv.w * (A)b.w;
      }
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    A a = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) red[k][warp] = (double)a;
  }
  __syncthreads();
  if ((int)threadIdx.x < nv) {
    double s = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[threadIdx.x][q];
    part[(int64_t)(v0 + threadIdx.x) * tk.n_task + t] = s;
  }
}

// h_c[i] = sum of component c's task shares; hcol (+)= h, hwork = h.  One warp per (c, i).
__global__ void seg_finalize_kernel(const double *part, int nvec, SegTasks tk, KState *kseg, const KState *st,
                                    int accumulate) {
  pdl_entry();
  if (finished(st)) return;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (gw >= (int64_t)tk.n_seg * nvec) return;
  const int c = (int)(gw / nvec), i = (int)(gw % nvec);
  double s = 0.0;
  for (int t = tk.task_off[c] + lane; t < tk.task_off[c + 1]; t += 32) s += part[(int64_t)i * tk.n_task + t];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    kseg[c].hwork[i] = s;
    kseg[c].hcol[i] = accumulate ? kseg[c].hcol[i] + s : s;
  }
}

// w -= sum_i h_c[i] v_i over each task's nodes; the task's share of |w|^2
template <class T>
__global__ void __launch_bounds__(kThreads) seg_maxpy_kernel(const T *Vb, int64_t ld, int nvec, T *w, SegTasks tk,
                                                             const KState *kseg, double *pn, const KState *st) {
  pdl_entry();
  if (finished(st)) return;
  using V4 = typename Vec4T<T>::type;
  using A = typename AccT<T>::type;
  __shared__ A h[kMaxRestart + 1];
  const int t = blockIdx.x;
  const KState &kc = kseg[tk.seg[t]];
  for (int i = threadIdx.x; i < nvec; i += blockDim.x) h[i] = (A)kc.hwork[i];
  __syncthreads();
  const int64_t ld4 = ld >> 2;
  V4 *w4 = reinterpret_cast<V4 *>(w);
  const V4 *b4 = reinterpret_cast<const V4 *>(Vb);
  A nrm = A(0);
  for (int64_t i = tk.lo[t] + threadIdx.x; i < tk.hi[t]; i += blockDim.x) {
    const V4 wv = w4[i];
    A a0 = (A)wv.x, a1 = (A)wv.y, a2 = (A)wv.z, a3 = (A)wv.w;
#pragma unroll 4
    for (int k = 0; k < nvec; ++k) {
      const V4 b = b4[(int64_t)k * ld4 + i];
      const A hk = h[k];
      a0 -= hk * (A)b.x;
      a1 -= hk * (A)b.y;
      a2 -= hk * (A)b.z;
      a3 -= hk * (A)b.w;
    }
    V4 o;
    o.x = (T)a0;
    o.y = (T)a1;
    o.z = (T)a2;
    o.w = (T)a3;
    w4[i] = o;
    nrm += a0 * a0 + a1 * a1 + a2 * a2 + a3 * a3;
  }
  const double s = cta_sum_t(nrm);
  if (threadIdx.x == 0) pn[t] = s;
}

// Arnoldi column j of every running component: h_{j+1,j} = ||w_c||, Givens rotations, residual
// estimate and stopping test; ks0 finishes when every component has, or at the restart length
// or the step limit.
__global__ void seg_givens_kernel(const double *pn, SegTasks tk, KState *kseg, KState *ks0, int j, int m, int maxit) {
  pdl_entry();
  if (finished(ks0)) return;
  __shared__ int all_done, any_bad;
  if (threadIdx.x == 0) {
    all_done = 1;
    any_bad = 0;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < tk.n_seg; c += blockDim.x) {
    KState &k = kseg[c];
    if (k.done) {
      k.scale = 0.0;
      continue;
    }
    const double hn = sqrt(seg_sum(pn, tk, c));
    double *H = k.H + (int64_t)j * (kMaxRestart + 1);
    for (int i = 0; i <= j; ++i) H[i] = k.hcol[i];
    H[j + 1] = hn;
    for (int i = 0; i < j; ++i) {
      const double q = k.cs[i] * H[i] + k.sn[i] * H[i + 1];
      H[i + 1] = -k.sn[i] * H[i] + k.cs[i] * H[i + 1];
      H[i] = q;
    }
    const double den = hypot(H[j], H[j + 1]);
    double cc = 1.0, sn = 0.0;
    if (den > 0.0) {
      cc = H[j] / den;
      sn = H[j + 1] / den;
    }
    k.cs[j] = cc;
    k.sn[j] = sn;
    H[j] = den;
    H[j + 1] = 0.0;
    k.g[j + 1] = -sn * k.g[j];
    k.g[j] = cc * k.g[j];
    const double res = fabs(k.g[j + 1]);
    k.j = j + 1;
    k.total += 1;
    k.res = res;
    k.scale = hn > 0.0 ? 1.0 / hn : 0.0;
    if (!isfinite(res) || !isfinite(hn)) {
      k.flag = 2;
      k.done = 1;
      atomicExch(&any_bad, 1);
    } else if (res <= k.tol_abs || hn == 0.0) {
      k.flag = 1;
      k.done = 1;
    }
    if (k.done) k.scale = 0.0;
    else atomicExch(&all_done, 0);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    ks0->j = j + 1;
    ks0->total += 1;
    ks0->flag = any_bad ? 2 : (all_done ? 1 : 0);
    if (all_done || any_bad || j + 1 >= m || ks0->total >= maxit) ks0->done = 1;
  }
}

// v_{j+1} = w scale_c (zero for components that have finished)
template <class T>
__global__ void __launch_bounds__(kThreads) seg_scale_kernel(const T *w, T *v, SegTasks tk, const KState *kseg,
                                                             const KState *st) {
  pdl_entry();
  if (finished(st)) return;
  using V4 = typename Vec4T<T>::type;
  using A = typename AccT<T>::type;
  const int t = blockIdx.x;
  const A s = (A)kseg[tk.seg[t]].scale;
  const V4 *w4 = reinterpret_cast<const V4 *>(w);
  V4 *v4 = reinterpret_cast<V4 *>(v);
  for (int64_t i = tk.lo[t] + threadIdx.x; i < tk.hi[t]; i += blockDim.x) {
    const V4 q = w4[i];
    V4 o;
    o.x = (T)((A)q.x * s);
    o.y = (T)((A)q.y * s);
    o.z = (T)((A)q.z * s);
    o.w = (T)((A)q.w * s);
    v4[i] = o;
  }
}

// y_c = H_c(0:j_c, 0:j_c)^-1 g_c by back substitution, one thread per component
__global__ void seg_trisolve_kernel(SegTasks tk, KState *kseg) {
  pdl_entry();
  for (int c = threadIdx.x; c < tk.n_seg; c += blockDim.x) {
    KState &k = kseg[c];
    const int j = k.j;
    for (int i = j - 1; i >= 0; --i) {
      double s = k.g[i];
      for (int q = i + 1; q < j; ++q) s -= k.H[(int64_t)q * (kMaxRestart + 1) + i] * k.y[q];
      const double d = k.H[(int64_t)i * (kMaxRestart + 1) + i];
      k.y[i] = d != 0.0 ? s / d : 0.0;   // d = 0 only after a breakdown (w = 0)
    }
  }
}

// x += sum_{i < j_c} y_c[i] z_i over each task's nodes
template <class T, class X>
__global__ void __launch_bounds__(kThreads) seg_update_x_kernel(const T *Zb, int64_t ld, X *x, SegTasks tk,
                                                                const KState *kseg) {
  pdl_entry();
  using A = typename AccT<T, X>::type;
  __shared__ A y[kMaxRestart];
  const int t = blockIdx.x;
  const KState &k = kseg[tk.seg[t]];
  const int j = k.j;
  for (int i = threadIdx.x; i < j; i += blockDim.x) y[i] = (A)k.y[i];
  __syncthreads();
  for (int64_t e = 4 * tk.lo[t] + threadIdx.x; e < 4 * tk.hi[t]; e += blockDim.x) {
    A a = (A)x[e];
#pragma unroll 4
    for (int i = 0; i < j; ++i) a += y[i] * (A)Zb[(int64_t)i * ld + e];
    x[e] = (X)a;
  }
}

// true residual per component (pn = task shares of |b - A x|^2): ks0->res = the largest
// ||r_c|| / ||b_c||, ks0->flag = 1 if every ||r_c|| <= 2 tol_c
__global__ void seg_confirm_kernel(const double *pn, SegTasks tk, const KState *kseg, KState *ks0) {
  pdl_entry();
  __shared__ double worst[kThreads];
  __shared__ int all_ok, any_bad;
  if (threadIdx.x == 0) {
    all_ok = 1;
    any_bad = 0;
  }
  __syncthreads();
  double w = 0.0;
  for (int c = threadIdx.x; c < tk.n_seg; c += blockDim.x) {
    const double tr = sqrt(seg_sum(pn, tk, c));
    const double b = kseg[c].bnorm;
    if (!isfinite(tr)) atomicExch(&any_bad, 1);
    if (!(tr <= 2.0 * kseg[c].tol_abs)) atomicExch(&all_ok, 0);
    if (b > 0.0) w = fmax(w, tr / b);
  }
  worst[threadIdx.x] = w;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int i = 0; i < (int)blockDim.x; ++i) m = fmax(m, worst[i]);
    ks0->res = any_bad ? NAN : m;
    ks0->flag = all_ok;
  }
}

// s[t] = w_t . x over the nodes of tag t (one CTA per tag)
template <class T>
__global__ void __launch_bounds__(kThreads) rank1_dot_kernel(Rank1View r, const T *x, double *s, const KState *st) {
  pdl_entry();
  if (finished(st)) return;
  const int t = blockIdx.x;
  double a = 0.0;
  for (int32_t k = r.dot_off[t] + threadIdx.x; k < r.dot_off[t + 1]; k += blockDim.x) {
    const int64_t nd = r.dot_node[k];
#pragma unroll
    for (int i = 0; i < 3; ++i) a += r.dot_w[3 * (int64_t)k + i] * (double)x[4 * nd + i];
  }
  a = cta_sum(a);
  if (threadIdx.x == 0) s[t] = a;
}

// y_row += sign cr[t] s[t] w_row over the listed rows
template <class T>
__global__ void rank1_axpy_kernel(Rank1View r, const double *s, T *y, double sign, const KState *st) {
  pdl_entry();
  if (finished(st)) return;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < r.n_ax; k += (int64_t)gridDim.x * blockDim.x) {
    const int t = r.ax_tag[k];
    const double c = sign * r.cr[t] * s[t];
    const int64_t nd = r.ax_node[k];
#pragma unroll
    for (int i = 0; i < 3; ++i) y[4 * nd + i] = (T)((double)y[4 * nd + i] + c * r.ax_w[3 * k + i]);
  }
}

inline int rows_grid(int64_t V) { return (int)((V * kRowGroup + kThreads - 1) / kThreads); }
// grid for a CSR kernel with G lanes per row over n rows
inline int lanes_grid(int64_t n, int G) { return (int)std::max<int64_t>(1, (n * G + kThreads - 1) / kThreads); }
inline int vec_grid(int64_t n) {
  int64_t g = (n + kThreads - 1) / kThreads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 8));
}

}  // namespace

// ==========================================================================================
// host side
// ==========================================================================================
template <class S, class T>
lfx_status launch_spmv(cudaStream_t st, const BsrView<S> &A, const T *x, const T *b, T *y, int mode,
                       double *part, int *n_part) {
  const int g = rows_grid(A.V);
  pdl_launch(spmv_kernel<S, T>, g, kThreads, 0, st, A, x, b, y, mode, part, nullptr);
  note_launches(1);
  if (n_part) *n_part = g;
  LFX_CUDA_TRY(cudaGetLastError());
  return LFX_OK;
}
template lfx_status launch_spmv<double, double>(cudaStream_t, const BsrView<double> &, const double *,
                                                const double *, double *, int, double *, int *);
template lfx_status launch_spmv<float, float>(cudaStream_t, const BsrView<float> &, const float *,
                                              const float *, float *, int, double *, int *);
template lfx_status launch_spmv<float, double>(cudaStream_t, const BsrView<float> &, const double *,
                                               const double *, double *, int, double *, int *);
template <>
lfx_status launch_spmv<DDMat, double>(cudaStream_t st, const BsrView<DDMat> &A, const double *x, const double *b,
                                      double *y, int mode, double *part, int *n_part) {
  pdl_launch(split_vec_kernel, vec_grid(A.V), kThreads, 0, st, A.V, x, A.xs_hi, A.xs_lo, nullptr);
  const int g = rows_grid(A.V);
  pdl_launch(spmv_dd_kernel, g, kThreads, 0, st, A, b, y, mode, part, nullptr);
  note_launches(2);
  if (n_part) *n_part = g;
  LFX_CUDA_TRY(cudaGetLastError());
  return LFX_OK;
}

lfx_status launch_norm_partials(cudaStream_t st, const double *v, int64_t n, double *part, int *n_part) {
  const int g = vec_grid(n);
  pdl_launch(norm_kernel<double>, g, kThreads, 0, st, v, n, part);
  note_launches(1);
  if (n_part) *n_part = g;
  LFX_CUDA_TRY(cudaGetLastError());
  return LFX_OK;
}
int norm_partials_capacity(int64_t V) { return std::max(rows_grid(V), vec_grid(4 * V)) + 64; }

lfx_status launch_split_vec(cudaStream_t st, int64_t V, const double *x, float4 *hi, float4 *lo) {
  pdl_launch(split_vec_kernel, vec_grid(V), kThreads, 0, st, V, x, hi, lo, nullptr);
  note_launches(1);
  LFX_CUDA_TRY(cudaGetLastError());
  return LFX_OK;
}

// The Arnoldi product w = A z_j (kernels return at once when the cycle has finished)
template <class S, class T>
static void arnoldi_spmv(cudaStream_t st, const BsrView<S> &A, const T *x, T *y, const KState *ks) {
  pdl_launch(spmv_kernel<S, T>, rows_grid(A.V), kThreads, 0, st, A, x, nullptr, y, 0, nullptr, ks);
  note_launches(1);
}
static void arnoldi_spmv(cudaStream_t st, const BsrView<DDMat> &A, const double *x, double *y, const KState *ks) {
  pdl_launch(split_vec_kernel, vec_grid(A.V), kThreads, 0, st, A.V, x, A.xs_hi, A.xs_lo, ks);
  pdl_launch(spmv_dd_kernel, rows_grid(A.V), kThreads, 0, st, A, nullptr, y, 0, nullptr, ks);
  note_launches(2);
}

template <class S, class T>
lfx_status ASimple<S, T>::init(int64_t V_, const SmootherConfig &cfg_) {
  V = V_;
  cfg = cfg_;
  const size_t vb = sizeof(T) * 4 * (size_t)V;
  LFX_TRY(dinvF.alloc(vb));
  LFX_TRY(dinvS.alloc(sizeof(T) * (size_t)V));
  LFX_TRY(X.alloc(vb));
  LFX_TRY(D0.alloc(vb));
  LFX_TRY(D1.alloc(vb));
  LFX_TRY(R.alloc(vb));
  LFX_TRY(W.alloc(vb));
  LFX_TRY(coef.alloc(sizeof(SmoothCoef)));
  LFX_TRY(part.alloc(sizeof(double) * (size_t)(rows_grid(V) + 1)));
  LFX_CUDA_TRY(cudaMemset(X.p, 0, vb));
  LFX_CUDA_TRY(cudaMemset(D0.p, 0, vb));
  LFX_CUDA_TRY(cudaMemset(D1.p, 0, vb));
  LFX_CUDA_TRY(cudaMemset(R.p, 0, vb));
  LFX_CUDA_TRY(cudaMemset(W.p, 0, vb));
  return LFX_OK;
}

template <class S, class T>
size_t ASimple<S, T>::scratch_bytes(int64_t V) {
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t vb = up(sizeof(T) * 4 * (size_t)V);
  return 6 * vb + up(sizeof(T) * (size_t)V) + up(sizeof(SmoothCoef)) + up(sizeof(double) * (size_t)(rows_grid(V) + 1));
}

template <class S, class T>
lfx_status ASimple<S, T>::init_borrowed(int64_t V_, const SmootherConfig &cfg_, void *base, size_t cap,
                                        cudaStream_t st) {
  V = V_;
  cfg = cfg_;
  if (scratch_bytes(V) > cap) {
    set_error("aSIMPLE: %zu bytes of work memory needed, %zu available", scratch_bytes(V), cap);
    return LFX_ERR_INVALID_ARG;
  }
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  char *p = static_cast<char *>(base);
  const size_t vb = up(sizeof(T) * 4 * (size_t)V);
  DBuf *vecs[6] = {&dinvF, &X, &D0, &D1, &R, &W};
  for (DBuf *d : vecs) {
    d->borrow(p, vb);
    p += vb;
  }
  dinvS.borrow(p, up(sizeof(T) * (size_t)V));
  p += up(sizeof(T) * (size_t)V);
  coef.borrow(p, up(sizeof(SmoothCoef)));
  p += up(sizeof(SmoothCoef));
  part.borrow(p, up(sizeof(double) * (size_t)(rows_grid(V) + 1)));
  // the memory keeps whatever the previous user left: clear the iterates that start at zero
  LFX_CUDA_TRY(cudaMemsetAsync(base, 0, scratch_bytes(V), st));
  return LFX_OK;
}

template <class S, class T>
size_t ASimple<S, T>::device_bytes() const {
  return dinvF.bytes + dinvS.bytes + X.bytes + D0.bytes + D1.bytes + R.bytes + W.bytes + coef.bytes + part.bytes +
         sF.bytes + sG.bytes + sDC.bytes + berr.bytes;
}

// Diagonals and (Chebyshev) eigenvalue estimates for the current matrix.
template <class S, class T>
template <class View>
lfx_status ASimple<S, T>::setup_view(cudaStream_t st, const View &A) {
  const int rg = rows_grid(V), vg = vec_grid(V);
  pdl_launch(diag_f_kernel<View, T>, vg, kThreads, 0, st, A, dinvF.as<T>());
  pdl_launch(diag_s_kernel<View, T>, rg, kThreads, 0, st, A, dinvF.as<T>(), dinvS.as<T>());
  SmoothCoef *cf = coef.as<SmoothCoef>();
  double *lam_f = &cf->lam_f, *lam_s = &cf->lam_s;
  const bool bound = cfg.n_power <= 0;
  if (bound) {
    // Gershgorin bounds (hold for every eigenvalue; no safety factor)
    pdl_launch(bound_kernel<View, T>, rg, kThreads, 0, st, A, dinvF.as<T>(), dinvS.as<T>(), W.as<T>(), part.as<double>(), 0);
    pdl_launch(reduce_kernel, 1, kThreads, 0, st, part.as<double>(), rg, lam_f, 2);
    pdl_launch(bound_kernel<View, T>, rg, kThreads, 0, st, A, dinvF.as<T>(), dinvS.as<T>(), W.as<T>(), part.as<double>(), 1);
    pdl_launch(bound_kernel<View, T>, rg, kThreads, 0, st, A, dinvF.as<T>(), dinvS.as<T>(), W.as<T>(), part.as<double>(), 2);
    pdl_launch(reduce_kernel, 1, kThreads, 0, st, part.as<double>(), rg, lam_s, 2);
    note_launches(5);
  }
  if (!bound && cfg.f_kind == LFX_SMOOTH_CHEBYSHEV) {
    // power iteration on diag(F)^-1 F from the normalised ones vector (velocity components)
    pdl_launch(fill_kernel<T>, vg, kThreads, 0, st, V, D0.as<T>(), 7, 1.0 / sqrt(3.0 * (double)V));
    for (int it = 0; it < cfg.n_power; ++it) {
      pdl_launch(f_step_kernel<View, T>, rg, kThreads, 0, st, A, dinvF.as<T>(), D0.as<T>(), D1.as<T>(), nullptr,
                                                   nullptr, cf, 0, 0, part.as<double>(), nullptr, nullptr);
      pdl_launch(reduce_kernel, 1, kThreads, 0, st, part.as<double>(), rg, lam_f, 1);
      pdl_launch(div_kernel<T>, vg, kThreads, 0, st, V, D1.as<T>(), D0.as<T>(), 7, lam_f);
    }
    note_launches(1 + 3 * cfg.n_power);
  }
  if (!bound && cfg.s_kind != LFX_SMOOTH_JACOBI) {
    pdl_launch(fill_kernel<T>, vg, kThreads, 0, st, V, D0.as<T>(), 8, 1.0 / sqrt((double)V));
    for (int it = 0; it < cfg.n_power; ++it) {
      pdl_launch(g_scaled_kernel<View, T>, rg, kThreads, 0, st, A, dinvF.as<T>(), D0.as<T>(), W.as<T>(), nullptr);
      pdl_launch(s_step_kernel<View, T>, rg, kThreads, 0, st, A, dinvS.as<T>(), D0.as<T>(), W.as<T>(), D1.as<T>(),
                                                   nullptr, nullptr, cf, 0, 0, part.as<double>(), nullptr);
      pdl_launch(reduce_kernel, 1, kThreads, 0, st, part.as<double>(), rg, lam_s, 1);
      pdl_launch(div_kernel<T>, vg, kThreads, 0, st, V, D1.as<T>(), D0.as<T>(), 8, lam_s);
    }
    note_launches(1 + 4 * cfg.n_power);
  }
  note_launches(3);
  pdl_launch(coef_kernel, 1, 32, 0, st, cf, cfg.f_kind, cfg.f_steps, cfg.f_omega, cfg.f_ratio, cfg.s_kind,
                                cfg.s_steps, cfg.s_omega, cfg.s_ratio, bound ? 1.0 : 1.1);
  LFX_CUDA_TRY(cudaGetLastError());
  return LFX_OK;
}

template <class S, class T>
lfx_status ASimple<S, T>::setup(cudaStream_t st, const BsrView<S> &A) {
  split = false;
  return setup_view(st, A);
}

// Sub-blocks stored apart in S, converted from the FP64 (or FP32) blocks; diagonals and bounds
// from them.
template <class S, class T>
lfx_status ASimple<S, T>::setup_split(cudaStream_t st, const BsrView<double> &A64, int64_t nnzb) {
  return setup_split_from(st, A64, nnzb);
}
template <class S, class T>
lfx_status ASimple<S, T>::setup_split(cudaStream_t st, const BsrView<float> &A32, int64_t nnzb) {
  return setup_split_from(st, A32, nnzb);
}
template <class S, class T>
template <class Src>
lfx_status ASimple<S, T>::setup_split_from(cudaStream_t st, const BsrView<Src> &A64, int64_t nnzb) {
  if (!sF.p || nnz_split != nnzb) {
    LFX_TRY(sF.alloc(sizeof(S) * 12 * (size_t)nnzb + 16));   // + 16: the staged pass copies whole 16-byte units
    LFX_TRY(sG.alloc(sizeof(S) * 4 * (size_t)nnzb));
    LFX_TRY(sDC.alloc(sizeof(S) * 4 * (size_t)nnzb));
    nnz_split = nnzb;
  }
  const int g = (int)std::max<int64_t>(1, std::min<int64_t>((nnzb + kThreads - 1) / kThreads, 152 * 16));
  pdl_launch(split_kernel<S, Src>, g, kThreads, 0, st, nnzb, A64.vals, A64.col, sF.as<S>(), sG.as<S>(), sDC.as<S>());
  note_launches(1);
  if (std::is_same<S, __nv_bfloat16>::value && !berr.p) {
    // error word of the staged velocity smoothing pass, and its host copy
    LFX_TRY(berr.alloc(16));
    LFX_CUDA_TRY(cudaMemsetAsync(berr.p, 0, 16, st));
    if (!berr_host) {
      LFX_CUDA_TRY(cudaMallocHost(&berr_host, sizeof(int)));
      *berr_host = 0;
    }
  }
  split = true;
  const SplitView<S> sv{A64.V, A64.rowptr, A64.col, A64.diag, A64.trans, sF.as<S>(), sG.as<S>(), sDC.as<S>()};
  return setup_view(st, sv);
}

// The staged pass serves BF16 sub-blocks stored apart, FP32 vectors, a pattern with row tiles.
template <class S, class T>
template <class View>
bool ASimple<S, T>::use_staged(const View &) const {
  if constexpr (std::is_same<View, SplitView<__nv_bfloat16>>::value && std::is_same<T, float>::value)
    return ftile != nullptr && n_ftile > 0 && berr.p != nullptr && (reinterpret_cast<uintptr_t>(sF.p) & 15u) == 0;
  return false;
}

template <class S, class T>
template <class View>
lfx_status ASimple<S, T>::launch_staged(cudaStream_t st, const View &A, bool first, int k, const T *d_old, T *d_new,
                                        const T *b0, const KState *ks) {
  if constexpr (std::is_same<View, SplitView<__nv_bfloat16>>::value && std::is_same<T, float>::value) {
    // one resident wave of persistent CTAs (the occupancy the kernel's shared memory allows)
    // (the attribute and the occupancy are per device: looked up again after a device switch)
    static int grid[2] = {0, 0}, grid_dev[2] = {-1, -1};
    const int f = first ? 1 : 0;
    int dev = 0;
    LFX_CUDA_TRY(cudaGetDevice(&dev));
    if (grid_dev[f] != dev) {
      auto kern = first ? f_step_staged_kernel<true> : f_step_staged_kernel<false>;
      LFX_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFStagedSmem));
      int sms = 0, per = 0;
      LFX_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
      LFX_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kFTileThreads, kFStagedSmem));
      grid[f] = std::max(1, sms * std::max(per, 1));
      grid_dev[f] = dev;
    }
    const int g = std::min(grid[f], n_ftile);
    const SmoothCoef *cf = coef.as<SmoothCoef>();
    const uint32_t polls = force_bulk_timeout ? 0u : kFWaitPolls;
    if (first)
      pdl_launch(f_step_staged_kernel<true>, g, kFTileThreads, kFStagedSmem, st, A, ftile, n_ftile, dinvF.as<float>(),
                 d_old, d_new, R.as<float>(), X.as<float>(), cf, k, ks, b0, berr.as<int>(), polls);
    else
      pdl_launch(f_step_staged_kernel<false>, g, kFTileThreads, kFStagedSmem, st, A, ftile, n_ftile, dinvF.as<float>(),
                 d_old, d_new, R.as<float>(), X.as<float>(), cf, k, ks, b0, berr.as<int>(), polls);
    return LFX_OK;   // counted by the caller with the plain passes it replaces
  } else {
    (void)st, (void)A, (void)first, (void)k, (void)d_old, (void)d_new, (void)b0, (void)ks;
    set_error("aSIMPLE: the staged velocity pass needs BF16 sub-blocks and FP32 vectors");
    return LFX_ERR_INVALID_ARG;
  }
}

// z = P^-1 r (aSIMPLE); r, z are [V][4] vectors of type T (they may not alias the work arrays).
template <class S, class T>
template <class View>
lfx_status ASimple<S, T>::apply_view(cudaStream_t st, const View &A, const T *r, T *z, const KState *ks) {
  const int rg = rows_grid(V), vg = vec_grid(V);
  const SmoothCoef *cf = coef.as<SmoothCoef>();
  T *d[2] = {D0.as<T>(), D1.as<T>()};
  // z_u* ~= F^-1 r_u
  bool pending_w = false;
  const bool staged = use_staged(A);
  if (cfg.f_steps >= 2 && staged) {
    LFX_TRY(launch_staged(st, A, true, 1, d[0], d[1], r, ks));
  } else if (cfg.f_steps >= 2) {
    // start of the smoothing fused into step 1 (d_old formed from r on the fly)
    pdl_launch(f_step_kernel<View, T, true>, rg, kThreads, 0, st, A, dinvF.as<T>(), d[0], d[1], R.as<T>(), X.as<T>(),
               cf, 1, 1, nullptr, ks, r);
  } else {
    pdl_launch(f_init_kernel<T>, vg, kThreads, 0, st, V, dinvF.as<T>(), r, R.as<T>(), d[0], X.as<T>(), cf, ks);
  }
  // one application per step is timed (the counter is reset per step): an event between two
  // launches costs the overlap of programmatic dependent launch there
  const bool timed = time_f && cfg.f_steps > 2 && n_fev == 0;
  if (timed) {
    if (n_fev + 2 > (int)fev.size())
      for (int q = 0; q < 32; ++q) {
        cudaEvent_t e;
        LFX_CUDA_TRY(cudaEventCreate(&e));
        fev.push_back(e);
      }
    LFX_CUDA_TRY(cudaEventRecord(fev[n_fev], st));
  }
  for (int k = 2; k < cfg.f_steps; ++k) {
    if (staged) LFX_TRY(launch_staged(st, A, false, k, d[(k - 1) & 1], d[k & 1], nullptr, ks));
    else
      pdl_launch(f_step_kernel<View, T>, rg, kThreads, 0, st, A, dinvF.as<T>(), d[(k - 1) & 1], d[k & 1], R.as<T>(),
                 X.as<T>(), cf, k, 1, nullptr, ks, nullptr);
  }
  if (timed) {
    LFX_CUDA_TRY(cudaEventRecord(fev[n_fev + 1], st));
    n_fev += 2;
  }
  // z_p ~= S^-1 (r_p - D z_u*): Chebyshev/Jacobi steps on S, or one AMG V-cycle
  if (cfg.s_kind == LFX_SMOOTH_AMG && !amg_ready) {
    set_error("aSIMPLE: the Schur AMG hierarchy has not been built");
    return LFX_ERR_INVALID_ARG;
  }
  pdl_launch(d_init_kernel<View, T>, rg, kThreads, 0, st, A, dinvS.as<T>(), r, R.as<T>(), d[0], X.as<T>(), cf, ks,
                                               amg_ready ? Bs.as<T>() : nullptr);
  for (int k = 1; k < cfg.s_steps; ++k) {
    pdl_launch(g_scaled_kernel<View, T>, rg, kThreads, 0, st, A, dinvF.as<T>(), d[(k - 1) & 1], W.as<T>(), ks);
    pdl_launch(s_step_kernel<View, T>, rg, kThreads, 0, st, A, dinvS.as<T>(), d[(k - 1) & 1], W.as<T>(), d[k & 1],
                                                 R.as<T>(), X.as<T>(), cf, k, 1, nullptr, ks);
  }
  if (cfg.s_kind == LFX_SMOOTH_AMG && amg.size() == 1) {
    // small problem: the hierarchy is the dense inverse of S itself
    pdl_launch(dense_mv_kernel<T>, (int)((V * 32 + kThreads - 1) / kThreads), kThreads, 0, st, 
        V, coarse_inv.as<T>(), Bs.as<T>(), 4, 3, X.as<T>(), 4, 3, ks);
    note_launches(1);
  } else if (cfg.s_kind == LFX_SMOOTH_AMG) {
    // residual of the pre-smoothed level-0 iterate, restriction, coarse V-cycle, prolongation
    pdl_launch(g_scaled_kernel<View, T>, rg, kThreads, 0, st, A, dinvF.as<T>(), X.as<T>(), W.as<T>(), ks);
    pdl_launch(s_resid_kernel<View, T>, rg, kThreads, 0, st, A, dinvS.as<T>(), X.as<T>(), W.as<T>(), Bs.as<T>(),
                                                  rr0.as<T>(), nullptr, nullptr, cf, 0, ks);
    const AmgDevLevel &L0 = amg[0];
    CsrV<T> R0{L0.nnext, L0.Rrp.as<int32_t>(), L0.Rci.as<int32_t>(), L0.Rv.as<T>()};
    pdl_launch(csr_spmv_kernel<T, 32>, (int)((L0.nnext * 32 + kThreads - 1) / kThreads), kThreads, 0, st, 
        R0, rr0.as<T>(), 1, 0, amg[1].b.as<T>(), 1, 0, 1.0, 0, ks);
    LFX_TRY(coarse_cycle(st, ks));
    CsrV<T> P0{V, L0.Prp.as<int32_t>(), L0.Pci.as<int32_t>(), L0.Pv.as<T>()};
    const T *x1 = coarse_x();
    pdl_launch(csr_spmv_kernel<T, 8>, lanes_grid(V, 8), kThreads, 0, st, P0, x1, 1, 0, X.as<T>(), 4, 3,
                                                            amg_alpha, 1, ks);
    // post-smoothing from the corrected iterate
    pdl_launch(g_scaled_kernel<View, T>, rg, kThreads, 0, st, A, dinvF.as<T>(), X.as<T>(), W.as<T>(), ks);
    pdl_launch(s_resid_kernel<View, T>, rg, kThreads, 0, st, A, dinvS.as<T>(), X.as<T>(), W.as<T>(), Bs.as<T>(), nullptr,
                                                  R.as<T>(), d[0], cf, 1, ks);
    if (cfg.s_steps == 1) {
      // x.w += d.w is left to the final pass, which reads x.w (own row and neighbours) as x.w + d.w
      pending_w = true;
    } else {
      pdl_launch(add_w_kernel<T>, vg, kThreads, 0, st, V, d[0], X.as<T>(), ks);
      note_launches(1);
    }
    for (int k = 1; k < cfg.s_steps; ++k) {
      pdl_launch(g_scaled_kernel<View, T>, rg, kThreads, 0, st, A, dinvF.as<T>(), d[(k - 1) & 1], W.as<T>(), ks);
      pdl_launch(s_step_kernel<View, T>, rg, kThreads, 0, st, A, dinvS.as<T>(), d[(k - 1) & 1], W.as<T>(), d[k & 1],
                                                   R.as<T>(), X.as<T>(), cf, k, 1, nullptr, ks);
    }
    note_launches(8 + 2 * (cfg.s_steps - 1));
  }
  // z_u = z_u* - diag(F)^-1 G z_p
  if (pending_w)
    pdl_launch(final_kernel<View, T, true>, rg, kThreads, 0, st, A, dinvF.as<T>(), X.as<T>(), z, ks, d[0]);
  else
    pdl_launch(final_kernel<View, T>, rg, kThreads, 0, st, A, dinvF.as<T>(), X.as<T>(), z, ks, nullptr);
  // start (or fused first step) + further F steps + d_init + final + extra Schur steps
  note_launches(3 + (cfg.f_steps >= 2 ? cfg.f_steps - 2 : 0) + 2 * (cfg.s_steps - 1));
  LFX_CUDA_TRY(cudaGetLastError());
  return LFX_OK;
}


static void cheb_coefs(double lam, double ratio, int steps, double &init, double *c1, double *c2) {
  const double lmax = lam, lmin = lmax / ratio;
  const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sigma1 = theta / delta;
  double rho = 1.0 / sigma1;
  init = 1.0 / theta;
  c1[0] = c2[0] = 0.0;
  for (int k = 1; k < steps; ++k) {
    const double rn = 1.0 / (2.0 * sigma1 - rho);
    c1[k] = rn * rho;
    c2[k] = 2.0 * rn / delta;
    rho = rn;
  }
}

template <class T>
static lfx_status upload_vec(DBuf &d, const std::vector<T> &h) {
  LFX_TRY(d.alloc(sizeof(T) * std::max<size_t>(h.size(), 1)));
  if (!h.empty()) LFX_CUDA_TRY(cudaMemcpy(d.p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice));
  return LFX_OK;
}
// FP64 host values uploaded in the preconditioner's arithmetic type
template <class T>
static lfx_status upload_as(DBuf &d, const std::vector<double> &h) {
  if (std::is_same<T, double>::value) return upload_vec(d, h);
  std::vector<T> c(h.begin(), h.end());
  return upload_vec(d, c);
}

template <class S, class T>
lfx_status ASimple<S, T>::upload_amg(const AmgHost &H) {
  amg_ready = false;
  const int L = (int)H.A.size();
  if (L < 1) {
    set_error("Schur AMG: empty hierarchy");
    return LFX_ERR_INVALID_ARG;
  }
  amg.clear();
  amg.resize(L);
  for (int l = 0; l < L; ++l) {
    AmgDevLevel &D = amg[l];
    D.n = H.A[l].n;
    if (l + 1 < L) {
      D.nnext = H.A[l + 1].n;
      LFX_TRY(upload_vec(D.Prp, H.P[l].rp));
      LFX_TRY(upload_vec(D.Pci, H.P[l].ci));
      LFX_TRY(upload_as<T>(D.Pv, H.P[l].v));
      LFX_TRY(upload_vec(D.Rrp, H.R[l].rp));
      LFX_TRY(upload_vec(D.Rci, H.R[l].ci));
      LFX_TRY(upload_as<T>(D.Rv, H.R[l].v));
      D.lam = H.lam[l];
      cheb_coefs(H.lam[l], cfg.s_ratio, cfg.s_steps, D.init, D.c1, D.c2);
    }
    if (l >= 1) {
      if (l + 1 < L) {
        LFX_TRY(upload_vec(D.rp, H.A[l].rp));
        LFX_TRY(upload_vec(D.ci, H.A[l].ci));
        LFX_TRY(upload_as<T>(D.v, H.A[l].v));
        LFX_TRY(upload_as<T>(D.dinv, H.dinv[l]));
      }
      const size_t vb = sizeof(T) * (size_t)std::max<int64_t>(D.n, 1);
      LFX_TRY(D.x.alloc(vb));
      LFX_TRY(D.b.alloc(vb));
      LFX_TRY(D.r.alloc(vb));
      LFX_TRY(D.d0.alloc(vb));
      LFX_TRY(D.d1.alloc(vb));
      LFX_TRY(D.rr.alloc(vb));
    }
  }
  nc = H.nc;
  lvl_rows.assign(L, 0);
  lvl_nnz.assign(L, 0);
  for (int l = 0; l < L; ++l) {
    lvl_rows[l] = H.A[l].n;
    lvl_nnz[l] = (int64_t)H.A[l].ci.size();
  }
  LFX_TRY(upload_as<T>(coarse_inv, H.coarse_inv));
  // arguments of the fused coarse V-cycle (one cooperative launch for levels 1..L-1)
  coop_grid = 0;
  int coop = 0, dev = 0, nsm = 0, per_sm = 0;
  LFX_CUDA_TRY(cudaGetDevice(&dev));
  LFX_CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  LFX_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  LFX_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, amg_coarse_kernel<T>, kThreads, 0));
  if (coop && per_sm > 0 && L >= 2 && L <= kMaxCoarse) {
    CoarseArgs<T> h{};
    h.L = L;
    h.s_steps = cfg.s_steps;
    h.alpha = amg_alpha;
    h.coarse_inv = coarse_inv.as<T>();
    h.nc = nc;
    for (int l = 1; l < L; ++l) {
      const AmgDevLevel &D = amg[l];
      CoarseLevel<T> &c = h.lv[l];
      c.n = D.n;
      c.nnext = D.nnext;
      c.rp = D.rp.as<int32_t>();
      c.ci = D.ci.as<int32_t>();
      c.v = D.v.as<T>();
      c.dinv = D.dinv.as<T>();
      c.Prp = D.Prp.as<int32_t>();
      c.Pci = D.Pci.as<int32_t>();
      c.Pv = D.Pv.as<T>();
      c.Rrp = D.Rrp.as<int32_t>();
      c.Rci = D.Rci.as<int32_t>();
      c.Rv = D.Rv.as<T>();
      c.x = D.x.as<T>();
      c.b = D.b.as<T>();
      c.r = D.r.as<T>();
      c.d0 = D.d0.as<T>();
      c.d1 = D.d1.as<T>();
      c.rr = D.rr.as<T>();
      c.xo = (cfg.s_steps == 1 && l < L - 1) ? D.d1.as<T>() : D.x.as<T>();
      c.init = D.init;
      for (int k = 0; k < kMaxSmooth; ++k) {
        c.c1[k] = D.c1[k];
        c.c2[k] = D.c2[k];
      }
    }
    LFX_TRY(coarse_args.alloc(sizeof(CoarseArgs<T>)));
    LFX_CUDA_TRY(cudaMemcpy(coarse_args.p, &h, sizeof(h), cudaMemcpyHostToDevice));
#ifndef LFX_COOP_PER_SM
#define LFX_COOP_PER_SM 4
#endif
    coop_grid = std::min(per_sm, LFX_COOP_PER_SM) * nsm;
  }
  if (!Bs.p) LFX_TRY(Bs.alloc(sizeof(T) * 4 * (size_t)V));
  if (!rr0.p) LFX_TRY(rr0.alloc(sizeof(T) * (size_t)V));
  LFX_CUDA_TRY(cudaMemset(Bs.p, 0, Bs.bytes));
  amg_ready = true;
  return LFX_OK;
}

template <class S, class T>
size_t ASimple<S, T>::amg_bytes() const {
  size_t b = Bs.bytes + rr0.bytes + coarse_inv.bytes;
  for (const auto &D : amg)
    b += D.rp.bytes + D.ci.bytes + D.v.bytes + D.dinv.bytes + D.Prp.bytes + D.Pci.bytes + D.Pv.bytes + D.Rrp.bytes +
         D.Rci.bytes + D.Rv.bytes + D.x.bytes + D.b.bytes + D.r.bytes + D.d0.bytes + D.d1.bytes + D.rr.bytes;
  return b;
}

static inline double H_nnz(const AmgDevLevel &D, size_t elem) { return (double)D.v.bytes / (double)elem; }

// One V-cycle on the explicit levels l >= 1 for amg[l].b -> amg[l].x
template <class S, class T>
lfx_status ASimple<S, T>::apply(cudaStream_t st, const BsrView<S> &A, const T *r, T *z, const KState *ks) {
  if (split) {
    const SplitView<S> sv{A.V, A.rowptr, A.col, A.diag, A.trans, sF.as<S>(), sG.as<S>(), sDC.as<S>()};
    return apply_view(st, sv, r, z, ks);
  }
  return apply_view(st, A, r, z, ks);
}

template <class S, class T>
lfx_status ASimple<S, T>::coarse_cycle(cudaStream_t st, const KState *ks) {
  if (coop_grid > 0) {
    const CoarseArgs<T> *ca = coarse_args.as<CoarseArgs<T>>();
    void *kargs[] = {(void *)&ca, (void *)&ks};
    LFX_CUDA_TRY(cudaLaunchCooperativeKernel((void *)amg_coarse_kernel<T>, dim3(coop_grid), dim3(kThreads), kargs,
                                             0, st));
    note_launches(1);
    return LFX_OK;
  }
  return vcycle(st, 1, ks);
}

// the level-1 iterate is in d1 when the coarse launch fused its last smoothing step
template <class S, class T>
const T *ASimple<S, T>::coarse_x() const {
  return (amg.size() > 2 && coop_grid > 0 && cfg.s_steps == 1) ? amg[1].d1.as<T>() : amg[1].x.as<T>();
}

template <class S, class T>
lfx_status ASimple<S, T>::vcycle(cudaStream_t st, int l, const KState *ks) {
  AmgDevLevel &D = amg[l];
  const int L = (int)amg.size();
  if (l == L - 1) {
    pdl_launch(dense_mv_kernel<T>, (int)((D.n * 32 + kThreads - 1) / kThreads), kThreads, 0, st, 
        D.n, coarse_inv.as<T>(), D.b.as<T>(), 1, 0, D.x.as<T>(), 1, 0, ks);
    note_launches(1);
    return LFX_OK;
  }
  CsrV<T> A{D.n, D.rp.as<int32_t>(), D.ci.as<int32_t>(), D.v.as<T>()};
  CsrV<T> P{D.n, D.Prp.as<int32_t>(), D.Pci.as<int32_t>(), D.Pv.as<T>()};
  CsrV<T> R{D.nnext, D.Rrp.as<int32_t>(), D.Rci.as<int32_t>(), D.Rv.as<T>()};
  const int vg = vec_grid(D.n), rg = lanes_grid(D.n, 8);
  T *d[2] = {D.d0.as<T>(), D.d1.as<T>()};
  const T *dinv = D.dinv.as<T>();
  const bool wide = D.rp.p && D.n > 0 && H_nnz(D, sizeof(T)) / (double)D.n > 24.0;
  const int rg32 = (int)((D.n * 32 + kThreads - 1) / kThreads);
  auto cheb_step = [&](int k) {
    if (wide)
      pdl_launch(csr_cheb_step_kernel<T, 32>, rg32, kThreads, 0, st, A, dinv, d[(k - 1) & 1], d[k & 1], D.r.as<T>(),
                                                             D.x.as<T>(), D.c1[k], D.c2[k], ks);
    else
      pdl_launch(csr_cheb_step_kernel<T, 8>, rg, kThreads, 0, st, A, dinv, d[(k - 1) & 1], d[k & 1], D.r.as<T>(),
                                                          D.x.as<T>(), D.c1[k], D.c2[k], ks);
  };
  auto resid = [&]() {
    if (wide)
      pdl_launch(csr_resid_kernel<T, 32>, rg32, kThreads, 0, st, A, D.x.as<T>(), D.b.as<T>(), D.rr.as<T>(), ks);
    else
      pdl_launch(csr_resid_kernel<T, 8>, rg, kThreads, 0, st, A, D.x.as<T>(), D.b.as<T>(), D.rr.as<T>(), ks);
  };
  pdl_launch(csr_cheb_init_kernel<T>, vg, kThreads, 0, st, D.n, dinv, D.b.as<T>(), D.r.as<T>(), d[0], D.x.as<T>(), D.init, 0, ks);
  for (int k = 1; k < cfg.s_steps; ++k) cheb_step(k);
  resid();
  pdl_launch(csr_spmv_kernel<T, 32>, (int)((D.nnext * 32 + kThreads - 1) / kThreads), kThreads, 0, st, 
      R, D.rr.as<T>(), 1, 0, amg[l + 1].b.as<T>(), 1, 0, 1.0, 0, ks);
  LFX_TRY(vcycle(st, l + 1, ks));
  pdl_launch(csr_spmv_kernel<T, 8>, rg, kThreads, 0, st, P, amg[l + 1].x.as<T>(), 1, 0, D.x.as<T>(), 1, 0, amg_alpha, 1, ks);
  resid();
  pdl_launch(csr_cheb_init_kernel<T>, vg, kThreads, 0, st, D.n, dinv, D.rr.as<T>(), D.r.as<T>(), d[0], D.x.as<T>(), D.init, 1, ks);
  for (int k = 1; k < cfg.s_steps; ++k) cheb_step(k);
  note_launches(6 + 2 * (cfg.s_steps - 1));
  LFX_CUDA_TRY(cudaGetLastError());
  return LFX_OK;
}

template <class S, class T>
ASimple<S, T>::~ASimple() {
  for (cudaEvent_t e : fev) cudaEventDestroy(e);
  if (berr_host) cudaFreeHost(berr_host);
}

template <class S, class T>
lfx_status ASimple<S, T>::queue_bulk_check(cudaStream_t st) {
  if (!berr.p || !berr_host) return LFX_OK;
  LFX_CUDA_TRY(cudaMemcpyAsync(berr_host, berr.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  LFX_CUDA_TRY(cudaMemsetAsync(berr.p, 0, sizeof(int), st));
  return LFX_OK;
}

template <class S, class T>
bool ASimple<S, T>::bulk_failed() {
  if (!berr_host || *berr_host == 0) return false;
  *berr_host = 0;
  return true;
}

// Median duration of one plain F pass over the applications timed since the last read (the
// median discards the applications queued after a solve had converged, whose kernels return at
// once), and the number of passes timed.
template <class S, class T>
lfx_status ASimple<S, T>::read_f_timing(float *median_ms_per_pass, int *passes) {
  std::vector<float> per;
  for (int i = 0; i + 1 < n_fev; i += 2) {
    LFX_CUDA_TRY(cudaEventSynchronize(fev[i + 1]));
    float t = 0.0f;
    LFX_CUDA_TRY(cudaEventElapsedTime(&t, fev[i], fev[i + 1]));
    per.push_back(t / (float)(cfg.f_steps - 2));
  }
  n_fev = 0;
  std::sort(per.begin(), per.end());
  if (median_ms_per_pass) *median_ms_per_pass = per.empty() ? 0.0f : per[per.size() / 2];
  if (passes) *passes = (int)per.size() * std::max(cfg.f_steps - 2, 0);
  return LFX_OK;
}

template <class S, class T>
lfx_status ASimple<S, T>::lambdas(double *lf, double *ls) const {
  SmoothCoef h;
  LFX_CUDA_TRY(cudaMemcpy(&h, coef.p, sizeof(SmoothCoef), cudaMemcpyDeviceToHost));
  const double f = cfg.n_power > 0 ? 1.1 : 1.0;
  if (lf) *lf = f * h.lam_f;
  if (ls) *ls = f * h.lam_s;
  return LFX_OK;
}

template struct ASimple<double, double>;
template struct ASimple<float, float>;
template struct ASimple<__nv_bfloat16, float>;

// ------------------------------------------------------------------------------------------
template <class S, class T>
lfx_status Gmres<S, T>::init(int64_t V_, int restart_) {
  V = V_;
  n = 4 * V;
  restart = std::min(restart_, kMaxRestart);
  if (restart < 1) restart = 1;
  const size_t vb = sizeof(T) * (size_t)n;
  LFX_TRY(basis.alloc(vb * (restart + 1)));
  LFX_TRY(zbasis.alloc(vb * restart));
  LFX_TRY(work.alloc(vb));
  nblk_dot = 152 * 4;
  LFX_TRY(part.alloc(sizeof(double) * (size_t)nblk_dot * (kMaxRestart + 1)));
  LFX_TRY(part_n.alloc(sizeof(double) * (size_t)std::max(rows_grid(V), vec_grid(n)) + 64));
  LFX_TRY(state.alloc(sizeof(KState)));
  LFX_CUDA_TRY(cudaMemset(state.p, 0, sizeof(KState)));
  LFX_CUDA_TRY(cudaMallocHost(&pinned, sizeof(int) * 8));
  for (int i = 0; i < 4; ++i) LFX_CUDA_TRY(cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming));
  return LFX_OK;
}

template <class S, class T>
lfx_status Gmres<S, T>::read_spmv_timing(float *ms, int *count) {
  float total = 0.0f;
  int c = 0;
  for (int i = 0; i + 1 < n_tev; i += 2) {
    LFX_CUDA_TRY(cudaEventSynchronize(tev[i + 1]));
    float t = 0.0f;
    LFX_CUDA_TRY(cudaEventElapsedTime(&t, tev[i], tev[i + 1]));
    total += t;
    ++c;
  }
  n_tev = 0;
  n_spmv_calls = 0;
  if (ms) *ms = total;
  if (count) *count = c;
  return LFX_OK;
}

template <class S, class T>
Gmres<S, T>::~Gmres() {
  for (cudaEvent_t e : tev) cudaEventDestroy(e);
  if (pinned) cudaFreeHost(pinned);
  for (int i = 0; i < 4; ++i)
    if (ev[i]) cudaEventDestroy(ev[i]);
}

template <class S, class T>
size_t Gmres<S, T>::device_bytes() const {
  return basis.bytes + zbasis.bytes + work.bytes + part.bytes + part_n.bytes + state.bytes + seg_lo.bytes +
         seg_hi.bytes + seg_id.bytes + seg_toff.bytes + seg_state.bytes + seg_part.bytes + seg_pn.bytes;
}

// Solve A x = b to ||b - A x|| <= rtol ||b|| from the x passed in.  Returns LFX_OK,
// LFX_ERR_NOT_CONVERGED or LFX_ERR_NONFINITE; *its_out = Arnoldi steps, *res_out = final
// relative residual (true residual of the last restart).
template <class S, class T>
lfx_status Gmres<S, T>::solve(cudaStream_t st, const BsrView<S> &A, const PrecFn<T> &pc, const T *b, T *x,
                              double rtol, int maxit, bool cgs2, int lag, bool x_zero, int *its_out,
                              double *res_out) {
  if (n_seg > 1) return solve_seg(st, A, pc, b, x, rtol, maxit, cgs2, lag, x_zero, its_out, res_out);
  if (lag < 0) lag = 0;
  if (lag > 2) lag = 2;
  KState *ks = state.as<KState>();
  T *Vb = basis.as<T>(), *Zb = zbasis.as<T>(), *w = work.as<T>();
  double *pn = part_n.as<double>();
  const int vg = vec_grid(n);
  // ||b|| and the tolerance on the device; x = 0 to start from, or as the solution when b = 0
  pdl_launch(norm_kernel<T>, vg, kThreads, 0, st, b, n, pn);
  pdl_launch(solve_start_kernel, 1, kThreads, 0, st, pn, vg, ks, rtol);
  if (x_zero) LFX_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(T) * n, st));
  pdl_launch(zero_if_b_zero_kernel<T>, vg, kThreads, 0, st, x, n, &ks->bnorm);
  note_launches(3);
  int total = 0;
  double rel = 1.0;
  lfx_status status = LFX_ERR_NOT_CONVERGED;
  KState hs;
  int ng = 0;
  bool have_r = false;   // w = b - A x and its partial sums are in place (from the previous cycle)
  for (int cycle = 0; cycle < 100000; ++cycle) {
    // r = b - A x -> w, beta, v0 = r / beta
    if (!have_r) LFX_TRY(residual(st, A, x, b, w, pn, &ng));
    pdl_launch(cycle_start_kernel, 1, kThreads, 0, st, pn, ng, ks);
    pdl_launch(scale_beta_kernel<T>, vg, kThreads, 0, st, w, Vb, n, ks);
    note_launches(2);
    LFX_TRY(arnoldi_cycle(st, A, pc, restart, maxit, cgs2, lag));
    pdl_launch(trisolve_kernel, 1, 32, 0, st, ks);
    pdl_launch(update_x_kernel<T, T>, vg, kThreads, 0, st, Zb, n, x, n, ks);
    // the true residual, which confirms convergence or starts the next cycle; one read of the
    // status header for both
    LFX_TRY(residual(st, A, x, b, w, pn, &ng));
    pdl_launch(reduce_kernel, 1, kThreads, 0, st, pn, ng, &ks->res, 1);
    note_launches(3);
    LFX_CUDA_TRY(cudaMemcpyAsync(&hs, ks, offsetof(KState, H), cudaMemcpyDeviceToHost, st));
    LFX_CUDA_TRY(cudaStreamSynchronize(st));
    LFX_CUDA_TRY(cudaGetLastError());
    total = hs.total;
    if (!std::isfinite(hs.bnorm)) {
      set_error("GMRES: right-hand side is not finite");
      status = LFX_ERR_NONFINITE;
      break;
    }
    if (hs.bnorm == 0.0) {   // x = 0
      total = 0;
      rel = 0.0;
      status = LFX_OK;
      break;
    }
    if (hs.flag == 2) {
      set_error("GMRES: non-finite residual after %d steps", total);
      status = LFX_ERR_NONFINITE;
      break;
    }
    rel = hs.res / hs.bnorm;
    if (!std::isfinite(rel)) {
      status = LFX_ERR_NONFINITE;
      set_error("GMRES: non-finite true residual");
      break;
    }
    if (hs.res <= 2.0 * hs.tol_abs) {
      status = LFX_OK;
      break;
    }
    if (total >= maxit) {
      set_error("GMRES: not converged after %d steps (relative residual %.3e)", total, rel);
      status = LFX_ERR_NOT_CONVERGED;
      break;
    }
    have_r = true;
  }
  if (its_out) *its_out = total;
  if (res_out) *res_out = rel;
  return status;
}


template <class S, class T>
lfx_status Gmres<S, T>::set_segments(const std::vector<int32_t> &comp_off) {
  const int ns = (int)comp_off.size() - 1;
  if (ns < 1 || comp_off[0] != 0 || comp_off[ns] != V) {
    set_error("GMRES: component offsets do not cover the %lld nodes", (long long)V);
    return LFX_ERR_INVALID_ARG;
  }
  std::vector<int64_t> lo, hi;
  std::vector<int32_t> id, toff(1, 0);
  for (int c = 0; c < ns; ++c) {
    const int64_t a = comp_off[c], b = comp_off[c + 1];
    if (b < a) {
      set_error("GMRES: component offsets are not increasing");
      return LFX_ERR_INVALID_ARG;
    }
    const int64_t nt = std::max<int64_t>(1, (b - a + kSegNodes - 1) / kSegNodes);
    for (int64_t t = 0; t < nt; ++t) {
      lo.push_back(a + (b - a) * t / nt);
      hi.push_back(a + (b - a) * (t + 1) / nt);
      id.push_back(c);
    }
    toff.push_back((int32_t)lo.size());
  }
  const int nt = (int)lo.size();
  LFX_TRY(seg_lo.alloc(sizeof(int64_t) * nt));
  LFX_TRY(seg_hi.alloc(sizeof(int64_t) * nt));
  LFX_TRY(seg_id.alloc(sizeof(int32_t) * nt));
  LFX_TRY(seg_toff.alloc(sizeof(int32_t) * (ns + 1)));
  LFX_TRY(seg_state.alloc(sizeof(KState) * (size_t)ns));
  LFX_TRY(seg_part.alloc(sizeof(double) * (size_t)nt * (kMaxRestart + 1)));
  LFX_TRY(seg_pn.alloc(sizeof(double) * (size_t)nt));
  LFX_CUDA_TRY(cudaMemcpy(seg_lo.p, lo.data(), sizeof(int64_t) * nt, cudaMemcpyHostToDevice));
  LFX_CUDA_TRY(cudaMemcpy(seg_hi.p, hi.data(), sizeof(int64_t) * nt, cudaMemcpyHostToDevice));
  LFX_CUDA_TRY(cudaMemcpy(seg_id.p, id.data(), sizeof(int32_t) * nt, cudaMemcpyHostToDevice));
  LFX_CUDA_TRY(cudaMemcpy(seg_toff.p, toff.data(), sizeof(int32_t) * (ns + 1), cudaMemcpyHostToDevice));
  LFX_CUDA_TRY(cudaMemset(seg_state.p, 0, sizeof(KState) * (size_t)ns));
  tasks = SegTasks{seg_lo.as<int64_t>(), seg_hi.as<int64_t>(), seg_id.as<int32_t>(), seg_toff.as<int32_t>(), nt, ns};
  n_seg = ns;
  return LFX_OK;
}

// The header of a KState (status words and scalars), read back by the host
static constexpr size_t kStateHead = offsetof(KState, H);

template <class S, class T>
lfx_status Gmres<S, T>::inner_tolerance(cudaStream_t st, double lo, double hi, double *eta) {
  const int ns = n_seg > 1 ? n_seg : 1;
  std::vector<KState> h(1);
  std::vector<char> heads((size_t)ns * kStateHead);
  const void *src = n_seg > 1 ? seg_state.p : state.p;
  LFX_CUDA_TRY(cudaMemcpy2DAsync(heads.data(), kStateHead, src, sizeof(KState), kStateHead, ns,
                                 cudaMemcpyDeviceToHost, st));
  LFX_CUDA_TRY(cudaStreamSynchronize(st));
  double e = hi;
  for (int c = 0; c < ns; ++c) {
    std::memcpy(h.data(), heads.data() + (size_t)c * kStateHead, kStateHead);
    const KState &k = h[0];
    if ((n_seg > 1 && k.done) || !(k.res > 0.0) || !(k.tol_abs > 0.0) || !std::isfinite(k.res)) continue;
    const double need = k.tol_abs / k.res;
    e = std::min(e, 0.5 * (k.j == 0 ? std::sqrt(need) : need));
  }
  *eta = std::max(lo, std::min(hi, e));
  return LFX_OK;
}

// Restarted GMRES over n_seg independent components (see set_segments); the same launches as
// solve, with every reduction and every small dense step done per component.
template <class S, class T>
lfx_status Gmres<S, T>::solve_seg(cudaStream_t st, const BsrView<S> &A, const PrecFn<T> &pc, const T *b, T *x,
                                  double rtol, int maxit, bool cgs2, int lag, bool x_zero, int *its_out,
                                  double *res_out) {
  if (lag < 0) lag = 0;
  if (lag > 2) lag = 2;
  KState *ks = state.as<KState>(), *kseg = seg_state.as<KState>();
  T *Vb = basis.as<T>(), *Zb = zbasis.as<T>(), *w = work.as<T>();
  double *pn = seg_pn.as<double>(), *pd = seg_part.as<double>();
  const SegTasks tk = tasks;
  const int nt = tk.n_task;
  // ||b_c||, tolerances; ks gets ||b||
  pdl_launch(seg_norm_kernel<T>, nt, kThreads, 0, st, b, tk, pn, nullptr);
  pdl_launch(seg_bnorm_kernel, 1, kThreads, 0, st, pn, tk, kseg, ks, rtol);
  note_launches(2);
  KState hs;
  LFX_CUDA_TRY(cudaMemcpyAsync(&hs, ks, kStateHead, cudaMemcpyDeviceToHost, st));
  LFX_CUDA_TRY(cudaStreamSynchronize(st));
  if (!std::isfinite(hs.bnorm)) {
    set_error("GMRES: right-hand side is not finite");
    return LFX_ERR_NONFINITE;
  }
  if (hs.bnorm == 0.0 || x_zero) LFX_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(T) * n, st));
  if (hs.bnorm == 0.0) {
    if (its_out) *its_out = 0;
    if (res_out) *res_out = 0.0;
    return LFX_OK;
  }
  if (!x_zero) {
    pdl_launch(seg_zero_x_kernel<T>, nt, kThreads, 0, st, x, tk, kseg);
    note_launches(1);
  }
  int total = 0;
  double rel = 1.0;
  lfx_status status = LFX_ERR_NOT_CONVERGED;
  const int fin_grid = (int)(((int64_t)n_seg * (restart + 1) * 32 + kThreads - 1) / kThreads);
  for (int cycle = 0; cycle < 100000; ++cycle) {
    // r = b - A x -> w; beta_c; v0 = r / beta_c
    LFX_TRY((launch_spmv<S, T>(st, A, x, b, w, 1, nullptr, nullptr)));
    pdl_launch(seg_norm_kernel<T>, nt, kThreads, 0, st, w, tk, pn, nullptr);
    pdl_launch(seg_cycle_start_kernel, 1, kThreads, 0, st, pn, tk, kseg, ks);
    pdl_launch(seg_scale_beta_kernel<T>, nt, kThreads, 0, st, w, Vb, tk, kseg);
    note_launches(3);
    for (int j = 0; j < restart; ++j) {
      T *vj = Vb + (int64_t)j * n, *vn = Vb + (int64_t)(j + 1) * n, *zj = Zb + (int64_t)j * n;
      LFX_TRY(pc(st, vj, zj, ks));
      LFX_TRY(timed_spmv(st, A, zj, w, ks));
      for (int pass = 0; pass < (cgs2 ? 2 : 1); ++pass) {
        pdl_launch(seg_mdot_kernel<T>, dim3(nt, (j + 8) / 8), kThreads, 0, st, Vb, n, j + 1, w, pd, tk, ks);
        pdl_launch(seg_finalize_kernel, fin_grid, kThreads, 0, st, pd, j + 1, tk, kseg, ks, pass);
        pdl_launch(seg_maxpy_kernel<T>, nt, kThreads, 0, st, Vb, n, j + 1, w, tk, kseg, pn, ks);
      }
      pdl_launch(seg_givens_kernel, 1, kThreads, 0, st, pn, tk, kseg, ks, j, restart, maxit);
      pdl_launch(seg_scale_kernel<T>, nt, kThreads, 0, st, w, vn, tk, kseg, ks);
      note_launches(2 + 3 * (cgs2 ? 2 : 1));
      LFX_CUDA_TRY(cudaMemcpyAsync(pinned + (j & 3), &ks->done, sizeof(int), cudaMemcpyDeviceToHost, st));
      LFX_CUDA_TRY(cudaEventRecord(ev[j & 3], st));
      if (j >= lag) {
        LFX_CUDA_TRY(cudaEventSynchronize(ev[(j - lag) & 3]));
        if (pinned[(j - lag) & 3]) break;
      }
    }
    pdl_launch(seg_trisolve_kernel, 1, kThreads, 0, st, tk, kseg);
    pdl_launch(seg_update_x_kernel<T, T>, nt, kThreads, 0, st, Zb, n, x, tk, kseg);
    note_launches(2);
    LFX_CUDA_TRY(cudaMemcpyAsync(&hs, ks, kStateHead, cudaMemcpyDeviceToHost, st));
    LFX_CUDA_TRY(cudaStreamSynchronize(st));
    LFX_CUDA_TRY(cudaGetLastError());
    total = hs.total;
    if (hs.flag == 2) {
      set_error("GMRES: non-finite residual after %d steps", total);
      status = LFX_ERR_NONFINITE;
      break;
    }
    if (hs.flag == 1 || total >= maxit) {
      // confirm with every component's true residual
      LFX_TRY((launch_spmv<S, T>(st, A, x, b, w, 1, nullptr, nullptr)));
      pdl_launch(seg_norm_kernel<T>, nt, kThreads, 0, st, w, tk, pn, nullptr);
      pdl_launch(seg_confirm_kernel, 1, kThreads, 0, st, pn, tk, kseg, ks);
      note_launches(2);
      LFX_CUDA_TRY(cudaMemcpyAsync(&hs, ks, kStateHead, cudaMemcpyDeviceToHost, st));
      LFX_CUDA_TRY(cudaStreamSynchronize(st));
      rel = hs.res;
      if (!std::isfinite(rel)) {
        status = LFX_ERR_NONFINITE;
        set_error("GMRES: non-finite true residual");
        break;
      }
      if (hs.flag == 1) {
        status = LFX_OK;
        break;
      }
      if (total >= maxit) {
        set_error("GMRES: not converged after %d steps (largest relative residual %.3e)", total, rel);
        status = LFX_ERR_NOT_CONVERGED;
        break;
      }
    }
  }
  if (its_out) *its_out = total;
  if (res_out) *res_out = rel;
  return status;
}

// w = b - A x (with the rank-one terms) and the partial sums of |w|^2 in pn (*ng of them)
template <class S, class T>
lfx_status Gmres<S, T>::residual(cudaStream_t st, const BsrView<S> &A, const T *x, const T *b, T *w, double *pn,
                                 int *ng) {
  if (r1.n_tags == 0) return launch_spmv<S, T>(st, A, x, b, w, 1, pn, ng);
  LFX_TRY((launch_spmv<S, T>(st, A, x, b, w, 1, nullptr, nullptr)));
  apply_rank1(st, x, w, -1.0, nullptr);
  const int vg = vec_grid(n);
  pdl_launch(norm_kernel<T>, vg, kThreads, 0, st, (const T *)w, n, pn);
  note_launches(1);
  *ng = vg;
  LFX_CUDA_TRY(cudaGetLastError());
  return LFX_OK;
}

template <class S, class T>
lfx_status Gmres<S, T>::set_rank1(const Rank1View &r) {
  if (n_seg > 1) {
    set_error("GMRES: rank-one terms need a single system");
    return LFX_ERR_INVALID_ARG;
  }
  r1 = r;
  if (r.n_tags > 0) LFX_TRY(r1_s.alloc(sizeof(double) * (size_t)r.n_tags));
  return LFX_OK;
}

template <class S, class T>
void Gmres<S, T>::apply_rank1(cudaStream_t st, const T *x, T *y, double sign, const KState *ks) {
  pdl_launch(rank1_dot_kernel<T>, r1.n_tags, kThreads, 0, st, r1, x, r1_s.as<double>(), ks);
  pdl_launch(rank1_axpy_kernel<T>, (int)std::max<int64_t>(1, (r1.n_ax + kThreads - 1) / kThreads), kThreads, 0, st, r1,
             (const double *)r1_s.as<double>(), y, sign, ks);
  note_launches(2);
}

// The Arnoldi product w = A z; the 3rd, 8th, 13th, ... of them after each reset of n_tev (at most
// kTimedSpmv) bracketed by CUDA events for the SpMV timing statistics.
constexpr int kTimedSpmv = 4;
template <class S, class T>
lfx_status Gmres<S, T>::timed_spmv(cudaStream_t st, const BsrView<S> &A, const T *z, T *w, const KState *ks) {
  const int call = n_spmv_calls++;
  if (n_tev >= 2 * kTimedSpmv || call % 5 != 2) {
    // one product in five is timed, up to kTimedSpmv per step: an event between two launches costs
    // the overlap of programmatic dependent launch there
    arnoldi_spmv(st, A, z, w, ks);
    if (r1.n_tags > 0) apply_rank1(st, z, w, 1.0, ks);
    return LFX_OK;
  }
  if (n_tev + 2 > (int)tev.size()) {
    for (int q = 0; q < 64; ++q) {
      cudaEvent_t e;
      LFX_CUDA_TRY(cudaEventCreate(&e));
      tev.push_back(e);
    }
  }
  LFX_CUDA_TRY(cudaEventRecord(tev[n_tev], st));
  arnoldi_spmv(st, A, z, w, ks);
  if (r1.n_tags > 0) apply_rank1(st, z, w, 1.0, ks);
  LFX_CUDA_TRY(cudaEventRecord(tev[n_tev + 1], st));
  n_tev += 2;
  return LFX_OK;
}

// Steps j = 0 .. m-1 of one Arnoldi cycle from v_0 (flexible: z_j = M^-1 v_j kept), classical
// Gram-Schmidt (twice with cgs2), Givens rotations and the stopping test on the device; the host
// reads the device's stop flag lag steps behind the launches, so the device always has queued work.
template <class S, class T>
lfx_status Gmres<S, T>::arnoldi_cycle(cudaStream_t st, const BsrView<S> &A, const PrecFn<T> &pc, int m, int maxit,
                                      bool cgs2, int lag) {
  KState *ks = state.as<KState>();
  T *Vb = basis.as<T>(), *Zb = zbasis.as<T>(), *w = work.as<T>();
  double *pn = part_n.as<double>();
  const int vg = vec_grid(n);
  for (int j = 0; j < m; ++j) {
    T *vj = Vb + (int64_t)j * n, *vn = Vb + (int64_t)(j + 1) * n, *zj = Zb + (int64_t)j * n;
    LFX_TRY(pc(st, vj, zj, ks));
    LFX_TRY(timed_spmv(st, A, zj, w, ks));
    for (int pass = 0; pass < (cgs2 ? 2 : 1); ++pass) {
      pdl_launch(mdot_kernel<T>, dim3(nblk_dot, (j + 8) / 8), kThreads, 0, st, Vb, n, j + 1, w, n, part.as<double>(),
                 nblk_dot, ks);
      pdl_launch(mdot_finalize_kernel, j + 1, 32, 0, st, part.as<double>(), nblk_dot, nblk_dot, j + 1, ks, pass);
      pdl_launch(maxpy_kernel<T>, vg, kThreads, 0, st, Vb, n, j + 1, w, n, pn, ks);
    }
    pdl_launch(givens_kernel, 1, kThreads, 0, st, pn, vg, ks, j, m, maxit);
    pdl_launch(scale_kernel<T>, vg, kThreads, 0, st, w, vn, n, &ks->scale, ks);
    note_launches(2 + 3 * (cgs2 ? 2 : 1));
    LFX_CUDA_TRY(cudaMemcpyAsync(pinned + (j & 3), &ks->done, sizeof(int), cudaMemcpyDeviceToHost, st));
    LFX_CUDA_TRY(cudaEventRecord(ev[j & 3], st));
    if (j >= lag) {
      LFX_CUDA_TRY(cudaEventSynchronize(ev[(j - lag) & 3]));
      if (pinned[(j - lag) & 3]) break;
    }
  }
  LFX_CUDA_TRY(cudaGetLastError());
  return LFX_OK;
}

template <class S, class T>
lfx_status Gmres<S, T>::solve_inner(cudaStream_t st, const BsrView<S> &A, const PrecFn<T> &pc, const T *b, T *x,
                                    double rtol, const KState *outer, double lo, double hi, int maxit, bool cgs2,
                                    int lag, int *its_pinned) {
  if (n_seg > 1 || maxit > restart) {
    set_error("GMRES: solve_inner needs one component and maxit <= restart");
    return LFX_ERR_INVALID_ARG;
  }
  if (lag < 0) lag = 0;
  if (lag > 2) lag = 2;
  KState *ks = state.as<KState>();
  T *Vb = basis.as<T>(), *Zb = zbasis.as<T>();
  double *pn = part_n.as<double>();
  const int vg = vec_grid(n);
  LFX_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(T) * n, st));
  // r = b: ||b||, tolerance, v0 = b / beta
  pdl_launch(norm_kernel<T>, vg, kThreads, 0, st, b, n, pn);
  pdl_launch(inner_start_kernel, 1, kThreads, 0, st, pn, vg, ks, outer, rtol, lo, hi);
  pdl_launch(scale_beta_kernel<T>, vg, kThreads, 0, st, b, Vb, n, ks);
  note_launches(3);
  LFX_TRY(arnoldi_cycle(st, A, pc, std::min(maxit, restart), maxit, cgs2, lag));
  pdl_launch(trisolve_kernel, 1, 32, 0, st, ks);
  pdl_launch(update_x_kernel<T, T>, vg, kThreads, 0, st, Zb, n, x, n, ks);
  note_launches(2);
  if (its_pinned) LFX_CUDA_TRY(cudaMemcpyAsync(its_pinned, &ks->total, sizeof(int), cudaMemcpyDeviceToHost, st));
  LFX_CUDA_TRY(cudaGetLastError());
  return LFX_OK;
}

template struct Gmres<double, double>;
template struct Gmres<float, float>;
template struct Gmres<DDMat, double>;

template <class A, class B>
lfx_status launch_convert(cudaStream_t st, const A *src, B *dst, int64_t n, const KState *ks) {
  pdl_launch(convert_kernel<A, B>, vec_grid(n), kThreads, 0, st, src, dst, n, ks);
  note_launches(1);
  LFX_CUDA_TRY(cudaGetLastError());
  return LFX_OK;
}
template lfx_status launch_convert<double, float>(cudaStream_t, const double *, float *, int64_t, const KState *);
template lfx_status launch_convert<float, double>(cudaStream_t, const float *, double *, int64_t, const KState *);
template lfx_status launch_convert<double, __nv_bfloat16>(cudaStream_t, const double *, __nv_bfloat16 *, int64_t,
                                                          const KState *);

}  // namespace lfx
