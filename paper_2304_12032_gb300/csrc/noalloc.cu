// lfx_asimple_apply_noalloc: the aSIMPLE preconditioner application (the same kernels as the
// step's preconditioner) for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need the preconditioner: code
// running while a CUDA graph is being captured (allocation is not allowed inside a capture),
// solvers embedded in a host framework that owns all device memory through its own pool, or
// time-critical loops that must not pay an allocation's latency or risk its failure midway.
// This entry point takes the caller's matrix and vectors and keeps every intermediate array
// (inverse diagonals, Chebyshev iterates, coefficients, reduction partials) in one file-scope
// static device array of fixed size, which exists on every GPU that loads the library until
// the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "lfx_internal.h"
#include "solver.h"

namespace {

constexpr int64_t kNoAllocMaxNodes = 65536;              // largest accepted matrix (block rows)
constexpr size_t kNoAllocScratchBytes = 16u << 20;        // 16 MiB of work memory per device
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_asimple_scratch[kNoAllocScratchBytes];

std::mutex g_scratch_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the static array on the current device, looked up once per device.  The
// array's name in host code is only a host-side stand-in, never a device address.
lfx_status scratch_address(void **out) {
  int dev = 0;
  LFX_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    lfx::set_error("lfx_asimple_apply_noalloc: device index %d out of range", dev);
    return LFX_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    LFX_CUDA_TRY(cudaGetSymbolAddress(&p, g_asimple_scratch));
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return LFX_OK;
}

}  // namespace

using namespace lfx;

extern "C" lfx_status lfx_asimple_apply_noalloc(int64_t n_nodes, const int32_t *row_ptr, const int32_t *col_idx,
                                                const int32_t *diag_idx, const int32_t *trans_idx,
                                                const double *blocks, const double *r, double *z,
                                                const lfx_options *opt, void *cuda_stream) {
  clear_error();
  if (!row_ptr || !col_idx || !diag_idx || !trans_idx || !blocks || !r || !z) {
    set_error("lfx_asimple_apply_noalloc: NULL argument");
    return LFX_ERR_INVALID_ARG;
  }
  if (n_nodes < 1 || n_nodes > kNoAllocMaxNodes) {
    set_error("lfx_asimple_apply_noalloc: n_nodes = %lld outside [1, %lld] (the fixed work memory holds "
              "matrices of at most %lld block rows)",
              (long long)n_nodes, (long long)kNoAllocMaxNodes, (long long)kNoAllocMaxNodes);
    return LFX_ERR_INVALID_ARG;
  }
  lfx_options o;
  if (opt) {
    o = *opt;
  } else {
    lfx_options_default(&o);
    o.s_smoother = LFX_SMOOTH_CHEBYSHEV;
    o.s_steps = 6;
  }
  if (o.f_smoother < 0 || o.f_smoother > 1 || o.s_smoother < 0 || o.s_smoother > 1 || o.f_steps < 1 ||
      o.f_steps > kMaxSmooth || o.s_steps < 1 || o.s_steps > kMaxSmooth || o.n_power < 0) {
    set_error("lfx_asimple_apply_noalloc: smoothers must be Jacobi or Chebyshev (the Schur AMG needs "
              "allocated set-up data) with 1..%d steps",
              kMaxSmooth);
    return LFX_ERR_INVALID_ARG;
  }
  void *scratch = nullptr;
  LFX_TRY(scratch_address(&scratch));
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
  cudaStream_t st = (cudaStream_t)cuda_stream;
  ASimple<double, double> pc;
  LFX_TRY(pc.init_borrowed(n_nodes, cfg, scratch, kNoAllocScratchBytes, st));
  const BsrView<double> A{n_nodes, row_ptr, col_idx, diag_idx, trans_idx, blocks};
  LFX_TRY(pc.setup(st, A));
  LFX_TRY(pc.apply(st, A, r, z, nullptr));
  LFX_CUDA_TRY(cudaGetLastError());
  return LFX_OK;
}
