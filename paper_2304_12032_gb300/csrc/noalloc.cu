// lfx_asimple_apply_noalloc: the aSIMPLE preconditioner application (the same kernels as the
// step's preconditioner) for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need the preconditioner: solvers
// embedded in a host framework that owns all device memory through its own pool (a second
// allocator would compete with it for the same HBM), and time-critical loops that must not pay an
// allocation's latency (cudaMalloc may synchronise the whole device) or risk its failure midway.
// This entry point takes the caller's matrix and vectors and keeps every intermediate array
// (inverse diagonals, Chebyshev iterates, coefficients, reduction partials) in one file-scope
// static device array of fixed size, which exists on every GPU that loads the library until
// the process exits.
#include <cuda.h>
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
// the array's device address per device, with the id of the context it was looked up in: a
// device reset (or any teardown and re-creation of the context) may load the module again at
// another address, so a lookup is only reused within the same context
struct ScratchAddr {
  void *ptr = nullptr;
  unsigned long long ctx_id = 0;
  bool valid = false;
};
ScratchAddr g_scratch[kMaxDevices];

// Id of the calling thread's current context (driver entry points resolved through the runtime,
// so that the library needs no link to the driver library); false if there is none or the
// driver does not offer the calls.
bool current_context_id(unsigned long long *id) {
  typedef CUresult (*GetCurrentFn)(CUcontext *);
  typedef CUresult (*GetIdFn)(CUcontext, unsigned long long *);
  static GetCurrentFn get_current = nullptr;
  static GetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = (GetCurrentFn)f;
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = (GetIdFn)f;
    (void)cudaGetLastError();
  });
  if (!get_current || !get_id) return false;
  CUcontext c = nullptr;
  if (get_current(&c) != CUDA_SUCCESS || !c) return false;
  return get_id(c, id) == CUDA_SUCCESS;
}

// Device address of the static array on the current device: looked up with cudaGetSymbolAddress
// once per device and context (the first call on a device, and the first after its context was
// reset), with that device current.  The array's name in host code is only a host-side stand-in,
// never a device address.
lfx_status scratch_address(void **out) {
  int dev = 0;
  LFX_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    lfx::set_error("lfx_asimple_apply_noalloc: device index %d out of range", dev);
    return LFX_ERR_INVALID_ARG;
  }
  unsigned long long id = 0;
  bool have_id = current_context_id(&id);
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  ScratchAddr &c = g_scratch[dev];
  if (have_id && c.valid && c.ctx_id == id) {
    *out = c.ptr;
    return LFX_OK;
  }
  void *p = nullptr;
  LFX_CUDA_TRY(cudaGetSymbolAddress(&p, g_asimple_scratch));
  if (!have_id) have_id = current_context_id(&id);   // the lookup may have made the context current
  c.ptr = p;
  c.ctx_id = id;
  c.valid = have_id;                                 // without a context id: look it up every call
  *out = p;
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
