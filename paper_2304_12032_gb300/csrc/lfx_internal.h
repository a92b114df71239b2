// Internal declarations shared by the host runtime (.cpp) and the CUDA kernels (.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "lfx.h"

namespace lfx {

// ---------------------------------------------------------------- errors
void set_error(const char *fmt, ...);
void clear_error();

#define LFX_CUDA_TRY(expr)                                                                 \
  do {                                                                                     \
    cudaError_t e_ = (expr);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      ::lfx::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__,     \
                       __LINE__);                                                          \
      return LFX_ERR_CUDA;                                                                 \
    }                                                                                      \
  } while (0)

#define LFX_TRY(expr)                 \
  do {                                \
    lfx_status s_ = (expr);           \
    if (s_ != LFX_OK) return s_;      \
  } while (0)

// ---------------------------------------------------------------- launch accounting
// Number of kernels this library has launched (diagnostic; read with lfx_launch_count).
void note_launches(int64_t n);

// ---------------------------------------------------------------- device memory
// Every allocation remembers the free function of the allocator that made it (lfx_set_allocator
// may switch allocators while buffers made by the previous one are still alive).
struct DFree {
  lfx_free_fn fn = nullptr;   // null: cudaFree
  void *ctx = nullptr;
};
void *dalloc(size_t bytes, DFree *how);   // nullptr on failure (error message set)
void dfree(void *p, const DFree &how);

// A device buffer that frees itself; tracks its size for admission control.
struct DBuf {
  void *p = nullptr;
  size_t bytes = 0;
  bool owned = true;   // false: a slice of memory owned elsewhere (never freed here)
  DFree how;           // how to free p
  DBuf() = default;
  DBuf(const DBuf &) = delete;
  DBuf &operator=(const DBuf &) = delete;
  DBuf(DBuf &&o) noexcept : p(o.p), bytes(o.bytes), owned(o.owned), how(o.how) {
    o.p = nullptr;
    o.bytes = 0;
  }
  DBuf &operator=(DBuf &&o) noexcept {
    if (this != &o) {
      release();
      p = o.p;
      bytes = o.bytes;
      owned = o.owned;
      how = o.how;
      o.p = nullptr;
      o.bytes = 0;
    }
    return *this;
  }
  ~DBuf() { release(); }
  void release() {
    if (p && owned) dfree(p, how);
    p = nullptr;
    bytes = 0;
    owned = true;
  }
  void borrow(void *ptr, size_t n) {
    release();
    p = ptr;
    bytes = n;
    owned = false;
  }
  lfx_status alloc(size_t n) {
    release();
    if (n == 0) n = 16;
    p = dalloc(n, &how);
    if (!p) return LFX_ERR_OOM;
    bytes = n;
    return LFX_OK;
  }
  template <class T> T *as() const { return static_cast<T *>(p); }
};

// ---------------------------------------------------------------- mesh (host + device)
struct Mesh {
  int64_t V = 0, T = 0, F = 0, nnzb = 0;
  int n_flipped = 0;
  bool uploaded = false;
  // renumbering
  std::vector<int32_t> node_old;     // internal node -> caller node
  std::vector<int32_t> node_new;     // caller node -> internal node
  std::vector<int32_t> elem_old;     // internal element (colour-sorted) -> caller element
  // geometry / topology, internal numbering
  std::vector<double> xyz;           // [V][3]
  std::vector<int32_t> tets;         // [T][4], positively oriented
  std::vector<int32_t> row_ptr;      // [V+1]
  std::vector<int32_t> col_idx;      // [nnzb], sorted per row
  std::vector<int32_t> diag_idx;     // [V] block index of (i,i)
  std::vector<int32_t> trans_idx;    // [nnzb] block index of (j,i) for block (i,j)
  std::vector<int32_t> slot;         // [T][16] block index of (node a, node b), a*4+b
  std::vector<uint16_t> first;       // [T] bit 4a+b: the element writes block (a, b) before any other
  bool all_blocks_touched = false;   // every block of the pattern belongs to some element
  bool all_nodes_touched = false;    // every node belongs to some element
  std::vector<int32_t> color_off;    // [n_colors+1] offsets into color_elems
  std::vector<int32_t> color_elems;  // [T] internal element ids listed colour by colour (Morton order inside)
  // chunked assembly: chunks of at most kChunkElems consecutive internal elements (a compact piece of
  // the Morton order); chunks coloured so that no two chunks of one colour share a node, the internal
  // element order running chunk by chunk, colour by colour.  Each chunk's (element, a, b) block
  // contributions are packed into passes of 4 kChunkElems slots, grouped in runs that share one
  // matrix block, no run straddling two passes.
  std::vector<int32_t> chunk_elem_off;   // [n_chunks+1] element ranges
  std::vector<int32_t> chunk_color_off;  // [n_chunk_colors+1] chunk ranges per colour
  std::vector<int32_t> chunk_pass_off;   // [n_chunks+1] pass ranges
  std::vector<uint16_t> pass_code;       // [n_passes][4 kChunkElems]: le << 4 | a << 2 | b, 0xffff idle
  std::vector<int32_t> pass_run_off;     // [n_passes+1] run ranges (diagonal runs first)
  std::vector<int32_t> pass_ndiag;       // [n_passes] diagonal runs (a == b: also the node's rhs row)
  std::vector<uint16_t> run_meta;        // slot start (bits 0-7) | length (8-13) | first writer (14) | diagonal (15)
  std::vector<int32_t> run_block;        // [runs] block index in the pattern
  std::vector<int32_t> run_node;         // [runs] node of a diagonal run (its rhs row), else -1
  // tiles of the staged velocity smoothing pass: consecutive block rows, at most kFTileRows rows and
  // kFTileBlocks blocks each ([n_tiles+1] row offsets; empty when some row alone exceeds the limit)
  std::vector<int32_t> ftile_row;
  std::vector<uint8_t> bad;          // [T] 1 if below the shape-quality threshold
  std::vector<int32_t> bfaces;       // [F][3] outward oriented, internal numbering
  std::vector<int32_t> btags;        // [F]
  std::vector<double> quality;       // [T] 6 sqrt2 |K| / e_rms^3
  int32_t n_comp = 1;                // connected components (batched independent meshes)
  std::vector<int32_t> comp_off;     // [n_comp+1] contiguous internal node range per component
  // device copies
  DBuf d_xyz;       // double4 [V] (x, y, z, 0)
  DBuf d_xyz_hi, d_xyz_lo;   // float4 [V]: d_xyz split into FP32 high and low parts
  DBuf d_conn;      // int4 [T]
  DBuf d_slot;      // int32 [T][16]
  DBuf d_rowptr;    // int32 [V+1]
  DBuf d_col;       // int32 [nnzb]
  DBuf d_diag;      // int32 [V]
  DBuf d_trans;     // int32 [nnzb]
  DBuf d_comp_off;  // int32 [n_comp+1]
  DBuf d_node_old;  // int32 [V] internal node -> caller node (host arrays in, solutions out)
  DBuf d_first;     // uint16 [T] (first)
  DBuf d_color_elems;
  DBuf d_chunk_elem_off, d_chunk_pass_off, d_pass_code, d_pass_run_off, d_pass_ndiag, d_run_meta, d_run_block,
      d_run_node;
  DBuf d_ftile_row;
  size_t device_bytes() const;
};

lfx_status build_mesh(const double *nodes, int64_t n_nodes, const int32_t *tets, int64_t n_tets,
                      const int32_t *bfaces, const int32_t *tags, int64_t n_bfaces, Mesh &m);
lfx_status upload_mesh(Mesh &m);

// ---------------------------------------------------------------- kernels' parameter blocks
constexpr int kMaxRiis = 8;
struct PhysParams {
  double rho, mu, dt, alpha, sigma, c_r;
  double f[3];
  int32_t n_riis, stab, diffusion, pad;
  double riis_r[kMaxRiis], riis_eps[kMaxRiis];
  // derived once on the host so that the kernels need no divisions
  double rho_dt;                 // rho / dt
  double rho_alpha_dt;           // rho alpha / dt
  double tau_t;                  // sigma^2 rho^2 / dt^2 (time part of tau_M^-2)
  double cr_mu2;                 // C_r mu^2
  double riis_coef[kMaxRiis];    // R_k / eps_k
  double riis_pi_eps[kMaxRiis];  // pi / eps_k
  double riis_inv2eps[kMaxRiis]; // 1 / (2 eps_k)
};

constexpr int kChunkElems = 32;     // elements per chunk (one CTA pass of the assembly kernels)
constexpr int kChunkMaxPasses = 8;  // passes of 4 kChunkElems slots a chunk may take (the kernels stage
                                    // a chunk's slot codes for this many in shared memory)
// tile limits of the staged velocity smoothing pass (its CTA handles kFTileRows rows with 4 lanes
// each, and stages at most kFTileBlocks 24-byte BF16 sub-block records in each of two buffers;
// measured on a 1M-tet mesh against 64-row tiles of 1536, 1024, 768 and 512 blocks: small buffers
// leave the SM's L1 to the gathers of the iterate)
constexpr int kFTileRows = 32;
constexpr int kFTileBlocks = 512;
// Chunks the chunked double-float assembly kernel processes in one wave (resident CTAs x SMs).
int64_t assemble_chunk_wave();
// Elements the double-float assembly kernel processes in one wave over the whole device (resident
// CTAs per SM x SMs x elements per CTA; GB300's 152 SMs x 3 x 32 when no device answers): the
// quantum the element colouring is balanced to.
int64_t assemble_wave_elements();

}  // namespace lfx

// opaque handles of the C ABI
struct lfx_mesh {
  lfx::Mesh m;
};
