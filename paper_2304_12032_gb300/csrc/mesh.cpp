// Host-side mesh set-up (once per mesh): validation and orientation, space-filling-curve
// renumbering of nodes and elements, the 4x4 block-CSR pattern of the node graph (the DoF
// pattern of P1-P1 with 4 unknowns per node, Section 2.3), the element -> block-slot map, the
// transpose map, outward boundary faces, and a greedy element colouring so that elements of one
// colour share no node and their block updates need no atomics.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "lfx_internal.h"

namespace lfx {

namespace {

// 21-bit-per-axis Morton code of a point inside the bounding box [lo, lo + span].
inline uint64_t spread3(uint64_t v) {
  v &= 0x1fffff;
  v = (v | v << 32) & 0x1f00000000ffffULL;
  v = (v | v << 16) & 0x1f0000ff0000ffULL;
  v = (v | v << 8) & 0x100f00f00f00f00fULL;
  v = (v | v << 4) & 0x10c30c30c30c30c3ULL;
  v = (v | v << 2) & 0x1249249249249249ULL;
  return v;
}
inline uint64_t morton(const double *p, const double *lo, double inv_span) {
  uint64_t c[3];
  for (int k = 0; k < 3; ++k) {
    double t = (p[k] - lo[k]) * inv_span;
    t = t < 0 ? 0 : (t > 1 ? 1 : t);
    c[k] = (uint64_t)(t * 2097151.0);
  }
  return spread3(c[0]) | (spread3(c[1]) << 1) | (spread3(c[2]) << 2);
}

// Colour sizes rebalanced toward whole waves of the assembly kernel.  A colour of s elements runs
// as ceil(s / W) waves of W elements (W = resident CTAs x elements per CTA over all SMs), and
// colours run one after another, so the greedy colouring's decreasing sizes (a 1M-tet mesh: 52.5
// waves of work in 38 colours, launched as 68 waves) waste most of a wave per colour.  The colour
// count stays (it is bounded below by the largest number of elements at one node); each colour
// gets a target of k_c >= 1 whole waves, the extra waves going to the colours with the most
// elements above their target, until the targets hold all T elements with a quarter wave to
// spare.  Elements then move from over-full colours to the under-full colour with the most room
// among those free at all four of their nodes (in practice from the large early colours up into
// the sparse late ones, which the greedy pass left free almost everywhere), so the colouring
// stays valid whatever the moves achieve.  Deterministic; returns the colour count.
// The same for any items with node sets (elements: 4 nodes; chunks: the nodes of their elements):
// nodes_of(e, n) returns a pointer to item e's n nodes.
template <class NodesOf>
int balance_colours(int64_t T, NodesOf nodes_of, const std::vector<int32_t> &eorder, std::vector<uint64_t> &used,
                    std::vector<int32_t> &color, int C, int kWords, int64_t W) {
  if (W <= 0 || C < 2) return C;
  std::vector<int64_t> sz(C, 0), k(C, 1);
  for (int64_t e = 0; e < T; ++e) sz[color[e]]++;
  if (*std::max_element(sz.begin(), sz.end()) <= W) return C;   // every colour is one wave or less
  int64_t waves = C;
  while (waves * W < T + W / 4) {
    int best = 0;
    for (int c = 1; c < C; ++c)
      if (sz[c] - k[c] * W > sz[best] - k[best] * W) best = c;
    ++k[best];
    ++waves;
  }
  auto bit = [&](int32_t n, int c) { return (used[(size_t)n * kWords + c / 64] >> (c % 64)) & 1ULL; };
  // passes of moves; when elements are left over, the last colour that can still grow (the late
  // colours are the ones free at most nodes) gets one more wave, while that beats the greedy sizes
  int64_t greedy_waves = 0;
  for (int c = 0; c < C; ++c) greedy_waves += (sz[c] + W - 1) / W;
  int grow = C - 1;
  for (int pass = 0; pass < 8; ++pass) {
    for (int64_t s = T - 1; s >= 0; --s) {
      const int32_t e = eorder[s];
      const int a = color[e];
      if (sz[a] <= k[a] * W) continue;
      int nn = 0;
      const int32_t *nd = nodes_of(e, nn);
      int b = -1;
      int64_t room = 0;
      for (int c = 0; c < C; ++c) {
        const int64_t r = k[c] * W - sz[c];
        if (c == a || r <= room) continue;
        bool busy = false;
        for (int q = 0; q < nn && !busy; ++q) busy = bit(nd[q], c);
        if (busy) continue;
        b = c;
        room = r;
      }
      if (b < 0) continue;
      for (int q = 0; q < nn; ++q) {
        used[(size_t)nd[q] * kWords + a / 64] &= ~(1ULL << (a % 64));
        used[(size_t)nd[q] * kWords + b / 64] |= 1ULL << (b % 64);
      }
      color[e] = b;
      --sz[a];
      ++sz[b];
    }
    int64_t now = 0;
    bool over = false;
    for (int c = 0; c < C; ++c) {
      now += (sz[c] + W - 1) / W;
      over |= sz[c] > k[c] * W;
    }
    if (!over || now + 1 >= greedy_waves || grow < 0) break;
    ++k[grow];
    grow = grow > 0 ? grow - 1 : C - 1;
  }
  int n = 0;
  for (int c = 0; c < C; ++c) n += sz[c] > 0;
  if (n < C) {   // (not expected: every target is at least one wave)
    std::vector<int> renum(C, -1);
    n = 0;
    for (int c = 0; c < C; ++c)
      if (sz[c] > 0) renum[c] = n++;
    for (int64_t e = 0; e < T; ++e) color[e] = renum[color[e]];
  }
  return n;
}

double signed_det(const double *x0, const double *x1, const double *x2, const double *x3) {
  double a[3], b[3], c[3];
  for (int k = 0; k < 3; ++k) {
    a[k] = x1[k] - x0[k];
    b[k] = x2[k] - x0[k];
    c[k] = x3[k] - x0[k];
  }
  return a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) +
         a[2] * (b[0] * c[1] - b[1] * c[0]);
}

}  // namespace

size_t Mesh::device_bytes() const {
  return d_xyz.bytes + d_xyz_hi.bytes + d_xyz_lo.bytes + d_conn.bytes + d_slot.bytes + d_rowptr.bytes + d_col.bytes + d_diag.bytes +
         d_trans.bytes + d_comp_off.bytes + d_node_old.bytes + d_first.bytes + d_color_elems.bytes +
         d_chunk_elem_off.bytes + d_chunk_pass_off.bytes + d_pass_code.bytes + d_pass_run_off.bytes +
         d_pass_ndiag.bytes + d_run_meta.bytes + d_run_block.bytes + d_run_node.bytes + d_ftile_row.bytes;
}

lfx_status build_mesh(const double *nodes, int64_t n_nodes, const int32_t *tets_in, int64_t n_tets,
                      const int32_t *bfaces_in, const int32_t *tags_in, int64_t n_bfaces,
                      Mesh &m) {
  if (!nodes || !tets_in || n_nodes < 4 || n_tets < 1 || n_bfaces < 0 ||
      (n_bfaces > 0 && (!bfaces_in || !tags_in))) {
    set_error("lfx_mesh_create: null array or size out of range");
    return LFX_ERR_INVALID_ARG;
  }
  if (n_nodes > (int64_t)INT32_MAX / 4 || n_tets > (int64_t)INT32_MAX / 16) {
    set_error("lfx_mesh_create: mesh too large for 32-bit indices");
    return LFX_ERR_INVALID_ARG;
  }
  const int64_t V = n_nodes, T = n_tets, F = n_bfaces;
  m.V = V;
  m.T = T;
  m.F = F;
  for (int64_t i = 0; i < 4 * T; ++i)
    if (tets_in[i] < 0 || tets_in[i] >= V) {
      set_error("lfx_mesh_create: tet %lld references node %d outside [0,%lld)",
                (long long)(i / 4), tets_in[i], (long long)V);
      return LFX_ERR_BAD_MESH;
    }
  for (int64_t i = 0; i < 3 * F; ++i)
    if (bfaces_in[i] < 0 || bfaces_in[i] >= V) {
      set_error("lfx_mesh_create: boundary face %lld references a node out of range",
                (long long)(i / 3));
      return LFX_ERR_BAD_MESH;
    }
  for (int64_t i = 0; i < 3 * V; ++i)
    if (!std::isfinite(nodes[i])) {
      set_error("lfx_mesh_create: non-finite node coordinate");
      return LFX_ERR_BAD_MESH;
    }

  // ---- node renumbering along a Morton curve
  double lo[3] = {nodes[0], nodes[1], nodes[2]}, hi[3] = {nodes[0], nodes[1], nodes[2]};
  for (int64_t i = 0; i < V; ++i)
    for (int k = 0; k < 3; ++k) {
      lo[k] = std::min(lo[k], nodes[3 * i + k]);
      hi[k] = std::max(hi[k], nodes[3 * i + k]);
    }
  double span = std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
  double inv_span = span > 0 ? 1.0 / span : 1.0;
  std::vector<uint64_t> key(V);
  for (int64_t i = 0; i < V; ++i) key[i] = morton(nodes + 3 * i, lo, inv_span);
  // connected components of the element graph (independent simulations batched in one mesh):
  // union-find over the element vertices, components numbered by their smallest caller node
  std::vector<int32_t> uf(V);
  std::iota(uf.begin(), uf.end(), 0);
  auto findr = [&](int32_t x) {
    while (uf[x] != x) {
      uf[x] = uf[uf[x]];
      x = uf[x];
    }
    return x;
  };
  for (int64_t e = 0; e < T; ++e)
    for (int a = 1; a < 4; ++a) {
      int32_t r0 = findr(tets_in[4 * e]), r1 = findr(tets_in[4 * e + a]);
      if (r0 != r1) uf[std::max(r0, r1)] = std::min(r0, r1);
    }
  std::vector<int32_t> comp_of_root(V, -1), comp_in(V);
  int32_t ncomp = 0;
  for (int64_t i = 0; i < V; ++i) {
    const int32_t r = findr((int32_t)i);
    if (comp_of_root[r] < 0) comp_of_root[r] = ncomp++;
    comp_in[i] = comp_of_root[r];
  }
  m.n_comp = ncomp;
  m.node_old.resize(V);
  std::iota(m.node_old.begin(), m.node_old.end(), 0);
  std::stable_sort(m.node_old.begin(), m.node_old.end(), [&](int32_t a, int32_t b) {
    return comp_in[a] != comp_in[b] ? comp_in[a] < comp_in[b] : key[a] < key[b];
  });
  m.node_new.assign(V, 0);
  for (int64_t i = 0; i < V; ++i) m.node_new[m.node_old[i]] = (int32_t)i;
  m.xyz.resize(3 * V);
  for (int64_t i = 0; i < V; ++i)
    for (int k = 0; k < 3; ++k) m.xyz[3 * i + k] = nodes[3 * (int64_t)m.node_old[i] + k];
  // contiguous node range of each component in the internal numbering
  m.comp_off.assign(ncomp + 1, 0);
  for (int64_t i = 0; i < V; ++i) m.comp_off[comp_in[m.node_old[i]] + 1]++;
  for (int c = 0; c < ncomp; ++c) m.comp_off[c + 1] += m.comp_off[c];

  // ---- elements: renumber nodes, orient, quality, Morton order of centroids
  std::vector<int32_t> tt(4 * T);
  std::vector<double> qual(T);
  m.n_flipped = 0;
  double scale = span > 0 ? span : 1.0;
  for (int64_t e = 0; e < T; ++e) {
    int32_t v[4];
    for (int a = 0; a < 4; ++a) v[a] = m.node_new[tets_in[4 * e + a]];
    const double *x[4];
    for (int a = 0; a < 4; ++a) x[a] = &m.xyz[3 * (int64_t)v[a]];
    double det = signed_det(x[0], x[1], x[2], x[3]);
    double e2 = 0;
    for (int a = 0; a < 4; ++a)
      for (int b = a + 1; b < 4; ++b)
        for (int k = 0; k < 3; ++k) e2 += (x[a][k] - x[b][k]) * (x[a][k] - x[b][k]);
    double erms = std::sqrt(e2 / 6.0);
    if (!(std::fabs(det) > 1e-15 * erms * erms * erms) || erms <= 1e-300 * scale) {
      set_error("lfx_mesh_create: tet %lld has zero volume", (long long)e);
      return LFX_ERR_BAD_MESH;
    }
    if (det < 0) {
      std::swap(v[2], v[3]);
      ++m.n_flipped;
    }
    qual[e] = std::fabs(det) / 6.0 * 6.0 * std::sqrt(2.0) / (erms * erms * erms);
    for (int a = 0; a < 4; ++a) tt[4 * e + a] = v[a];
  }
  std::vector<uint64_t> ekey(T);
  for (int64_t e = 0; e < T; ++e) {
    double c[3] = {0, 0, 0};
    for (int a = 0; a < 4; ++a)
      for (int k = 0; k < 3; ++k) c[k] += 0.25 * m.xyz[3 * (int64_t)tt[4 * e + a] + k];
    ekey[e] = morton(c, lo, inv_span);
  }
  std::vector<int32_t> eorder(T);
  std::iota(eorder.begin(), eorder.end(), 0);
  std::stable_sort(eorder.begin(), eorder.end(),
                   [&](int32_t a, int32_t b) { return ekey[a] < ekey[b]; });

  // ---- greedy colouring in Morton order: smallest colour unused at the element's 4 nodes
  constexpr int kWords = 4;  // up to 256 colours
  std::vector<uint64_t> used((size_t)V * kWords, 0);
  std::vector<int32_t> color(T);
  int n_colors = 0;
  for (int64_t s = 0; s < T; ++s) {
    int32_t e = eorder[s];
    int c = -1;
    for (int w = 0; w < kWords && c < 0; ++w) {
      uint64_t busy = 0;
      for (int a = 0; a < 4; ++a) busy |= used[(size_t)tt[4 * e + a] * kWords + w];
      if (~busy) c = 64 * w + __builtin_ctzll(~busy);
    }
    if (c < 0) {
      set_error("lfx_mesh_create: element colouring needs more than %d colours", 64 * kWords);
      return LFX_ERR_BAD_MESH;
    }
    color[e] = c;
    for (int a = 0; a < 4; ++a) used[(size_t)tt[4 * e + a] * kWords + c / 64] |= 1ULL << (c % 64);
    n_colors = std::max(n_colors, c + 1);
  }
  n_colors = balance_colours(
      T, [&](int32_t e, int &n) { n = 4; return &tt[4 * (int64_t)e]; }, eorder, used, color, n_colors, kWords,
      assemble_wave_elements());

  // ---- chunks: kChunkElems consecutive elements of the Morton order, coloured greedily so that no
  // two chunks of one colour share a node; the internal element order runs chunk by chunk in
  // colour order (Morton order inside each chunk)
  const int NE = kChunkElems;
  const int64_t nch = (T + NE - 1) / NE;
  std::vector<int32_t> ccolor(nch);
  int n_ccolors = 0;
  {
    std::vector<uint64_t> cused((size_t)V * kWords, 0);
    std::vector<int32_t> cn_off(nch + 1, 0), cn;
    for (int64_t k = 0; k < nch; ++k) {
      const size_t b0 = cn.size();
      for (int64_t q = k * NE; q < std::min<int64_t>(T, (k + 1) * NE); ++q)
        for (int a = 0; a < 4; ++a) cn.push_back(tt[4 * (int64_t)eorder[q] + a]);
      std::sort(cn.begin() + b0, cn.end());
      cn.erase(std::unique(cn.begin() + b0, cn.end()), cn.end());
      cn_off[k + 1] = (int32_t)cn.size();
      int c = -1;
      for (int w = 0; w < kWords && c < 0; ++w) {
        uint64_t busy = 0;
        for (size_t i = b0; i < cn.size(); ++i) busy |= cused[(size_t)cn[i] * kWords + w];
        if (~busy) c = 64 * w + __builtin_ctzll(~busy);
      }
      if (c < 0) {
        set_error("lfx_mesh_create: chunk colouring needs more than %d colours", 64 * kWords);
        return LFX_ERR_BAD_MESH;
      }
      ccolor[k] = c;
      for (size_t i = b0; i < cn.size(); ++i) cused[(size_t)cn[i] * kWords + c / 64] |= 1ULL << (c % 64);
      n_ccolors = std::max(n_ccolors, c + 1);
    }
    // chunk colours balanced to whole waves of the chunk kernel (one chunk per resident CTA)
    std::vector<int32_t> korder(nch);
    std::iota(korder.begin(), korder.end(), 0);
    n_ccolors = balance_colours(
        nch, [&](int32_t k, int &n) { n = cn_off[k + 1] - cn_off[k]; return cn.data() + cn_off[k]; }, korder, cused,
        ccolor, n_ccolors, kWords, assemble_chunk_wave());
  }
  std::vector<int32_t> corder(nch);
  std::iota(corder.begin(), corder.end(), 0);
  std::stable_sort(corder.begin(), corder.end(), [&](int32_t a, int32_t b) { return ccolor[a] < ccolor[b]; });
  m.chunk_color_off.assign(n_ccolors + 1, 0);
  for (int64_t k = 0; k < nch; ++k) m.chunk_color_off[ccolor[k] + 1]++;
  for (int c = 0; c < n_ccolors; ++c) m.chunk_color_off[c + 1] += m.chunk_color_off[c];
  m.elem_old.resize(T);
  m.chunk_elem_off.assign(nch + 1, 0);
  {
    int64_t w = 0;
    for (int64_t i = 0; i < nch; ++i) {
      const int64_t k = corder[i];
      for (int64_t q = k * NE; q < std::min<int64_t>(T, (k + 1) * NE); ++q) m.elem_old[w++] = eorder[q];
      m.chunk_elem_off[i + 1] = (int32_t)w;
    }
  }
  std::vector<int32_t> elem_new(T);
  for (int64_t i = 0; i < T; ++i) elem_new[m.elem_old[i]] = (int32_t)i;
  // element colours (for the per-colour kernels): internal ids listed colour by colour, Morton order
  // inside each colour
  m.color_off.assign(n_colors + 1, 0);
  for (int64_t e = 0; e < T; ++e) m.color_off[color[e] + 1]++;
  for (int c = 0; c < n_colors; ++c) m.color_off[c + 1] += m.color_off[c];
  {
    std::vector<int32_t> fill(m.color_off.begin(), m.color_off.end() - 1);
    m.color_elems.resize(T);
    for (int64_t q = 0; q < T; ++q) {
      const int32_t e = eorder[q];
      m.color_elems[fill[color[e]]++] = elem_new[e];
    }
  }
  m.tets.resize(4 * T);
  m.quality.resize(T);
  for (int64_t i = 0; i < T; ++i) {
    int32_t e = m.elem_old[i];
    for (int a = 0; a < 4; ++a) m.tets[4 * i + a] = tt[4 * (int64_t)e + a];
    m.quality[i] = qual[e];
  }

  // ---- node -> element adjacency (internal numbering)
  std::vector<int32_t> n2e_ptr(V + 1, 0), n2e;
  for (int64_t i = 0; i < 4 * T; ++i) n2e_ptr[m.tets[i] + 1]++;
  for (int64_t i = 0; i < V; ++i) n2e_ptr[i + 1] += n2e_ptr[i];
  n2e.resize(4 * T);
  {
    std::vector<int32_t> f(n2e_ptr.begin(), n2e_ptr.end() - 1);
    for (int64_t e = 0; e < T; ++e)
      for (int a = 0; a < 4; ++a) n2e[f[m.tets[4 * e + a]]++] = (int32_t)e;
  }
  for (int64_t i = 0; i < V; ++i)
    if (n2e_ptr[i + 1] == n2e_ptr[i]) {
      set_error("lfx_mesh_create: node %d belongs to no tetrahedron", m.node_old[i]);
      return LFX_ERR_BAD_MESH;
    }

  // ---- block pattern: row i = sorted unique nodes of the elements around i
  m.row_ptr.assign(V + 1, 0);
  m.col_idx.clear();
  m.col_idx.reserve((size_t)V * 16);
  std::vector<int32_t> buf;
  for (int64_t i = 0; i < V; ++i) {
    buf.clear();
    for (int32_t k = n2e_ptr[i]; k < n2e_ptr[i + 1]; ++k)
      for (int a = 0; a < 4; ++a) buf.push_back(m.tets[4 * (int64_t)n2e[k] + a]);
    std::sort(buf.begin(), buf.end());
    buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
    m.col_idx.insert(m.col_idx.end(), buf.begin(), buf.end());
    if ((int64_t)m.col_idx.size() > (int64_t)INT32_MAX) {
      set_error("lfx_mesh_create: pattern too large");
      return LFX_ERR_INVALID_ARG;
    }
    m.row_ptr[i + 1] = (int32_t)m.col_idx.size();
  }
  m.nnzb = (int64_t)m.col_idx.size();
  auto find = [&](int32_t r, int32_t c) -> int32_t {
    const int32_t *b = m.col_idx.data() + m.row_ptr[r], *e = m.col_idx.data() + m.row_ptr[r + 1];
    const int32_t *p = std::lower_bound(b, e, c);
    return (p != e && *p == c) ? (int32_t)(p - m.col_idx.data()) : -1;
  };
  m.diag_idx.resize(V);
  for (int64_t i = 0; i < V; ++i) m.diag_idx[i] = find((int32_t)i, (int32_t)i);
  m.trans_idx.resize(m.nnzb);
  for (int64_t i = 0; i < V; ++i)
    for (int32_t k = m.row_ptr[i]; k < m.row_ptr[i + 1]; ++k)
      m.trans_idx[k] = find(m.col_idx[k], (int32_t)i);
  // row tiles of the staged velocity smoothing pass, greedily as long as both limits hold
  m.ftile_row.assign(1, 0);
  for (int64_t r0 = 0; r0 < V;) {
    int64_t r1 = r0;
    while (r1 < V && r1 - r0 < kFTileRows && m.row_ptr[r1 + 1] - m.row_ptr[r0] <= kFTileBlocks) ++r1;
    if (r1 == r0) {   // one row alone is over the block limit: no tiles, the plain pass runs
      m.ftile_row.clear();
      break;
    }
    m.ftile_row.push_back((int32_t)r1);
    r0 = r1;
  }
  m.slot.resize((size_t)T * 16);
  for (int64_t e = 0; e < T; ++e)
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b)
        m.slot[16 * e + 4 * a + b] = find(m.tets[4 * e + a], m.tets[4 * e + b]);
  // First writers: colours are assembled in the order of color_elems, so the first element of that
  // order touching a block writes it first and can store its terms instead of adding them to a
  // cleared matrix; the first writer of a node's right-hand-side row is the first writer of its
  // diagonal block.
  m.first.assign(T, 0);
  {
    std::vector<uint8_t> seen(m.nnzb, 0), node(V, 0);
    int64_t blocks = 0, nodes = 0;
    for (int64_t i = 0; i < T; ++i) {
      const int64_t e = m.color_elems[i];
      for (int q = 0; q < 16; ++q) {
        const int32_t s = m.slot[16 * e + q];
        if (!seen[s]) {
          seen[s] = 1;
          ++blocks;
          m.first[e] |= (uint16_t)(1u << q);
        }
      }
      for (int a = 0; a < 4; ++a)
        if (!node[m.tets[4 * e + a]]) {
          node[m.tets[4 * e + a]] = 1;
          ++nodes;
        }
    }
    m.all_blocks_touched = blocks == m.nnzb;
    m.all_nodes_touched = nodes == V;
  }
  // ---- chunk tables: each chunk's 16 block contributions per element grouped into runs by matrix
  // block, packed first-fit-decreasing into passes of 4 NE slots (no run straddles two passes),
  // diagonal runs first in each pass; a run's first-writer flag marks the first chunk (in
  // processing order) touching its block
  {
    const int PS = 4 * NE;
    std::vector<uint8_t> seenb(m.nnzb, 0);
    m.chunk_pass_off.assign(nch + 1, 0);
    m.pass_code.clear();
    m.pass_run_off.assign(1, 0);
    m.pass_ndiag.clear();
    m.run_meta.clear();
    m.run_block.clear();
    m.run_node.clear();
    struct Run {
      int32_t block, node, start, len;
      bool diag;
    };
    std::vector<std::pair<int32_t, uint16_t>> cs;
    std::vector<Run> runs;
    std::vector<std::vector<int>> passes;
    std::vector<int> fillp;
    for (int64_t k = 0; k < nch; ++k) {
      const int64_t e0 = m.chunk_elem_off[k], e1 = m.chunk_elem_off[k + 1];
      cs.clear();
      for (int64_t e = e0; e < e1; ++e)
        for (int a = 0; a < 4; ++a)
          for (int b = 0; b < 4; ++b)
            cs.push_back({m.slot[16 * e + 4 * a + b], (uint16_t)(((e - e0) << 4) | (a << 2) | b)});
      std::stable_sort(cs.begin(), cs.end(),
                       [](const std::pair<int32_t, uint16_t> &x, const std::pair<int32_t, uint16_t> &y) {
                         return x.first < y.first;
                       });
      runs.clear();
      for (size_t i = 0; i < cs.size();) {
        size_t j = i;
        while (j < cs.size() && cs[j].first == cs[i].first) ++j;
        const uint16_t c0 = cs[i].second;
        const int a = (c0 >> 2) & 3, b = c0 & 3;
        Run r{cs[i].first, -1, (int32_t)i, (int32_t)(j - i), a == b};
        if (r.diag) r.node = m.tets[4 * (e0 + (c0 >> 4)) + a];
        runs.push_back(r);
        i = j;
      }
      std::vector<int> ord(runs.size());
      std::iota(ord.begin(), ord.end(), 0);
      std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return runs[x].len > runs[y].len; });
      passes.clear();
      fillp.clear();
      for (int ri : ord) {
        size_t p = 0;
        while (p < passes.size() && fillp[p] + runs[ri].len > PS) ++p;
        if (p == passes.size()) {
          passes.emplace_back();
          fillp.push_back(0);
        }
        passes[p].push_back(ri);
        fillp[p] += runs[ri].len;
      }
      for (auto &pl : passes) {
        std::stable_sort(pl.begin(), pl.end(), [&](int x, int y) { return runs[x].diag && !runs[y].diag; });
        const size_t base = m.pass_code.size();
        m.pass_code.resize(base + PS, 0xffff);
        int at = 0, ndiag = 0;
        for (int ri : pl) {
          const Run &r = runs[ri];
          for (int q = 0; q < r.len; ++q) m.pass_code[base + at + q] = cs[r.start + q].second;
          const bool first = !seenb[r.block];
          seenb[r.block] = 1;
          m.run_meta.push_back((uint16_t)(at | (r.len << 8) | (first ? 1 << 14 : 0) | (r.diag ? 1 << 15 : 0)));
          m.run_block.push_back(r.block);
          m.run_node.push_back(r.node);
          ndiag += r.diag;
          at += r.len;
        }
        m.pass_ndiag.push_back(ndiag);
        m.pass_run_off.push_back((int32_t)m.run_block.size());
      }
      if ((int)passes.size() > kChunkMaxPasses) {
        set_error("lfx_mesh_create: a chunk needs %d passes (more than %d)", (int)passes.size(), kChunkMaxPasses);
        return LFX_ERR_INVALID_ARG;
      }
      m.chunk_pass_off[k + 1] = m.chunk_pass_off[k] + (int32_t)passes.size();
    }
  }

  // ---- boundary faces: internal numbering, outward orientation from the owning tetrahedron
  m.bfaces.resize(3 * F);
  m.btags.assign(tags_in, tags_in + F);
  for (int64_t f = 0; f < F; ++f) {
    int32_t v[3];
    for (int k = 0; k < 3; ++k) v[k] = m.node_new[bfaces_in[3 * f + k]];
    int32_t owner = -1, opp = -1;
    for (int32_t k = n2e_ptr[v[0]]; k < n2e_ptr[v[0] + 1] && owner < 0; ++k) {
      const int32_t *t = &m.tets[4 * (int64_t)n2e[k]];
      int hits = 0, other = -1;
      for (int a = 0; a < 4; ++a) {
        if (t[a] == v[0] || t[a] == v[1] || t[a] == v[2]) ++hits;
        else other = t[a];
      }
      if (hits == 3) {
        owner = n2e[k];
        opp = other;
      }
    }
    if (owner < 0) {
      set_error("lfx_mesh_create: boundary face %lld is not a face of any tetrahedron",
                (long long)f);
      return LFX_ERR_BAD_MESH;
    }
    const double *a = &m.xyz[3 * (int64_t)v[0]], *b = &m.xyz[3 * (int64_t)v[1]],
                 *c = &m.xyz[3 * (int64_t)v[2]], *d = &m.xyz[3 * (int64_t)opp];
    if (signed_det(a, b, c, d) > 0) std::swap(v[1], v[2]);
    for (int k = 0; k < 3; ++k) m.bfaces[3 * f + k] = v[k];
  }
  return LFX_OK;
}

lfx_status upload_mesh(Mesh &m) {
  const int64_t V = m.V, T = m.T;
  std::vector<double> x4(4 * V);
  for (int64_t i = 0; i < V; ++i) {
    for (int k = 0; k < 3; ++k) x4[4 * i + k] = m.xyz[3 * i + k];
    x4[4 * i + 3] = 0.0;
  }
  LFX_TRY(m.d_xyz.alloc(sizeof(double) * 4 * V));
  LFX_TRY(m.d_conn.alloc(sizeof(int32_t) * 4 * T));
  LFX_TRY(m.d_slot.alloc(sizeof(int32_t) * 16 * T));
  LFX_TRY(m.d_rowptr.alloc(sizeof(int32_t) * (V + 1)));
  LFX_TRY(m.d_col.alloc(sizeof(int32_t) * m.nnzb));
  LFX_TRY(m.d_diag.alloc(sizeof(int32_t) * V));
  LFX_TRY(m.d_trans.alloc(sizeof(int32_t) * m.nnzb));
  LFX_TRY(m.d_comp_off.alloc(sizeof(int32_t) * m.comp_off.size()));
  LFX_TRY(m.d_node_old.alloc(sizeof(int32_t) * V));
  LFX_TRY(m.d_first.alloc(sizeof(uint16_t) * std::max<int64_t>(T, 1)));
  if (T > 0) LFX_CUDA_TRY(cudaMemcpy(m.d_first.p, m.first.data(), sizeof(uint16_t) * T, cudaMemcpyHostToDevice));
  auto up = [](DBuf &d, const void *src, size_t bytes) -> lfx_status {
    LFX_TRY(d.alloc(std::max<size_t>(bytes, 16)));
    if (bytes) LFX_CUDA_TRY(cudaMemcpy(d.p, src, bytes, cudaMemcpyHostToDevice));
    return LFX_OK;
  };
  LFX_TRY(up(m.d_color_elems, m.color_elems.data(), sizeof(int32_t) * m.color_elems.size()));
  LFX_TRY(up(m.d_chunk_elem_off, m.chunk_elem_off.data(), sizeof(int32_t) * m.chunk_elem_off.size()));
  LFX_TRY(up(m.d_chunk_pass_off, m.chunk_pass_off.data(), sizeof(int32_t) * m.chunk_pass_off.size()));
  LFX_TRY(up(m.d_pass_code, m.pass_code.data(), sizeof(uint16_t) * m.pass_code.size()));
  LFX_TRY(up(m.d_pass_run_off, m.pass_run_off.data(), sizeof(int32_t) * m.pass_run_off.size()));
  LFX_TRY(up(m.d_pass_ndiag, m.pass_ndiag.data(), sizeof(int32_t) * m.pass_ndiag.size()));
  LFX_TRY(up(m.d_run_meta, m.run_meta.data(), sizeof(uint16_t) * m.run_meta.size()));
  LFX_TRY(up(m.d_run_block, m.run_block.data(), sizeof(int32_t) * m.run_block.size()));
  LFX_TRY(up(m.d_run_node, m.run_node.data(), sizeof(int32_t) * m.run_node.size()));
  LFX_TRY(up(m.d_ftile_row, m.ftile_row.data(), sizeof(int32_t) * m.ftile_row.size()));
  LFX_CUDA_TRY(cudaMemcpy(m.d_node_old.p, m.node_old.data(), sizeof(int32_t) * V, cudaMemcpyHostToDevice));
  LFX_CUDA_TRY(cudaMemcpy(m.d_xyz.p, x4.data(), m.d_xyz.bytes, cudaMemcpyHostToDevice));
  // FP32 high and low parts of the coordinates (x = hi + lo to 48 bits) for double-float assembly
  std::vector<float> xh(4 * V), xl(4 * V);
  for (int64_t i = 0; i < 4 * V; ++i) {
    xh[i] = (float)x4[i];
    xl[i] = (float)(x4[i] - (double)xh[i]);
  }
  LFX_TRY(m.d_xyz_hi.alloc(sizeof(float) * 4 * V));
  LFX_TRY(m.d_xyz_lo.alloc(sizeof(float) * 4 * V));
  LFX_CUDA_TRY(cudaMemcpy(m.d_xyz_hi.p, xh.data(), m.d_xyz_hi.bytes, cudaMemcpyHostToDevice));
  LFX_CUDA_TRY(cudaMemcpy(m.d_xyz_lo.p, xl.data(), m.d_xyz_lo.bytes, cudaMemcpyHostToDevice));
  LFX_CUDA_TRY(cudaMemcpy(m.d_conn.p, m.tets.data(), sizeof(int32_t) * 4 * T, cudaMemcpyHostToDevice));
  LFX_CUDA_TRY(cudaMemcpy(m.d_slot.p, m.slot.data(), sizeof(int32_t) * 16 * T, cudaMemcpyHostToDevice));
  LFX_CUDA_TRY(cudaMemcpy(m.d_rowptr.p, m.row_ptr.data(), sizeof(int32_t) * (V + 1), cudaMemcpyHostToDevice));
  LFX_CUDA_TRY(cudaMemcpy(m.d_col.p, m.col_idx.data(), sizeof(int32_t) * m.nnzb, cudaMemcpyHostToDevice));
  LFX_CUDA_TRY(cudaMemcpy(m.d_diag.p, m.diag_idx.data(), sizeof(int32_t) * V, cudaMemcpyHostToDevice));
  LFX_CUDA_TRY(cudaMemcpy(m.d_trans.p, m.trans_idx.data(), sizeof(int32_t) * m.nnzb, cudaMemcpyHostToDevice));
  LFX_CUDA_TRY(cudaMemcpy(m.d_comp_off.p, m.comp_off.data(), sizeof(int32_t) * m.comp_off.size(),
                          cudaMemcpyHostToDevice));
  return LFX_OK;
}

}  // namespace lfx
