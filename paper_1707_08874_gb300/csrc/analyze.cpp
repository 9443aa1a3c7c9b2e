// Host symbolic analysis, done once per lattice shape: geometric nested
// dissection of the Ns^3 x Nt torus, the supernodal elimination tree, the front
// index maps and the fixed launch schedule of the factorisation and of the
// selected-inversion sweep (Sec. 3: "sparse LU followed by a selected
// inversion"; the paper's solver does not describe its ordering).
#include <algorithm>
#include <array>
#include <cstdlib>
#include <functional>
#include <stdexcept>

#include "plan.hpp"

namespace cl {
namespace {

struct Box {
  std::array<int, 4> lo, n;
  std::array<bool, 4> per;
};

struct Geo {
  int Ns, Nt;
  std::array<int, 4> L;
  int site(const std::array<int, 4>& c) const { return ((c[3] * Ns + c[2]) * Ns + c[1]) * Ns + c[0]; }
  std::array<int, 4> coords(int s) const {
    std::array<int, 4> c;
    c[0] = s % Ns; s /= Ns;
    c[1] = s % Ns; s /= Ns;
    c[2] = s % Ns; s /= Ns;
    c[3] = s;
    return c;
  }
  int nbr(int s, int nu, int dir) const {
    auto c = coords(s);
    c[nu] = (c[nu] + dir + L[nu]) % L[nu];
    return site(c);
  }
  bool in_box(const Box& b, int s) const {
    auto c = coords(s);
    for (int d = 0; d < 4; ++d) {
      if (b.per[d]) continue;
      int rel = ((c[d] - b.lo[d]) % L[d] + L[d]) % L[d];
      if (rel >= b.n[d]) return false;
    }
    return true;
  }
  std::vector<int> sites(const Box& b) const {
    std::vector<int> out;
    std::array<int, 4> c;
    for (int t = 0; t < b.n[3]; ++t)
      for (int z = 0; z < b.n[2]; ++z)
        for (int y = 0; y < b.n[1]; ++y)
          for (int x = 0; x < b.n[0]; ++x) {
            c = {(b.lo[0] + x) % L[0], (b.lo[1] + y) % L[1], (b.lo[2] + z) % L[2], (b.lo[3] + t) % L[3]};
            out.push_back(site(c));
          }
    std::sort(out.begin(), out.end());
    return out;
  }
};

// Recursive geometric nested dissection.  A periodic extent is cut by two
// opposite hyperplanes, an open one by its middle hyperplane; the cut with the
// smallest separator wins (ties: the longer extent, then the lower direction).
// Nodes are appended in postorder; `boxes` keeps each node's subtree domain.
int dissect(const Geo& g, const Box& b, std::vector<SNode>& nodes, std::vector<Box>& boxes) {
  int64_t nsites = 1;
  for (int d = 0; d < 4; ++d) nsites *= b.n[d];
  int best = -1;
  int64_t best_sz = 0;
  for (int d = 0; d < 4; ++d) {
    int64_t other = nsites / b.n[d], sz;
    if (b.per[d]) {
      if (b.n[d] < 4) continue;
      sz = 2 * other;
    } else {
      if (b.n[d] < 2) continue;
      sz = other;
    }
    if (best < 0 || sz < best_sz || (sz == best_sz && b.n[d] > b.n[best])) {
      best = d;
      best_sz = sz;
    }
  }
  SNode nd;
  if (nsites <= kLeafSites || best < 0) {
    nd.sep = g.sites(b);
    nodes.push_back(nd);
    boxes.push_back(b);
    return (int)nodes.size() - 1;
  }
  const int d = best, lo = b.lo[d], n = b.n[d];
  std::vector<int> planes;
  std::vector<std::pair<int, int>> pieces;
  if (b.per[d]) {
    planes = {lo, lo + n / 2};
    pieces = {{lo + 1, n / 2 - 1}, {lo + n / 2 + 1, n - n / 2 - 1}};
  } else {
    int mid = lo + n / 2;
    planes = {mid};
    pieces = {{lo, n / 2}, {mid + 1, n - n / 2 - 1}};
  }
  std::vector<int> kids;
  for (auto& pc : pieces) {
    if (pc.second <= 0) continue;
    Box c = b;
    c.lo[d] = pc.first % g.L[d];
    c.n[d] = pc.second;
    c.per[d] = false;
    kids.push_back(dissect(g, c, nodes, boxes));
  }
  for (int pl : planes) {
    Box c = b;
    c.lo[d] = pl % g.L[d];
    c.n[d] = 1;
    c.per[d] = false;
    auto s = g.sites(c);
    nd.sep.insert(nd.sep.end(), s.begin(), s.end());
  }
  std::sort(nd.sep.begin(), nd.sep.end());
  nd.children = kids;
  nodes.push_back(nd);
  boxes.push_back(b);
  int id = (int)nodes.size() - 1;
  for (int c : kids) nodes[c].parent = id;
  return id;
}

int64_t tiles(int M, int N) {
  return (int64_t)((M + kTileM - 1) / kTileM) * ((N + kTileN - 1) / kTileN);
}

void check_shape(int Ns, int Nt) {
  if (Ns < 4 || Nt < 4 || (Ns & 1) || (Nt & 1)) throw std::invalid_argument("Ns, Nt must be even and >= 4");
  if (Ns > 64 || Nt > 128) throw std::invalid_argument("lattice too large");
}

int check_precision_panel(int precision, int panel) {
  if (precision != CL_FP64 && precision != CL_MIXED_FP32 && precision != CL_FP64_EMU &&
      precision != CL_MIXED_BF16X3)
    throw std::invalid_argument("precision");
  if (panel != 0 && (panel < 3 || panel > 48 || panel % 3 != 0)) throw std::invalid_argument("panel");
  return panel ? panel : (precision == CL_FP64 ? kPanelFP64 : digit_gemms(precision) ? kPanelEmu : kPanelFP32);
}

// Everything of the analysis that depends on one lattice shape: the
// supernodal elimination tree (postorder), front offsets inside the shape's
// own pool, the block tables of D and G, the extend-add and gather site maps
// (SNode::ea_map / ga_map index `maps`) and the flop counts at panel width b.
struct Tree {
  int Ns = 0, Nt = 0, V = 0;
  std::vector<SNode> nodes;
  int n_levels = 0;
  int64_t pool_elems = 0;
  double factor_flops = 0, selinv_flops = 0;
  std::vector<int64_t> off;  // diagonal [V] | forward [4V] | backward [4V]
  std::vector<int> ld;
  std::vector<int> maps;
};

void build_tree(Tree& t, int Ns, int Nt, int b) {
  check_shape(Ns, Nt);
  t.Ns = Ns;
  t.Nt = Nt;
  t.V = Ns * Ns * Ns * Nt;
  Geo g{Ns, Nt, {Ns, Ns, Ns, Nt}};
  const int V = t.V;

  // ---- elimination tree -------------------------------------------------
  std::vector<Box> boxes;
  Box whole{{0, 0, 0, 0}, {Ns, Ns, Ns, Nt}, {true, true, true, true}};
  t.nodes.clear();
  dissect(g, whole, t.nodes, boxes);
  auto& nodes = t.nodes;
  const int nn = (int)nodes.size();
  std::vector<int> sn(V, -1);
  for (int i = 0; i < nn; ++i)
    for (int s : nodes[i].sep) {
      if (sn[s] != -1) throw std::logic_error("site in two supernodes");
      sn[s] = i;
    }
  for (int s = 0; s < V; ++s)
    if (sn[s] < 0) throw std::logic_error("site in no supernode");

  // ---- boundaries, ordered by position in the parent's front (preorder) ----
  std::vector<int> pos(V, -1);
  for (int i = nn - 1; i >= 0; --i) {  // reverse postorder: parents before children
    SNode& P = nodes[i];
    std::vector<int> front = P.sep;
    front.insert(front.end(), P.bnd.begin(), P.bnd.end());
    for (size_t q = 0; q < front.size(); ++q) pos[front[q]] = (int)q;
    for (int c : P.children) {
      std::vector<int> bb;
      for (int s : g.sites(boxes[c]))
        for (int nu = 0; nu < 4; ++nu)
          for (int dir = -1; dir <= 1; dir += 2) {
            int y = g.nbr(s, nu, dir);
            if (!g.in_box(boxes[c], y)) bb.push_back(y);
          }
      std::sort(bb.begin(), bb.end());
      bb.erase(std::unique(bb.begin(), bb.end()), bb.end());
      for (int s : bb)
        if (pos[s] < 0) throw std::logic_error("boundary outside the parent front");
      std::sort(bb.begin(), bb.end(), [&](int a, int c2) { return pos[a] < pos[c2]; });
      nodes[c].bnd = bb;
    }
    for (int s : front) pos[s] = -1;
  }

  // ---- sizes, levels, front offsets ---------------------------------------
  t.n_levels = 0;
  int64_t off = 0;
  for (int i = 0; i < nn; ++i) {
    SNode& n = nodes[i];
    n.k = 3 * (int)n.sep.size();
    n.r = 3 * (int)n.bnd.size();
    n.nf = n.k + n.r;
    n.level = 0;
    for (int c : n.children) n.level = std::max(n.level, nodes[c].level + 1);
    t.n_levels = std::max(t.n_levels, n.level + 1);
    n.off = off;
    off += ((int64_t)n.nf * n.nf + 15) / 16 * 16;
  }
  t.pool_elems = off;

  // ---- flop counts (complex multiply-add = 8 real flops) ------------------
  t.factor_flops = t.selinv_flops = 0;
  for (auto& n : nodes) {
    for (int c0 = 0; c0 < n.k; c0 += b) {
      double bp = std::min(b, n.k - c0), nf = n.nf;
      t.factor_flops += 8.0 * (bp * bp * bp + 2 * nf * bp * bp + nf * nf * bp);
    }
    double k = n.k, r = n.r;
    t.selinv_flops += 8.0 * (2 * r * r * k + k * k * r);
  }

  // ---- assembly / extraction tables -----------------------------------------
  // position of a site in a front: sep sites by their own index, boundary
  // sites through a per-node table sorted by site
  std::vector<int> sep_pos(V);
  for (int i = 0; i < nn; ++i)
    for (size_t q = 0; q < nodes[i].sep.size(); ++q) sep_pos[nodes[i].sep[q]] = (int)q;
  std::vector<std::vector<std::pair<int, int>>> bnd_sorted(nn);
  for (int i = 0; i < nn; ++i) {
    auto& v = bnd_sorted[i];
    for (size_t q = 0; q < nodes[i].bnd.size(); ++q) v.push_back({nodes[i].bnd[q], (int)q});
    std::sort(v.begin(), v.end());
  }
  auto front_pos = [&](int node, int s) -> int {
    if (sn[s] == node) return sep_pos[s];
    const auto& v = bnd_sorted[node];
    auto it = std::lower_bound(v.begin(), v.end(), std::make_pair(s, -1));
    if (it == v.end() || it->first != s) throw std::logic_error("site not in front");
    return (int)nodes[node].sep.size() + it->second;
  };
  auto block_off = [&](int x, int y, int64_t& o, int& l) {
    int node = std::min(sn[x], sn[y]);  // the supernode eliminated first (postorder)
    const SNode& n = nodes[node];
    o = n.off + (int64_t)3 * front_pos(node, x) * n.nf + 3 * front_pos(node, y);
    l = n.nf;
  };
  t.off.assign(9 * (size_t)V, 0);
  t.ld.assign(9 * (size_t)V, 0);
  for (int s = 0; s < V; ++s) {
    block_off(s, s, t.off[s], t.ld[s]);
    for (int nu = 0; nu < 4; ++nu) {
      int y = g.nbr(s, nu, +1);
      block_off(s, y, t.off[V + 4 * s + nu], t.ld[V + 4 * s + nu]);
      block_off(y, s, t.off[5 * V + 4 * s + nu], t.ld[5 * V + 4 * s + nu]);
    }
  }

  // ---- site maps of the extend-add (parent front site -> child boundary
  // index or -1) and of the selected-inversion gather (child boundary index
  // -> parent front site) ---------------------------------------------------
  t.maps.clear();
  for (int i = 0; i < nn; ++i) {
    SNode& P = nodes[i];
    if (P.children.size() > 2) throw std::logic_error("more than two children");
    const size_t nfs = P.sep.size() + P.bnd.size();
    for (size_t q = 0; q < P.children.size(); ++q) {
      const SNode& C = nodes[P.children[q]];
      P.ea_map[q] = (int)t.maps.size();
      std::vector<int> inv(nfs, -1);
      for (size_t j = 0; j < C.bnd.size(); ++j) inv[front_pos(i, C.bnd[j])] = (int)j;
      t.maps.insert(t.maps.end(), inv.begin(), inv.end());
    }
  }
  for (int i = 0; i < nn; ++i) {
    SNode& C = nodes[i];
    if (C.parent < 0 || C.r == 0) continue;
    C.ga_map = (int)t.maps.size();
    for (int s : C.bnd) t.maps.push_back(front_pos(C.parent, s));
  }
}

// A front of the merged schedule: one supernode of one lattice, at its
// offset in the arena (fronts of every lattice of a ragged plan side by side).
struct FNode {
  int64_t off = 0, tmp = 0;
  int nf = 0, k = 0, r = 0, level = 0;
  int nchild = 0;
  int child[2] = {-1, -1};
  int ea_map[2] = {-1, -1};
  int ga_map = -1;
  int site0 = 0;  // separator sites at p.vsites[site0 ..]
};

// appends the separator sites of a node (offset by site_base) to p.vsites
FNode fnode_of(Plan& p, const SNode& n, int64_t base, int index_base, int maps_base, int64_t site_base) {
  FNode f;
  f.site0 = (int)p.vsites.size();
  for (int s : n.sep) p.vsites.push_back((int)(site_base + s));
  f.off = base + n.off;
  f.nf = n.nf;
  f.k = n.k;
  f.r = n.r;
  f.level = n.level;
  f.nchild = (int)n.children.size();
  for (int q = 0; q < f.nchild; ++q) {
    f.child[q] = index_base + n.children[q];
    f.ea_map[q] = maps_base + n.ea_map[q];
  }
  f.ga_map = n.ga_map >= 0 ? maps_base + n.ga_map : -1;
  return f;
}

// The fixed launch schedule of the factorisation and the selected-inversion
// sweep over the fronts F (by level: every front of a level, of every lattice,
// in the same launches), the workspace layout after p.pool_elems and the
// digit workspace of the tensor-core GEMMs.  p.panel, p.pool_elems and p.maps
// are set by the caller.
void build_schedule(Plan& p, std::vector<FNode>& F, int n_levels, int precision) {
  const int nn = (int)F.size();
  const int b = p.panel;
  p.n_levels = n_levels;

  // per-node workspace inside its level (panel temps / selected-inversion temps)
  std::vector<int64_t> level_tmp(n_levels, 0);
  for (int i = 0; i < nn; ++i) {
    FNode& n = F[i];
    int64_t need = std::max<int64_t>(4LL * b * n.nf, 2LL * n.r * n.k);  // two TR/TC sets (look-ahead)
    need = (need + 15) / 16 * 16;
    n.tmp = p.pool_elems + level_tmp[n.level];
    level_tmp[n.level] += need;
  }
  p.tmp_elems = 0;
  for (auto t : level_tmp) p.tmp_elems = std::max(p.tmp_elems, t);
  p.arena_elems = (p.pool_elems + p.tmp_elems + 63) / 64 * 64;

  // ---- schedule ----------------------------------------------------------
  p.gemm.clear();
  p.panels.clear();
  p.copies.clear();
  p.extadd.clear();
  p.gather.clear();
  p.factor_ops.clear();
  p.selinv_ops.clear();
  std::vector<std::vector<int>> by_level(n_levels);
  for (int i = 0; i < nn; ++i) by_level[F[i].level].push_back(i);

  const Mask2 none{0, 0, 0, 0};
  auto add_gemm = [&](int blk, int64_t a, int lda, int64_t bb, int ldb, int64_t c, int ldc, int M, int N,
                      int K, int neg, int beta, Mask2 rm, Mask2 cm, int trans = 0) {
    GemmDesc d{a, bb, c, lda, ldb, ldc, M, N, K, neg, beta, rm, cm, blk, (N + kTileN - 1) / kTileN, trans};
    p.gemm.push_back(d);
    return (int)tiles(M, N);
  };
  // The digit GEMMs tile C in 128-row blocks: a product with few rows (the
  // TR panel products, b x nf) is issued transposed (nf x b) there, with
  // every operand read and C written through the transposed strides.
  const bool tr_short = digit_gemms(precision);
  // digits per operand of the digit GEMMs: factorisation (panel products and
  // Schur updates), off-diagonal and diagonal blocks of the selected inversion
  // (CLSELINV_EMU_DIGITS=7 gives CL_FP64_EMU the accuracy of an FP64 GEMM
  // instead, for accuracy / speed comparisons)
  int nd_fp64 = kDigitsFP64;
  if (const char* v = std::getenv("CLSELINV_EMU_DIGITS")) nd_fp64 = std::atoi(v) == 7 ? 7 : kDigitsFP64;
  // mixed form: the panel products TR = Y A_p* and TC = -A_*p Y apply the FP64
  // pivot-block inverse Y and keep its accuracy (7 digits); the Schur updates
  // (bulk and next-panel strips) and the off-diagonal selected-inverse
  // products are split-BF16x3 (3 digits)
  const bool mixed = precision == CL_MIXED_BF16X3;
  const int nd_panel = mixed ? kDigitsDiag : nd_fp64;
  const int nd_factor = mixed ? kDigitsMixed : nd_fp64;
  const int nd_offdiag = nd_factor;
  const int nd_diag = mixed ? kDigitsDiag : nd_fp64;
  auto add_copy = [&](int blk, int64_t src, int lds, int64_t dst, int ldd, int rows, int cols, Mask2 rm,
                      Mask2 cm) {
    CopyDesc d{src, dst, lds, ldd, rows, cols, rm, cm, blk};
    p.copies.push_back(d);
    return (int)(((int64_t)rows * cols + 255) / 256);
  };

  // permutation workspace: per node a slot for its running row permutation
  // (k ints, kept by host executors of the exported schedule only), then per
  // panel its local permutation of the candidate rows (nc ints)
  p.unperm.clear();
  int64_t perm_ints = 0;
  std::vector<int> pi_off(nn);
  for (int i = 0; i < nn; ++i) {
    pi_off[i] = (int)perm_ints;
    perm_ints += F[i].k;
  }

  p.factor_ops.push_back(Op{OP_ZERO, 0, 0, 0, -1});
  int assemble_blocks = 0;
  for (const Segment& sg : p.segs) assemble_blocks = std::max(assemble_blocks, (4 * sg.V + 127) / 128);
  p.factor_ops.push_back(Op{OP_ASSEMBLE, 0, 0, assemble_blocks, -1});
  std::vector<int> level_last_copy(n_levels, -1);
  for (int h = 0; h < n_levels; ++h) {
    const auto& lv = by_level[h];
    if (h > 0) {
      Op op{OP_EXTADD, (int)p.extadd.size(), 0, 0, h};
      op.wait = level_last_copy[h - 1];  // the children's Schur complements are complete
      int blk = 0;
      for (int i : lv) {
        const FNode& P = F[i];
        if (P.nchild == 0) continue;
        ExtAddDesc d{};
        d.parent = P.off;
        d.nfp = P.nf;
        d.nchild = P.nchild;
        for (int q = 0; q < d.nchild; ++q) {
          const FNode& C = F[P.child[q]];
          d.child[q] = C.off;
          d.nfc[q] = C.nf;
          d.kc[q] = C.k;
          d.map[q] = P.ea_map[q];
        }
        d.blk0 = blk;
        blk += (int)(((int64_t)P.nf * P.nf + 255) / 256);
        p.extadd.push_back(d);
      }
      op.d1 = (int)p.extadd.size();
      op.blocks = blk;
      if (op.d1 > op.d0) p.factor_ops.push_back(op);
    }
    // Blocked sweep of the pivot panels with a one-panel look-ahead.  Stream 0
    // (critical): panel inverse, row swap, panel products TR/TC, the update
    // of the next two panels' rows and of the next panel's column strip, and
    // the entries the next step reads from the current one.  Stream 1: the
    // bulk rank-b update of the rest of the front and the write-back of the
    // panel.  TR/TC alternate
    // between two workspace sets by panel parity.
    int maxk = 0;
    for (int i : lv) maxk = std::max(maxk, F[i].k);
    int last_copy = -1;  // op index of the previous step's stream-1 write-back
    // copies of the previous step's swept entries that the next panel's
    // products read: launched with the next panel inverses, which read only
    // their diagonal blocks (disjoint from the copied entries)
    int pend_x0 = 0, pend_x1 = 0, pend_blocks = 0;
    for (int c0 = 0, step = 0; c0 < maxk; c0 += b, ++step) {
      const int set = step & 1;
      auto tR_of = [&](const FNode& n) { return n.tmp + (int64_t)set * 2 * b * n.nf; };
      auto tC_of = [&](const FNode& n) { return tR_of(n) + (int64_t)b * n.nf; };
      Op pinv{OP_PANEL, (int)p.panels.size(), 0, 0, h};
      Op g1{OP_GEMM, (int)p.gemm.size(), 0, 0, h};
      g1.ndig = nd_panel;
      int blk1 = 0, blk_sw = 0;
      for (int i : lv) {
        const FNode& n = F[i];
        if (c0 >= n.k) continue;
        const int bp = std::min(b, n.k - c0);
        // pivots among the rows of this panel and of the next one in the supernode
        const int nc = std::min(bp + b, n.k - c0);
        PanelDesc pd{n.off + (int64_t)c0 * n.nf + c0, n.nf, bp, i, c0, nc, (int)perm_ints, pi_off[i], blk_sw};
        perm_ints += nc;
        if (nc > bp) blk_sw += (n.nf + kSwapCols - 1) / kSwapCols;  // rows from the next panel may come in
        p.panels.push_back(pd);
        if (n.nf == bp) continue;  // nothing outside the panel
        // TR = Y * R_old (bp x nf), TC = -C_old * Y (nf x bp)
        if (tr_short)  // TR^T = R_old^T Y^T
          blk1 += add_gemm(blk1, n.off + (int64_t)c0 * n.nf, n.nf, n.off + (int64_t)c0 * n.nf + c0, n.nf, tR_of(n),
                           n.nf, n.nf, bp, bp, 0, 0, none, none, 7);
        else
          blk1 += add_gemm(blk1, n.off + (int64_t)c0 * n.nf + c0, n.nf, n.off + (int64_t)c0 * n.nf, n.nf, tR_of(n),
                           n.nf, bp, n.nf, bp, 0, 0, none, none);
        blk1 += add_gemm(blk1, n.off + c0, n.nf, n.off + (int64_t)c0 * n.nf + c0, n.nf, tC_of(n), bp, n.nf, bp, bp,
                         1, 0, none, none);
      }
      pinv.d1 = (int)p.panels.size();
      pinv.blocks = pinv.d1 - pinv.d0;
      pinv.x0 = pend_x0;
      pinv.x1 = pend_x1;
      pinv.xblocks = pend_blocks;
      pend_x0 = pend_x1 = pend_blocks = 0;
      p.factor_ops.push_back(pinv);
      // the panel's row permutation applied to the columns outside the panel.
      // The candidate rows (panels p and p+1) took their updates of step p-1
      // from its strips on this stream, and those of the steps before from
      // bulk updates that the strips of step p-1 waited for: no wait here
      if (blk_sw > 0) p.factor_ops.push_back(Op{OP_SWAP, pinv.d0, pinv.d1, blk_sw, h});
      g1.d1 = (int)p.gemm.size();
      g1.blocks = blk1;
      if (g1.d1 == g1.d0) continue;
      g1.signal = true;
      const int g1_idx = (int)p.factor_ops.size();
      p.factor_ops.push_back(g1);
      // strips and the entries the next panel reads (stream 0).  The row strip
      // covers the rows of panels p+1 and p+2, the candidate pivot rows of
      // step p+1: their update of step p is then ordered before the row swap
      // of step p+1 on this stream, and that swap need not wait for the bulk
      // update of step p
      Op st{OP_GEMM, (int)p.gemm.size(), 0, 0, h};
      st.ndig = nd_factor;
      Op ec{OP_COPY, (int)p.copies.size(), 0, 0, h};
      int blks = 0, blke = 0;
      for (int i : lv) {
        const FNode& n = F[i];
        if (c0 >= n.k) continue;
        const int bp = std::min(b, n.k - c0), c1 = c0 + b;
        if (n.nf == bp || c1 >= n.k) continue;
        const int b1 = std::min(b, n.k - c1), r2 = std::min(2 * b, n.k - c1);
        const int64_t tR = tR_of(n), tC = tC_of(n);
        // row strip: A[c1 .. c1+r2, j] -= C_old[c1 .., :] TR[:, j], j outside panel p
        if (tr_short)  // (A[c1.., :])^T -= TR^T C_old[c1.., :]^T
          blks += add_gemm(blks, tR, n.nf, n.off + (int64_t)c1 * n.nf + c0, n.nf, n.off + (int64_t)c1 * n.nf, n.nf,
                           n.nf, r2, bp, 1, 1, Mask2{c0, c0 + bp, 0, 0}, none, 7);
        else
          blks += add_gemm(blks, n.off + (int64_t)c1 * n.nf + c0, n.nf, tR, n.nf, n.off + (int64_t)c1 * n.nf, n.nf,
                           r2, n.nf, bp, 1, 1, none, Mask2{c0, c0 + bp, 0, 0});
        // column strip: A[r, c1..] -= C_old[r, :] TR[:, c1..], r outside panels p .. p+2
        blks += add_gemm(blks, n.off + c0, n.nf, tR + c1, n.nf, n.off + c1, n.nf, n.nf, b1, bp, 1, 1,
                         Mask2{c0, c0 + bp, c1, c1 + r2}, none);
        // swept entries of panel p that the next step reads or swaps:
        // A[c1 .. c1+r2, c0..] = TC, A[c0.., c1..] = TR
        blke += add_copy(blke, tC + (int64_t)c1 * bp, bp, n.off + (int64_t)c1 * n.nf + c0, n.nf, r2, bp, none, none);
        blke += add_copy(blke, tR + c1, n.nf, n.off + (int64_t)c0 * n.nf + c1, n.nf, bp, b1, none, none);
      }
      st.d1 = (int)p.gemm.size();
      st.blocks = blks;
      ec.d1 = (int)p.copies.size();
      ec.blocks = blke;
      int strips_idx = -1;
      if (st.d1 > st.d0) {
        st.wait = last_copy;  // the previous bulk update and write-back touched these strips
        st.signal = true;
        strips_idx = (int)p.factor_ops.size();
        p.factor_ops.push_back(st);
        // the copies overwrite entries the strips read (C_old of panel p+1):
        // they run with the next panel op, after the strips on stream 0
        pend_x0 = ec.d0;
        pend_x1 = ec.d1;
        pend_blocks = ec.blocks;
      }
      // bulk update and write-back of panel p (stream 1)
      Op g2{OP_GEMM, (int)p.gemm.size(), 0, 0, h};
      g2.ndig = nd_factor;
      Op cp{OP_COPY, (int)p.copies.size(), 0, 0, h};
      int blk2 = 0, blk3 = 0;
      for (int i : lv) {
        const FNode& n = F[i];
        if (c0 >= n.k) continue;
        const int bp = std::min(b, n.k - c0), c1 = c0 + b;
        if (n.nf == bp) continue;
        const int b1 = c1 < n.k ? std::min(b, n.k - c1) : 0;
        const int r2 = c1 < n.k ? std::min(2 * b, n.k - c1) : 0;
        const Mask2 rows{c0, c0 + bp, c1, c1 + r2};  // panels p .. p+2 (row strip)
        const Mask2 cols{c0, c0 + bp, c1, c1 + b1};  // panels p and p+1 (column strip)
        const int64_t tR = tR_of(n), tC = tC_of(n);
        blk2 += add_gemm(blk2, n.off + c0, n.nf, tR, n.nf, n.off, n.nf, n.nf, n.nf, bp, 1, 1, rows, cols);
        blk3 += add_copy(blk3, tC, bp, n.off + c0, n.nf, n.nf, bp, rows, none);
        blk3 += add_copy(blk3, tR, n.nf, n.off + (int64_t)c0 * n.nf, n.nf, bp, n.nf, none, cols);
      }
      g2.d1 = (int)p.gemm.size();
      g2.blocks = blk2;
      g2.stream = 1;
      g2.wait = g1_idx;
      cp.d1 = (int)p.copies.size();
      cp.blocks = blk3;
      cp.stream = 1;
      cp.signal = true;
      // the column strip reads the old column panel that this write-back replaces
      if (strips_idx >= 0) cp.wait = strips_idx;
      p.factor_ops.push_back(g2);
      last_copy = (int)p.factor_ops.size();
      p.factor_ops.push_back(cp);
    }
    level_last_copy[h] = last_copy;
  }

  // selected inversion: root to leaves
  std::vector<int> parent(nn, -1);
  for (int i = 0; i < nn; ++i)
    for (int q = 0; q < F[i].nchild; ++q) parent[F[i].child[q]] = i;
  // columns of the level's pivot rows back in the supernodes' original order,
  // once the level's G is complete (before the level below gathers from it)
  // each supernode's panels in step order
  std::vector<int> pan0(nn, 0), npan(nn, 0);
  {
    std::vector<std::vector<int>> by_node(nn);
    for (int d = 0; d < (int)p.panels.size(); ++d) by_node[p.panels[d].node].push_back(d);
    p.node_panels.clear();
    for (int i = 0; i < nn; ++i) {
      pan0[i] = (int)p.node_panels.size();
      npan[i] = (int)by_node[i].size();
      p.node_panels.insert(p.node_panels.end(), by_node[i].begin(), by_node[i].end());
    }
  }
  auto push_unperm = [&](int h) {
    Op up{OP_UNPERM, (int)p.unperm.size(), 0, 0, h};
    int blk = 0;
    for (int i : by_level[h]) {
      const FNode& n = F[i];
      if (n.k == 0) continue;
      p.unperm.push_back(UnpermDesc{n.off, n.nf, n.k, pan0[i], npan[i], blk});
      blk += (n.nf + kUnpermRows - 1) / kUnpermRows;
    }
    up.d1 = (int)p.unperm.size();
    up.blocks = blk;
    if (blk > 0) p.selinv_ops.push_back(up);
  };
  for (int h = n_levels - 1; h >= 0; --h) {
    const auto& lv = by_level[h];
    if (h == n_levels - 1) push_unperm(h);  // the root level's G is the factorisation's inverse
    Op ga{OP_GATHER, (int)p.gather.size(), 0, 0, h};
    int blk = 0;
    for (int i : lv) {
      const FNode& C = F[i];
      if (parent[i] < 0 || C.r == 0) continue;
      const FNode& P = F[parent[i]];
      GatherDesc d{C.off, P.off, C.nf, C.k, P.nf, C.r / 3, C.ga_map, blk};
      blk += (int)(((int64_t)C.r * C.r + 255) / 256);
      p.gather.push_back(d);
    }
    ga.d1 = (int)p.gather.size();
    ga.blocks = blk;
    if (ga.d1 == ga.d0) {  // only roots on this level (their G is the factorisation's inverse)
      if (h != n_levels - 1) push_unperm(h);
      continue;
    }
    p.selinv_ops.push_back(ga);
    Op g1{OP_GEMM, (int)p.gemm.size(), 0, 0, h};
    g1.ndig = nd_offdiag;
    int blk1 = 0;
    for (int i : lv) {
      const FNode& n = F[i];
      if (n.r == 0) continue;
      int64_t tSJ = n.tmp, tJS = n.tmp + (int64_t)n.r * n.k;
      int64_t SS = n.off + (int64_t)n.k * n.nf + n.k, SJ = n.off + (int64_t)n.k * n.nf, JS = n.off + n.k;
      blk1 += add_gemm(blk1, SS, n.nf, SJ, n.nf, tSJ, n.k, n.r, n.k, n.r, 0, 0, none, none);  // G_SJ = G_SS (-Lhat)
      blk1 += add_gemm(blk1, JS, n.nf, SS, n.nf, tJS, n.r, n.k, n.r, n.r, 1, 0, none, none);  // G_JS = -Uhat G_SS
    }
    g1.d1 = (int)p.gemm.size();
    g1.blocks = blk1;
    p.selinv_ops.push_back(g1);
    Op g2{OP_GEMM, (int)p.gemm.size(), 0, 0, h};
    g2.ndig = nd_diag;
    Op cp{OP_COPY, (int)p.copies.size(), 0, 0, h};
    int blk2 = 0, blk3 = 0;
    for (int i : lv) {
      const FNode& n = F[i];
      if (n.r == 0) continue;
      int64_t tSJ = n.tmp, tJS = n.tmp + (int64_t)n.r * n.k;
      int64_t SJ = n.off + (int64_t)n.k * n.nf, JS = n.off + n.k;
      // G_JJ = Ainv - Uhat G_SJ = Ainv + G_JS (-Lhat)... written as Ainv + tJS * F_SJ
      blk2 += add_gemm(blk2, tJS, n.r, SJ, n.nf, n.off, n.nf, n.k, n.k, n.r, 0, 1, none, none);
      blk3 += add_copy(blk3, tSJ, n.k, SJ, n.nf, n.r, n.k, none, none);
      blk3 += add_copy(blk3, tJS, n.r, JS, n.nf, n.k, n.r, none, none);
    }
    g2.d1 = (int)p.gemm.size();
    g2.blocks = blk2;
    cp.d1 = (int)p.copies.size();
    cp.blocks = blk3;
    p.selinv_ops.push_back(g2);
    p.selinv_ops.push_back(cp);
    push_unperm(h);
  }
  p.selinv_ops.push_back(Op{OP_EXTRACT, 0, 0, assemble_blocks, -1});
  p.perm_ints = perm_ints;

  // row-vector solves (stochastic estimator): nodes by level, front-vector
  // workspace offsets, CTA offsets of the level launches (128 elements per CTA)
  {
    std::vector<int64_t> vec(nn);
    int64_t v = 0;
    for (int i = 0; i < nn; ++i) {
      vec[i] = v;
      v += F[i].nf;
    }
    p.vec_elems = v;
    p.vnodes.clear();
    p.vlevel.assign(1, 0);
    p.vblk_nf.clear();
    p.vblk_r.clear();
    for (int h = 0; h < n_levels; ++h) {
      int bnf = 0, br = 0;
      for (int i : by_level[h]) {
        const FNode& n = F[i];
        VecNode x{};
        x.front = n.off;
        x.vec = vec[i];
        x.parent_vec = parent[i] >= 0 ? vec[parent[i]] : -1;
        x.nf = n.nf;
        x.k = n.k;
        x.r = n.r;
        x.level = h;
        x.nchild = n.nchild;
        x.pan0 = pan0[i];
        x.npan = npan[i];
        for (int q = 0; q < 2; ++q) {
          x.child_vec[q] = q < n.nchild ? vec[n.child[q]] : -1;
          x.child_k[q] = q < n.nchild ? F[n.child[q]].k : 0;
          x.ea_map[q] = n.ea_map[q];
        }
        x.ga_map = n.ga_map;
        x.site0 = n.site0;
        x.blk_nf = bnf;
        x.blk_r = br;
        bnf += (n.nf + 127) / 128;
        br += (n.r + 127) / 128;
        p.vnodes.push_back(x);
      }
      p.vlevel.push_back((int)p.vnodes.size());
      p.vblk_nf.push_back(bnf);
      p.vblk_r.push_back(br);
    }
  }

  // split-digit workspace of the digit GEMMs: per GEMM launch the problems
  // are laid out one after the other from the start of that launch's stream
  // region (launches of one stream run in order; the factorisation's second
  // stream gets a region of its own after the first one's)
  p.emu.clear();
  p.emu_words = p.emu_ints = 0;
  if (digit_gemms(precision)) {
    p.emu.resize(p.gemm.size());
    int64_t max_w[2] = {0, 0}, max_in[2] = {0, 0};
    for (auto* ops : {&p.factor_ops, &p.selinv_ops})
      for (auto& op : *ops) {
        if (op.kind != OP_GEMM) continue;
        int64_t w = 0, in = 0;
        int it = 0, blk = 0;
        for (int d = op.d0; d < op.d1; ++d) {
          GemmDesc& g = p.gemm[d];
          EmuDesc& e = p.emu[d];
          e.Mp = (g.M + kEmuTileM - 1) / kEmuTileM * kEmuTileM;
          e.Np = (g.N + 31) / 32 * 32;
          e.Kp = (g.K + 31) / 32 * 32;
          const int64_t nch = e.Kp / 32;
          e.adig = w;
          w += ((int64_t)op.ndig * e.Mp * e.Kp + 63) / 64 * 64;
          e.bdig = w;
          w += ((int64_t)op.ndig * 2 * e.Np * e.Kp + 63) / 64 * 64;
          e.aexp = in;
          in += nch * e.Mp;
          e.bexp = in;
          in += nch * e.Np;
          e.it0 = it;
          e.items = (int)(e.Mp * nch + e.Np * nch);
          it += e.items;
          // this precision tiles the GEMMs by kEmuTileM rows
          g.blk0 = blk;
          g.tilesN = e.Np / 16;  // 16 complex columns per CTA
          blk += (e.Mp / kEmuTileM) * g.tilesN;
        }
        op.blocks = blk;
        op.single_chunk = true;
        for (int d = op.d0; d < op.d1; ++d) op.single_chunk &= p.emu[d].Kp == 32;  // one exponent chunk
        max_w[op.stream] = std::max(max_w[op.stream], w);
        max_in[op.stream] = std::max(max_in[op.stream], in);
      }
    for (auto& op : p.factor_ops) {
      if (op.kind != OP_GEMM || op.stream == 0) continue;
      for (int d = op.d0; d < op.d1; ++d) {
        p.emu[d].adig += max_w[0];
        p.emu[d].bdig += max_w[0];
        p.emu[d].aexp += max_in[0];
        p.emu[d].bexp += max_in[0];
      }
    }
    p.emu_words = max_w[0] + max_w[1];
    p.emu_ints = max_in[0] + max_in[1];
  }
}

}  // namespace

void analyze_host(Plan& p, int Ns, int Nt, int batch, int precision, int panel) {
  check_shape(Ns, Nt);
  p.panel = check_precision_panel(precision, panel);
  p.precision = precision;
  Tree t;
  build_tree(t, Ns, Nt, p.panel);
  p.Ns = Ns;
  p.Nt = Nt;
  p.V = t.V;
  p.N = 3 * t.V;
  p.batch = batch;
  p.fbatch = batch;
  p.ragged = false;
  p.nodes = t.nodes;
  p.pool_elems = t.pool_elems;
  p.factor_flops = t.factor_flops;
  p.selinv_flops = t.selinv_flops;
  const int V = t.V;
  p.off_diag.assign(t.off.begin(), t.off.begin() + V);
  p.off_fwd.assign(t.off.begin() + V, t.off.begin() + 5 * V);
  p.off_bwd.assign(t.off.begin() + 5 * V, t.off.end());
  p.ld_diag.assign(t.ld.begin(), t.ld.begin() + V);
  p.ld_fwd.assign(t.ld.begin() + V, t.ld.begin() + 5 * V);
  p.ld_bwd.assign(t.ld.begin() + 5 * V, t.ld.end());
  p.off_all = t.off;
  p.ld_all = t.ld;
  p.maps = t.maps;
  p.segs.assign(1, Segment{Ns, Nt, V, batch, 0, 0, 0, 0});
  p.vsites.clear();
  std::vector<FNode> F;
  F.reserve(t.nodes.size());
  for (const SNode& n : t.nodes) F.push_back(fnode_of(p, n, 0, 0, 0, 0));
  build_schedule(p, F, t.n_levels, precision);
  for (size_t i = 0; i < F.size(); ++i) p.nodes[i].tmp = F[i].tmp;
  p.segs[0].rep_stride = p.arena_elems;  // each replica: its own fronts and workspace (grid.y)
}

void analyze_ragged(Plan& p, int nshapes, const int* Ns, const int* Nt, const int* count, int precision,
                    int panel) {
  if (nshapes < 1 || !Ns || !Nt || !count) throw std::invalid_argument("shapes");
  int64_t lattices = 0, sites = 0;
  for (int s = 0; s < nshapes; ++s) {
    check_shape(Ns[s], Nt[s]);
    if (count[s] < 1) throw std::invalid_argument("count");
    lattices += count[s];
    sites += (int64_t)count[s] * Ns[s] * Ns[s] * Ns[s] * Nt[s];
  }
  if (lattices > 65535 || sites * 3 > (1LL << 31) - 1) throw std::invalid_argument("too many lattices");
  p.panel = check_precision_panel(precision, panel);
  p.precision = precision;
  p.ragged = true;
  p.fbatch = 1;
  p.batch = (int)lattices;
  p.V = (int)sites;
  p.N = 3 * p.V;
  p.Ns = p.Nt = 0;
  p.nodes.clear();
  p.maps.clear();
  p.off_all.clear();
  p.ld_all.clear();
  p.off_diag.clear();
  p.off_fwd.clear();
  p.off_bwd.clear();
  p.ld_diag.clear();
  p.ld_fwd.clear();
  p.ld_bwd.clear();
  p.segs.clear();
  p.vsites.clear();
  p.factor_flops = p.selinv_flops = 0;
  std::vector<FNode> F;
  int n_levels = 0;
  int64_t base = 0, table_base = 0, site_base = 0;
  for (int s = 0; s < nshapes; ++s) {
    Tree t;
    build_tree(t, Ns[s], Nt[s], p.panel);
    const int maps_base = (int)p.maps.size();
    p.maps.insert(p.maps.end(), t.maps.begin(), t.maps.end());
    p.off_all.insert(p.off_all.end(), t.off.begin(), t.off.end());
    p.ld_all.insert(p.ld_all.end(), t.ld.begin(), t.ld.end());
    p.segs.push_back(Segment{Ns[s], Nt[s], t.V, count[s], base, t.pool_elems, table_base, site_base});
    for (int r = 0; r < count[s]; ++r) {
      const int index_base = (int)F.size();
      for (const SNode& n : t.nodes)
        F.push_back(fnode_of(p, n, base, index_base, maps_base, site_base + (int64_t)r * t.V));
      base += t.pool_elems;
    }
    p.nodes.insert(p.nodes.end(), t.nodes.begin(), t.nodes.end());
    n_levels = std::max(n_levels, t.n_levels);
    table_base += 9LL * t.V;
    site_base += (int64_t)count[s] * t.V;
    p.factor_flops += count[s] * t.factor_flops;
    p.selinv_flops += count[s] * t.selinv_flops;
  }
  // flops per lattice (averaged), so that info.batch x flops is the plan's work
  p.factor_flops /= (double)lattices;
  p.selinv_flops /= (double)lattices;
  p.pool_elems = base;
  build_schedule(p, F, n_levels, precision);
}

}  // namespace cl
