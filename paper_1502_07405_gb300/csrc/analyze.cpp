// Geometric nested dissection and symbolic factorization (host C++).
//
// Ordering rules (Sections 3.1, 4.2 and 6.1 of the paper, with the readings
// where it is silent):
//   - boxes are half-open per axis; a box with every side <= nd_leaf is a
//     leaf of the elimination tree;
//   - otherwise the longest side is cut (ties: lowest axis) at
//     mid = lo + len / 2; the plane at mid is the separator, the children
//     are [lo, mid) and [mid + 1, hi);
//   - postorder numbering: left subtree, right subtree, separator;
//   - the vertices of a separator (or leaf box) are ordered by recursive
//     bisection of its box with the same cut rule into [lo, mid) and
//     [mid, hi) until a piece has <= hss_leaf vertices; pieces in order, x
//     fastest inside a piece.  The bisection tree is the F11 cluster tree.
// Symbolic (Section 5.4): I^upd of a front is the set of vertices numbered
// after its separator that are adjacent to the separator or in a child's
// I^upd, ascending.  The F22 cluster tree halves the I^upd list at
// floor(n/2) until a node has <= hss_leaf indices; the front tree is
// root -> [F11 tree, F22 tree] (the F11 tree alone without I^upd).
// Several independent grids (a block-diagonal matrix, grid s owning the
// natural indices [sys_off[s], sys_off[s+1])) are ordered one after the other:
// the elimination forest is the concatenation of their trees in postorder and
// a front's level is its height, so one level schedule covers every system.
#include "analyze.h"

#include <algorithm>
#include <array>
#include <cstdlib>
#include <cstdio>

namespace hssmf {
namespace {

using Box = std::array<int, 6>;  // lo x, lo y, lo z, hi x, hi y, hi z

int cut_axis(const Box& b, int* len) {
  for (int a = 0; a < 3; ++a) len[a] = b[3 + a] - b[a];
  int best = 0;
  for (int a = 1; a < 3; ++a)
    if (len[a] > len[best]) best = a;
  return best;
}

struct Builder {
  int nx, ny, nz, nd_leaf, hss_leaf;
  std::vector<int> perm;
  std::vector<FrontSym> fronts;
  int base = 0;  // natural index of vertex (0, 0, 0) of the grid being ordered

  void box_vertices(const Box& b) {
    for (int z = b[2]; z < b[5]; ++z)
      for (int y = b[1]; y < b[4]; ++y)
        for (int x = b[0]; x < b[3]; ++x) perm.push_back(base + x + nx * (y + ny * z));
  }

  // Recursive bisection of a box into pieces; appends vertices and adds the
  // cluster nodes (postorder) to tree with ranges offset by the local start.
  int bisect(const Box& b, ClusterTree& tree, int& local) {
    long vol = (long)(b[3] - b[0]) * (b[4] - b[1]) * (b[5] - b[2]);
    if (vol <= hss_leaf) {
      int lo = local;
      box_vertices(b);
      local += (int)vol;
      return tree.add(lo, local);
    }
    int len[3];
    int a = cut_axis(b, len);
    int mid = b[a] + len[a] / 2;
    Box l = b, r = b;
    l[3 + a] = mid;
    r[a] = mid;
    int lo = local;
    int t1 = bisect(l, tree, local);
    int t2 = bisect(r, tree, local);
    return tree.add(lo, local, t1, t2);
  }

  int add_front(const Box& sepbox, int first, int c1, int c2) {
    FrontSym f;
    f.first = first;
    f.sep_begin = (int)perm.size();
    int local = 0;
    f.k_node = bisect(sepbox, f.tree, local);
    f.sep_end = (int)perm.size();
    if (c1 >= 0) {
      f.child[0] = c1;
      f.child[1] = c2;
      f.nchild = 2;
    }
    fronts.push_back(std::move(f));
    int me = (int)fronts.size() - 1;
    if (c1 >= 0) {
      fronts[c1].parent = me;
      fronts[c2].parent = me;
    }
    return me;
  }

  int rec(const Box& b) {
    int len[3];
    int a = cut_axis(b, len);
    int first = (int)perm.size();
    if (len[0] <= nd_leaf && len[1] <= nd_leaf && len[2] <= nd_leaf)
      return add_front(b, first, -1, -1);
    int mid = b[a] + len[a] / 2;
    Box l = b, r = b, s = b;
    l[3 + a] = mid;
    r[a] = mid + 1;
    s[a] = mid;
    s[3 + a] = mid + 1;
    int c1 = rec(l);
    int c2 = rec(r);
    return add_front(s, first, c1, c2);
  }
};

int halving(ClusterTree& t, int lo, int hi, int b) {
  if (hi - lo <= b) return t.add(lo, hi);
  int mid = lo + (hi - lo) / 2;
  int l = halving(t, lo, mid, b);
  int r = halving(t, mid, hi, b);
  return t.add(lo, hi, l, r);
}

// Algebraic nested dissection of a structurally symmetric pattern (no
// geometry).  Connected components are separate trees of the forest.  In a
// connected vertex set, the level structure of a breadth-first search from a
// pseudo-peripheral vertex (the last vertex reached by a first search) gives
// the separator: the level at which the cumulative count passes half the set;
// a separator vertex with no neighbour beyond that level moves to the near
// side.  A disconnected set (left behind by a level separator) is split into
// two groups of whole components of about equal size by a one-vertex
// separator taken from the second group.  Sets of at most leaf_max vertices
// are leaves.  Separator vertices keep their search order; the F11 cluster
// tree halves that order down to hss_leaf.
struct AlgebraicND {
  const int* rp;
  const int* ci;
  int leaf_max, hss_leaf;
  std::vector<int> perm;
  std::vector<FrontSym> fronts;
  std::vector<int> mark, lev;  // set membership stamp, search level
  int stamp = 0;

  // breadth-first search inside the set stamped st, from s; returns the
  // visit order, levels in lev[]
  void bfs(int s, int st, std::vector<int>& order) {
    order.clear();
    order.push_back(s);
    lev[s] = 0;
    mark[s] = -st;  // visited
    for (size_t h = 0; h < order.size(); ++h) {
      const int u = order[h];
      for (int p = rp[u]; p < rp[u + 1]; ++p) {
        const int w = ci[p];
        if (mark[w] == st) {
          mark[w] = -st;
          lev[w] = lev[u] + 1;
          order.push_back(w);
        }
      }
    }
  }
  void restamp(const std::vector<int>& V, int st) {
    for (int v : V) mark[v] = st;
  }
  int add_front(const std::vector<int>& sep, int c1, int c2) {
    FrontSym f;
    f.first = (int)perm.size();
    f.sep_begin = (int)perm.size();
    perm.insert(perm.end(), sep.begin(), sep.end());
    f.sep_end = (int)perm.size();
    f.k_node = halving(f.tree, 0, f.ns(), hss_leaf);
    if (c1 >= 0) f.child[f.nchild++] = c1;
    if (c2 >= 0) f.child[f.nchild++] = c2;
    fronts.push_back(std::move(f));
    const int me = (int)fronts.size() - 1;
    for (int k = 0; k < fronts[me].nchild; ++k) fronts[fronts[me].child[k]].parent = me;
    return me;
  }
  // components of V (V stamped st on entry; every vertex visited on exit)
  void components(const std::vector<int>& V, int st, std::vector<std::vector<int>>& comps) {
    std::vector<int> order;
    for (int v : V)
      if (mark[v] == st) {
        bfs(v, st, order);
        comps.push_back(order);
      }
  }
  int rec(std::vector<int> V) {
    if ((int)V.size() <= leaf_max) return add_front(V, -1, -1);
    const int st = ++stamp;
    restamp(V, st);
    std::vector<int> order;
    bfs(V[0], st, order);
    std::vector<int> S, A, B;
    if (order.size() < V.size()) {  // disconnected: two groups of whole components
      restamp(V, st);
      std::vector<std::vector<int>> comps;
      components(V, st, comps);
      std::stable_sort(comps.begin(), comps.end(),  // equal sizes keep their discovery order
                       [](const std::vector<int>& a, const std::vector<int>& b) { return a.size() > b.size(); });
      size_t na = 0, nb = 0;
      std::vector<int> ga, gb;
      for (auto& c : comps) {  // largest first, each to the smaller group
        auto& g = na <= nb ? ga : gb;
        g.insert(g.end(), c.begin(), c.end());
        (na <= nb ? na : nb) += c.size();
      }
      S.push_back(gb.back());  // any vertex of the second group separates the groups
      gb.pop_back();
      A = std::move(ga);
      B = std::move(gb);
    } else {
      restamp(V, st);
      bfs(order.back(), st, order);  // from a pseudo-peripheral vertex
      const int depth = lev[order.back()];
      if (depth < 2) return add_front(V, -1, -1);  // no level separates two non-empty sides
      std::vector<int> cnt(depth + 1, 0);
      for (int v : order) ++cnt[lev[v]];
      int l = 1, cum = cnt[0];
      while (l < depth - 1 && 2 * (cum + cnt[l]) <= (int)V.size()) cum += cnt[l++];
      for (int v : order) {
        if (lev[v] < l) A.push_back(v);
        else if (lev[v] > l) B.push_back(v);
        else {
          bool far = false;
          for (int p = rp[v]; p < rp[v + 1] && !far; ++p) {
            const int w = ci[p];
            far = mark[w] == -st && lev[w] > l;
          }
          (far ? S : A).push_back(v);
        }
      }
    }
    const int c1 = A.empty() ? -1 : rec(std::move(A));
    const int c2 = B.empty() ? -1 : rec(std::move(B));
    return add_front(S, c1, c2);
  }
};

}  // namespace

// Shared tail of every analysis: from the ordering (out.perm) and the fronts
// (separator ranges, children, F11 cluster trees) to iperm, I^upd, levels,
// the F22 trees, the positions in the parents and the local sparse parts.
// Fails if a front's I^upd is not inside its parent's index set (the
// separator tree is then not an elimination structure of the pattern).
static std::string finish_symbolic(const int* rowptr, const int* colind, int hss_leaf, Symbolic& out) {
  const int n = out.n;
  if ((int)out.perm.size() != n) return "internal: ordering size mismatch";
  out.iperm.assign(n, -1);
  for (int v = 0; v < n; ++v) out.iperm[out.perm[v]] = v;

  // symbolic factorization, bottom-up (fronts are in postorder)
  std::vector<int> buf;
  for (size_t fi = 0; fi < out.fronts.size(); ++fi) {
    FrontSym& f = out.fronts[fi];
    buf.clear();
    for (int v = f.sep_begin; v < f.sep_end; ++v) {
      int o = out.perm[v];
      for (int p = rowptr[o]; p < rowptr[o + 1]; ++p) {
        int g = out.iperm[colind[p]];
        if (g >= f.sep_end) buf.push_back(g);
      }
    }
    for (int c = 0; c < f.nchild; ++c)
      for (int g : out.fronts[f.child[c]].upd)
        if (g >= f.sep_end) buf.push_back(g);
    std::sort(buf.begin(), buf.end());
    buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
    f.upd = buf;
    f.height = 0;
    for (int c = 0; c < f.nchild; ++c)
      f.height = std::max(f.height, out.fronts[f.child[c]].height + 1);
  }
  int maxh = 0;
  for (auto& f : out.fronts) maxh = std::max(maxh, f.height);
  out.levels.assign(maxh + 1, {});
  for (size_t fi = 0; fi < out.fronts.size(); ++fi) out.levels[out.fronts[fi].height].push_back((int)fi);

  // local index of a new index g in front f (-1 if absent)
  auto local_index = [&](const FrontSym& f, int g) -> int {
    if (g >= f.sep_begin && g < f.sep_end) return g - f.sep_begin;
    auto it = std::lower_bound(f.upd.begin(), f.upd.end(), g);
    if (it == f.upd.end() || *it != g) return -1;
    return f.ns() + (int)(it - f.upd.begin());
  };

  for (size_t fi = 0; fi < out.fronts.size(); ++fi) {
    FrontSym& f = out.fronts[fi];
    // cluster tree: F11 already built by bisect(); add F22 and the root
    if (f.nu() > 0) {
      f.q_node = halving(f.tree, f.ns(), f.nf(), hss_leaf);
      f.tree.add(0, f.nf(), f.k_node, f.q_node);
    }
    // positions of I^upd in the parent's I
    if (f.parent >= 0) {
      const FrontSym& p = out.fronts[f.parent];
      f.pos_in_parent.resize(f.nu());
      for (int j = 0; j < f.nu(); ++j) {
        int l = local_index(p, f.upd[j]);
        if (l < 0) return "a front's I^upd is not inside its parent's index set (not an elimination tree of the pattern)";
        f.pos_in_parent[j] = l;
      }
    } else if (f.nu() > 0) {
      return "a root front has a non-empty I^upd (not an elimination tree of the pattern)";
    }
    // local sparse part A_i = [A(sep, I) ; A(upd, sep)]
    int nf = f.nf(), ns = f.ns();
    std::vector<std::vector<std::pair<int, int>>> rows(nf);
    for (int r = 0; r < ns; ++r) {
      int o = out.perm[f.sep_begin + r];
      for (int p = rowptr[o]; p < rowptr[o + 1]; ++p) {
        int g = out.iperm[colind[p]];
        int c = local_index(f, g);
        if (c >= 0) {
          rows[r].push_back({c, p});
          if (c >= ns) rows[c].push_back({r, out.tpos[p]});  // A(upd, sep) via the transpose entry
        } else if (g >= f.sep_end) {
          return "internal: separator neighbour outside the front";
        }
      }
    }
    f.a_rowptr.assign(nf + 1, 0);
    for (int r = 0; r < nf; ++r) {
      std::sort(rows[r].begin(), rows[r].end());
      f.a_rowptr[r + 1] = f.a_rowptr[r] + (int)rows[r].size();
    }
    f.a_col.resize(f.a_rowptr[nf]);
    f.a_val.resize(f.a_rowptr[nf]);
    for (int r = 0, k = 0; r < nf; ++r)
      for (auto& e : rows[r]) { f.a_col[k] = e.first; f.a_val[k] = e.second; ++k; }
  }
  return "";
}

std::string analyze_grid(int nx, int ny, int nz, int n, const int* rowptr, const int* colind,
                         int nd_leaf, int hss_leaf, Symbolic& out) {
  const int dims[3] = {nx, ny, nz};
  return analyze_grids(1, dims, n, rowptr, colind, nd_leaf, hss_leaf, out);
}

std::string analyze_grids(int nsys, const int* dims, int n, const int* rowptr, const int* colind,
                          int nd_leaf, int hss_leaf, Symbolic& out) {
  if (nsys < 1 || !dims) return "at least one grid is required";
  std::vector<int> off(nsys + 1, 0);
  for (int s = 0; s < nsys; ++s) {
    const int* d = dims + 3 * s;
    if (d[0] < 1 || d[1] < 1 || d[2] < 1) return "grid sides must be positive";
    const long long ns = (long long)d[0] * d[1] * d[2];
    if (off[s] + ns > 0x7fffffffLL) return "total grid size exceeds 2^31 - 1";
    off[s + 1] = off[s] + (int)ns;
  }
  if (off[nsys] != n) return "grid dims do not match n";
  if (nd_leaf < 1 || hss_leaf < 1) return "nd_leaf and hss_leaf must be positive";
  if (!rowptr || !colind) return "null CSR pattern";
  if (rowptr[0] != 0) return "rowptr[0] must be 0";
  for (int i = 0; i < n; ++i)
    if (rowptr[i + 1] < rowptr[i]) return "rowptr not monotone";
  out = Symbolic();
  out.nx = dims[0]; out.ny = dims[1]; out.nz = dims[2]; out.n = n;
  out.nsys = nsys;
  out.sys_off = off;
  out.nnz = rowptr[n];
  out.nd_leaf = nd_leaf;
  out.hss_leaf = hss_leaf;
  // pattern checks: in range, ascending, neighbours in the same grid,
  // structurally symmetric
  out.tpos.assign(out.nnz, -1);
  for (int s = 0; s < nsys; ++s) {
    const int nx = dims[3 * s], ny = dims[3 * s + 1], b0 = off[s], b1 = off[s + 1];
    for (int i = b0; i < b1; ++i) {
      const int li = i - b0;
      const int xi = li % nx, yi = (li / nx) % ny, zi = li / (nx * ny);
      for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
        int j = colind[p];
        if (j < 0 || j >= n) return "column index out of range";
        if (p > rowptr[i] && colind[p - 1] >= j) return "column indices not ascending";
        if (j < b0 || j >= b1) return "pattern edge joins two grids";
        const int lj = j - b0;
        const int xj = lj % nx, yj = (lj / nx) % ny, zj = lj / (nx * ny);
        if (std::abs(xi - xj) > 1 || std::abs(yi - yj) > 1 || std::abs(zi - zj) > 1)
          return "pattern edge joins vertices that are not grid neighbours";
        const int* b = colind + rowptr[j];
        const int* e = colind + rowptr[j + 1];
        const int* f = std::lower_bound(b, e, i);
        if (f == e || *f != i) return "pattern is not structurally symmetric";
        out.tpos[p] = (int)(f - colind);
      }
    }
  }
  Builder B{dims[0], dims[1], dims[2], nd_leaf, hss_leaf, {}, {}};
  B.perm.reserve(n);
  for (int s = 0; s < nsys; ++s) {
    B.nx = dims[3 * s];
    B.ny = dims[3 * s + 1];
    B.nz = dims[3 * s + 2];
    B.base = off[s];
    B.rec(Box{0, 0, 0, B.nx, B.ny, B.nz});
  }
  out.perm = std::move(B.perm);
  out.fronts = std::move(B.fronts);
  return finish_symbolic(rowptr, colind, hss_leaf, out);
}

// Pattern checks of a general matrix: indices in range, ascending,
// structurally symmetric; fills out.tpos.
static std::string check_csr(int n, const int* rowptr, const int* colind, Symbolic& out) {
  if (n < 1) return "n must be positive";
  if (!rowptr || !colind) return "null CSR pattern";
  if (rowptr[0] != 0) return "rowptr[0] must be 0";
  for (int i = 0; i < n; ++i)
    if (rowptr[i + 1] < rowptr[i]) return "rowptr not monotone";
  out.tpos.assign(rowptr[n], -1);
  for (int i = 0; i < n; ++i)
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
      const int j = colind[p];
      if (j < 0 || j >= n) return "column index out of range";
      if (p > rowptr[i] && colind[p - 1] >= j) return "column indices not ascending";
      const int* b = colind + rowptr[j];
      const int* e = colind + rowptr[j + 1];
      const int* f = std::lower_bound(b, e, i);
      if (f == e || *f != i) return "pattern is not structurally symmetric";
      out.tpos[p] = (int)(f - colind);
    }
  return "";
}

std::string analyze_csr(int n, const int* rowptr, const int* colind, int nfronts, const int* perm,
                        const int* sep_ptr, const int* parent, int nd_leaf, int hss_leaf, Symbolic& out) {
  if (nd_leaf < 1 || hss_leaf < 1) return "nd_leaf and hss_leaf must be positive";
  out = Symbolic();
  std::string e = check_csr(n, rowptr, colind, out);
  if (!e.empty()) return e;
  out.n = n;
  out.nx = n; out.ny = out.nz = 1;
  out.nsys = 1;
  out.sys_off = {0, n};
  out.nnz = rowptr[n];
  out.nd_leaf = nd_leaf;
  out.hss_leaf = hss_leaf;
  if (!perm) {  // algebraic nested dissection, one tree per connected component
    AlgebraicND nd{rowptr, colind, std::max(16, nd_leaf * nd_leaf), hss_leaf, {}, {}, {}, {}};
    nd.mark.assign(n, 0);
    nd.lev.assign(n, 0);
    nd.perm.reserve(n);
    std::vector<int> all(n);
    for (int v = 0; v < n; ++v) all[v] = v;
    const int st = ++nd.stamp;
    nd.restamp(all, st);
    std::vector<std::vector<int>> comps;
    nd.components(all, st, comps);
    for (auto& c : comps) nd.rec(std::move(c));
    out.perm = std::move(nd.perm);
    out.fronts = std::move(nd.fronts);
  } else {  // the caller's ordering and separator tree
    if (nfronts < 1 || !sep_ptr || !parent) return "nfronts, sep_ptr and parent are required with perm";
    std::vector<char> seen(n, 0);
    for (int v = 0; v < n; ++v) {
      if (perm[v] < 0 || perm[v] >= n || seen[perm[v]]) return "perm is not a permutation";
      seen[perm[v]] = 1;
    }
    if (sep_ptr[0] != 0 || sep_ptr[nfronts] != n) return "sep_ptr must run from 0 to n";
    std::vector<int> nch(nfronts, 0);
    for (int f = 0; f < nfronts; ++f) {
      if (sep_ptr[f + 1] <= sep_ptr[f]) return "every front needs at least one separator vertex";
      if (parent[f] != -1 && (parent[f] <= f || parent[f] >= nfronts))
        return "fronts must be in postorder (parent index above the child's, -1 for roots)";
      if (parent[f] >= 0 && ++nch[parent[f]] > 2) return "a front may have at most two children";
    }
    out.perm.assign(perm, perm + n);
    out.fronts.resize(nfronts);
    for (int f = 0; f < nfronts; ++f) {
      FrontSym& fs = out.fronts[f];
      fs.sep_begin = fs.first = sep_ptr[f];
      fs.sep_end = sep_ptr[f + 1];
      fs.parent = parent[f];
      fs.k_node = halving(fs.tree, 0, fs.ns(), hss_leaf);
      if (parent[f] >= 0) {
        FrontSym& p = out.fronts[parent[f]];
        p.child[p.nchild++] = f;
      }
    }
  }
  return finish_symbolic(rowptr, colind, hss_leaf, out);
}

}  // namespace hssmf
