// Host-side symbolic phase: geometric nested dissection, separator
// reordering, elimination tree, I^upd, front HSS trees and index maps.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace hssmf {

// Binary cluster tree of one front, nodes in postorder, front-local ranges.
struct ClusterTree {
  std::vector<int> lo, hi, c1, c2, parent;
  int root() const { return (int)lo.size() - 1; }
  int size() const { return (int)lo.size(); }
  bool leaf(int t) const { return c1[t] < 0; }
  int add(int l, int h, int a = -1, int b = -1) {
    int t = (int)lo.size();
    lo.push_back(l); hi.push_back(h); c1.push_back(a); c2.push_back(b); parent.push_back(-1);
    if (a >= 0) { parent[a] = t; parent[b] = t; }
    return t;
  }
};

struct FrontSym {
  int sep_begin = 0, sep_end = 0, first = 0;
  int child[2] = {-1, -1};
  int nchild = 0;
  int parent = -1;
  int height = 0;
  std::vector<int> upd;  // I^upd, ascending new indices
  int ns() const { return sep_end - sep_begin; }
  int nu() const { return (int)upd.size(); }
  int nf() const { return ns() + nu(); }
  // Local sparse part A_i: rows 0..nf-1, entries (col, value index into CSR values)
  std::vector<int> a_rowptr, a_col, a_val;
  // Position of each of this front's I^upd entries inside the parent's I (ascending).
  std::vector<int> pos_in_parent;
  ClusterTree tree;
  int k_node = -1, q_node = -1;
  // Nested piece structure from the separator bisection (pre-order encoding):
  // used only while building the tree.
};

struct Symbolic {
  int nx = 0, ny = 0, nz = 0, n = 0, nnz = 0;  // grid sides: those of the first grid
  int nsys = 1;                 // independent grids (block-diagonal systems)
  std::vector<int> sys_off;     // natural index range of grid s: [sys_off[s], sys_off[s+1])
  int nd_leaf = 8, hss_leaf = 128;
  std::vector<int> perm;   // perm[new] = natural
  std::vector<int> iperm;  // iperm[natural] = new
  std::vector<FrontSym> fronts;  // postorder
  std::vector<std::vector<int>> levels;  // fronts by height (0 = leaves)
  std::vector<int> tpos;  // CSR position of the transposed entry
};

// Returns an empty string on success, else an error message.
std::string analyze_grid(int nx, int ny, int nz, int n, const int* rowptr, const int* colind,
                         int nd_leaf, int hss_leaf, Symbolic& out);
// nsys grids (dims: 3 sides per grid) of one block-diagonal matrix, grid s
// owning the natural indices after those of grids 0..s-1: one elimination
// forest with a common level schedule.
std::string analyze_grids(int nsys, const int* dims, int n, const int* rowptr, const int* colind,
                          int nd_leaf, int hss_leaf, Symbolic& out);
// A general structurally symmetric pattern.  perm == nullptr: algebraic
// nested dissection (one tree per connected component).  Otherwise the
// caller's ordering (perm[new] = old) and separator tree: front f owns the
// new indices [sep_ptr[f], sep_ptr[f+1]), parent[f] > f or -1, at most two
// children per front.
std::string analyze_csr(int n, const int* rowptr, const int* colind, int nfronts, const int* perm,
                        const int* sep_ptr, const int* parent, int nd_leaf, int hss_leaf, Symbolic& out);

}  // namespace hssmf
