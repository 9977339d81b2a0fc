// HSS frontal matrices on the device: host orchestration (Section 4).
//
// All HSS fronts of one elimination-tree level are processed together, and
// inside them all nodes of one HSS-tree height: every step below is one
// batched launch over (front, node) jobs.
//
// Per level:
//   1. R_i(r, c) = G(seed, I_i(r), c) (the child blocks R(I^upd_child, :) are
//      generated from the child's global indices, which is eq. Rmerge);
//      S^r = A_i R (+) U_child R_child, S^c = A_i^T R (+) U_child^T R_child
//      (eq. FtimesR; children's update matrices are dense in HBM).
//   2. Algorithm 1 bottom-up, heights of the front trees in order.  A round
//      processes every node whose children are compressed with all d
//      columns; IDs already accepted are kept (Section 2.2.1).  A node fails
//      if its rank exceeds d - p and its size; then d += dd for its front
//      and the next round samples only the new columns.
//   3. ULV-like factorization of F11 (Section 2.3), low-rank Schur update
//      Theta^* Phi (Section 4.4), and the dense update matrix
//      F22 - Theta^* Phi for the parent.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <type_traits>
#include <vector>

#include "hss.h"
#include "hss_kernels.h"

namespace hssmf {

namespace {

constexpr size_t ALIGN = 256;
// IDs with d * m at least this large run on a thread-block cluster
// (measured on GB300: one CTA is fastest for nodes of <= 256 columns, 8-CTA
// clusters for d * m up to ~1M, 16-CTA clusters beyond)
constexpr long long kClusterIdWork = 64 * 1024;
constexpr long long kClusterIdWork16 = 1024 * 1024;  // ... and on 16 CTAs from this size
constexpr long long kTinyIdBytes = 32 * 1024;        // one CTA per job up to this matrix size

struct Pool {  // device bump allocator over large chunks
  std::vector<std::pair<char*, size_t>> chunks;
  size_t ci = 0, off = 0, used = 0, peak = 0;
  char* alloc(size_t bytes) {
    bytes = std::max<size_t>((bytes + ALIGN - 1) / ALIGN * ALIGN, ALIGN);
    for (;;) {
      if (ci < chunks.size()) {
        if (off + bytes <= chunks[ci].second) {
          char* p = chunks[ci].first + off;
          off += bytes;
          used += bytes;
          peak = std::max(peak, used);
          return p;
        }
        ++ci;
        off = 0;
        continue;
      }
      size_t sz = std::max<size_t>(bytes, (size_t)256 << 20);
      char* p = nullptr;
      if (cudaMalloc(&p, sz) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
      }
      chunks.push_back({p, sz});
    }
  }
  void reset() { ci = 0; off = 0; used = 0; }
  void release() {
    for (auto& c : chunks) cudaFree(c.first);
    chunks.clear();
    reset();
  }
};

struct Ring {  // job descriptors: pinned host staging -> device, reused after a sync
  char* h = nullptr;
  char* d = nullptr;
  size_t cap = 0, off = 0;
  const cudaStream_t* side = nullptr;  // other streams whose launches read the ring
  int nside = 0;
  bool grow(size_t need) {
    if (h) cudaFreeHost(h);
    if (d) cudaFree(d);
    h = d = nullptr;
    cap = std::max(need, (size_t)64 << 20);
    if (cudaMallocHost(&h, cap) != cudaSuccess || cudaMalloc(&d, cap) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    off = 0;
    return true;
  }
  template <class J>
  const J* put(const std::vector<J>& v, cudaStream_t s) {
    size_t bytes = std::max<size_t>((v.size() * sizeof(J) + ALIGN - 1) / ALIGN * ALIGN, ALIGN);
    if (off + bytes > cap) {
      cudaStreamSynchronize(s);
      for (int q = 0; q < nside; ++q) cudaStreamSynchronize(side[q]);
      off = 0;
      if (bytes > cap && !grow(bytes)) return nullptr;
    }
    if (!v.empty()) {
      std::memcpy(h + off, v.data(), v.size() * sizeof(J));
      cudaMemcpyAsync(d + off, h + off, v.size() * sizeof(J), cudaMemcpyHostToDevice, s);
    }
    const J* p = (const J*)(d + off);
    off += bytes;
    return p;
  }
  void release() {
    if (h) cudaFreeHost(h);
    if (d) cudaFree(d);
    h = d = nullptr;
    cap = off = 0;
  }
};

// leading dimension of a child's sampling matrix R(I^upd_child, :) stored as
// BF16 in the FP32 form: 16-byte aligned columns for 16-byte copies
inline int rch_ld(int nu) { return (nu + 7) & ~7; }

struct NodeRt {
  int m = 0, mc = 0, n = 0;  // ID row counts (S^r, S^c) and node size
  int kr = 0, kc = 0;
  bool done = false, extracted = false;
  void *D = nullptr, *B12 = nullptr, *B21 = nullptr;
  int *piv_r = nullptr, *piv_c = nullptr;
  void *Xr = nullptr, *Xc = nullptr;
  int *Ir = nullptr, *Ic = nullptr;
  int slot = -1;
  // compression: Y (this round's rows of the samples before the ID); S^r, S^c
  // after the ID and R^r, R^c (rows 0..dk-1 computed, leading dimension dk,
  // carried from round to round so that a later round adds only the rows of
  // the new sample columns)
  void *Yr = nullptr, *Yc = nullptr, *Srp = nullptr, *Scp = nullptr, *Rrp = nullptr, *Rcp = nullptr;
  int dk = 0;
  // factor
  void *Uexp = nullptr, *Vexp = nullptr, *Dt = nullptr, *Vt = nullptr, *tau = nullptr, *Tq = nullptr;
  int* lupiv = nullptr;
  int* luperm = nullptr;
  // transposed generators (D^T; B21^T and B12^T, the B12 and B21 of the
  // transposed matrix) and the ULV factorization of the transposed F11,
  // built at the first solve_T after a factorization; swap_view exchanges
  // them with the fields above
  void *DT = nullptr, *Bt12 = nullptr, *Bt21 = nullptr;
  void *DtT = nullptr, *VtT = nullptr, *tauT = nullptr, *TqT = nullptr;
  int* lupivT = nullptr;
  int* lupermT = nullptr;
  void *Ubig = nullptr, *Vbig = nullptr;
  // solve scratch
  void *bt = nullptr, *bo = nullptr, *w = nullptr, *x = nullptr;
};

struct FrontRt {
  int f = -1, nf = 0, ns = 0, nu = 0;
  int d = 0, dprev = 0, dalloc = 0, rounds = 0;
  bool compressed = false, failed = false;
  void *R = nullptr, *Sr = nullptr, *Sc = nullptr;
  void* Rch[2] = {nullptr, nullptr};
  long long gidx_off = 0;
  long long pos_off[2] = {-1, -1};  // ints offset of the children's positions in I_i
  long long rch_off[2] = {-1, -1};  // ints offset of the children's I^upd, grid-local (keys of R)
  std::vector<NodeRt> nd;
  std::vector<int> height;
  int tree_h = 0;
  // low-rank Schur and solve data
  void* Z = nullptr;
  void* ZT = nullptr;  // the same for the transposed front (solve_T)
  int k = -1, q = -1, root = -1;
  std::vector<int> f11;  // F11 subtree nodes in postorder
};

// Exchanges the generators of the front's HSS matrix with those of its
// transpose (row and column IDs, bases and ranks, D <-> D^T, B12 <-> B21^T,
// B21 <-> B12^T) and the ULV data with the transposed ULV data: every
// routine that works on the view then works on the transposed front.
// Applying it twice restores the front.
void swap_view(FrontRt& F) {
  for (NodeRt& N : F.nd) {
    std::swap(N.kr, N.kc);
    std::swap(N.m, N.mc);
    std::swap(N.piv_r, N.piv_c);
    std::swap(N.Xr, N.Xc);
    std::swap(N.Ir, N.Ic);
    std::swap(N.Uexp, N.Vexp);
    std::swap(N.Ubig, N.Vbig);
    std::swap(N.D, N.DT);
    std::swap(N.B12, N.Bt12);
    std::swap(N.B21, N.Bt21);
    std::swap(N.Dt, N.DtT);
    std::swap(N.Vt, N.VtT);
    std::swap(N.tau, N.tauT);
    std::swap(N.Tq, N.TqT);
    std::swap(N.lupiv, N.lupivT);
    std::swap(N.luperm, N.lupermT);
  }
  std::swap(F.Z, F.ZT);
}

struct ViewGuard {  // transposed view of the listed fronts for a scope
  std::vector<FrontRt*> fs;
  bool on;
  ViewGuard(const std::vector<FrontRt*>& f, bool t) : fs(f), on(t) {
    if (on)
      for (FrontRt* F : fs) swap_view(*F);
  }
  ~ViewGuard() {
    if (on)
      for (FrontRt* F : fs) swap_view(*F);
  }
};

}  // namespace

struct HssState {
  Pool fac, lvl, rnd, sol;
  // node samples kept across compression rounds, alternating by round: round
  // i writes keep[i & 1] and reads round i-1's arrays in the other pool
  Pool keep[2];
  Pool gws;  // split-K partial tiles of one GEMM launch (reused by the next)
  bool transposed_ready = false;  // ULV of the transposed F11 trees built
  Ring ring;
  // side streams of the ID launches of one batch (independent nodes, run
  // concurrently): fork marks the batch's job arrays on the device, join[k]
  // the end of side stream k's launches; side_state 0 = not created yet,
  // 1 = ready, -1 = unavailable (every launch stays on the main stream)
  static constexpr int kSide = 16;
  cudaStream_t side[kSide] = {};
  cudaEvent_t fork = nullptr, join[kSide] = {};
  int side_state = 0;
  int* d_ranks = nullptr;
  int* h_ranks = nullptr;
  int rank_cap = 0;
  long long iota_off = 0;
  std::vector<int> index;  // front id -> slot in fronts (-1 if dense)
  std::vector<FrontRt> fronts;
  int sol_nrhs = -1;
  double flops = 0.0, bytes = 0.0;
};

hssmf_status hss_prepare(hssmf_ctx& c) {
  hss_release(c);
  if (c.n_hss == 0) return HSSMF_OK;
  HssState* H = new HssState();
  c.hss = H;
  const Symbolic& S = c.sym;
  H->index.assign(S.fronts.size(), -1);
  c.hss_first_level = -1;
  for (size_t h = 0; h < c.plan.size() && c.hss_first_level < 0; ++h)
    if (!c.plan[h].hss.empty()) c.hss_first_level = (int)h;
  int max_nf = 0;
  for (size_t i = 0; i < S.fronts.size(); ++i) max_nf = std::max(max_nf, S.fronts[i].nf());
  H->iota_off = (long long)c.ints_host.size();
  for (int i = 0; i < max_nf; ++i) c.ints_host.push_back(i);
  for (size_t i = 0; i < S.fronts.size(); ++i) {
    if (!c.is_hss[i]) continue;
    const FrontSym& f = S.fronts[i];
    H->index[i] = (int)H->fronts.size();
    H->fronts.emplace_back();
    FrontRt& F = H->fronts.back();
    F.f = (int)i;
    F.nf = f.nf();
    F.ns = f.ns();
    F.nu = f.nu();
    // R is keyed by the row's index inside its own grid, so a grid factored
    // in a batch draws the same sketch as when factored alone
    const int base = S.sys_off.empty()
                         ? 0
                         : *(std::upper_bound(S.sys_off.begin(), S.sys_off.end(), f.sep_begin) - 1);
    F.gidx_off = (long long)c.ints_host.size();
    for (int v = f.sep_begin; v < f.sep_end; ++v) c.ints_host.push_back(v - base);
    for (int g : f.upd) c.ints_host.push_back(g - base);
    for (int k = 0; k < f.nchild; ++k) {
      const FrontSym& ch = S.fronts[f.child[k]];
      F.pos_off[k] = (long long)c.ints_host.size();
      c.ints_host.insert(c.ints_host.end(), ch.pos_in_parent.begin(), ch.pos_in_parent.end());
      F.rch_off[k] = (long long)c.ints_host.size();
      for (int g : ch.upd) c.ints_host.push_back(g - base);
    }
    const ClusterTree& t = f.tree;
    F.nd.assign(t.size(), NodeRt());
    F.height.assign(t.size(), 0);
    for (int u = 0; u < t.size(); ++u) {
      F.nd[u].n = t.hi[u] - t.lo[u];
      if (!t.leaf(u)) F.height[u] = 1 + std::max(F.height[t.c1[u]], F.height[t.c2[u]]);
    }
    F.tree_h = F.height[t.root()];
    F.k = f.k_node;
    F.q = f.q_node;
    F.root = t.root();
    // F11 subtree in postorder (nodes are stored in postorder, the subtree is contiguous)
    std::vector<int> st{F.k};
    while (!st.empty()) {
      int u = st.back();
      st.pop_back();
      F.f11.push_back(u);
      if (!t.leaf(u)) {
        st.push_back(t.c1[u]);
        st.push_back(t.c2[u]);
      }
    }
    std::sort(F.f11.begin(), F.f11.end());
  }
  return HSSMF_OK;
}

hssmf_status hss_device_init(hssmf_ctx& c) {
  if (!c.hss) return HSSMF_OK;
  HssState& H = *c.hss;
  if (!H.ring.grow((size_t)64 << 20)) return c.fail(HSSMF_ERR_OOM, "job ring allocation failed");
  H.rank_cap = 1 << 20;
  if (cudaMalloc(&H.d_ranks, sizeof(int) * H.rank_cap) != cudaSuccess ||
      cudaMallocHost(&H.h_ranks, sizeof(int) * H.rank_cap) != cudaSuccess) {
    cudaGetLastError();
    return c.fail(HSSMF_ERR_OOM, "rank buffer allocation failed");
  }
  return HSSMF_OK;
}

void hss_release(hssmf_ctx& c) {
  if (!c.hss) return;
  HssState& H = *c.hss;
  for (int k = 0; k < HssState::kSide; ++k) {
    if (H.side[k]) {
      cudaStreamSynchronize(H.side[k]);
      cudaStreamDestroy(H.side[k]);
    }
    if (H.join[k]) cudaEventDestroy(H.join[k]);
  }
  if (H.fork) cudaEventDestroy(H.fork);
  H.fac.release();
  H.lvl.release();
  H.keep[0].release();
  H.keep[1].release();
  H.rnd.release();
  H.sol.release();
  H.gws.release();
  H.ring.release();
  if (H.d_ranks) cudaFree(H.d_ranks);
  if (H.h_ranks) cudaFreeHost(H.h_ranks);
  delete c.hss;
  c.hss = nullptr;
}

namespace {

bool ensure_side_streams(HssState& H) {
  if (H.side_state != 0) return H.side_state > 0;
  H.side_state = -1;  // partial creations are released with the state
  if (cudaEventCreateWithFlags(&H.fork, cudaEventDisableTiming) != cudaSuccess) {
    H.fork = nullptr;
    cudaGetLastError();
    return false;
  }
  for (int k = 0; k < HssState::kSide; ++k) {
    if (cudaStreamCreateWithFlags(&H.side[k], cudaStreamNonBlocking) != cudaSuccess) {
      H.side[k] = nullptr;
      cudaGetLastError();
      return false;
    }
    if (cudaEventCreateWithFlags(&H.join[k], cudaEventDisableTiming) != cudaSuccess) {
      H.join[k] = nullptr;
      cudaGetLastError();
      return false;
    }
  }
  H.ring.side = H.side;
  H.ring.nside = HssState::kSide;
  H.side_state = 1;
  return true;
}

// The main stream waits for every side stream that received a launch.
struct SideJoin {
  HssState& H;
  cudaStream_t main;
  bool used[HssState::kSide] = {};
  ~SideJoin() {
    for (int k = 0; k < HssState::kSide; ++k)
      if (used[k]) {
        cudaEventRecord(H.join[k], H.side[k]);
        cudaStreamWaitEvent(main, H.join[k], 0);
      }
  }
};

template <typename T>
struct Ctx {  // per-call helpers
  hssmf_ctx& c;
  HssState& H;
  cudaStream_t s;
  bool oom = false;
  std::vector<GemmJob> gj;
  std::vector<CopyJob> cj;
  explicit Ctx(hssmf_ctx& cc) : c(cc), H(*cc.hss), s(cc.stream) {}
  T* arena() { return static_cast<T*>(c.d_arena); }
  T* A(Pool& p, long long elems) {
    char* q = p.alloc(sizeof(T) * (size_t)std::max(elems, 1LL));
    if (!q) oom = true;
    return (T*)q;
  }
  int* I(Pool& p, long long n) {
    char* q = p.alloc(sizeof(int) * (size_t)std::max(n, 1LL));
    if (!q) oom = true;
    return (int*)q;
  }
  const int* ints(long long off) const { return c.d_ints + off; }
  // C = alpha op(A) op(B) + beta C
  // b_exact: the values of B are exactly BF16 (the sampling matrix of the
  // FP32 form), which halves the tensor-core products
  void gemm(const void* A_, long long lda, int ta, const void* B_, long long ldb, int tb, void* C_,
            long long ldc, int M, int N, int K, double alpha, double beta, const int* crow = nullptr,
            int b_exact = 0) {
    if (M <= 0 || N <= 0) return;
    if (K <= 0 && beta == 1.0) return;
    GemmJob j;
    std::memset(&j, 0, sizeof(j));
    j.A = A_; j.B = B_; j.C = C_; j.crow = crow;
    j.lda = lda; j.ldb = ldb; j.ldc = ldc;
    j.M = M; j.N = N; j.K = std::max(K, 0);
    j.ta = ta; j.tb = tb; j.alpha = alpha; j.beta = beta;
    j.b_exact = b_exact;
    gj.push_back(j);
    H.flops += 2.0 * M * N * std::max(K, 0);
  }
  // Matrix-vector products (N <= GEMV_MAX_N, the solves) run on the
  // memory-bound GEMV kernel; other FP32 products on the tensor cores (128 x
  // 128 tiles), FP64 products on the DFMA kernel (64 x 64 tiles)
  enum { K_GEMV = 0, K_TILES = 1 };
  void flush_gemm() {
    if (gj.empty()) return;
    constexpr bool tc = std::is_same<T, float>::value;
    for (int pass = 0; pass < 2; ++pass) {
      std::vector<Tile> tiles, rtiles;
      if (pass == K_TILES && tc) split_k();
      for (size_t i = 0; i < gj.size(); ++i) {
        const bool mv = gj[i].N <= GEMV_MAX_N && gj[i].b_exact != 2;  // BF16 B: tensor-core tiles only
        if (mv != (pass == K_GEMV)) continue;
        if (mv) {
          const int rows = gj[i].ta ? GEMV_ROWS_T : GEMV_ROWS_N;
          for (int a = 0; a < ceil_div(gj[i].M, rows); ++a) tiles.push_back(Tile{(int)i, a, 0, 0});
          continue;
        }
        const int tile = tc ? GEMM_TILE_TC : GEMM_TILE;
        const int tm = ceil_div(gj[i].M, tile), tn = ceil_div(gj[i].N, tile);
        const int ks = std::max(gj[i].ksplit, 1);
        for (int q = 0; q < ks; ++q)
          for (int b = 0; b < tn; ++b)
            for (int a = 0; a < tm; ++a) tiles.push_back(Tile{(int)i, a, b, q});
        if (ks > 1)
          for (int b = 0; b < tn; ++b)
            for (int a = 0; a < tm; ++a) rtiles.push_back(Tile{(int)i, a, b, 0});
      }
      if (tiles.empty()) continue;
      const GemmJob* dj = H.ring.put(gj, s);
      const Tile* dt = H.ring.put(tiles, s);
      const Tile* dr = rtiles.empty() ? nullptr : H.ring.put(rtiles, s);
      if (!dj || !dt || (!rtiles.empty() && !dr)) { oom = true; gj.clear(); return; }
      if (pass == K_GEMV) {
        Kern<T>::gemv(dj, dt, (int)tiles.size(), s);
      } else if (tc) {
        gemm_tc(dj, dt, (int)tiles.size(), c.d_status, s);
        if (dr) gemm_tc_reduce(dj, dr, (int)rtiles.size(), s);
      } else {
        Kern<T>::gemm(dj, dt, (int)tiles.size(), s);
      }
    }
    gj.clear();
  }
  // Tensor-core launches with fewer tiles than about two CTAs per SM split
  // the K range of their long-K jobs (partials summed in split order)
  // K split of a tensor-core launch: the tiles run about two CTAs per SM, so
  // t tiles take ceil(t / slots) waves; splitting K in S shortens each CTA
  // about S times but multiplies the CTAs and adds a reduction of S t
  // partial tiles, so S (1..8) minimizes, in units of one unsplit CTA,
  // ceil(S t / slots) / S + 0.03 S t / slots (S > 1); a job is split at most
  // K / 128 ways (eight 16-deep steps per part at least).
  void split_k() {
    static int nsm = 0;
    if (!nsm) {
      int dev = 0;
      cudaGetDevice(&dev);
      if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) nsm = 148;
    }
    long long t0 = 0;
    for (const GemmJob& j : gj)
      if (j.N > GEMV_MAX_N) t0 += (long long)ceil_div(j.M, GEMM_TILE_TC) * ceil_div(j.N, GEMM_TILE_TC);
    if (t0 == 0) return;
    const long long slots = 2LL * nsm;
    int S = 1;
    double best = 1e300;
    for (int q = 1; q <= 8; ++q) {
      const double cost = (double)((q * t0 + slots - 1) / slots) / q + (q > 1 ? 0.03 * q * t0 / slots : 0.0);
      if (cost < best - 1e-9) {
        best = cost;
        S = q;
      }
    }
    if (S < 2) return;
    H.gws.reset();
    for (GemmJob& j : gj) {
      if (j.N <= GEMV_MAX_N) continue;
      const int sj = std::min(S, j.K / 128);
      if (sj < 2) continue;
      const int tm = ceil_div(j.M, GEMM_TILE_TC), tn = ceil_div(j.N, GEMM_TILE_TC);
      float* ws = (float*)H.gws.alloc(sizeof(float) * (size_t)tm * tn * sj * GEMM_TILE_TC * GEMM_TILE_TC);
      if (!ws) continue;  // no room: this job runs unsplit
      j.ws = ws;
      j.ksplit = sj;
      j.tiles_m = tm;
    }
  }
  void copy(const void* src, long long lds, int trans, void* dst, long long ldd, int rows, int cols,
            const int* rmap = nullptr, const int* cmap = nullptr, const void* src2 = nullptr,
            long long lds2 = 0, int split = 0) {
    if (rows <= 0 || cols <= 0) return;
    CopyJob j;
    std::memset(&j, 0, sizeof(j));
    j.src = src; j.src2 = src2; j.lds2 = lds2; j.split = split;
    j.dst = dst; j.rmap = rmap; j.cmap = cmap; j.lds = lds; j.ldd = ldd;
    j.rows = rows; j.cols = cols; j.src_trans = trans;
    cj.push_back(j);
  }
  void flush_copy() {
    if (cj.empty()) return;
    std::vector<Tile> tiles;
    for (size_t i = 0; i < cj.size(); ++i)
      for (int b = 0; b < ceil_div(cj[i].cols, 32); b += COPY_TN)
        for (int a = 0; a < ceil_div(cj[i].rows, 32); ++a) tiles.push_back(Tile{(int)i, a, b});
    const CopyJob* d = H.ring.put(cj, s);
    const Tile* t = H.ring.put(tiles, s);
    if (!d || !t) { oom = true; cj.clear(); return; }
    HssKern<T>::copy(d, t, (int)tiles.size(), s);
    cj.clear();
  }
  template <class J, class F>
  void launch(std::vector<J>& v, F f) {
    if (v.empty()) return;
    const J* d = H.ring.put(v, s);
    if (!d) { oom = true; v.clear(); return; }
    f(d, (int)v.size());
    v.clear();
  }
};

// Columns [dprev, d) of R, R(I^upd_child, :), S^r and S^c of every listed
// front (eq. FtimesR; eq. Rmerge holds because R depends only on the row's
// index, taken inside its grid).
template <typename T>
void sample_fronts(Ctx<T>& X, const std::vector<FrontRt*>& fs) {
  hssmf_ctx& c = X.c;
  const Symbolic& S = c.sym;
  std::vector<PhiloxJob> pj;
  std::vector<SampleAJob> sj;
  int max_rows = 0, max_nf = 0;
  for (FrontRt* F : fs) {
    const FrontSym& f = S.fronts[F->f];
    const int c0 = F->dprev, c1 = F->d;
    if (c1 <= c0) continue;
    pj.push_back(PhiloxJob{X.ints(F->gidx_off), F->R, F->nf, F->nf, c0, c1, 0});
    max_rows = std::max(max_rows, F->nf);
    max_nf = std::max(max_nf, F->nf);
    for (int k = 0; k < f.nchild; ++k) {
      const DFront& ch = c.fronts_host[f.child[k]];
      if (ch.nu == 0) continue;
      const bool b16 = std::is_same<T, float>::value;
      pj.push_back(PhiloxJob{X.ints(F->rch_off[k]), F->Rch[k], b16 ? rch_ld(ch.nu) : ch.nu, ch.nu, c0, c1,
                             b16 ? 1 : 0});
      max_rows = std::max(max_rows, ch.nu);
    }
    sj.push_back(SampleAJob{F->Sr, F->Sc, F->R, F->nf, F->f, c0, c1, 0});
  }
  X.c.prof.mark(PH_SAMPLE, X.s);
  X.launch(pj, [&](const PhiloxJob* d, int n) { HssKern<T>::philox(d, n, max_rows, c.opts.seed, X.s); });
  X.launch(sj, [&](const SampleAJob* d, int n) { HssKern<T>::sample_a(c.ds, c.d_values, d, n, max_nf, X.s); });
  for (int k = 0; k < 2; ++k) {  // one launch per child slot: deterministic order of the sums
    for (FrontRt* F : fs) {
      const FrontSym& f = S.fronts[F->f];
      if (k >= f.nchild) continue;
      const DFront& ch = c.fronts_host[f.child[k]];
      const int c0 = F->dprev, w = F->d - F->dprev;
      if (ch.nu == 0 || w <= 0) continue;
      const T* U = X.arena() + ch.u_off;
      // FP32 form: R_child in BF16 (b_exact 2); FP64 form: R_child in T
      const bool b16 = std::is_same<T, float>::value;
      const long long ldr = b16 ? rch_ld(ch.nu) : ch.nu;
      const void* Rk = (const char*)F->Rch[k] + (b16 ? 2 : sizeof(T)) * (size_t)c0 * ldr;
      const int* pos = X.ints(F->pos_off[k]);
      X.gemm(U, ch.u_ld, 0, Rk, ldr, 0, (T*)F->Sr + (long long)c0 * F->nf, F->nf, ch.nu, w, ch.nu,
             1.0, 1.0, pos, b16 ? 2 : 1);
      X.gemm(U, ch.u_ld, 1, Rk, ldr, 0, (T*)F->Sc + (long long)c0 * F->nf, F->nf, ch.nu, w, ch.nu,
             1.0, 1.0, pos, b16 ? 2 : 1);
    }
    X.flush_gemm();
  }
}

// Room for d columns in R, R_child, S^r, S^c (old columns copied over).
template <typename T>
void ensure_cols(Ctx<T>& X, FrontRt& F, const FrontSym& f) {
  if (F.d <= F.dalloc) return;
  const int na = std::min(F.nf, F.d + X.c.opts.dd);
  auto grow = [&](void*& p, int rows) {
    T* q = X.A(X.H.lvl, (long long)rows * na);
    if (p && F.dprev > 0 && q)
      cudaMemcpyAsync(q, p, sizeof(T) * (size_t)rows * F.dprev, cudaMemcpyDeviceToDevice, X.s);
    p = q;
  };
  grow(F.R, F.nf);
  grow(F.Sr, F.nf);
  grow(F.Sc, F.nf);
  for (int k = 0; k < f.nchild; ++k) {
    const int nu = X.c.fronts_host[f.child[k]].nu;
    if (std::is_same<T, float>::value) {  // BF16, leading dimension rch_ld (16-byte aligned columns)
      const int ld = rch_ld(nu);
      void* q = X.H.lvl.alloc(2 * (size_t)ld * na);
      if (!q) X.oom = true;
      if (F.Rch[k] && F.dprev > 0 && q)
        cudaMemcpyAsync(q, F.Rch[k], 2 * (size_t)ld * F.dprev, cudaMemcpyDeviceToDevice, X.s);
      F.Rch[k] = q;
    } else {
      grow(F.Rch[k], nu);
    }
  }
  F.dalloc = na;
}

// Algorithm 1 with the adaptive rank scheme over all fronts of a level.
template <typename T>
hssmf_status compress_level(Ctx<T>& X, const std::vector<FrontRt*>& fs) {
  hssmf_ctx& c = X.c;
  HssState& H = X.H;
  const Symbolic& S = c.sym;
  const int p = c.opts.oversample_p;
  const double eps = c.opts.hss_tol;
  const int* iota = X.ints(H.iota_off);
  for (FrontRt* F : fs) {
    for (auto& N : F->nd) {
      int n = N.n;
      N = NodeRt();
      N.n = n;
    }
    F->d = std::min(c.opts.d0, F->nf);
    F->dprev = 0;
    F->dalloc = 0;
    F->rounds = 0;
    F->compressed = false;
    F->R = F->Sr = F->Sc = nullptr;
    F->Rch[0] = F->Rch[1] = nullptr;
    F->Z = F->ZT = nullptr;
    ensure_cols(X, *F, S.fronts[F->f]);
  }
  std::vector<FrontRt*> todo = fs;
  sample_fronts(X, todo);
  struct Item {
    FrontRt* F;
    int t;
  };
  H.keep[0].reset();
  H.keep[1].reset();
  for (int iter = 0; !todo.empty(); ++iter) {
    if (X.oom) return c.fail(HSSMF_ERR_OOM, "device memory exhausted during HSS compression");
    // every compressed node of an unfinished front gets new arrays in every
    // round, so round iter-2's arrays are dead
    Pool& keep = H.keep[iter & 1];
    if (iter >= 2) keep.reset();
    int maxh = 0;
    for (FrontRt* F : todo) maxh = std::max(maxh, F->tree_h);
    for (int lv = 0; lv < maxh; ++lv) {
      std::vector<Item> batch;
      for (FrontRt* F : todo) {
        const ClusterTree& tr = S.fronts[F->f].tree;
        for (int t = 0; t < tr.size(); ++t) {
          if (t == tr.root() || F->height[t] != lv) continue;
          if (!tr.leaf(t) && !(F->nd[tr.c1[t]].done && F->nd[tr.c2[t]].done)) continue;
          batch.push_back({F, t});
        }
      }
      if (batch.empty()) continue;
      for (auto& it : batch) {
        const ClusterTree& tr = S.fronts[it.F->f].tree;
        NodeRt& N = it.F->nd[it.t];
        if (tr.leaf(it.t)) {
          N.m = N.mc = N.n;
        } else {
          const NodeRt &a = it.F->nd[tr.c1[it.t]], &b = it.F->nd[tr.c2[it.t]];
          N.m = a.kr + b.kr;
          N.mc = a.kc + b.kc;
        }
      }
      c.prof.mark(PH_EXTRACT, X.s);
      // (a) D of the leaves, B of the sibling pairs: submatrices of F_i
      std::vector<ExtractJob> ej;
      for (auto& it : batch) {
        const ClusterTree& tr = S.fronts[it.F->f].tree;
        NodeRt& N = it.F->nd[it.t];
        if (N.extracted) continue;
        N.extracted = true;
        if (tr.leaf(it.t)) {
          N.D = X.A(H.fac, (long long)N.n * N.n);
          ej.push_back(ExtractJob{iota + tr.lo[it.t], iota + tr.lo[it.t], N.D, N.n, it.F->f, N.n, N.n, 0});
        } else {
          const NodeRt &a = it.F->nd[tr.c1[it.t]], &b = it.F->nd[tr.c2[it.t]];
          N.B12 = X.A(H.fac, (long long)a.kr * b.kc);
          N.B21 = X.A(H.fac, (long long)b.kr * a.kc);
          if (a.kr > 0 && b.kc > 0)
            ej.push_back(ExtractJob{a.Ir, b.Ic, N.B12, a.kr, it.F->f, a.kr, b.kc, 0});
          if (b.kr > 0 && a.kc > 0)
            ej.push_back(ExtractJob{b.Ir, a.Ic, N.B21, b.kr, it.F->f, b.kr, a.kc, 0});
        }
      }
      X.launch(ej, [&](const ExtractJob* d, int n) {
        HssKern<T>::extract(c.ds, c.d_values, X.arena(), d, n, X.s);
      });
      c.prof.mark(PH_PREID, X.s);
      // (b) samples of the node before the ID, stored transposed (sample rows
      // x node rows): all d rows for a node still to compress, only the rows
      // dk..d-1 of the new sample columns for a node compressed in an earlier
      // round (its children's arrays hold all d rows, leading dimension d)
      for (auto& it : batch) {
        const ClusterTree& tr = S.fronts[it.F->f].tree;
        FrontRt& F = *it.F;
        NodeRt& N = F.nd[it.t];
        const int d = F.d, lo = tr.lo[it.t];
        const int r0 = N.done ? N.dk : 0, rows = d - r0;
        if (rows <= 0) continue;
        N.Yr = X.A(H.rnd, (long long)rows * N.m);
        N.Yc = X.A(H.rnd, (long long)rows * N.mc);
        if (tr.leaf(it.t)) {
          X.copy((T*)F.Sr + lo + (long long)r0 * F.nf, F.nf, 1, N.Yr, rows, rows, N.m);
          X.copy((T*)F.Sc + lo + (long long)r0 * F.nf, F.nf, 1, N.Yc, rows, rows, N.mc);
        } else {
          const NodeRt &a = F.nd[tr.c1[it.t]], &b = F.nd[tr.c2[it.t]];
          X.copy((T*)a.Srp + r0, d, 0, N.Yr, rows, rows, a.kr);
          X.copy((T*)b.Srp + r0, d, 0, (T*)N.Yr + (long long)a.kr * rows, rows, rows, b.kr);
          X.copy((T*)a.Scp + r0, d, 0, N.Yc, rows, rows, a.kc);
          X.copy((T*)b.Scp + r0, d, 0, (T*)N.Yc + (long long)a.kc * rows, rows, rows, b.kc);
        }
      }
      X.flush_copy();
      for (auto& it : batch) {
        const ClusterTree& tr = S.fronts[it.F->f].tree;
        FrontRt& F = *it.F;
        NodeRt& N = F.nd[it.t];
        const int d = F.d, lo = tr.lo[it.t];
        const int r0 = N.done ? N.dk : 0, rows = d - r0;
        if (rows <= 0) continue;
        if (tr.leaf(it.t)) {  // S^r - D R, S^c - D^* R (transposed)
          const T* Rt = (const T*)F.R + lo + (long long)r0 * F.nf;
          X.gemm(Rt, F.nf, 1, N.D, N.n, 1, N.Yr, rows, rows, N.m, N.n, -1.0, 1.0);
          X.gemm(Rt, F.nf, 1, N.D, N.n, 0, N.Yc, rows, rows, N.mc, N.n, -1.0, 1.0);
        } else {  // [S^r_1 - B12 R^r_2; S^r_2 - B21 R^r_1], [S^c_1 - B21^* R^c_2; S^c_2 - B12^* R^c_1]
          const NodeRt &a = F.nd[tr.c1[it.t]], &b = F.nd[tr.c2[it.t]];
          X.gemm((T*)b.Rrp + r0, d, 0, N.B12, std::max(a.kr, 1), 1, N.Yr, rows, rows, a.kr, b.kc, -1.0, 1.0);
          X.gemm((T*)a.Rrp + r0, d, 0, N.B21, std::max(b.kr, 1), 1, (T*)N.Yr + (long long)a.kr * rows, rows,
                 rows, b.kr, a.kc, -1.0, 1.0);
          X.gemm((T*)b.Rcp + r0, d, 0, N.B21, std::max(b.kr, 1), 0, N.Yc, rows, rows, a.kc, b.kr, -1.0, 1.0);
          X.gemm((T*)a.Rcp + r0, d, 0, N.B12, std::max(a.kr, 1), 0, (T*)N.Yc + (long long)a.kc * rows, rows,
                 rows, b.kc, a.kr, -1.0, 1.0);
        }
      }
      X.flush_gemm();
      c.prof.mark(PH_ID, X.s);
      // (c) interpolative decompositions of the nodes not yet compressed
      std::vector<IdJob> ij;
      std::vector<Item> idn;
      int maxm = 0;
      for (auto& it : batch) {
        FrontRt& F = *it.F;
        NodeRt& N = F.nd[it.t];
        if (N.done) continue;
        const int d = F.d;
        if (!N.piv_r) {
          N.piv_r = X.I(H.fac, N.m);
          N.piv_c = X.I(H.fac, N.mc);
          N.Xr = X.A(H.fac, (long long)N.m * N.m / 4 + 1);
          N.Xc = X.A(H.fac, (long long)N.mc * N.mc / 4 + 1);
        }
        T* Wr = X.A(H.rnd, (long long)d * N.m);
        T* Wc = X.A(H.rnd, (long long)d * N.mc);
        const int slot = (int)idn.size();
        ij.push_back(IdJob{N.Yr, Wr, N.piv_r, N.Xr, H.d_ranks + 2 * slot, d, N.m});
        ij.push_back(IdJob{N.Yc, Wc, N.piv_c, N.Xc, H.d_ranks + 2 * slot + 1, d, N.mc});
        maxm = std::max(maxm, std::max(N.m, N.mc));
        idn.push_back(it);
        H.flops += 4.0 * d * (double)N.m * std::min(N.m, d) + 4.0 * d * (double)N.mc * std::min(N.mc, d);
      }
      if (X.oom) return c.fail(HSSMF_ERR_OOM, "device memory exhausted during HSS compression");
      if (!ij.empty()) {
        if ((int)ij.size() > H.rank_cap) return c.fail(HSSMF_ERR_ARG, "too many IDs in one level");
        // Routing: FP32 nodes that fit in the registers of a cluster no larger
        // than their shared-memory cluster run register-resident; other nodes
        // run with their matrix in the shared memory of a cluster of 1..16
        // CTAs (overflow columns in global memory); tiny nodes one per CTA
        // (more CTAs per SM).  The L2-resident cluster kernels remain the
        // fallback where a cluster cannot be scheduled.
        std::vector<IdJob> tier[3], smem_tier[5];
        std::vector<int> tier_ix[3], smem_ix[5];  // positions in ij, for the ID trace
        int tm[3] = {0, 0, 0}, td[3] = {0, 0, 0}, sm_m[5] = {0, 0, 0, 0, 0}, sm_d[5] = {0, 0, 0, 0, 0};
        std::map<int, std::vector<IdJob>> rr_tier;  // register-resident (FP32), by configuration
        std::map<int, std::pair<int, int>> rr_md;
        // kernel that ran each ID (ID trace): 100 * family + CTAs per job, family
        // 0 = one CTA in L2, 1 = shared memory, 2 = registers, 3 = L2 cluster,
        // 4 = registers with one exchange per pivot step
        std::vector<int> route(ij.size(), 0);
        auto route_old = [&](size_t ji) {
          const IdJob& j = ij[ji];
          // registers hold less than shared memory: the register-resident
          // kernel only where it needs no larger cluster
          const int rr = HssKern<T>::id_rr_config(j.d, j.m);
          const int cl_sm = HssKern<T>::id_smem_cluster_size(j.d, j.m);
          if (rr > 0 && (cl_sm == 0 || (rr & 31) <= cl_sm)) {
            rr_tier[rr].push_back(j);
            route[ji] = 200 + (rr & 31);
            auto& md = rr_md[rr];
            md.first = std::max(md.first, j.m);
            md.second = std::max(md.second, j.d);
            return;
          }
          // shared-memory kernel on the smallest cluster that holds the
          // matrix; past 16 CTAs the overflow columns stay in global memory
          const long long w = (long long)j.d * j.m;
          const int cl = cl_sm > 0 ? cl_sm : 16;
          if (w * (long long)sizeof(T) > kTinyIdBytes) {
            const int ti = cl == 1 ? 0 : cl == 2 ? 1 : cl == 4 ? 2 : cl == 8 ? 3 : 4;
            smem_tier[ti].push_back(j);
            smem_ix[ti].push_back((int)ji);
            route[ji] = 100 + cl;
            sm_m[ti] = std::max(sm_m[ti], j.m);
            sm_d[ti] = std::max(sm_d[ti], j.d);
            return;
          }
          const int t = (w >= kClusterIdWork16 && j.m > 256) ? 2 : (w >= kClusterIdWork && j.m > 256) ? 1 : 0;
          tier[t].push_back(j);
          tier_ix[t].push_back((int)ji);
          route[ji] = t == 0 ? 1 : t == 1 ? 308 : 316;
          tm[t] = std::max(tm[t], j.m);
          td[t] = std::max(td[t], j.d);
        };
        // FP32 nodes that need a cluster go to the register-resident kernel
        // with one exchange per pivot step where they fit (family 4 in the
        // trace); the others, and any batch that cannot be scheduled, to the
        // kernels above
        std::map<int, std::vector<IdJob>> rx_tier;
        std::map<int, std::vector<int>> rx_ix;
        std::map<int, std::pair<int, int>> rx_md;
        // The exchange kernel takes every node that needs a cluster (it may
        // use more CTAs per node than the shared-memory kernels, registers
        // holding less than shared memory; measured at 64^3 it is faster
        // whether or not the launch fits in one wave of the GPU).
        std::vector<int> rx_cfg(ij.size(), 0), old_cl(ij.size(), 1);
        for (size_t ji = 0; ji < ij.size(); ++ji) {
          const IdJob& j = ij[ji];
          const int rx = std::is_same<T, float>::value ? id_rx_config(j.d, j.m) : 0;
          const int rr = HssKern<T>::id_rr_config(j.d, j.m);
          const int cl_sm = HssKern<T>::id_smem_cluster_size(j.d, j.m);
          old_cl[ji] = (rr > 0 && (cl_sm == 0 || (rr & 31) <= cl_sm)) ? (rr & 31)
                       : (long long)j.d * j.m * (long long)sizeof(T) > kTinyIdBytes ? (cl_sm > 0 ? cl_sm : 16)
                                                                                    : 1;
          if (rx > 0 && (old_cl[ji] > 1 || (rx & 31) > 1)) rx_cfg[ji] = rx;
        }
        for (size_t ji = 0; ji < ij.size(); ++ji) {
          const IdJob& j = ij[ji];
          const int rx = rx_cfg[ji];
          if (rx == 0) {
            route_old(ji);
            continue;
          }
          rx_tier[rx].push_back(j);
          rx_ix[rx].push_back((int)ji);
          route[ji] = 400 + (rx & 31);
          auto& md = rx_md[rx];
          md.first = std::max(md.first, j.m);
          md.second = std::max(md.second, j.d);
        }
        c.prof.mark(PH_IDK, X.s);
        {
          // The launches of a batch hold independent nodes: each runs on a side
          // stream of its own once the batch's job arrays (copied on the main
          // stream) are on the device, the longest first, so that a launch of a
          // few large clusters does not keep the rest of the GPU idle until it
          // ends; the main stream waits for all of them (at the end of this
          // scope, also on an early return) before it reads the ranks.
          const bool side = ensure_side_streams(H);
          SideJoin join{H, X.s};
          int n_side = 0;
          auto next_stream = [&]() -> cudaStream_t {
            if (!side) return X.s;
            const int k = n_side++ % HssState::kSide;
            cudaEventRecord(H.fork, X.s);
            cudaStreamWaitEvent(H.side[k], H.fork, 0);
            join.used[k] = true;
            return H.side[k];
          };
          // with profiling on, every ID launch is timed by its own events
          auto timed = [&](int code, int cl, int nj, int dmax, int mmax, auto&& launch) -> int {
            const cudaStream_t ss = next_stream();
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            const bool rec = c.prof.on && cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
            if (rec) cudaEventRecord(e0, ss);
            const int r = launch(ss);
            if (rec) {
              cudaEventRecord(e1, ss);
              c.id_ev.push_back({e0, e1});
              const double desc[5] = {(double)code, (double)cl, (double)nj, (double)dmax, (double)mmax};
              c.id_ev_desc.insert(c.id_ev_desc.end(), desc, desc + 5);
            }
            return r;
          };
          // shared-memory kernels (the largest nodes, the longest launches)
          // first; jobs a failed launch below adds to a tier after its launch go
          // in a second launch of that tier
          size_t smem_done[5] = {0, 0, 0, 0, 0};
          auto launch_smem = [&](int ti) -> bool {
            const size_t from = smem_done[ti];
            if (smem_tier[ti].size() <= from) return true;
            smem_done[ti] = smem_tier[ti].size();
            const std::vector<IdJob> jobs(smem_tier[ti].begin() + from, smem_tier[ti].end());
            const int cl = 1 << ti, nj = (int)jobs.size();
            int mm = 0, dd = 0;
            for (const IdJob& j : jobs) {
              mm = std::max(mm, j.m);
              dd = std::max(dd, j.d);
            }
            double* rdiag = (double*)H.rnd.alloc(sizeof(double) * nj * std::max(std::min(mm, dd), 1));
            int* order = (int*)H.rnd.alloc(sizeof(int) * nj * std::max(mm, 1));
            const IdJob* dj = H.ring.put(jobs, X.s);
            if (!dj || !rdiag || !order) return false;
            if (timed(100 + cl, cl, nj, dd, mm, [&](cudaStream_t ss) {
                  return HssKern<T>::batched_id_smem(dj, nj, mm, dd, eps, rdiag, order, cl, ss, p);
                }) < 0) {
              for (size_t q = from; q < smem_tier[ti].size(); ++q) {  // not schedulable: the L2-resident kernels
                const IdJob& j = smem_tier[ti][q];
                const int t = j.m > 256 ? 1 : 0;
                tier[t].push_back(j);
                tier_ix[t].push_back(smem_ix[ti][q]);
                route[smem_ix[ti][q]] = t == 0 ? 1 : 308;
                tm[t] = std::max(tm[t], j.m);
                td[t] = std::max(td[t], j.d);
              }
            } else {
              ++c.id_launches;
            }
            return true;
          };
          for (int ti = 4; ti >= 0; --ti)
            if (!launch_smem(ti)) return c.fail(HSSMF_ERR_OOM, "ID scratch");
          // exchange kernels, longest first (pivot steps x waves of clusters)
          std::vector<int> rx_keys;
          for (auto& kv : rx_tier) rx_keys.push_back(kv.first);
          auto rx_len = [&](int key) {
            return (double)rx_md[key].second * std::ceil((double)rx_tier[key].size() * (key & 31) / c.num_sms);
          };
          std::stable_sort(rx_keys.begin(), rx_keys.end(), [&](int a, int b) { return rx_len(a) > rx_len(b); });
          for (int key : rx_keys) {
            const std::vector<IdJob>& jobs = rx_tier[key];
            const int mm = rx_md[key].first, dd = rx_md[key].second;
            double* rdiag = (double*)H.rnd.alloc(sizeof(double) * jobs.size() * std::max(std::min(mm, dd), 1));
            int* order = (int*)H.rnd.alloc(sizeof(int) * jobs.size() * std::max(mm, 1));
            const IdJob* dj = H.ring.put(jobs, X.s);
            if (!dj || !rdiag || !order) return c.fail(HSSMF_ERR_OOM, "ID scratch");
            if (timed(400 + (key & 31), key & 31, (int)jobs.size(), dd, mm, [&](cudaStream_t ss) {
                  return batched_id_rx(dj, (int)jobs.size(), mm, dd, eps, rdiag, order, key, ss, 0, -1, p);
                }) < 0) {
              for (int q : rx_ix[key]) route_old((size_t)q);  // not schedulable: the other kernels
            } else {
              ++c.id_launches;
            }
          }
          for (auto& kv : rr_tier) {
            const int mm = rr_md[kv.first].first, dd = rr_md[kv.first].second;
            double* rdiag = (double*)H.rnd.alloc(sizeof(double) * kv.second.size() * std::max(std::min(mm, dd), 1));
            int* order = (int*)H.rnd.alloc(sizeof(int) * kv.second.size() * std::max(mm, 1));
            const IdJob* dj = H.ring.put(kv.second, X.s);
            if (!dj || !rdiag || !order) return c.fail(HSSMF_ERR_OOM, "ID scratch");
            if (timed(200 + (kv.first & 31), kv.first & 31, (int)kv.second.size(), dd, mm, [&](cudaStream_t ss) {
                  return HssKern<T>::batched_id_rr(dj, (int)kv.second.size(), mm, dd, eps, rdiag, order, kv.first, ss);
                }) < 0)
              return c.fail(HSSMF_ERR_CUDA, "register-resident ID launch failed");
            ++c.id_launches;
          }
          for (int ti = 4; ti >= 0; --ti)  // nodes of failed exchange launches
            if (!launch_smem(ti)) return c.fail(HSSMF_ERR_OOM, "ID scratch");
          for (int t = 2; t >= 1; --t) {
            if (tier[t].empty()) continue;
            const int bk = std::max(std::min(tm[t], td[t]), 1);
            double* rdiag = (double*)H.rnd.alloc(sizeof(double) * tier[t].size() * bk);
            int* order = (int*)H.rnd.alloc(sizeof(int) * tier[t].size() * std::max(tm[t], 1));
            const IdJob* dj = H.ring.put(tier[t], X.s);
            if (!dj || !rdiag || !order) return c.fail(HSSMF_ERR_OOM, "ID scratch");
            if (timed(t == 2 ? 316 : 308, t == 2 ? 16 : 8, (int)tier[t].size(), td[t], tm[t], [&](cudaStream_t ss) {
                  return HssKern<T>::batched_id_cluster(dj, (int)tier[t].size(), tm[t], td[t], eps, rdiag, order, ss,
                                                        t == 2 ? 16 : 8);
                }) < 0) {
              tier[0].insert(tier[0].end(), tier[t].begin(), tier[t].end());  // one CTA per job
              for (int q : tier_ix[t]) route[q] = 1;
              tm[0] = std::max(tm[0], tm[t]);
              td[0] = std::max(td[0], td[t]);
            }
          }
          if (!tier[0].empty()) {
            const IdJob* dj = H.ring.put(tier[0], X.s);
            if (!dj) return c.fail(HSSMF_ERR_OOM, "job ring");
            if (timed(1, 1, (int)tier[0].size(), td[0], tm[0], [&](cudaStream_t ss) {
                  return HssKern<T>::batched_id(dj, (int)tier[0].size(), tm[0], td[0], eps, ss);
                }) < 0)
              return c.fail(HSSMF_ERR_ARG, "an HSS node is too large for the ID kernel");
          }
        }
        c.prof.mark(PH_ID, X.s);
        hssmf_status st = c.cuda_check(cudaMemcpyAsync(H.h_ranks, H.d_ranks, sizeof(int) * ij.size(),
                                                       cudaMemcpyDeviceToHost, X.s), "ranks");
        if (st) return st;
        if ((st = c.cuda_check(cudaStreamSynchronize(X.s), "ID"))) return st;
        H.ring.off = 0;
        c.prof.resolve();
        for (size_t q = 0; q < c.id_ev.size(); ++q) {  // the stream is synchronized: launch times are final
          float ms = -1.f;
          if (cudaEventElapsedTime(&ms, c.id_ev[q].first, c.id_ev[q].second) != cudaSuccess) cudaGetLastError();
          c.id_launch_trace.insert(c.id_launch_trace.end(), c.id_ev_desc.begin() + 5 * q,
                                   c.id_ev_desc.begin() + 5 * q + 5);
          c.id_launch_trace.push_back(ms);
          cudaEventDestroy(c.id_ev[q].first);
          cudaEventDestroy(c.id_ev[q].second);
        }
        c.id_ev.clear();
        c.id_ev_desc.clear();
        for (int t = 0; t < 3; ++t) c.id_launches += tier[t].empty() ? 0 : 1;
        for (size_t i = 0; i < idn.size(); ++i) {
          FrontRt& F = *idn[i].F;
          NodeRt& N = F.nd[idn[i].t];
          const int kr = H.h_ranks[2 * i], kc = H.h_ranks[2 * i + 1], d = F.d;
          if (kr < 0 || kc < 0) return c.fail(HSSMF_ERR_TIMEOUT, "a bounded wait in an ID kernel ran out");
          for (int side = 0; side < 2; ++side) {  // algorithmic work of the two IDs
            const double mm = side ? N.mc : N.m, kk = side ? kc : kr;
            c.id_bytes += sizeof(T) * (mm * d + kk * (mm - kk));
            c.id_flops += 4.0 * mm * d * kk - 2.0 * kk * kk * (mm + d) + 4.0 * kk * kk * kk / 3.0;
          }
          const bool cap = d >= F.nf;
          const bool ok_r = kr <= d - p || kr == N.m || cap;
          const bool ok_c = kc <= d - p || kc == N.mc || cap;
          if (c.prof.on) {
            const int rec[kIdTraceFields] = {F.f, idn[i].t, F.rounds, d, N.m, N.mc, kr, kc, (int)(ok_r && ok_c),
                                             route[2 * i], route[2 * i + 1]};
            c.id_trace.insert(c.id_trace.end(), rec, rec + kIdTraceFields);
          }
          if (ok_r && ok_c) {
            N.done = true;
            N.kr = kr;
            N.kc = kc;
            N.slot = 1;  // newly compressed: skeleton lists still to build
            c.hss_max_rank = std::max(c.hss_max_rank, std::max(kr, kc));
          }
        }
      }
      c.prof.mark(PH_POSTID, X.s);
      // (d) after the ID: S <- S(J, :), R^r = V^* R, R^c = U^* R, skeleton sets
      std::vector<IntGatherJob> ig;
      std::vector<int> r0s(batch.size(), 0);
      for (size_t bi = 0; bi < batch.size(); ++bi) {
        const Item& it = batch[bi];
        const ClusterTree& tr = S.fronts[it.F->f].tree;
        FrontRt& F = *it.F;
        NodeRt& N = F.nd[it.t];
        if (!N.done) continue;
        const int d = F.d, lo = tr.lo[it.t];
        const int r0 = N.dk, rows = d - r0;  // rows 0..r0-1 were computed in earlier rounds
        r0s[bi] = r0;
        if (rows <= 0) continue;
        T* Srp = X.A(keep, (long long)d * N.kr);
        T* Scp = X.A(keep, (long long)d * N.kc);
        T* Rpc = X.A(keep, (long long)d * N.mc);
        T* Rpr = X.A(keep, (long long)d * N.m);
        if (r0 > 0) {  // the finished rows move to the arrays of leading dimension d
          X.copy(N.Srp, r0, 0, Srp, d, r0, N.kr);
          X.copy(N.Scp, r0, 0, Scp, d, r0, N.kc);
          X.copy(N.Rrp, r0, 0, Rpc, d, r0, N.kc);
          X.copy(N.Rcp, r0, 0, Rpr, d, r0, N.kr);
        }
        X.copy(N.Yr, rows, 0, Srp + r0, d, rows, N.kr, nullptr, N.piv_r);
        X.copy(N.Yc, rows, 0, Scp + r0, d, rows, N.kc, nullptr, N.piv_c);
        if (tr.leaf(it.t)) {
          const T* Rt = (const T*)F.R + lo + (long long)r0 * F.nf;
          X.copy(Rt, F.nf, 1, Rpc + r0, d, rows, N.mc, nullptr, N.piv_c);
          X.copy(Rt, F.nf, 1, Rpr + r0, d, rows, N.m, nullptr, N.piv_r);
        } else {
          const NodeRt &a = F.nd[tr.c1[it.t]], &b = F.nd[tr.c2[it.t]];
          X.copy((T*)a.Rrp + r0, d, 0, Rpc + r0, d, rows, N.mc, nullptr, N.piv_c, (T*)b.Rrp + r0, d, a.kc);
          X.copy((T*)a.Rcp + r0, d, 0, Rpr + r0, d, rows, N.m, nullptr, N.piv_r, (T*)b.Rcp + r0, d, a.kr);
        }
        N.Srp = Srp;
        N.Scp = Scp;
        N.Rrp = Rpc;
        N.Rcp = Rpr;
        if (N.slot == 1) {
          N.slot = 0;
          N.Ir = X.I(H.fac, N.kr);
          N.Ic = X.I(H.fac, N.kc);
          if (tr.leaf(it.t)) {
            if (N.kr) ig.push_back(IntGatherJob{iota + lo, iota + lo, N.piv_r, N.Ir, N.kr, N.m});
            if (N.kc) ig.push_back(IntGatherJob{iota + lo, iota + lo, N.piv_c, N.Ic, N.kc, N.mc});
          } else {
            const NodeRt &a = F.nd[tr.c1[it.t]], &b = F.nd[tr.c2[it.t]];
            if (N.kr) ig.push_back(IntGatherJob{a.Ir, b.Ir, N.piv_r, N.Ir, N.kr, a.kr});
            if (N.kc) ig.push_back(IntGatherJob{a.Ic, b.Ic, N.piv_c, N.Ic, N.kc, a.kc});
          }
        }
      }
      X.flush_copy();
      for (size_t bi = 0; bi < batch.size(); ++bi) {
        FrontRt& F = *batch[bi].F;
        NodeRt& N = F.nd[batch[bi].t];
        if (!N.done) continue;
        const int d = F.d, r0 = r0s[bi], rows = d - r0;
        if (rows <= 0) continue;
        X.gemm((T*)N.Rrp + (long long)N.kc * d + r0, d, 0, N.Xc, std::max(N.kc, 1), 1, (T*)N.Rrp + r0, d, rows,
               N.kc, N.mc - N.kc, 1.0, 1.0);
        X.gemm((T*)N.Rcp + (long long)N.kr * d + r0, d, 0, N.Xr, std::max(N.kr, 1), 1, (T*)N.Rcp + r0, d, rows,
               N.kr, N.m - N.kr, 1.0, 1.0);
        N.dk = d;
      }
      X.flush_gemm();
      X.launch(ig, [&](const IntGatherJob* d, int n) { HssKern<T>::int_gather(d, n, X.s); });
    }
    c.prof.mark(PH_EXTRACT, X.s);
    // end of the round: fronts with every non-root node compressed are done
    std::vector<ExtractJob> ej;
    std::vector<FrontRt*> next;
    for (FrontRt* F : todo) {
      const ClusterTree& tr = S.fronts[F->f].tree;
      bool all = true;
      for (int t = 0; t < tr.size(); ++t)
        if (t != tr.root()) all = all && F->nd[t].done;
      if (all) {
        const int r = tr.root();
        NodeRt& N = F->nd[r];
        if (tr.leaf(r)) {
          N.m = N.mc = N.n;
          N.D = X.A(H.fac, (long long)N.n * N.n);
          ej.push_back(ExtractJob{iota, iota, N.D, N.n, F->f, N.n, N.n, 0});
        } else {
          const NodeRt &a = F->nd[tr.c1[r]], &b = F->nd[tr.c2[r]];
          N.m = a.kr + b.kr;
          N.mc = a.kc + b.kc;
          N.B12 = X.A(H.fac, (long long)a.kr * b.kc);
          N.B21 = X.A(H.fac, (long long)b.kr * a.kc);
          if (a.kr > 0 && b.kc > 0) ej.push_back(ExtractJob{a.Ir, b.Ic, N.B12, a.kr, F->f, a.kr, b.kc, 0});
          if (b.kr > 0 && a.kc > 0) ej.push_back(ExtractJob{b.Ir, a.Ic, N.B21, b.kr, F->f, b.kr, a.kc, 0});
        }
        F->compressed = true;
        c.hss_max_d = std::max(c.hss_max_d, F->d);
        c.hss_rounds += F->rounds;
      } else {
        F->dprev = F->d;
        F->d = std::min(F->d + c.opts.dd, F->nf);
        F->rounds++;
        ensure_cols(X, *F, S.fronts[F->f]);
        next.push_back(F);
      }
    }
    X.launch(ej, [&](const ExtractJob* d, int n) { HssKern<T>::extract(c.ds, c.d_values, X.arena(), d, n, X.s); });
    hssmf_status st = c.cuda_check(cudaStreamSynchronize(X.s), "compression round");
    if (st) return st;
    H.ring.off = 0;
    H.rnd.reset();  // the round's scratch is dead
    todo.swap(next);
    if (!todo.empty()) sample_fronts(X, todo);
  }
  return X.oom ? c.fail(HSSMF_ERR_OOM, "device memory exhausted during HSS compression") : HSSMF_OK;
}

// ULV solve of F11 (postorder up the F11 tree, root LU, back down), for
// every listed front: x = F11^-1 b, nrhs[i] columns, in and out with their
// own leading dimensions (may alias).  Scratch from ``pool``.
template <typename T>
void ulv_solve(Ctx<T>& X, const std::vector<FrontRt*>& fs, const std::vector<const T*>& bin,
               const std::vector<long long>& ldin, const std::vector<T*>& xout,
               const std::vector<long long>& ldout, const std::vector<int>& nrhs, Pool& pool) {
  const Symbolic& S = X.c.sym;
  int maxh = 0, maxnr = 1, maxm = 1;
  for (size_t i = 0; i < fs.size(); ++i) {
    FrontRt& F = *fs[i];
    maxh = std::max(maxh, F.height[F.k]);
    maxnr = std::max(maxnr, nrhs[i]);
    for (int t : F.f11) {
      NodeRt& N = F.nd[t];
      maxm = std::max(maxm, N.m);
      N.bt = X.A(pool, (long long)N.m * nrhs[i]);
      N.bo = X.A(pool, (long long)N.m * nrhs[i]);
      N.w = X.A(pool, (long long)std::max(N.kc, 1) * nrhs[i]);
      N.x = X.A(pool, (long long)N.m * nrhs[i]);
    }
  }
  if (X.oom) return;
  for (int lv = 0; lv <= maxh; ++lv) {
    std::vector<UlvFwdJob> jobs;
    for (size_t i = 0; i < fs.size(); ++i) {
      FrontRt& F = *fs[i];
      const ClusterTree& tr = S.fronts[F.f].tree;
      for (int t : F.f11) {
        if (F.height[t] != lv) continue;
        NodeRt& N = F.nd[t];
        UlvFwdJob j;
        std::memset(&j, 0, sizeof(j));
        j.Dt = N.Dt;
        j.is_root = t == F.k;
        j.piv = j.is_root ? N.luperm : N.piv_r;
        j.X = N.Xr;
        j.Vt = N.Vt;
        j.leaf = tr.leaf(t);
        j.m = N.m;
        j.k = N.kr;
        j.kc = N.kc;
        j.mc = N.mc;
        j.nrhs = nrhs[i];
        if (j.leaf) {
          j.bsrc = bin[i] + tr.lo[t];
          j.ldbsrc = ldin[i];
        } else {
          const NodeRt &a = F.nd[tr.c1[t]], &b = F.nd[tr.c2[t]];
          j.Vloc = N.Vexp;
          j.B12 = N.B12;
          j.B21 = N.B21;
          j.bh1 = (const T*)a.bo + (a.m - a.kr);
          j.bh2 = (const T*)b.bo + (b.m - b.kr);
          j.ldbh1 = a.m;
          j.ldbh2 = b.m;
          j.wc1 = a.w;
          j.wc2 = b.w;
          j.k1 = a.kr;
          j.k2 = b.kr;
          j.kc1 = a.kc;
          j.kc2 = b.kc;
        }
        j.bt = N.bt;
        j.bo = N.bo;
        j.w = N.w;
        jobs.push_back(j);
      }
    }
    X.launch(jobs, [&](const UlvFwdJob* d, int n) {
      if (HssKern<T>::ulv_fwd(d, n, maxnr, maxm, X.s) < 0) X.oom = true;
    });
  }
  for (int lv = maxh; lv >= 0; --lv) {
    std::vector<UlvBwdJob> jobs;
    for (size_t i = 0; i < fs.size(); ++i) {
      FrontRt& F = *fs[i];
      const ClusterTree& tr = S.fronts[F.f].tree;
      for (int t : F.f11) {
        if (F.height[t] != lv) continue;
        NodeRt& N = F.nd[t];
        if (t == F.k) {
          if (tr.leaf(t)) X.copy(N.bo, N.m, 0, xout[i] + tr.lo[t], ldout[i], N.m, nrhs[i]);
          continue;
        }
        const int P = tr.parent[t];
        const NodeRt& PN = F.nd[P];
        const T* xpar = (const T*)(P == F.k ? PN.bo : PN.x);
        const int off = (t == tr.c1[P]) ? 0 : F.nd[tr.c1[P]].kr;
        UlvBwdJob j;
        std::memset(&j, 0, sizeof(j));
        j.Dt = N.Dt;
        j.Tq = N.Tq;
        j.x1 = N.bo;
        j.xh2 = xpar + off;
        j.ldxh2 = PN.m;
        if (tr.leaf(t)) {
          j.out = xout[i] + tr.lo[t];
          j.ldout = ldout[i];
        } else {
          j.out = N.x;
          j.ldout = N.m;
        }
        j.m = N.m;
        j.k = N.kr;
        j.nrhs = nrhs[i];
        jobs.push_back(j);
      }
    }
    X.flush_copy();
    X.launch(jobs, [&](const UlvBwdJob* d, int n) {
      if (HssKern<T>::ulv_bwd(d, n, maxnr, maxm, X.s) < 0) X.oom = true;
    });
  }
}

// ULV-like factorization of F11 (Section 2.3), then Theta^* Phi and the dense
// update matrix F22 - Theta^* Phi of every front of the level (Section 4.4).
// ULV-like factorization of the F11 trees of the listed fronts (Section 2.3),
// bottom-up; reads the node generators (D, B, the row IDs, the explicit
// column bases) and writes Dt, Vt, tau, Tq and the root LU.
template <typename T>
hssmf_status ulv_factor_f11(Ctx<T>& X, const std::vector<FrontRt*>& fs) {
  hssmf_ctx& c = X.c;
  HssState& H = X.H;
  const Symbolic& S = c.sym;
  // ULV, bottom-up over the F11 trees
  int maxh = 0;
  for (FrontRt* F : fs) maxh = std::max(maxh, F->height[F->k]);
  for (int lv = 0; lv <= maxh; ++lv) {
    std::vector<std::pair<FrontRt*, int>> items;
    for (FrontRt* F : fs)
      for (int t : F->f11)
        if (F->height[t] == lv) items.push_back({F, t});
    if (items.empty()) continue;
    // merged diagonal block [[Dh1, B12 Vh2^T], [B21 Vh1^T, Dh2]] (leaf: D)
    std::vector<T*> Dm(items.size());
    for (size_t i = 0; i < items.size(); ++i) {
      FrontRt& F = *items[i].first;
      const int t = items[i].second;
      const ClusterTree& tr = S.fronts[F.f].tree;
      NodeRt& N = F.nd[t];
      const int m = N.m;
      const bool root = t == F.k;
      Dm[i] = X.A(root ? H.fac : H.lvl, (long long)m * m);
      if (tr.leaf(t)) {
        X.copy(N.D, m, 0, Dm[i], m, m, m);
      } else {
        const NodeRt &a = F.nd[tr.c1[t]], &b = F.nd[tr.c2[t]];
        const long long oa = (a.m - a.kr) + (long long)(a.m - a.kr) * a.m;
        const long long ob = (b.m - b.kr) + (long long)(b.m - b.kr) * b.m;
        X.copy((const T*)a.Dt + oa, a.m, 0, Dm[i], m, a.kr, a.kr);
        X.copy((const T*)b.Dt + ob, b.m, 0, Dm[i] + a.kr + (long long)a.kr * m, m, b.kr, b.kr);
      }
    }
    X.flush_copy();
    for (size_t i = 0; i < items.size(); ++i) {
      FrontRt& F = *items[i].first;
      const int t = items[i].second;
      const ClusterTree& tr = S.fronts[F.f].tree;
      if (tr.leaf(t)) continue;
      NodeRt& N = F.nd[t];
      const NodeRt &a = F.nd[tr.c1[t]], &b = F.nd[tr.c2[t]];
      const int m = N.m;
      const T* Vh1 = (const T*)a.Vt + (a.m - a.kr);
      const T* Vh2 = (const T*)b.Vt + (b.m - b.kr);
      X.gemm(N.B12, std::max(a.kr, 1), 0, Vh2, b.m, 1, Dm[i] + (long long)a.kr * m, m, a.kr, b.kr, b.kc, 1.0, 0.0);
      X.gemm(N.B21, std::max(b.kr, 1), 0, Vh1, a.m, 1, Dm[i] + a.kr, m, b.kr, a.kr, a.kc, 1.0, 0.0);
    }
    X.flush_gemm();
    // Omega: rows piv[k:] minus E rows piv[:k] on top, rows piv[:k] below; root: LU
    std::vector<LuJob> lu;
    for (size_t i = 0; i < items.size(); ++i) {
      FrontRt& F = *items[i].first;
      const int t = items[i].second;
      NodeRt& N = F.nd[t];
      const int m = N.m, k = N.kr;
      if (t == F.k) {
        N.Dt = Dm[i];
        N.lupiv = X.I(H.fac, m);
        N.luperm = X.I(H.fac, m);
        if (m > 0) lu.push_back(LuJob{N.Dt, N.lupiv, N.luperm, m, 0});
        continue;
      }
      N.Dt = X.A(H.fac, (long long)m * m);
      X.copy(Dm[i], m, 0, N.Dt, m, m - k, m, N.piv_r + k);
      X.copy(Dm[i], m, 0, (T*)N.Dt + (m - k), m, k, m, N.piv_r);
    }
    X.flush_copy();
    for (size_t i = 0; i < items.size(); ++i) {
      FrontRt& F = *items[i].first;
      const int t = items[i].second;
      if (t == F.k) continue;
      NodeRt& N = F.nd[t];
      const int m = N.m, k = N.kr;
      X.gemm(N.Xr, std::max(k, 1), 1, (const T*)N.Dt + (m - k), m, 0, N.Dt, m, m - k, m, k, -1.0, 1.0);
    }
    X.flush_gemm();
    // V merged: leaf V_t; non-leaf diag(Vh1, Vh2) V_t
    for (size_t i = 0; i < items.size(); ++i) {
      FrontRt& F = *items[i].first;
      const int t = items[i].second;
      const ClusterTree& tr = S.fronts[F.f].tree;
      if (t == F.k) continue;
      NodeRt& N = F.nd[t];
      N.Vt = X.A(H.fac, (long long)N.m * std::max(N.kc, 1));
      if (tr.leaf(t)) {
        X.copy(N.Vexp, N.mc, 0, N.Vt, N.m, N.m, N.kc);
      } else {
        const NodeRt &a = F.nd[tr.c1[t]], &b = F.nd[tr.c2[t]];
        const T* Vh1 = (const T*)a.Vt + (a.m - a.kr);
        const T* Vh2 = (const T*)b.Vt + (b.m - b.kr);
        X.gemm(Vh1, a.m, 0, N.Vexp, std::max(N.mc, 1), 0, N.Vt, N.m, a.kr, N.kc, a.kc, 1.0, 0.0);
        X.gemm(Vh2, b.m, 0, (const T*)N.Vexp + a.kc, std::max(N.mc, 1), 0, (T*)N.Vt + a.kr, N.m, b.kr,
               N.kc, b.kc, 1.0, 0.0);
      }
    }
    X.flush_copy();
    X.flush_gemm();
    // LQ of the top m - k rows, blocked: panel reflectors on one CTA per
    // node, block-reflector updates of the rows below and of V_t as GEMMs
    constexpr int NBQ = 32;
    std::vector<LqJob> lq;
    std::vector<T*> W1, W2, Z1, Z2;
    int max_nk = 0;
    for (size_t i = 0; i < items.size(); ++i) {
      FrontRt& F = *items[i].first;
      const int t = items[i].second;
      if (t == F.k) continue;
      NodeRt& N = F.nd[t];
      N.tau = X.A(H.fac, std::max(N.m - N.kr, 1));
      if (N.m - N.kr <= 0) continue;
      T* Vb = X.A(H.lvl, (long long)NBQ * N.m);
      N.Tq = X.A(H.fac, (long long)NBQ * NBQ * ceil_div(N.m - N.kr, NBQ));
      lq.push_back(LqJob{N.Dt, N.Vt, N.tau, Vb, N.Tq, N.m, N.kr, N.kc, 0});
      W1.push_back(X.A(H.lvl, (long long)N.m * NBQ));
      W2.push_back(X.A(H.lvl, (long long)N.m * NBQ));
      Z1.push_back(X.A(H.lvl, (long long)NBQ * std::max(N.kc, 1)));
      Z2.push_back(X.A(H.lvl, (long long)NBQ * std::max(N.kc, 1)));
      max_nk = std::max(max_nk, N.m - N.kr);
    }
    if (X.oom) return c.fail(HSSMF_ERR_OOM, "device memory exhausted during the ULV factorization");
    for (int j0 = 0; j0 < max_nk; j0 += NBQ) {
      std::vector<LqJob> cur = lq;  // staged again each step: the job ring may wrap
      int max_n = 0;
      for (const LqJob& J : lq)
        if (j0 < J.m - J.k) max_n = std::max(max_n, J.m - j0);
      X.launch(cur, [&](const LqJob* d, int n) { HssKern<T>::lq_panel(d, n, j0, NBQ, max_n, X.s); });
      for (size_t q = 0; q < lq.size(); ++q) {
        const LqJob& J = lq[q];
        const int nk = J.m - J.k;
        if (j0 >= nk) continue;
        const int j1 = std::min(j0 + NBQ, nk), w = j1 - j0, n = J.m - j0, rows = J.m - j1;
        T* D = (T*)J.Dt;
        X.gemm(D + j1 + (long long)j0 * J.m, J.m, 0, J.Vb, NBQ, 1, W1[q], J.m, rows, w, n, 1.0, 0.0);
        X.gemm(J.Vb, NBQ, 0, (T*)J.V + j0, J.m, 0, Z1[q], NBQ, w, J.kc, n, 1.0, 0.0);
      }
      X.flush_gemm();
      for (size_t q = 0; q < lq.size(); ++q) {
        const LqJob& J = lq[q];
        const int nk = J.m - J.k;
        if (j0 >= nk) continue;
        const int j1 = std::min(j0 + NBQ, nk), w = j1 - j0, rows = J.m - j1;
        const T* Tb = (const T*)J.Tb + (long long)(j0 / NBQ) * NBQ * NBQ;
        X.gemm(W1[q], J.m, 0, Tb, NBQ, 0, W2[q], J.m, rows, w, w, 1.0, 0.0);
        X.gemm(Tb, NBQ, 1, Z1[q], NBQ, 0, Z2[q], NBQ, w, J.kc, w, 1.0, 0.0);
      }
      X.flush_gemm();
      for (size_t q = 0; q < lq.size(); ++q) {
        const LqJob& J = lq[q];
        const int nk = J.m - J.k;
        if (j0 >= nk) continue;
        const int j1 = std::min(j0 + NBQ, nk), w = j1 - j0, n = J.m - j0, rows = J.m - j1;
        T* D = (T*)J.Dt;
        X.gemm(W2[q], J.m, 0, J.Vb, NBQ, 0, D + j1 + (long long)j0 * J.m, J.m, rows, n, w, -1.0, 1.0);
        X.gemm(J.Vb, NBQ, 1, Z2[q], NBQ, 0, (T*)J.V + j0, J.m, n, J.kc, w, -1.0, 1.0);
      }
      X.flush_gemm();
    }
    // root LU of the F11 tree, blocked: panel + row block of U on one CTA
    // per root, trailing update as GEMMs
    int max_m = 0;
    for (const LuJob& J : lu) max_m = std::max(max_m, J.m);
    for (int k0 = 0; k0 < max_m; k0 += NBQ) {
      std::vector<LuJob> cur = lu;
      int max_n = 0;
      for (const LuJob& J : lu)
        if (k0 < J.m) max_n = std::max(max_n, J.m - k0);
      X.launch(cur, [&](const LuJob* d, int n) { HssKern<T>::lu_panel(d, n, k0, NBQ, c.d_status, max_n, X.s); });
      cur = lu;
      X.launch(cur, [&](const LuJob* d, int n) { HssKern<T>::lu_trsm(d, n, k0, NBQ, max_m, X.s); });
      for (const LuJob& J : lu) {
        const int k1 = k0 + NBQ;
        if (J.m <= k1) continue;
        T* A = (T*)J.A;
        X.gemm(A + k1 + (long long)k0 * J.m, J.m, 0, A + k0 + (long long)k1 * J.m, J.m, 0,
               A + k1 + (long long)k1 * J.m, J.m, J.m - k1, J.m - k1, NBQ, -1.0, 1.0);
      }
      X.flush_gemm();
    }
    X.launch(lu, [&](const LuJob* d, int n) { HssKern<T>::lu_perm(d, n, X.s); });
  }
  return X.oom ? c.fail(HSSMF_ERR_OOM, "device memory exhausted during the ULV factorization") : HSSMF_OK;
}

// Z = F11^-1 U^big_k of every front with an update block (Section 4.4).
template <typename T>
void ulv_z(Ctx<T>& X, const std::vector<FrontRt*>& fs) {
  HssState& H = X.H;
  // Z = F11^-1 U^big_k for fronts with an update block
  std::vector<FrontRt*> sf;
  std::vector<const T*> bin;
  std::vector<long long> ldin, ldout;
  std::vector<T*> xout;
  std::vector<int> nr;
  for (FrontRt* F : fs) {
    if (F->nu == 0 || F->nd[F->k].kr == 0) continue;
    F->Z = X.A(H.fac, (long long)F->ns * F->nd[F->k].kr);
    sf.push_back(F);
    bin.push_back((const T*)F->nd[F->k].Ubig);
    ldin.push_back(F->ns);
    xout.push_back((T*)F->Z);
    ldout.push_back(F->ns);
    nr.push_back(F->nd[F->k].kr);
  }
  if (!sf.empty()) ulv_solve(X, sf, bin, ldin, xout, ldout, nr, H.lvl);
}

template <typename T>
hssmf_status factor_ulv_schur(Ctx<T>& X, const std::vector<FrontRt*>& fs) {
  hssmf_ctx& c = X.c;
  HssState& H = X.H;
  const Symbolic& S = c.sym;
  c.prof.mark(PH_ULV, X.s);
  // explicit interpolative bases U = Pi_r [I; E_r], V = Pi_c [I; E_c]
  std::vector<BasisJob> bj;
  for (FrontRt* F : fs) {
    const ClusterTree& tr = S.fronts[F->f].tree;
    for (int t = 0; t < tr.size(); ++t) {
      if (t == tr.root()) continue;
      NodeRt& N = F->nd[t];
      N.Uexp = X.A(H.fac, (long long)N.m * N.kr);
      N.Vexp = X.A(H.fac, (long long)N.mc * N.kc);
      if (N.kr) bj.push_back(BasisJob{N.piv_r, N.Xr, N.Uexp, std::max(N.m, 1), N.m, N.kr});
      if (N.kc) bj.push_back(BasisJob{N.piv_c, N.Xc, N.Vexp, std::max(N.mc, 1), N.mc, N.kc});
    }
  }
  X.launch(bj, [&](const BasisJob* d, int n) { HssKern<T>::basis(d, n, X.s); });
  hssmf_status st = ulv_factor_f11(X, fs);
  if (st) return st;
  c.prof.mark(PH_SCHUR, X.s);
  // nested bases U^big, V^big of every non-root node, bottom-up
  int th = 0;
  for (FrontRt* F : fs) th = std::max(th, F->tree_h);
  for (int lv = 0; lv < th; ++lv) {
    for (FrontRt* F : fs) {
      const ClusterTree& tr = S.fronts[F->f].tree;
      for (int t = 0; t < tr.size(); ++t) {
        if (t == tr.root() || F->height[t] != lv) continue;
        NodeRt& N = F->nd[t];
        if (tr.leaf(t)) {
          N.Ubig = N.Uexp;
          N.Vbig = N.Vexp;
          continue;
        }
        const NodeRt &a = F->nd[tr.c1[t]], &b = F->nd[tr.c2[t]];
        N.Ubig = X.A(H.fac, (long long)N.n * std::max(N.kr, 1));
        N.Vbig = X.A(H.fac, (long long)N.n * std::max(N.kc, 1));
        X.gemm(a.Ubig, a.n, 0, N.Uexp, std::max(N.m, 1), 0, N.Ubig, N.n, a.n, N.kr, a.kr, 1.0, 0.0);
        X.gemm(b.Ubig, b.n, 0, (const T*)N.Uexp + a.kr, std::max(N.m, 1), 0, (T*)N.Ubig + a.n, N.n, b.n,
               N.kr, b.kr, 1.0, 0.0);
        X.gemm(a.Vbig, a.n, 0, N.Vexp, std::max(N.mc, 1), 0, N.Vbig, N.n, a.n, N.kc, a.kc, 1.0, 0.0);
        X.gemm(b.Vbig, b.n, 0, (const T*)N.Vexp + a.kc, std::max(N.mc, 1), 0, (T*)N.Vbig + a.n, N.n, b.n,
               N.kc, b.kc, 1.0, 0.0);
      }
    }
    X.flush_gemm();
  }
  ulv_z(X, fs);
  // W = V^big_k^* Z, Theta^* = U^big_q B_qk W, Phi^* = V^big_q B_kq^*
  std::vector<T*> Wk(fs.size()), G2(fs.size()), Th(fs.size()), Ph(fs.size());
  for (size_t i = 0; i < fs.size(); ++i) {
    FrontRt& F = *fs[i];
    if (F.nu == 0) continue;
    const NodeRt &K = F.nd[F.k], &Q = F.nd[F.q], &Rt = F.nd[F.root];
    const int r = K.kr;
    Wk[i] = X.A(H.lvl, (long long)std::max(K.kc, 1) * std::max(r, 1));
    G2[i] = X.A(H.lvl, (long long)std::max(Q.kr, 1) * std::max(r, 1));
    Th[i] = X.A(H.lvl, (long long)F.nu * std::max(r, 1));
    Ph[i] = X.A(H.lvl, (long long)F.nu * std::max(r, 1));
    if (r > 0) X.gemm(K.Vbig, F.ns, 1, F.Z, F.ns, 0, Wk[i], std::max(K.kc, 1), K.kc, r, F.ns, 1.0, 0.0);
  }
  X.flush_gemm();
  for (size_t i = 0; i < fs.size(); ++i) {
    FrontRt& F = *fs[i];
    if (F.nu == 0) continue;
    const NodeRt &K = F.nd[F.k], &Q = F.nd[F.q], &Rt = F.nd[F.root];
    const int r = K.kr;
    X.gemm(Rt.B21, std::max(Q.kr, 1), 0, Wk[i], std::max(K.kc, 1), 0, G2[i], std::max(Q.kr, 1), Q.kr, r,
           K.kc, 1.0, 0.0);
    X.gemm(Q.Vbig, F.nu, 0, Rt.B12, std::max(K.kr, 1), 1, Ph[i], F.nu, F.nu, r, Q.kc, 1.0, 0.0);
  }
  X.flush_gemm();
  for (size_t i = 0; i < fs.size(); ++i) {
    FrontRt& F = *fs[i];
    if (F.nu == 0) continue;
    const NodeRt &K = F.nd[F.k], &Q = F.nd[F.q];
    X.gemm(Q.Ubig, F.nu, 0, G2[i], std::max(Q.kr, 1), 0, Th[i], F.nu, F.nu, K.kr, Q.kr, 1.0, 0.0);
  }
  X.flush_gemm();
  // dense F22 (HSS expansion) into the update matrix, then -= Theta^* Phi
  struct Blk {
    FrontRt* F;
    int t;
    T* t1;
    T* t2;
  };
  std::vector<Blk> blks;
  for (FrontRt* F : fs) {
    if (F->nu == 0) continue;
    const ClusterTree& tr = S.fronts[F->f].tree;
    T* Ui = X.arena() + c.fronts_host[F->f].u_off;
    for (int t = 0; t < tr.size(); ++t) {
      if (t == tr.root() || tr.lo[t] < F->ns) continue;  // F22 subtree only
      NodeRt& N = F->nd[t];
      const long long o = (tr.lo[t] - F->ns) * (1LL + F->nu);
      if (tr.leaf(t)) {
        X.copy(N.D, N.n, 0, Ui + o, F->nu, N.n, N.n);
        continue;
      }
      const NodeRt &a = F->nd[tr.c1[t]], &b = F->nd[tr.c2[t]];
      Blk bk{F, t, X.A(H.lvl, (long long)std::max(a.kr, 1) * b.n), X.A(H.lvl, (long long)std::max(b.kr, 1) * a.n)};
      X.gemm(N.B12, std::max(a.kr, 1), 0, b.Vbig, b.n, 1, bk.t1, std::max(a.kr, 1), a.kr, b.n, b.kc, 1.0, 0.0);
      X.gemm(N.B21, std::max(b.kr, 1), 0, a.Vbig, a.n, 1, bk.t2, std::max(b.kr, 1), b.kr, a.n, a.kc, 1.0, 0.0);
      blks.push_back(bk);
    }
  }
  X.flush_copy();
  X.flush_gemm();
  for (auto& bk : blks) {
    FrontRt& F = *bk.F;
    const ClusterTree& tr = S.fronts[F.f].tree;
    T* Ui = X.arena() + c.fronts_host[F.f].u_off;
    const int c1 = tr.c1[bk.t], c2 = tr.c2[bk.t];
    const NodeRt &a = F.nd[c1], &b = F.nd[c2];
    const long long r1 = tr.lo[c1] - F.ns, r2 = tr.lo[c2] - F.ns;
    X.gemm(a.Ubig, a.n, 0, bk.t1, std::max(a.kr, 1), 0, Ui + r1 + r2 * F.nu, F.nu, a.n, b.n, a.kr, 1.0, 0.0);
    X.gemm(b.Ubig, b.n, 0, bk.t2, std::max(b.kr, 1), 0, Ui + r2 + r1 * F.nu, F.nu, b.n, a.n, b.kr, 1.0, 0.0);
  }
  X.flush_gemm();
  for (size_t i = 0; i < fs.size(); ++i) {
    FrontRt& F = *fs[i];
    if (F.nu == 0) continue;
    T* Ui = X.arena() + c.fronts_host[F.f].u_off;
    X.gemm(Th[i], F.nu, 0, Ph[i], F.nu, 1, Ui, F.nu, F.nu, F.nu, F.nd[F.k].kr, -1.0, 1.0);
  }
  X.flush_gemm();
  return X.oom ? c.fail(HSSMF_ERR_OOM, "device memory exhausted in the HSS Schur update") : HSSMF_OK;
}

std::vector<FrontRt*> level_fronts(HssState& H, const LevelPlan& L) {
  std::vector<FrontRt*> fs;
  for (int f : L.hss) fs.push_back(&H.fronts[H.index[f]]);
  return fs;
}

}  // namespace

void hss_begin_factor(hssmf_ctx& c) {
  c.hss_max_rank = c.hss_max_d = c.hss_rounds = 0;
  c.id_launches = 0;
  c.id_bytes = c.id_flops = 0.0;
  c.id_trace.clear();
  c.id_launch_trace.clear();
  c.hss_flops = c.hss_bytes = 0.0;
  if (!c.hss) return;
  c.hss->transposed_ready = false;
  c.hss->fac.reset();
  c.hss->sol.reset();
  c.hss->sol_nrhs = -1;
  c.hss->flops = 0.0;
}

template <typename T>
hssmf_status hss_factor_level(hssmf_ctx& c, int level) {
  if (!c.hss) return c.fail(HSSMF_ERR_ARG, "internal: no HSS state");
  Ctx<T> X(c);
  HssState& H = X.H;
  H.lvl.reset();
  std::vector<FrontRt*> fs = level_fronts(H, c.plan[level]);
  hssmf_status st = compress_level(X, fs);
  if (st) return st;
  if ((st = factor_ulv_schur(X, fs))) return st;
  if ((st = c.cuda_check(cudaStreamSynchronize(c.stream), "HSS level"))) return st;
  H.ring.off = 0;
  c.hss_flops = H.flops;
  c.hss_bytes = (double)H.fac.used;
  return HSSMF_OK;
}

// ULV factorization of the transposed F11 of every HSS front and Z^T =
// F11^-T V^big_k (solve_T, Section 3.3): the same routines run on the
// transposed view of each front after transposed copies of D, B12, B21.
template <typename T>
hssmf_status ensure_transposed(hssmf_ctx& c) {
  HssState& H = *c.hss;
  if (H.transposed_ready) return HSSMF_OK;
  const Symbolic& S = c.sym;
  for (size_t h = 0; h < c.plan.size(); ++h) {
    if (c.plan[h].hss.empty()) continue;
    Ctx<T> X(c);
    H.lvl.reset();
    std::vector<FrontRt*> fs = level_fronts(H, c.plan[h]);
    for (FrontRt* F : fs) {
      const ClusterTree& tr = S.fronts[F->f].tree;
      for (int t = 0; t < tr.size(); ++t) {
        NodeRt& N = F->nd[t];
        if (tr.leaf(t)) {
          if (!N.D) continue;
          N.DT = X.A(H.fac, (long long)N.n * N.n);
          X.copy(N.D, N.n, 1, N.DT, N.n, N.n, N.n);
        } else {
          const NodeRt &a = F->nd[tr.c1[t]], &b = F->nd[tr.c2[t]];
          N.Bt12 = X.A(H.fac, (long long)std::max(a.kc, 1) * std::max(b.kr, 1));  // B21^T
          N.Bt21 = X.A(H.fac, (long long)std::max(b.kc, 1) * std::max(a.kr, 1));  // B12^T
          X.copy(N.B21, std::max(b.kr, 1), 1, N.Bt12, std::max(a.kc, 1), a.kc, b.kr);
          X.copy(N.B12, std::max(a.kr, 1), 1, N.Bt21, std::max(b.kc, 1), b.kc, a.kr);
        }
      }
    }
    X.flush_copy();
    if (X.oom) return c.fail(HSSMF_ERR_OOM, "device memory exhausted building the transposed ULV");
    hssmf_status st;
    {
      ViewGuard view(fs, true);
      st = ulv_factor_f11(X, fs);
      if (!st) ulv_z(X, fs);
    }
    if (st) return st;
    if (X.oom) return c.fail(HSSMF_ERR_OOM, "device memory exhausted building the transposed ULV");
    if ((st = c.cuda_check(cudaStreamSynchronize(c.stream), "transposed ULV"))) return st;
    H.ring.off = 0;
  }
  H.transposed_ready = true;
  return HSSMF_OK;
}

// Forward multifrontal step of the HSS fronts of a level (Section 4.4);
// with transpose, the same on the transposed fronts (solve_T).
template <typename T>
hssmf_status hss_solve_fwd_level(hssmf_ctx& c, int level, T* W, int nrhs, int transpose) {
  if (transpose) {
    hssmf_status st = ensure_transposed<T>(c);
    if (st) return st;
  }
  Ctx<T> X(c);
  HssState& H = X.H;
  std::vector<FrontRt*> fs = level_fronts(H, c.plan[level]);
  ViewGuard view(fs, transpose != 0);
  // scratch for this level is taken from the solve pool; the pool is reset
  // at the first (bottom) HSS level of every solve
  if (level == c.hss_first_level) H.sol.reset();
  std::vector<const T*> bin;
  std::vector<T*> xout;
  std::vector<long long> ld;
  std::vector<int> nr;
  for (FrontRt* F : fs) {
    const DFront& d = c.fronts_host[F->f];
    bin.push_back(W + d.w_off);
    xout.push_back(W + d.w_off);
    ld.push_back(d.nf);
    nr.push_back(nrhs);
  }
  ulv_solve(X, fs, bin, ld, xout, ld, nr, H.sol);
  // b_u -= U^big_q B_qk (V^big_k)^* y
  std::vector<T*> t1(fs.size()), t2(fs.size());
  for (size_t i = 0; i < fs.size(); ++i) {
    FrontRt& F = *fs[i];
    if (F.nu == 0) continue;
    const DFront& d = c.fronts_host[F.f];
    const NodeRt &K = F.nd[F.k], &Q = F.nd[F.q];
    t1[i] = X.A(H.sol, (long long)std::max(K.kc, 1) * nrhs);
    t2[i] = X.A(H.sol, (long long)std::max(Q.kr, 1) * nrhs);
    X.gemm(K.Vbig, F.ns, 1, W + d.w_off, d.nf, 0, t1[i], std::max(K.kc, 1), K.kc, nrhs, F.ns, 1.0, 0.0);
  }
  X.flush_gemm();
  for (size_t i = 0; i < fs.size(); ++i) {
    FrontRt& F = *fs[i];
    if (F.nu == 0) continue;
    const NodeRt &K = F.nd[F.k], &Q = F.nd[F.q], &Rt = F.nd[F.root];
    X.gemm(Rt.B21, std::max(Q.kr, 1), 0, t1[i], std::max(K.kc, 1), 0, t2[i], std::max(Q.kr, 1), Q.kr, nrhs,
           K.kc, 1.0, 0.0);
  }
  X.flush_gemm();
  for (size_t i = 0; i < fs.size(); ++i) {
    FrontRt& F = *fs[i];
    if (F.nu == 0) continue;
    const DFront& d = c.fronts_host[F.f];
    const NodeRt& Q = F.nd[F.q];
    X.gemm(Q.Ubig, F.nu, 0, t2[i], std::max(Q.kr, 1), 0, W + d.w_off + F.ns, d.nf, F.nu, nrhs, Q.kr, -1.0, 1.0);
  }
  X.flush_gemm();
  return X.oom ? c.fail(HSSMF_ERR_OOM, "device memory exhausted in the HSS solve") : HSSMF_OK;
}

template <typename T>
hssmf_status hss_solve_bwd_level(hssmf_ctx& c, int level, T* W, T* xp, int nrhs, int transpose) {
  Ctx<T> X(c);
  HssState& H = X.H;
  std::vector<FrontRt*> fs = level_fronts(H, c.plan[level]);
  ViewGuard view(fs, transpose != 0);
  // x_s = y - Z B_kq (V^big_q)^* x_u
  std::vector<T*> t3(fs.size()), t4(fs.size());
  for (size_t i = 0; i < fs.size(); ++i) {
    FrontRt& F = *fs[i];
    if (F.nu == 0 || !F.Z) continue;
    const DFront& d = c.fronts_host[F.f];
    const NodeRt &K = F.nd[F.k], &Q = F.nd[F.q];
    t3[i] = X.A(H.sol, (long long)std::max(Q.kc, 1) * nrhs);
    t4[i] = X.A(H.sol, (long long)std::max(K.kr, 1) * nrhs);
    X.gemm(Q.Vbig, F.nu, 1, W + d.w_off + F.ns, d.nf, 0, t3[i], std::max(Q.kc, 1), Q.kc, nrhs, F.nu, 1.0, 0.0);
  }
  X.flush_gemm();
  for (size_t i = 0; i < fs.size(); ++i) {
    FrontRt& F = *fs[i];
    if (F.nu == 0 || !F.Z) continue;
    const NodeRt &K = F.nd[F.k], &Q = F.nd[F.q], &Rt = F.nd[F.root];
    X.gemm(Rt.B12, std::max(K.kr, 1), 0, t3[i], std::max(Q.kc, 1), 0, t4[i], std::max(K.kr, 1), K.kr, nrhs,
           Q.kc, 1.0, 0.0);
  }
  X.flush_gemm();
  for (size_t i = 0; i < fs.size(); ++i) {
    FrontRt& F = *fs[i];
    if (F.nu == 0 || !F.Z) continue;
    const DFront& d = c.fronts_host[F.f];
    const NodeRt& K = F.nd[F.k];
    X.gemm(F.Z, F.ns, 0, t4[i], std::max(K.kr, 1), 0, W + d.w_off, d.nf, F.ns, nrhs, K.kr, -1.0, 1.0);
  }
  X.flush_gemm();
  for (FrontRt* F : fs) {
    const DFront& d = c.fronts_host[F->f];
    X.copy(W + d.w_off, d.nf, 0, xp + d.sep_begin, c.sym.n, F->ns, nrhs);
  }
  X.flush_copy();
  return X.oom ? c.fail(HSSMF_ERR_OOM, "device memory exhausted in the HSS solve") : HSSMF_OK;
}

template hssmf_status hss_factor_level<double>(hssmf_ctx&, int);
template hssmf_status hss_factor_level<float>(hssmf_ctx&, int);
template hssmf_status hss_solve_fwd_level<double>(hssmf_ctx&, int, double*, int, int);
template hssmf_status hss_solve_fwd_level<float>(hssmf_ctx&, int, float*, int, int);
template hssmf_status hss_solve_bwd_level<double>(hssmf_ctx&, int, double*, double*, int, int);
template hssmf_status hss_solve_bwd_level<float>(hssmf_ctx&, int, float*, float*, int, int);

}  // namespace hssmf
