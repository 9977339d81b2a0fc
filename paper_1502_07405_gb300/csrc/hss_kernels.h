// Job descriptors and launchers of the HSS-front kernels.
#pragma once
#include "kernels.h"

namespace hssmf {

constexpr int COPY_TN = 4;  // 32-column tiles of one copy CTA

struct CopyJob {  // dst(i, j) = src'(rmap[i], cmap[j]); source columns >= split come from src2
  const void* src;
  const void* src2;  // second source (columns split.. of the concatenation), lds2
  long long lds2;
  int split, pad2;
  void* dst;
  const int* rmap;  // nullptr: identity
  const int* cmap;  // nullptr: identity
  long long lds, ldd;
  int rows, cols;
  int src_trans;  // src'(a, b) = src[b + a * lds] instead of src[a + b * lds]
  int scale_neg;  // 1: dst = -src'
};

struct IntGatherJob {  // out[i] = cat(a, b)[idx[i]], cat(a, b)[p] = p < split ? a[p] : b[p - split]
  const int* a;
  const int* b;
  const int* idx;
  int* out;
  int n, split;
};

struct PhiloxJob {  // out(i, c) = G(seed, gidx[i], c), c in [c0, c1)
  const int* gidx;
  void* out;
  long long ld;
  int rows, c0, c1;
  int bf16;  // FP32 form: out holds BF16 values (G is BF16-rounded there, so exactly)
};

struct SampleAJob {  // Sr(:, c) = A_i R(:, c), Sc(:, c) = A_i^T R(:, c), c in [c0, c1)
  void* Sr;
  void* Sc;
  const void* R;
  long long ld;
  int front, c0, c1, pad;
};

struct ExtractJob {  // out(i, j) = F_front(rows[i], cols[j]) from A_i and the children's updates
  const int* rows;
  const int* cols;
  void* out;
  long long ld;
  int front, nr, nc, pad;
};

struct IdJob {  // ID of the columns of Y (d x m): rank, piv, X = R1^-1 R2 (k x (m-k), ld k)
  const void* Y;
  void* W;  // d x m work copy
  int* piv;
  void* X;
  int* rank;
  int d, m;
};

struct BasisJob {  // out (m x k, ld ldo) = Pi [I; X^T]
  const int* piv;
  const void* X;
  void* out;
  long long ldo;
  int m, k;
};

struct LqJob {  // LQ of the top m-k rows of Dt (m x m): Dt <- Dt Q, V <- Q^T V; taus
  void* Dt;
  void* V;
  void* tau;
  void* Vb;  // blocked form: panel reflectors (nb x m, ld nb) and their T (nb x nb)
  void* Tb;  // T of panel b at Tb + b nb^2 (kept for the solve)
  int m, k, kc, pad;
};

struct LuJob {  // in-place partial-pivoting LU of A (m x m, ld m)
  void* A;
  int* piv;
  int* perm;  // after the factorization: row i of P A is row perm[i] of A
  int m, pad;
};

// Forward ULV step of one HSS node (one CTA per job, all nrhs columns):
//   b_t   = leaf: bsrc rows; non-leaf: [bh1 - B12 wc2; bh2 - B21 wc1]
//   bo    = Omega b_t (rows piv[k:] minus E rows piv[:k]; then rows piv[:k])
//   x1    = L^-1 bo[0:m-k], bhat = bo[m-k:] - D21 x1 (one column sweep of Dt)
//   w     = V_t^T [wc1; wc2] + Vt_top^T x1
// At the root of the F11 tree: x1 = LU^-1 b_t (m rows).
struct UlvFwdJob {
  const void* Dt;     // m x m, ld m: [L 0; D21 Dhat] (root: LU factors)
  const int* piv;     // Pi (m); root: LU row interchanges
  const void* X;      // k x (m - k), ld k: E = X^T
  const void* Vt;     // Q^T V_merged (m x kc, ld m)
  const void* Vloc;   // V_t explicit (mc x kc, ld mc), non-leaf only
  const void* B12;    // k1 x kc2, ld k1
  const void* B21;    // k2 x kc1, ld k2
  const void* bsrc;   // leaf: m x nrhs, ld ldbsrc
  const void* bh1;    // non-leaf: children's bhat (k1 x nrhs, ld k1) and (k2 x nrhs, ld k2)
  const void* bh2;
  const void* wc1;    // children's w (kc1 x nrhs, ld kc1) and (kc2 x nrhs, ld kc2)
  const void* wc2;
  void* bt;           // scratch m x nrhs, ld m
  void* bo;           // out m x nrhs, ld m: [x1; bhat] (root: the solution)
  void* w;            // out kc x nrhs, ld kc
  long long ldbsrc;
  int m, k, kc, mc, k1, k2, kc1, kc2, leaf, is_root, ldbh1, ldbh2, nrhs, pad;
};
// (root: piv holds the row permutation of the LU, row i of P b is b[piv[i]])

// Backward ULV step: x_t = Q [x1; xhat2] with Q the product of the LQ
// reflectors stored in the rows of Dt; x1 = bo[0:m-k] of the forward job.
struct UlvBwdJob {
  const void* Dt;
  const void* Tq;   // T of each 32-reflector panel (32 x 32, upper), panel b at Tq + 1024 b
  const void* x1;   // (m - k) x nrhs, ld m
  const void* xh2;  // k x nrhs, ld ldxh2 (slice of the parent's x)
  void* out;        // m x nrhs, ld ldout
  long long ldxh2, ldout;
  int m, k, nrhs, pad;
};

// Register-resident ID of FP32 nodes on clusters of 1..16 CTAs with one
// exchange round per pivot step (k_id_rx.cu).  id_rx_config: 0 if a d x m
// node does not fit, else a configuration code for batched_id_rx (family 0:
// 256-thread CTAs, 255 registers a thread; 1: 512-thread CTAs).  rdiag
// (njobs x min(max_m, max_d) doubles) and order (njobs x max_m ints) are
// scratch.  spin bounds every wait (0: the default); hang_rank >= 0 makes
// that CTA of every cluster withhold its first proposal, so that the waits
// run out (tests of the timeout path; -1 otherwise).  fail_p >= 0 stops an
// ID as soon as its rank exceeds d - fail_p with m > d (the adaptive scheme
// rejects it whatever follows): it reports that rank, d - fail_p + 1, and
// leaves X and piv unwritten; -1 runs every ID to its rank.  Returns -1 if
// the configuration cannot be launched (the caller falls back).
int id_rx_config(int d, int m, int family = 0);
int batched_id_rx(const IdJob* jobs, int njobs, int max_m, int max_d, double eps, double* rdiag, int* order,
                  int cfg, cudaStream_t s, int spin = 0, int hang_rank = -1, int fail_p = -1);

template <typename T>
struct HssKern {
  // tiles: destination strips (job, tm, tn) of 32 rows x COPY_TN 32-column
  // tiles starting at tile column tn (a multiple of COPY_TN)
  static void copy(const CopyJob* jobs, const Tile* tiles, int ntiles, cudaStream_t s);
  static void int_gather(const IntGatherJob* jobs, int njobs, cudaStream_t s);
  static void philox(const PhiloxJob* jobs, int njobs, int max_rows, unsigned long long seed,
                     cudaStream_t s);
  static void sample_a(const DevSym& ds, const double* values, const SampleAJob* jobs, int njobs,
                       int max_rows, cudaStream_t s);
  static void extract(const DevSym& ds, const double* values, const T* arena, const ExtractJob* jobs,
                      int njobs, cudaStream_t s);
  // returns -1 if max_m exceeds the shared-memory bound of the kernel
  static int batched_id(const IdJob* jobs, int njobs, int max_m, int max_d, double eps, cudaStream_t s);
  // one thread-block cluster of cl (8 or 16) CTAs per job; rdiag (njobs x min(max_m, max_d)
  // doubles) and order (njobs x max_m ints) are scratch.  Returns -1 if no launch is possible.
  static int batched_id_cluster(const IdJob* jobs, int njobs, int max_m, int max_d, double eps,
                                double* rdiag, int* order, cudaStream_t s, int cl = 8);
  // Shared-memory-resident ID on clusters of cl CTAs (1, 2, 4, 8, 16); the
  // smallest cl whose shared memory holds a d x m node, 0 if none does.
  static int id_smem_cluster_size(int d, int m);
  // register-resident ID (FP32 only): 0 if (d, m) does not fit, else a
  // configuration code for batched_id_rr (cluster size, + 32 for the
  // 16-rows-per-lane layout)
  static int id_rr_config(int d, int m);
  static int batched_id_rr(const IdJob* jobs, int njobs, int max_m, int max_d, double eps, double* rdiag,
                           int* order, int cfg, cudaStream_t s);
  // fail_p >= 0: a job with m > d stops, with no X and no pivots, as soon
  // as its rank passes d - fail_p (an ID the adaptive scheme rejects)
  static int batched_id_smem(const IdJob* jobs, int njobs, int max_m, int max_d, double eps, double* rdiag,
                             int* order, int cl, cudaStream_t s, int fail_p = -1);
  static void basis(const BasisJob* jobs, int njobs, cudaStream_t s);
  static void lu(const LuJob* jobs, int njobs, unsigned* status, cudaStream_t s);
  // Blocked LQ, panel of rows [j0, j0 + nb) of every job with m - k > j0:
  // reflectors of the panel rows (applied inside the panel), the block
  // reflector's V (nb x (m - j0), ld nb, explicit ones and zeros) into
  // Vb + vb_off[j] and its triangular factor T (nb x nb) into Tb + t_off[j].
  // (max_n: the largest m - j0 of the jobs still in range: sizes the
  // shared-memory form of the kernel)
  static void lq_panel(const LqJob* jobs, int njobs, int j0, int nb, int max_n, cudaStream_t s);
  // Blocked LU: panel columns [k0, k0 + nb) (pivot search over all rows),
  // then the row block of U right of the panel.
  static void lu_panel(const LuJob* jobs, int njobs, int k0, int nb, unsigned* status, int max_n, cudaStream_t s);
  static void lu_trsm(const LuJob* jobs, int njobs, int k0, int nb, int max_m, cudaStream_t s);
  // row permutation of each finished LU from its interchanges
  static void lu_perm(const LuJob* jobs, int njobs, cudaStream_t s);
  // max_m bounds the node sizes (shared-memory vectors); -1 if too large
  static int ulv_fwd(const UlvFwdJob* jobs, int njobs, int max_nrhs, int max_m, cudaStream_t s);
  static int ulv_bwd(const UlvBwdJob* jobs, int njobs, int max_nrhs, int max_m, cudaStream_t s);
};

}  // namespace hssmf
