/*
 * hssmf.h -- C ABI of a GB300 (sm_103a) HSS-structured multifrontal sparse
 * solver with randomized sampling (Ghysels, Li, Rouet, Williams, Napov,
 * "An efficient multi-core implementation of a novel HSS-structured
 * multifrontal solver using randomized sampling", arXiv 1502.07405).
 *
 * The problem is the paper's: solve a sparse system A x = b by
 * reordering (nested dissection, Section 3.1), numerical factorization with
 * dense or HSS frontal matrices (Sections 3.2 and 4), and a solve used
 * directly, through iterative refinement or as a GMRES(30) preconditioner
 * (Sections 3.3, 4.6 and 6.1).
 *
 * Conventions for every entry point:
 *   - Pointers named *_host are host memory.  Matrix values, right-hand
 *     sides and solutions may be host or device memory (detected with
 *     cudaPointerGetAttributes); device memory is read or written on the
 *     context's stream, host memory is copied through it.
 *   - Dense blocks are column-major with the leading dimension given.
 *   - Every call returns an hssmf_status and never aborts or traps.  On an
 *     error, hssmf_last_error() describes it.  Device-side failures (a zero
 *     pivot, a non-finite value, a wait that ran out) are recorded in a
 *     device status word and reported by the call that launched the work.
 *   - A context is used by one host thread at a time.
 */
#ifndef HSSMF_H
#define HSSMF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hssmf_ctx hssmf_ctx;

typedef enum {
  HSSMF_OK = 0,
  HSSMF_ERR_ARG = 1,       /* bad argument or call order */
  HSSMF_ERR_CUDA = 2,      /* a CUDA runtime call failed */
  HSSMF_ERR_SINGULAR = 3,  /* zero or non-finite pivot in a frontal factorization */
  HSSMF_ERR_NOCONV = 4,    /* the outer iteration did not reach rtol within maxit */
  HSSMF_ERR_OOM = 5,       /* device memory exhausted */
  HSSMF_ERR_TIMEOUT = 6    /* a bounded device-side wait ran out */
} hssmf_status;

/* Arithmetic of the factorization.  The outer iteration, the sparse
 * residual product and the ID pivot/truncation decisions are FP64 in every
 * mode. */
typedef enum {
  HSSMF_PREC_FP64 = 0,  /* plain FP64 method */
  HSSMF_PREC_FP32 = 1   /* FP32 fronts, sampling, ID and ULV; FP64 outer loop */
} hssmf_precision;

typedef struct {
  double hss_tol;      /* relative ID tolerance eps (Section 5.3 rule) */
  int d0;              /* initial number of random sample columns */
  int dd;              /* sample columns added when an ID fails (Section 4.3) */
  int oversample_p;    /* an ID succeeds if rank <= d - p (default 10) */
  int hss_min_front;   /* fronts with n_f >= this are HSS (replaces l_s, Section 4.1) */
  int hss_leaf;        /* HSS leaf size b (default 128, Section 4.2) */
  int nd_leaf;         /* nested dissection stops at boxes of this side (default 8) */
  uint64_t seed;       /* key of the counter-based generator of R */
  int precision;       /* hssmf_precision */
  int gmres_restart;   /* default 30 (Section 6.1) */
  int maxit;           /* outer iterations; 0 = apply the factorization once */
  double rtol;         /* relative residual target ||b - A x|| / ||b|| (default 1e-10) */
} hssmf_opts;

typedef struct {
  int n;                 /* matrix order */
  int n_fronts;          /* elimination-tree nodes */
  int n_levels;          /* elimination-tree levels */
  int n_hss_fronts;      /* fronts stored in HSS form */
  int max_front;         /* largest n_f */
  int max_rank;          /* largest HSS rank found (row or column) */
  int max_d;             /* largest number of sample columns used */
  int adaptive_rounds;   /* total extra sampling rounds over all fronts */
  int iterations;        /* outer iterations of the last solve (max over rhs) */
  double relres;         /* final true relative residual (max over rhs) */
  double factor_flops;   /* algorithmic flops of the last factorization */
  double factor_bytes;   /* bytes of the stored factors */
  double t_analyze_ms;   /* host wall time of analyze */
  double t_factor_ms;    /* device time of the last factor (CUDA events) */
  double t_solve_ms;     /* device time of the last solve (CUDA events) */
  int gpu_launches;      /* kernels launched by the last factor + solve */
  int id_launches;       /* interpolative-decomposition kernel launches of the last factor */
  double id_bytes;       /* their algorithmic bytes: sum of m d + k (m - k) elements */
  double id_flops;       /* their algorithmic flops: sum of 4mdk - 2k^2(m + d) + 4k^3/3 */
} hssmf_stats;

/* Fill *opts with the defaults named above (hss_tol 1e-4, d0 128, dd 64,
 * p 10, hss_min_front 1024, hss_leaf 128, nd_leaf 8, seed 0, FP64,
 * restart 30, maxit 300, rtol 1e-10). */
void hssmf_default_opts(hssmf_opts* opts);

/* Create a context on the current CUDA device.  cuda_stream is a
 * cudaStream_t (NULL = legacy default stream).  The context owns every
 * device allocation it makes; hssmf_destroy frees them. */
hssmf_status hssmf_create(hssmf_ctx** ctx, const hssmf_opts* opts, void* cuda_stream);

/* Symbolic phase for a matrix on an nx x ny x nz grid (nz = 1 in 2D) whose
 * pattern is given in CSR form in natural numbering x + nx*(y + ny*z)
 * (host arrays, n + 1 and nnz entries, column indices ascending per row).
 * The pattern must be structurally symmetric and every edge must join grid
 * neighbours (|dx|, |dy|, |dz| <= 1).  Computes the geometric nested
 * dissection and separator reordering (Sections 3.1, 4.2, 6.1), the
 * elimination tree, I^sep / I^upd of every front (Section 5.4), the HSS
 * trees of the fronts and all index maps, and uploads them once. */
hssmf_status hssmf_analyze_grid(hssmf_ctx* ctx, int nx, int ny, int nz, int n,
                                const int* rowptr_host, const int* colind_host);

/* Symbolic phase for nsys independent grid problems solved together as one
 * block-diagonal matrix.  dims holds 3 sides per grid (host, 3 * nsys ints);
 * grid s owns the natural indices after those of grids 0..s-1, numbered
 * x + nx*(y + ny*z) inside the grid; n is the total size.  No pattern edge
 * may join two grids (HSSMF_ERR_ARG).  Each grid is ordered as by
 * hssmf_analyze_grid; the elimination forest is their trees side by side
 * and every level of the factorization and of the solve is one batch over
 * the fronts of all grids at that height.  hssmf_solve then runs iterative
 * refinement (FP64 residuals, the factorization as M^-1) on all grids at
 * once until every grid's relative residual is <= rtol for every column
 * (HSSMF_ERR_NOCONV after maxit applications); nsys * nrhs <= 131072. */
hssmf_status hssmf_analyze_grids(hssmf_ctx* ctx, int nsys, const int* dims_host, int n,
                                 const int* rowptr_host, const int* colind_host);

/* Symbolic phase for a general n x n matrix with a structurally symmetric
 * pattern (host CSR, column indices ascending per row).  perm == NULL: the
 * library orders it by algebraic nested dissection (no geometry: each
 * connected component is a separate elimination tree; in a connected set,
 * the separator is the middle level of a breadth-first level structure from
 * a pseudo-peripheral vertex, trimmed of vertices with no neighbour beyond
 * it; sets of at most max(16, nd_leaf^2) vertices are leaf fronts); nfronts,
 * sep_ptr and parent are then ignored.  Otherwise the caller gives the
 * ordering and the separator tree of Sections 3.1 and 5.4: perm[new] = old
 * (n entries), front f owns the new indices [sep_ptr[f], sep_ptr[f+1])
 * (nfronts + 1 entries, 0 to n, every front non-empty), parent[f] > f or -1
 * for a root (postorder), at most two children per front.  The tree must be
 * an elimination structure of the pattern: every front's I^upd must lie in
 * its parent's index set (HSSMF_ERR_ARG otherwise).  HSS cluster trees halve
 * each front's index range down to hss_leaf.  Factor and solve are as after
 * hssmf_analyze_grid. */
hssmf_status hssmf_analyze_csr(hssmf_ctx* ctx, int n, const int* rowptr_host, const int* colind_host,
                               int nfronts, const int* perm_host, const int* sep_ptr_host,
                               const int* parent_host);

/* Numerical factorization (Sections 3.2 and 4): values are the nnz matrix
 * entries in the CSR order given to analyze (host or device, FP64).
 * Fronts below hss_min_front are assembled by extend-add and partially
 * factored by LU with partial pivoting inside F11; larger fronts are
 * sampled by the skinny extend-add, compressed by Algorithm 1 with the
 * adaptive rank scheme and ULV-factored with a low-rank Schur update.
 * HSSMF_ERR_SINGULAR if a pivot is zero or not finite. */
hssmf_status hssmf_factor(hssmf_ctx* ctx, const double* values);

/* Solve A X = B for nrhs columns (B, X: n x nrhs, leading dimension ldb,
 * host or device, FP64, natural numbering; X may alias B).  With
 * opts.maxit == 0 the factorization is applied once (forward then backward
 * sweep, Section 3.3).  Otherwise iterative refinement (no HSS front) or
 * right-preconditioned GMRES(restart) with modified Gram-Schmidt and
 * x0 = 0 (HSS fronts present) runs every column until its true relative
 * residual is <= rtol; HSSMF_ERR_NOCONV if one does not within maxit.
 * After hssmf_analyze_grids with nsys > 1: refinement with per-grid
 * residuals (see there). */
hssmf_status hssmf_solve(hssmf_ctx* ctx, const double* B, double* X, int nrhs, int ldb);

/* Same for A^T X = B (Section 3.3 applied to A^T): dense fronts apply
 * U^T, then L^T with the row interchanges; HSS fronts use the ULV
 * factorization of the transposed HSS matrix (D^T, row and column
 * generators exchanged, B12 <-> B21^T) and Z^T = F11^-T V^big_k, built on
 * the device at the first solve_T after each factorization and kept until
 * the next one (the first call takes about as long as the ULV part of the
 * factorization); the outer iteration runs on A^T. */
hssmf_status hssmf_solve_T(hssmf_ctx* ctx, const double* B, double* X, int nrhs, int ldb);

hssmf_status hssmf_get_stats(const hssmf_ctx* ctx, hssmf_stats* out);

/* Copy out the symbolic structure (host arrays sized by the caller):
 *   perm[n]: perm[new] = natural index;
 *   sep_begin[n_fronts], sep_end[n_fronts], parent[n_fronts] (-1 at the
 *   root), n_upd[n_fronts]: fronts in postorder, separators in new numbering.
 * Any pointer may be NULL. */
hssmf_status hssmf_get_symbolic(const hssmf_ctx* ctx, int* perm, int* sep_begin, int* sep_end,
                                int* parent, int* n_upd);

/* I^upd of front f (ascending new indices) into upd[n_upd[f]]. */
hssmf_status hssmf_get_upd(const hssmf_ctx* ctx, int f, int* upd);

/* Per-phase device times of the last factor + solve (CUDA events, ms), in
 * this order: 0 dense-front assembly and partial LU, 1 sampling (R, A_i R,
 * child-update GEMMs), 2 element extraction, 3 pre-ID sample updates,
 * 4 interpolative-decomposition steps outside the ID kernels (job set-up
 * gaps, rank read-back), 5 post-ID updates, 6 ULV factorization, 7 nested
 * bases, Theta^* Phi and update matrices, 8 multifrontal solve (all
 * preconditioner applications), 9 outer-iteration kernels, 10 the ID kernel
 * launches themselves.  Writes min(n, 11) values; phase timing is recorded
 * only after hssmf_set_profiling(ctx, 1). */
hssmf_status hssmf_get_phase_times(const hssmf_ctx* ctx, double* ms, int n);
hssmf_status hssmf_set_profiling(hssmf_ctx* ctx, int on);

/* Gradient of a loss L(x) with respect to the stored entries of A, for
 * x = A^-1 b (the adjoint of hssmf_solve): with lambda = A^-T dL/dx (from
 * hssmf_solve_T), dL/dA_ij = -sum_c lambda_i,c x_j,c, written in the order
 * of the CSR pattern given to hssmf_analyze_grid (natural numbering):
 * out[p] for the entry (row(p), colind[p]).  lambda and x are n x nrhs
 * column-major device arrays with leading dimension ld; out is a device
 * array of nnz doubles.  The paper has no counterpart; the differentiation
 * interface of the library.  HSSMF_ERR_ARG before a factorization, for host
 * pointers or ld < n; synchronizes the stream. */
hssmf_status hssmf_pattern_grad(hssmf_ctx* ctx, const double* lambda, const double* x, int nrhs, int ld,
                                double* out);

/* Records of every interpolative decomposition of the last factorization
 * run with profiling on (Algorithm 1 with the adaptive scheme of Section
 * 2.2.1): 11 ints per node attempt -- front, HSS node, adaptive round of
 * the front, sample columns d, rows m of the row ID, rows of the column ID,
 * row rank, column rank, 1 if both IDs were accepted, and the kernel that
 * ran the row ID and the column ID, coded 100 * family + CTAs per ID
 * (family 0: one CTA, matrix in L2; 1: matrix in shared memory; 2: matrix
 * in registers; 3: L2-resident cluster; 4: matrix in registers, one
 * exchange of proposals per pivot step).  Copies at most
 * max_records records into rec (host, may be NULL) and returns the number
 * available, or -1 for a NULL context. */
int hssmf_get_id_trace(const hssmf_ctx* ctx, int* rec, int max_records);

/* One record per ID kernel launch of the last factorization run with
 * profiling on (the paper has no counterpart; a profiling aid): 6 doubles --
 * kernel code (as in hssmf_get_id_trace), CTAs per ID, IDs in the launch,
 * largest d, largest m, device time in ms (CUDA events around the launch).
 * Copies at most max_records records into rec (host, may be NULL) and
 * returns the number available, or -1 for a NULL context. */
int hssmf_get_id_launch_trace(const hssmf_ctx* ctx, double* rec, int max_records);

/* Autotuner of the dense fronts (the paper has no counterpart; it replaces
 * the task scheduling of Section 5 for batched levels).  The dense fronts of
 * every elimination-tree level are split by size: the larger ones take the
 * blocked panel LU (assembly tiles, 32-column panels, batched GEMMs), the
 * others one persistent launch whose CTAs take fronts from a work queue and
 * assemble and factor each in shared memory.  With autotuning on (the
 * default), the first factorization after an analysis times every distinct
 * split of each level among a fixed set of size bounds, with 128 or 256
 * threads per CTA, and keeps the fastest; later factorizations reuse it.
 * Off: levels not tuned yet keep the default split (every front that fits
 * the shared memory takes the persistent kernel, 256 threads); splits
 * already chosen are kept until the next analysis. */
hssmf_status hssmf_set_autotune(hssmf_ctx* ctx, int on);

/* The split chosen per elimination-tree level (bottom level first): 6 ints
 * per level -- dense fronts, fronts on the panel path (the largest), size
 * bound of the persistent kernel, its threads per CTA, 1 if tuned by timed
 * trials, the tuned level's time in microseconds.  Copies at most
 * max_levels records into rec (host, may be NULL) and returns the number of
 * levels, or -1 for a NULL context. */
int hssmf_get_tuning(const hssmf_ctx* ctx, int* rec, int max_levels);

/* Kernel-level entry point: a batch of interpolative decompositions
 * (Section 2.2, ID definitions; rank rule of Section 5.3).  Job j selects
 * columns of Y_j (d_j x m_j, column-major, leading dimension d_j, device
 * memory at Y + y_off[j] elements, arithmetic T = double for prec 0, float
 * for prec 1) by column-pivoted Householder QR with column norms recomputed
 * from the trailing rows at every step and the first largest norm winning;
 * the rank k_j is the first i with |R_{i+1,i+1}| <= eps |R_11| (0 if
 * R_11 = 0), else min(d_j, m_j).  Norms are sums in T: FP64 for prec 0; for
 * prec 1 the squared norms and the pivot choice are FP32, and the rank rule
 * is the FP64 comparison (its threshold eps^2 |R_11|^2 is formed in FP64 and
 * rounded down to FP32, which decides every FP32 norm exactly as FP64
 * would).  Outputs: rank_host[j];
 * piv + p_off[j] (m_j ints, device): the k_j skeleton columns first, in
 * pivot order; X + x_off[j] (device, k_j x (m_j - k_j), leading dimension
 * k_j, room for m_j * m_j / 4 + 1 elements): X = R1^-1 R2 for the
 * non-skeleton columns in the order piv[k_j:], so Y ~ Y(:, piv[:k]) [I X]
 * and the interpolative basis is Pi [I; X^T].  y_off, m, d, p_off, x_off
 * are host arrays.  use_cluster = 0 runs every job on one CTA; 1..8 on a
 * thread-block cluster of 8 CTAs, 16 on a cluster of 16 CTAs (where the
 * device can schedule it, else 8), all working on the matrix in L2;
 * use_cluster = -1 keeps every matrix in the shared memory of a cluster of
 * 1..16 CTAs sized for the largest job (past 16 CTAs the columns that do not
 * fit stay in global memory);
 * use_cluster = -100 - c (c = 2, 4, 8, 16) runs the shared-memory kernel on
 * clusters of c CTAs whatever the size; use_cluster = -3 (prec 1 only) keeps
 * every matrix in the registers of a cluster of CTAs of 256 threads with one
 * exchange of proposals per pivot step: lanes hold 32 r rows (r the smallest
 * even number with d <= 32 r, at least 4; d <= 832) and a warp c columns
 * (c = 32, 24, 16, 16, 14, 12, 10, 9, 8, 8, 7, 7 for r = 4, 6, ..., 26), on
 * the smallest cluster of 1..16 CTAs with m <= 8 c x CTAs, else
 * HSSMF_ERR_ARG; use_cluster = -4 the same on CTAs of 512 threads (m up to
 * 2048, 1024 or 768 for d <= 256, 512, 832);
 * use_cluster = -2 (prec 1 only) keeps
 * every matrix in the registers of a
 * cluster of 1..16 CTAs, for d <= 512 and m <= 2048 (d <= 256) or m <= 1024
 * (d <= 512), else HSSMF_ERR_ARG.
 * Y is not modified.  Synchronizes the stream. */
hssmf_status hssmf_batched_id(int prec, int njobs, const void* Y, const long long* y_off,
                              const int* m, const int* d, double eps, int* rank_host, int* piv,
                              const long long* p_off, void* X, const long long* x_off,
                              int use_cluster, void* cuda_stream);

/* Test of the failure path of the bounded waits (the paper has no
 * counterpart): one FP32 ID on the register-resident cluster kernel with
 * cl CTAs (2 to 16) in which CTA 0 withholds its first proposal, so
 * that every wait of the cluster runs out after spin polls.  The kernel
 * then stops, meets its cluster barriers and reports rank -1; the call
 * returns HSSMF_ERR_TIMEOUT (HSSMF_OK would mean the wait did not run out),
 * HSSMF_ERR_ARG for invalid arguments.  Allocates and frees its own small
 * device buffers; synchronizes the device. */
hssmf_status hssmf_id_timeout_test(int cl, int spin);

/* Kernel-level entry point: the FP32 GEMM of the FP32 factorization,
 * C = alpha op(A) op(B) + beta C with op(A) m x k and op(B) k x n
 * (transa/transb = 1: use the transpose), column-major device arrays with
 * leading dimensions lda, ldb, ldc.  It runs on the tensor cores
 * (tcgen05, 128 x 128 tiles, accumulator in tensor memory): every FP32
 * operand value is split into three BF16 terms and the six term products of
 * order >= 2^-16 are accumulated in FP32, which gives FP32-level accuracy.
 * b_exact = 1 declares that every value of B is exactly a BF16 number
 * (as the FP32 form's sampling matrix R is, Section 4.3), which drops the
 * products to three; values of B that are not BF16 are then rounded.  The
 * paper's products S = F R of eq. FtimesR, the sample updates of
 * Algorithm 1 and the Schur complements of Sections 3.2 and 4.4 use this
 * kernel in the FP32 form.
 *   - HSSMF_ERR_ARG for negative sizes, null arrays or leading dimensions
 *     below the stored rows; m, n or k = 0 is valid (C = beta C).
 *   - HSSMF_ERR_TIMEOUT if a bounded wait inside the kernel ran out.
 *   - The operands are split once into BF16 term arrays and the product runs
 *     as a TMA-fed tcgen05 pipeline (K split when the output has few tiles).
 *     b_exact + 2 (bit 1 set) runs instead the kernel the factorization
 *     uses, which stages the FP32 tiles in shared memory and splits them
 *     inside its loop (tests and profiling of that kernel).
 *   - Device scratch (term arrays, job and tile lists) is kept by the library
 *     between calls and reused; calls are serialized; synchronizes the
 *     stream. */
hssmf_status hssmf_gemm_f32(int transa, int transb, int m, int n, int k, float alpha,
                            const float* A, long long lda, const float* B, long long ldb,
                            float beta, float* C, long long ldc, int b_exact, void* cuda_stream);

/* Allocation-free form of hssmf_batched_id for callers that must not
 * allocate device memory while they run: cudaMalloc/cudaFree synchronize
 * the whole device, an application's memory pool may already own the
 * device memory, or a policy may forbid allocation after start-up.  The
 * paper has no counterpart; this is a property of the library.
 * Same arguments, results and one-CTA kernel as hssmf_batched_id with
 * use_cluster = 0, but every scratch word (job descriptors, ranks and the
 * d_j x m_j work copies) lives in one fixed 32 MiB array compiled into the
 * library, held on each GPU that loads it until the process exits.  No
 * device memory is allocated or freed.
 *   - HSSMF_ERR_ARG if the batch needs more than 32 MiB of scratch
 *     (256-byte-rounded job and rank arrays plus sum(d_j * m_j) elements of
 *     T), or if a node is too large for the kernel's shared memory.
 *   - The first call on a device looks up the array's device address (once
 *     per device, with that device current); make that first call before
 *     any stream capture.  The address is kept for the life of the process:
 *     do not use this entry point after cudaDeviceReset on that device.
 *   - Every call shares the array: calls that overlap on the GPU (other
 *     streams, other host threads) race and must be serialized by the
 *     caller.  Nothing in the array needs clearing between calls.
 *   - Synchronizes the stream. */
hssmf_status hssmf_batched_id_noalloc(int prec, int njobs, const void* Y, const long long* y_off,
                                      const int* m, const int* d, double eps, int* rank_host,
                                      int* piv, const long long* p_off, void* X,
                                      const long long* x_off, void* cuda_stream);

const char* hssmf_last_error(const hssmf_ctx* ctx);
void hssmf_destroy(hssmf_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* HSSMF_H */
