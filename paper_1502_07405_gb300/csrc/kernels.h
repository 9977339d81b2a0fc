// Host-callable launchers of the device kernels (one set per arithmetic T).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

#include <atomic>

namespace hssmf {

// Kernels launched by this library since load (read by the stats).
extern std::atomic<long long> g_launches;
// Set when a launch is rejected (bad configuration, no resources); launchers
// that probe a configuration clear the error state themselves, so every launch
// is checked here, right after it is issued.
extern std::atomic<int> g_launch_error;
inline void count_launch(int k = 1) {
  g_launches.fetch_add(k, std::memory_order_relaxed);
  if (cudaPeekAtLastError() != cudaSuccess) g_launch_error.store(1, std::memory_order_relaxed);
}

// Kernel attributes (the dynamic shared-memory limit, non-portable cluster
// sizes) belong to a device, not to the process: each (device, kernel,
// attribute, value) is set once on the current device, under a lock so that
// host threads do not race.  Returns false if the runtime refuses it (the
// error state is cleared: a launch that needed the attribute is then rejected
// and caught by count_launch, or the caller falls back).
bool set_func_attr(const void* func, cudaFuncAttribute attr, int value);

// Per-front table uploaded once after analyze (all offsets in elements).
struct DFront {
  long long off;       // front storage F (nf x nf, T) in the factor arena (dense fronts)
  long long u_off;     // update matrix (nu x nu, T) consumed by the parent
  long long piv_off;   // ns pivots (dense fronts)
  long long inv_off;   // nchild * nf ints: parent-local -> child I^upd index or -1
  long long arow_off;  // nf + 1 local CSR row pointers of A_i
  long long upd_off;   // nu ints: I^upd (new numbering)
  long long w_off;     // solve workspace (nf x nrhs, T), per solve
  int nf, ns, nu, u_ld;
  int sep_begin, nchild, child0, child1;
  int is_hss;
  int pad;
};

struct DevSym {  // device copies of the symbolic structure
  DFront* fronts;
  int* ints;          // inv maps, local CSR, upd lists
  int* perm;          // n
  int* rowptr;        // natural CSR (n + 1)
  int* colind;        // nnz
  int* tpos;          // nnz: position of the transposed entry
  int n, nnz;
};

template <typename T>
struct Kern {
  static void gemm(const GemmJob* jobs, const Tile* tiles, int ntiles, cudaStream_t s);
  // jobs with N <= GEMV_MAX_N; tile tm = row block (GEMV_ROWS_N rows, or
  // GEMV_ROWS_T for op(A) = A^T)
  static void gemv(const GemmJob* jobs, const Tile* tiles, int ntiles, cudaStream_t s);
  // dense fronts ---------------------------------------------------------
  static void assemble(const DevSym& ds, T* arena, const double* values, const Tile* tiles,
                       int ntiles, cudaStream_t s);
  static void panel_lu(const DevSym& ds, T* arena, int* piv, const int* flist, int nfr, int k0,
                       int nb, unsigned* status, cudaStream_t s);
  static void panel_trsm(const DevSym& ds, T* arena, const int* flist, int nfr, int k0, int nb,
                         int max_chunks, cudaStream_t s);
  // persistent assembly + partial LU of the listed fronts (nf <= max_nf, the
  // front held in shared memory): as many CTAs of `threads` (128 or 256) as
  // can be resident on the nsm SMs take fronts from the work counter (device
  // int, reset here); -1 if the front does not fit or the launch is refused
  static int front_lu(const DevSym& ds, T* arena, const double* values, int* piv, const int* flist, int nfr,
                      int max_nf, int threads, int nsm, int* counter, unsigned* status, cudaStream_t s);
  // solve --------------------------------------------------------------------
  static void permute_in(const double* b, long long ldb, T* bp, const int* perm, int n, int nrhs,
                         cudaStream_t s);
  static void permute_out(const T* xp, double* x, long long ldx, const int* perm, int n, int nrhs,
                          cudaStream_t s);
  static void solve_gather(const DevSym& ds, T* W, const T* bp, const int* flist, int nfr,
                           int max_rows, int nrhs, cudaStream_t s);
  // max_nf: largest dense front of the list (sizes the shared-memory staging)
  static void solve_fwd_dense(const DevSym& ds, const T* arena, const int* piv, T* W,
                              const int* flist, int nfr, int max_nf, int nrhs, int transpose, cudaStream_t s);
  static void solve_bwd_gather(const DevSym& ds, T* W, const T* xp, const int* flist, int nfr,
                               int max_nu, int nrhs, cudaStream_t s);
  static void solve_bwd_dense(const DevSym& ds, const T* arena, const int* piv, T* W, T* xp,
                              const int* flist, int nfr, int max_nf, int nrhs, int transpose, cudaStream_t s);
};

// FP32 GEMM over a tile list of 128 x 128 tiles on the tensor cores
// (three-term BF16 split, FP32 accumulation in tensor memory); status gets
// ST_TIMEOUT if a bounded wait ran out.
void gemm_tc(const GemmJob* jobs, const Tile* tiles, int ntiles, unsigned* status, cudaStream_t s);
// C = alpha sum_ks partial_ks + beta C for the split-K jobs (one tile per output tile)
void gemm_tc_reduce(const GemmJob* jobs, const Tile* tiles, int ntiles, cudaStream_t s);

// out[p] = -sum_c lam[row(p) + c ld] x[col(p) + c ld] (gradient on the pattern)
void pattern_grad(const DevSym& ds, const double* lam, const double* x, long long ld, int nrhs, double* out,
                  cudaStream_t s);

// FP64 outer-iteration kernels ------------------------------------------------
void spmv(const DevSym& ds, const double* values, const double* x, double* y, int nrhs,
          int transpose, cudaStream_t s);
// r = b - A x
void residual(const DevSym& ds, const double* values, const double* b, long long ldb,
              const double* x, double* r, int nrhs, int transpose, cudaStream_t s);
// out[j] = sum_i x[i + j*n] y[i + j*n]  (deterministic two-pass), partial has
// at least 64 * nrhs doubles
void dots(const double* x, const double* y, int n, int nrhs, double* partial, double* out,
          long long ostride, cudaStream_t s);
// out[g + nseg * j] = sum over rows off[g] <= i < off[g+1] of x[i + j*n]^2
// (off on device, nseg + 1 entries; deterministic)
void seg_norms2(const double* x, int n, int nrhs, const int* off, int nseg, double* out, cudaStream_t s);
// y[:, j] += alpha_sign * a[j * astride] * x[:, j] for active columns (a on device)
void axpy_dev(double* y, const double* x, const double* a, long long astride, double alpha_sign,
              int n, int nrhs, const int* active, cudaStream_t s);
// y[:, j] = x[:, j] / a[j * astride] (a on device; 0 if a == 0)
void scale_dev(double* y, const double* x, const double* a, long long astride, int n, int nrhs,
               cudaStream_t s);
// a[j * astride] = sqrt(a[j * astride])
void sqrt_dev(double* a, long long astride, int nrhs, cudaStream_t s);
void copy_cols(double* y, long long ldy, const double* x, long long ldx, int n, int nrhs,
               cudaStream_t s);
// y[:, j] += x[:, j] for active columns
void add_cols(double* y, const double* x, int n, int nrhs, const int* active, cudaStream_t s);
// GMRES: apply previous rotations to column j of H, new rotation, update g;
// per rhs column (H is (m+1) x m x nrhs).
void givens_step(double* H, double* cs, double* sn, double* g, int m, int j, int nrhs,
                 const int* active, cudaStream_t s);
// y = H(0:j,0:j)^-1 g(0:j) (upper triangular back substitution), per rhs
void hess_solve(const double* H, const double* g, double* y, int m, int j, int nrhs,
                const int* active, cudaStream_t s);
// X[:, c] += sum_i Z_i[:, c] y[i, c]
void update_x(double* X, const double* Z, long long zstride, const double* y, int m, int j, int n,
              int nrhs, const int* active, cudaStream_t s);

}  // namespace hssmf
