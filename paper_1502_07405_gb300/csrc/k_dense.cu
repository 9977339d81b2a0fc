// Dense-front kernels: batched GEMM, front assembly by extend-add
// (Section 3.2, eq. extend-add), blocked partial LU with row partial
// pivoting restricted to F11 (Section 3.2).
#include <algorithm>
#include <cfloat>

#include "kernels.h"

namespace hssmf {

// ---------------------------------------------------------------------------
// Batched variable-size GEMM over a tile list (64 x 64 tiles, 256 threads,
// 4 x 4 outputs per thread, K staged through shared memory 16 at a time).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_gemm(const GemmJob* __restrict__ jobs,
                                              const Tile* __restrict__ tiles) {
  const Tile tl = tiles[blockIdx.x];
  const GemmJob jb = jobs[tl.job];
  const T* A = static_cast<const T*>(jb.A);
  const T* B = static_cast<const T*>(jb.B);
  T* C = static_cast<T*>(jb.C);
  const int m0 = tl.tm * 64, n0 = tl.tn * 64;
  __shared__ T As[16][64 + 1];
  __shared__ T Bs[16][64 + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  for (int k0 = 0; k0 < jb.K; k0 += 16) {
    // A tile: op(A)(m0 + i, k0 + k), i < 64, k < 16
    for (int e = threadIdx.x; e < 1024; e += 256) {
      int i, k;
      if (!jb.ta) { i = e & 63; k = e >> 6; } else { k = e & 15; i = e >> 4; }
      int gi = m0 + i, gk = k0 + k;
      T v = T(0);
      if (gi < jb.M && gk < jb.K) v = jb.ta ? A[gk + (long long)gi * jb.lda] : A[gi + (long long)gk * jb.lda];
      As[k][i] = v;
    }
    // B tile: op(B)(k0 + k, n0 + j), k < 16, j < 64
    for (int e = threadIdx.x; e < 1024; e += 256) {
      int j, k;
      if (!jb.tb) { k = e & 15; j = e >> 4; } else { j = e & 63; k = e >> 6; }
      int gj = n0 + j, gk = k0 + k;
      T v = T(0);
      if (gj < jb.N && gk < jb.K) v = jb.tb ? B[gj + (long long)gk * jb.ldb] : B[gk + (long long)gj * jb.ldb];
      Bs[k][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][tx + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[k][ty + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
  }
  const T alpha = T(jb.alpha), beta = T(jb.beta);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    int gj = n0 + ty + 16 * j;
    if (gj >= jb.N) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int gi = m0 + tx + 16 * i;
      if (gi >= jb.M) continue;
      long long r = jb.crow ? jb.crow[gi] : gi;
      T* c = C + r + (long long)gj * jb.ldc;
      *c = (jb.beta == 0.0) ? alpha * acc[i][j] : alpha * acc[i][j] + beta * (*c);
    }
  }
}

template <typename T>
void Kern<T>::gemm(const GemmJob* jobs, const Tile* tiles, int ntiles, cudaStream_t s) {
  if (ntiles <= 0) return;
  k_gemm<T><<<ntiles, 256, 0, s>>>(jobs, tiles);
  count_launch();
}

// ---------------------------------------------------------------------------
// Batched matrix-vector products (N <= GEMV_MAX_N right-hand columns) of the
// same job list: memory-bound, so every element of op(A) is read once with
// coalesced loads and used for all N columns.  op(A) = A: a CTA takes 32 rows
// (lanes), its 8 warps split K and combine in shared memory; op(A) = A^T: a
// warp per row, lanes over the contiguous K.  Deterministic sums.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_gemv(const GemmJob* __restrict__ jobs, const Tile* __restrict__ tiles) {
  const Tile tl = tiles[blockIdx.x];
  const GemmJob jb = jobs[tl.job];
  const T* A = static_cast<const T*>(jb.A);
  const T* B = static_cast<const T*>(jb.B);
  T* C = static_cast<T*>(jb.C);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int N = jb.N;
  const long long bk = jb.tb ? jb.ldb : 1, bc = jb.tb ? 1 : jb.ldb;  // op(B)(k, c) = B[k bk + c bc]
  T acc[GEMV_MAX_N];
#pragma unroll
  for (int c = 0; c < GEMV_MAX_N; ++c) acc[c] = T(0);
  int r;
  if (!jb.ta) {
    __shared__ T red[8][GEMV_MAX_N][33];
    r = tl.tm * 32 + lane;
    if (r < jb.M) {
#pragma unroll 8
      for (int k = wid; k < jb.K; k += 8) {
        const T a = A[r + (long long)k * jb.lda];
#pragma unroll
        for (int c = 0; c < GEMV_MAX_N; ++c)
          if (c < N) acc[c] += a * B[k * bk + c * bc];
      }
    }
#pragma unroll
    for (int c = 0; c < GEMV_MAX_N; ++c) red[wid][c][lane] = acc[c];
    __syncthreads();
    if (wid != 0) return;
#pragma unroll
    for (int c = 0; c < GEMV_MAX_N; ++c) {
      T s2 = T(0);
      for (int w = 0; w < 8; ++w) s2 += red[w][c][lane];
      acc[c] = s2;
    }
  } else {
    r = tl.tm * 8 + wid;
    if (r >= jb.M) return;
    const T* a_r = A + (long long)r * jb.lda;
#pragma unroll 4
    for (int k = lane; k < jb.K; k += 32) {
      const T a = a_r[k];
#pragma unroll
      for (int c = 0; c < GEMV_MAX_N; ++c)
        if (c < N) acc[c] += a * B[k * bk + c * bc];
    }
#pragma unroll
    for (int c = 0; c < GEMV_MAX_N; ++c)
      for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
    if (lane != 0) return;
  }
  if (r >= jb.M) return;
  const T alpha = T(jb.alpha), beta = T(jb.beta);
  const long long row = jb.crow ? jb.crow[r] : r;
#pragma unroll
  for (int c = 0; c < GEMV_MAX_N; ++c) {
    if (c >= N) break;
    T* cp = C + row + (long long)c * jb.ldc;
    *cp = (jb.beta == 0.0) ? alpha * acc[c] : alpha * acc[c] + beta * *cp;
  }
}

template <typename T>
void Kern<T>::gemv(const GemmJob* jobs, const Tile* tiles, int ntiles, cudaStream_t s) {
  if (ntiles <= 0) return;
  k_gemv<T><<<ntiles, 256, 0, s>>>(jobs, tiles);
  count_launch();
}

// ---------------------------------------------------------------------------
// Front assembly (A3): F_i = A_i (+) U_child0 (+) U_child1, written once per
// element as a gather over the children's update matrices (children in
// order: deterministic, no atomics), then the entries of A_i of the tile's
// rows are added.  Tiles are 32 x 32; tile list entries (front, tm, tn).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_assemble(const DFront* __restrict__ fr,
                                                  const int* __restrict__ ints, T* __restrict__ ar,
                                                  const double* __restrict__ values,
                                                  const Tile* __restrict__ tiles) {
  const Tile tl = tiles[blockIdx.x];
  const DFront f = fr[tl.job];
  __shared__ T tile[32][33];
  const int r = tl.tm * 32 + (threadIdx.x & 31);
  const int cbase = tl.tn * 32;
  for (int cc = threadIdx.x >> 5; cc < 32; cc += 8) {
    int c = cbase + cc;
    T v = T(0);
    if (r < f.nf && c < f.nf) {
      for (int k = 0; k < f.nchild; ++k) {
        const DFront ch = fr[k == 0 ? f.child0 : f.child1];
        const int* inv = ints + f.inv_off + (long long)k * f.nf;
        int ir = inv[r], ic = inv[c];
        if (ir >= 0 && ic >= 0) v += ar[ch.u_off + ir + (long long)ic * ch.u_ld];
      }
    }
    tile[threadIdx.x & 31][cc] = v;
  }
  __syncthreads();
  if (threadIdx.x < 32 && r < f.nf) {
    const int* arow = ints + f.arow_off;
    const int nnz_f = arow[f.nf];
    const int* acol = arow + f.nf + 1;
    const int* aval = acol + nnz_f;
    for (int p = arow[r]; p < arow[r + 1]; ++p) {
      int c = acol[p] - cbase;
      if (c >= 0 && c < 32) tile[threadIdx.x][c] += T(values[aval[p]]);
    }
  }
  __syncthreads();
  for (int cc = threadIdx.x >> 5; cc < 32; cc += 8) {
    int c = cbase + cc;
    if (r < f.nf && c < f.nf) ar[f.off + r + (long long)c * f.nf] = tile[threadIdx.x & 31][cc];
  }
}

template <typename T>
void Kern<T>::assemble(const DevSym& ds, T* arena, const double* values, const Tile* tiles,
                       int ntiles, cudaStream_t s) {
  if (ntiles <= 0) return;
  k_assemble<T><<<ntiles, 256, 0, s>>>(ds.fronts, ds.ints, arena, values, tiles);
  count_launch();
}

// ---------------------------------------------------------------------------
// Panel factorization of columns [k0, k0 + nb) of every listed front: pivot
// search restricted to rows < ns (first maximum of |a| wins), full-row swap
// across all nf columns, scaling of the column below the pivot and rank-1
// update of the remaining panel columns.  One CTA per front.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_panel(const DFront* __restrict__ fr, T* __restrict__ ar,
                                               int* __restrict__ piv, const int* __restrict__ flist,
                                               int k0, int nb, unsigned* status) {
  const DFront f = fr[flist[blockIdx.x]];
  if (k0 >= f.ns) return;
  const int k1 = min(k0 + nb, f.ns);
  T* F = ar + f.off;
  const long long ld = f.nf;
  __shared__ T s_val[8];
  __shared__ int s_idx[8];
  __shared__ int s_p;
  for (int j = k0; j < k1; ++j) {
    // pivot search over rows j .. ns-1 of column j
    T best = T(-1);
    int bi = f.ns;
    for (int r = j + threadIdx.x; r < f.ns; r += blockDim.x) {
      T a = tabs(F[r + j * ld]);
      if (a > best) { best = a; bi = r; }  // ascending r per thread: first max kept
    }
    for (int o = 16; o > 0; o >>= 1) {
      T ob = __shfl_down_sync(0xffffffffu, best, o);
      int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if ((threadIdx.x & 31) == 0) { s_val[threadIdx.x >> 5] = best; s_idx[threadIdx.x >> 5] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
      T b = s_val[0];
      int i = s_idx[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
        if (s_val[w] > b || (s_val[w] == b && s_idx[w] < i)) { b = s_val[w]; i = s_idx[w]; }
      if (!(b > T(0)) || !isfinite((double)b)) {
        set_status(status, b == T(0) ? ST_ZERO_PIVOT : ST_NONFINITE);
        i = j;
      }
      s_p = i;
      piv[f.piv_off + j] = i;
    }
    __syncthreads();
    const int p = s_p;
    if (p != j) {
      for (int c = threadIdx.x; c < f.nf; c += blockDim.x) {
        T t = F[j + c * ld];
        F[j + c * ld] = F[p + c * ld];
        F[p + c * ld] = t;
      }
    }
    __syncthreads();
    const T d = F[j + j * ld];
    const T inv = (d != T(0)) ? T(1) / d : T(0);
    for (int r = j + 1 + threadIdx.x; r < f.nf; r += blockDim.x) {
      T l = F[r + j * ld] * inv;
      F[r + j * ld] = l;
      for (int c = j + 1; c < k1; ++c) F[r + c * ld] -= l * F[j + c * ld];
    }
    __syncthreads();
  }
}

template <typename T>
void Kern<T>::panel_lu(const DevSym& ds, T* arena, int* piv, const int* flist, int nfr, int k0,
                       int nb, unsigned* status, cudaStream_t s) {
  if (nfr <= 0) return;
  k_panel<T><<<nfr, 256, 0, s>>>(ds.fronts, arena, piv, flist, k0, nb, status);
  count_launch();
}

// ---------------------------------------------------------------------------
// Row block of U12 after a panel: rows [k0, k1), columns [k1, nf) are
// replaced by L_panel^-1 times themselves (unit lower, nb <= 32).  Grid:
// (front, chunk of 128 columns); one column per thread.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(128) k_panel_trsm(const DFront* __restrict__ fr,
                                                    T* __restrict__ ar,
                                                    const int* __restrict__ flist, int k0, int nb) {
  const DFront f = fr[flist[blockIdx.x]];
  if (k0 >= f.ns) return;
  const int k1 = min(k0 + nb, f.ns);
  const int w = k1 - k0;
  T* F = ar + f.off;
  const long long ld = f.nf;
  __shared__ T L[32][33];
  for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
    int i = e & 31, j = e >> 5;
    L[i][j] = (i < w && j < w) ? F[(k0 + i) + (k0 + j) * ld] : T(0);
  }
  __syncthreads();
  const int c = k1 + blockIdx.y * 128 + threadIdx.x;
  if (c >= f.nf) return;
  T x[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) x[i] = (i < w) ? F[(k0 + i) + c * ld] : T(0);
#pragma unroll
  for (int i = 0; i < 32; ++i) {
#pragma unroll
    for (int r = i + 1; r < 32; ++r) x[r] -= L[r][i] * x[i];
  }
#pragma unroll
  for (int i = 0; i < 32; ++i)
    if (i < w) F[(k0 + i) + c * ld] = x[i];
}

template <typename T>
void Kern<T>::panel_trsm(const DevSym& ds, T* arena, const int* flist, int nfr, int k0, int nb,
                         int max_chunks, cudaStream_t s) {
  if (nfr <= 0 || max_chunks <= 0) return;
  dim3 g(nfr, max_chunks);  // fronts on x (no 65535 limit)
  k_panel_trsm<T><<<g, 128, 0, s>>>(ds.fronts, arena, flist, k0, nb);
  count_launch();
}

// ---------------------------------------------------------------------------
// Persistent per-level factorization of the small dense fronts (Section 3.2):
// a work queue over the level's fronts (largest first, an atomic counter);
// the CTA that takes a front assembles it in shared memory (extend-add of
// the children's update matrices in child order, then the entries of A_i,
// as k_assemble), factors F11 by the blocked partial LU with row pivoting
// inside F11 (first maximum of |a| wins, full-row swaps; L21, U12 and the
// update F22 - L21 U12 come out in place), and writes the front back.  One
// launch covers every front with nf <= the level's shared-memory bound.
// ---------------------------------------------------------------------------
template <typename T, int NT>
__global__ void __launch_bounds__(NT) k_front_lu(const DFront* __restrict__ fr, const int* __restrict__ ints,
                                                  T* __restrict__ ar, const double* __restrict__ values,
                                                  int* __restrict__ piv, const int* __restrict__ flist, int nfr,
                                                  int* __restrict__ counter, unsigned* status) {
  extern __shared__ __align__(16) unsigned char fl_smem[];
  T* Fs = reinterpret_cast<T*>(fl_smem);
  __shared__ T s_val[NT / 32];
  __shared__ int s_idx[NT / 32];
  __shared__ int s_front, s_p;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (;;) {
    if (threadIdx.x == 0) s_front = atomicAdd(counter, 1);
    __syncthreads();
    const int q = s_front;
    if (q >= nfr) break;
    const DFront f = fr[flist[q]];
    const int nf = f.nf, ns = f.ns;
    // assembly
    for (int e = threadIdx.x; e < nf * nf; e += NT) {
      const int r = e % nf, c = e / nf;
      T v = T(0);
      for (int k = 0; k < f.nchild; ++k) {
        const DFront ch = fr[k == 0 ? f.child0 : f.child1];
        const int* inv = ints + f.inv_off + (long long)k * nf;
        const int ir = inv[r], ic = inv[c];
        if (ir >= 0 && ic >= 0) v += ar[ch.u_off + ir + (long long)ic * ch.u_ld];
      }
      Fs[e] = v;
    }
    __syncthreads();
    {
      const int* arow = ints + f.arow_off;
      const int nnz_f = arow[nf];
      const int* acol = arow + nf + 1;
      const int* aval = acol + nnz_f;
      for (int r = threadIdx.x; r < nf; r += NT)  // one thread per row: the row's entries in CSR order
        for (int p = arow[r]; p < arow[r + 1]; ++p) Fs[r + acol[p] * nf] += T(values[aval[p]]);
    }
    __syncthreads();
    // the blocked partial LU of the panel path (32-column panels: panel LU,
    // U12 rows by forward substitution, trailing update with the panel's
    // products summed first), in the same operation order, so that either
    // path gives the same factors bit for bit
    for (int k0 = 0; k0 < ns; k0 += 32) {
      const int k1 = min(k0 + 32, ns), w = k1 - k0;
      for (int j = k0; j < k1; ++j) {
        T best = T(-1);
        int bi = ns;
        for (int r = j + threadIdx.x; r < ns; r += NT) {
          const T a = tabs(Fs[r + j * nf]);
          if (a > best) { best = a; bi = r; }
        }
        for (int o = 16; o > 0; o >>= 1) {
          const T ob = __shfl_down_sync(0xffffffffu, best, o);
          const int oi = __shfl_down_sync(0xffffffffu, bi, o);
          if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (lane == 0) { s_val[wid] = best; s_idx[wid] = bi; }
        __syncthreads();
        if (threadIdx.x == 0) {
          T b = s_val[0];
          int i = s_idx[0];
          for (int w2 = 1; w2 < NT / 32; ++w2)
            if (s_val[w2] > b || (s_val[w2] == b && s_idx[w2] < i)) { b = s_val[w2]; i = s_idx[w2]; }
          if (!(b > T(0)) || !isfinite((double)b)) {
            set_status(status, b == T(0) ? ST_ZERO_PIVOT : ST_NONFINITE);
            i = j;
          }
          s_p = i;
          piv[f.piv_off + j] = i;
        }
        __syncthreads();
        const int p = s_p;
        if (p != j)
          for (int c = threadIdx.x; c < nf; c += NT) {
            const T t = Fs[j + c * nf];
            Fs[j + c * nf] = Fs[p + c * nf];
            Fs[p + c * nf] = t;
          }
        __syncthreads();
        const T d = Fs[j + j * nf];
        const T inv = (d != T(0)) ? T(1) / d : T(0);
        for (int r = j + 1 + threadIdx.x; r < nf; r += NT) {
          const T l = Fs[r + j * nf] * inv;
          Fs[r + j * nf] = l;
          for (int c = j + 1; c < k1; ++c) Fs[r + c * nf] -= l * Fs[j + c * nf];
        }
        __syncthreads();
      }
      // rows k0..k1-1 of the columns right of the panel: L_panel^-1 times them
      for (int c = k1 + threadIdx.x; c < nf; c += NT) {
        T x[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) x[i] = i < w ? Fs[(k0 + i) + c * nf] : T(0);
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const T xi = x[i];
#pragma unroll
          for (int r = i + 1; r < 32; ++r) x[r] -= (r < w && i < w ? Fs[(k0 + r) + (k0 + i) * nf] : T(0)) * xi;
        }
#pragma unroll
        for (int i = 0; i < 32; ++i)
          if (i < w) Fs[(k0 + i) + c * nf] = x[i];
      }
      __syncthreads();
      // trailing update: F22 block -= sum over the panel columns, summed first
      const int m1 = nf - k1;
      for (int e = threadIdx.x; e < m1 * m1; e += NT) {
        const int r = k1 + e % m1, c = k1 + e / m1;
        T acc = T(0);
        for (int k = 0; k < w; ++k) acc += Fs[r + (k0 + k) * nf] * Fs[(k0 + k) + c * nf];
        Fs[r + c * nf] = T(-1) * acc + T(1) * Fs[r + c * nf];
      }
      __syncthreads();
    }
    for (int e = threadIdx.x; e < nf * nf; e += NT) ar[f.off + e] = Fs[e];
    __syncthreads();  // Fs and s_front are reused by the next front
  }
}

template <typename T>
int Kern<T>::front_lu(const DevSym& ds, T* arena, const double* values, int* piv, const int* flist, int nfr,
                      int max_nf, int threads, int nsm, int* counter, unsigned* status, cudaStream_t s) {
  if (nfr <= 0) return 0;
  const size_t smem = sizeof(T) * (size_t)max_nf * max_nf;
  if (smem > kFrontLuSmemMax || nsm <= 0) return -1;
  const void* kern = threads == 128 ? (const void*)k_front_lu<T, 128> : (const void*)k_front_lu<T, 256>;
  if (!set_func_attr(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFrontLuSmemMax)) return -1;
  // a persistent grid: every CTA that can be resident at once, at most one per front
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem) != cudaSuccess || occ < 1) {
    cudaGetLastError();
    return -1;
  }
  const int grid = (int)std::min<long long>(nfr, (long long)nsm * occ);
  if (cudaMemsetAsync(counter, 0, sizeof(int), s) != cudaSuccess) return -1;
  if (threads == 128)
    k_front_lu<T, 128><<<grid, 128, smem, s>>>(ds.fronts, ds.ints, arena, values, piv, flist, nfr, counter, status);
  else
    k_front_lu<T, 256><<<grid, 256, smem, s>>>(ds.fronts, ds.ints, arena, values, piv, flist, nfr, counter, status);
  count_launch();
  return 0;
}

template struct Kern<double>;
template struct Kern<float>;

}  // namespace hssmf
