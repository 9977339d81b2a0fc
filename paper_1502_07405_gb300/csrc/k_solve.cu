// Multifrontal solve kernels for dense fronts (Section 3.3) and the FP64
// kernels of the outer iteration (sparse product, GMRES(30) with modified
// Gram-Schmidt, iterative refinement; Sections 4.6 and 6.1).
#include <algorithm>

#include "kernels.h"

namespace hssmf {

template <typename Tin, typename Tout>
__global__ void k_permute_in(const Tin* __restrict__ b, long long ldb, Tout* __restrict__ bp,
                             const int* __restrict__ perm, int n, int nrhs) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long tot = (long long)n * nrhs;
  for (; t < tot; t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t % n), j = (int)(t / n);
    bp[i + (long long)j * n] = Tout(b[perm[i] + j * ldb]);
  }
}

template <typename Tin, typename Tout>
__global__ void k_permute_out(const Tin* __restrict__ xp, Tout* __restrict__ x, long long ldx,
                              const int* __restrict__ perm, int n, int nrhs) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long tot = (long long)n * nrhs;
  for (; t < tot; t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t % n), j = (int)(t / n);
    x[perm[i] + j * ldx] = Tout(xp[i + (long long)j * n]);
  }
}

static int grid_for(long long work, int block = 256) {
  long long g = (work + block - 1) / block;
  if (g > 152 * 32) g = 152 * 32;
  return (int)(g < 1 ? 1 : g);
}

template <typename T>
void Kern<T>::permute_in(const double* b, long long ldb, T* bp, const int* perm, int n, int nrhs,
                         cudaStream_t s) {
  k_permute_in<double, T><<<grid_for((long long)n * nrhs), 256, 0, s>>>(b, ldb, bp, perm, n, nrhs);
  count_launch();
}

template <typename T>
void Kern<T>::permute_out(const T* xp, double* x, long long ldx, const int* perm, int n, int nrhs,
                          cudaStream_t s) {
  k_permute_out<T, double><<<grid_for((long long)n * nrhs), 256, 0, s>>>(xp, x, ldx, perm, n, nrhs);
  count_launch();
}

// ---------------------------------------------------------------------------
// Forward solve, assembly of the front right-hand side: W_f = [b(I^sep); 0]
// (+) the children's updated I^upd parts (extend-add of vectors, children in
// order).  Grid (front, row chunk of 256): fronts on x, which has no 65535
// limit.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_solve_gather(const DFront* __restrict__ fr, const int* __restrict__ ints,
                               T* __restrict__ W, const T* __restrict__ bp,
                               const int* __restrict__ flist, int n, int nrhs) {
  const DFront f = fr[flist[blockIdx.x]];
  const int r = blockIdx.y * blockDim.x + threadIdx.x;
  if (r >= f.nf) return;
  int ir[2] = {-1, -1};
  for (int k = 0; k < f.nchild; ++k) ir[k] = ints[f.inv_off + (long long)k * f.nf + r];
  for (int j = 0; j < nrhs; ++j) {
    T v = r < f.ns ? bp[f.sep_begin + r + (long long)j * n] : T(0);
    for (int k = 0; k < f.nchild; ++k) {
      if (ir[k] < 0) continue;
      const DFront ch = fr[k == 0 ? f.child0 : f.child1];
      v += W[ch.w_off + ch.ns + ir[k] + (long long)j * ch.nf];
    }
    W[f.w_off + r + (long long)j * f.nf] = v;
  }
}

template <typename T>
void Kern<T>::solve_gather(const DevSym& ds, T* W, const T* bp, const int* flist, int nfr,
                           int max_rows, int nrhs, cudaStream_t s) {
  if (nfr <= 0) return;
  dim3 g(nfr, (max_rows + 255) / 256);
  k_solve_gather<T><<<g, 256, 0, s>>>(ds.fronts, ds.ints, W, bp, flist, ds.n, nrhs);
  count_launch();
}

// block-wide sum (blockDim multiple of 32, <= 1024)
template <typename T>
__device__ T block_sum(T v, T* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  T s = T(0);
  if (threadIdx.x == 0) {
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    sh[32] = s;
  }
  __syncthreads();
  s = sh[32];
  __syncthreads();
  return s;
}

// ---------------------------------------------------------------------------
// Forward sweep of a dense front, one CTA per front.
//   transpose = 0: row interchanges, then column-oriented unit-lower
//     substitution over all nf rows, which gives y = L11^-1 P b_s and
//     b_u -= L21 y in one pass over the first ns columns of F.
//   transpose = 1: y = U11^-T b_s (dot-product form over the columns of
//     U11), then b_u -= U12^T y.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_solve_fwd_dense(const DFront* __restrict__ fr,
                                                         const T* __restrict__ ar,
                                                         const int* __restrict__ piv,
                                                         T* __restrict__ W,
                                                         const int* __restrict__ flist, int nrhs,
                                                         int transpose) {
  const DFront f = fr[flist[blockIdx.x]];
  if (f.is_hss) return;
  const T* F = ar + f.off;
  const long long ld = f.nf;
  T* w = W + f.w_off;
  __shared__ T sh[33];
  for (int j = blockIdx.y; j < nrhs; j += gridDim.y) {  // columns are independent
    T* x = w + (long long)j * f.nf;
    if (!transpose) {
      if (threadIdx.x == 0) {
        for (int i = 0; i < f.ns; ++i) {
          int p = piv[f.piv_off + i];
          if (p != i) { T t = x[i]; x[i] = x[p]; x[p] = t; }
        }
      }
      __syncthreads();
      for (int c = 0; c < f.ns; ++c) {
        const T xc = x[c];
        for (int r = c + 1 + threadIdx.x; r < f.nf; r += blockDim.x) x[r] -= F[r + c * ld] * xc;
        __syncthreads();
      }
    } else {
      for (int c = 0; c < f.ns; ++c) {  // U11^T is lower triangular: y_c = (b_c - U(0:c,c).y)/U(c,c)
        T part = T(0);
        for (int r = threadIdx.x; r < c; r += blockDim.x) part += F[r + c * ld] * x[r];
        T s = block_sum(part, sh);
        if (threadIdx.x == 0) x[c] = (x[c] - s) / F[c + c * ld];
        __syncthreads();
      }
      // b_u -= U12^T y : one warp per column of U12
      const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
      for (int c = f.ns + wid; c < f.nf; c += nw) {
        T part = T(0);
        for (int r = lane; r < f.ns; r += 32) part += F[r + c * ld] * x[r];
        for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
        if (lane == 0) x[c] -= part;
      }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------
// Several right-hand sides: one warp per column, the column staged in shared
// memory, so a substitution step needs only the warp (no CTA barrier) and the
// CTA's 8 warps share the front's factor through L1.  Same substitution
// forms as the one-CTA-per-column kernels above and below.
// ---------------------------------------------------------------------------
constexpr int WC_WARPS = 8;
constexpr size_t kWarpColSmem = 160 * 1024;

template <typename T>
__device__ __forceinline__ T warp_allsum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__global__ void __launch_bounds__(256) k_solve_fwd_dense_wc(const DFront* __restrict__ fr,
                                                            const T* __restrict__ ar,
                                                            const int* __restrict__ piv,
                                                            T* __restrict__ W,
                                                            const int* __restrict__ flist, int nrhs,
                                                            int max_nf, int transpose) {
  const DFront f = fr[flist[blockIdx.x]];
  if (f.is_hss) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int j = blockIdx.y * WC_WARPS + wid;
  if (j >= nrhs) return;
  extern __shared__ __align__(16) unsigned char wc_raw[];
  T* xw = reinterpret_cast<T*>(wc_raw) + (size_t)wid * max_nf;
  const T* F = ar + f.off;
  const long long ld = f.nf;
  T* x = W + f.w_off + (long long)j * f.nf;
  for (int r = lane; r < f.nf; r += 32) xw[r] = x[r];
  __syncwarp();
  if (!transpose) {
    if (lane == 0)
      for (int i = 0; i < f.ns; ++i) {
        const int p = piv[f.piv_off + i];
        if (p != i) { const T t = xw[i]; xw[i] = xw[p]; xw[p] = t; }
      }
    __syncwarp();
    for (int c = 0; c < f.ns; ++c) {  // unit lower, column-oriented over all nf rows
      const T xc = xw[c];
      const T* Fc = F + c * ld;
      for (int r = c + 1 + lane; r < f.nf; r += 32) xw[r] -= Fc[r] * xc;
      __syncwarp();
    }
  } else {
    for (int c = 0; c < f.ns; ++c) {  // U11^T: y_c = (b_c - U(0:c, c) . y) / U(c, c)
      const T* Fc = F + c * ld;
      T part = T(0);
      for (int r = lane; r < c; r += 32) part += Fc[r] * xw[r];
      part = warp_allsum(part);
      if (lane == 0) xw[c] = (xw[c] - part) / Fc[c];
      __syncwarp();
    }
    for (int c = f.ns; c < f.nf; ++c) {  // b_u -= U12^T y
      const T* Fc = F + c * ld;
      T part = T(0);
      for (int r = lane; r < f.ns; r += 32) part += Fc[r] * xw[r];
      part = warp_allsum(part);
      if (lane == 0) xw[c] -= part;
    }
    __syncwarp();
  }
  for (int r = lane; r < f.nf; r += 32) x[r] = xw[r];
}

template <typename T>
static bool warp_cols_fit(int max_nf, int nrhs) {
  return nrhs >= 4 && max_nf > 0 && (size_t)WC_WARPS * max_nf * sizeof(T) <= kWarpColSmem;
}

// ---------------------------------------------------------------------------
// Blocked sweeps of the dense fronts: the triangular factors in 32 x 32
// diagonal blocks (solved by one warp per right-hand side from a shared-
// memory copy of the block), each followed by the update of the remaining
// rows (or columns) with the block's 32 columns (rows): a product read once
// with coalesced loads, so the sweep is bound by reading the factor, not by
// one dependent step per column.  A CTA takes nc <= 8 right-hand sides of a
// front, staged in shared memory.
// ---------------------------------------------------------------------------
constexpr int BLK_NC = 8;
constexpr size_t kBlkSolveSmem = 192 * 1024;

template <typename T>
__global__ void __launch_bounds__(256) k_solve_fwd_blk(const DFront* __restrict__ fr, const T* __restrict__ ar,
                                                       const int* __restrict__ piv, T* __restrict__ W,
                                                       const int* __restrict__ flist, int nrhs, int nc_max,
                                                       int max_nf, int transpose) {
  const DFront f = fr[flist[blockIdx.x]];
  if (f.is_hss) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int j0 = blockIdx.y * nc_max, nc = min(nc_max, nrhs - j0);
  if (nc <= 0) return;
  extern __shared__ __align__(16) unsigned char blk_raw[];
  T* xs = reinterpret_cast<T*>(blk_raw);  // nc x max_nf
  int* pv = reinterpret_cast<int*>(xs + (size_t)nc * max_nf);  // max_nf: the front's pivots
  __shared__ T B[32][33];
  const T* F = ar + f.off;
  const long long ld = f.nf;
  const int nf = f.nf, ns = f.ns;
  T* w = W + f.w_off + (long long)j0 * nf;
  for (int e = threadIdx.x; e < nc * nf; e += blockDim.x) xs[(e / nf) * max_nf + e % nf] = w[e];
  if (!transpose)
    for (int i = threadIdx.x; i < ns; i += blockDim.x) pv[i] = piv[f.piv_off + i];
  __syncthreads();
  if (!transpose && threadIdx.x < nc) {  // P b_s: the interchanges in order, one thread per column
    T* x = xs + threadIdx.x * max_nf;
    for (int i = 0; i < ns; ++i) {
      const int p = pv[i];
      if (p != i) { const T t = x[i]; x[i] = x[p]; x[p] = t; }
    }
  }
  __syncthreads();
  for (int cb = 0; cb < ns; cb += 32) {
    const int cw = min(32, ns - cb);
    for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
      const int t = e & 31, k = e >> 5;
      B[t][k] = (t < cw && k < cw) ? F[(cb + t) + (long long)(cb + k) * ld] : T(0);
    }
    __syncthreads();
    for (int q = wid; q < nc; q += blockDim.x >> 5) {  // the diagonal block, one warp per column
      T* x = xs + q * max_nf + cb;
      T v = lane < cw ? x[lane] : T(0);
      if (!transpose) {  // unit lower: x_t -= L(t, k) x_k
        for (int k = 0; k < cw; ++k) {
          const T xk = __shfl_sync(0xffffffffu, v, k);
          if (lane > k) v -= B[lane][k] * xk;
        }
      } else {  // U^T (lower): y_k = x_k / U(k, k), then x_t -= U(k, t) y_k
        for (int k = 0; k < cw; ++k) {
          const T yk = __shfl_sync(0xffffffffu, v, k) / B[k][k];
          if (lane == k) v = yk;
          if (lane > k) v -= B[k][lane] * yk;
        }
      }
      if (lane < cw) x[lane] = v;
    }
    __syncthreads();
    if (!transpose) {  // rows below the block: x_r -= L(r, block) x_block (also b_u -= L21 y)
      for (int r = cb + cw + threadIdx.x; r < nf; r += blockDim.x) {
        T acc[BLK_NC];
#pragma unroll
        for (int q = 0; q < BLK_NC; ++q) acc[q] = T(0);
        for (int k = 0; k < cw; ++k) {
          const T l = F[r + (long long)(cb + k) * ld];
#pragma unroll
          for (int q = 0; q < BLK_NC; ++q)
            if (q < nc) acc[q] += l * xs[q * max_nf + cb + k];
        }
#pragma unroll
        for (int q = 0; q < BLK_NC; ++q)
          if (q < nc) xs[q * max_nf + r] -= acc[q];
      }
    } else {  // columns right of the block: x_c -= U(block, c)^T y_block (also b_u -= U12^T y)
      for (int c = cb + cw + threadIdx.x; c < nf; c += blockDim.x) {
        T acc[BLK_NC];
#pragma unroll
        for (int q = 0; q < BLK_NC; ++q) acc[q] = T(0);
        const T* Fc = F + (long long)c * ld + cb;
        for (int k = 0; k < cw; ++k) {
          const T u = Fc[k];
#pragma unroll
          for (int q = 0; q < BLK_NC; ++q)
            if (q < nc) acc[q] += u * xs[q * max_nf + cb + k];
        }
#pragma unroll
        for (int q = 0; q < BLK_NC; ++q)
          if (q < nc) xs[q * max_nf + c] -= acc[q];
      }
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < nc * nf; e += blockDim.x) w[e] = xs[(e / nf) * max_nf + e % nf];
}

template <typename T>
__global__ void __launch_bounds__(256) k_solve_bwd_blk(const DFront* __restrict__ fr, const T* __restrict__ ar,
                                                       const int* __restrict__ piv, T* __restrict__ W,
                                                       T* __restrict__ xp, const int* __restrict__ flist, int n,
                                                       int nrhs, int nc_max, int max_nf, int transpose) {
  const DFront f = fr[flist[blockIdx.x]];
  if (f.is_hss) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int j0 = blockIdx.y * nc_max, nc = min(nc_max, nrhs - j0);
  if (nc <= 0) return;
  extern __shared__ __align__(16) unsigned char blk_raw[];
  T* xs = reinterpret_cast<T*>(blk_raw);  // nc x max_nf
  int* pv = reinterpret_cast<int*>(xs + (size_t)nc * max_nf);  // max_nf: the front's pivots
  __shared__ T B[32][33];
  const T* F = ar + f.off;
  const long long ld = f.nf;
  const int nf = f.nf, ns = f.ns;
  const T* w = W + f.w_off + (long long)j0 * nf;
  for (int e = threadIdx.x; e < nc * nf; e += blockDim.x) xs[(e / nf) * max_nf + e % nf] = w[e];
  if (transpose)
    for (int i = threadIdx.x; i < ns; i += blockDim.x) pv[i] = piv[f.piv_off + i];
  __syncthreads();
  if (!transpose) {  // y -= U12 x_u, thread per row
    for (int r = threadIdx.x; r < ns; r += blockDim.x) {
      T acc[BLK_NC];
#pragma unroll
      for (int q = 0; q < BLK_NC; ++q) acc[q] = T(0);
      for (int c = ns; c < nf; ++c) {
        const T u = F[r + (long long)c * ld];
#pragma unroll
        for (int q = 0; q < BLK_NC; ++q)
          if (q < nc) acc[q] += u * xs[q * max_nf + c];
      }
#pragma unroll
      for (int q = 0; q < BLK_NC; ++q)
        if (q < nc) xs[q * max_nf + r] -= acc[q];
    }
  } else {  // y -= L21^T x_u, warp per row of the result (column of L21)
    for (int r = wid; r < ns; r += blockDim.x >> 5) {
      const T* Fr = F + (long long)r * ld;
      T acc[BLK_NC];
#pragma unroll
      for (int q = 0; q < BLK_NC; ++q) acc[q] = T(0);
      for (int c = ns + lane; c < nf; c += 32) {
        const T l = Fr[c];
#pragma unroll
        for (int q = 0; q < BLK_NC; ++q)
          if (q < nc) acc[q] += l * xs[q * max_nf + c];
      }
#pragma unroll
      for (int q = 0; q < BLK_NC; ++q) {
        if (q >= nc) break;
        const T sum = warp_allsum(acc[q]);
        if (lane == 0) xs[q * max_nf + r] -= sum;
      }
    }
  }
  __syncthreads();
  for (int cb = ((ns - 1) / 32) * 32; cb >= 0 && ns > 0; cb -= 32) {
    const int cw = min(32, ns - cb);
    for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
      const int t = e & 31, k = e >> 5;
      B[t][k] = (t < cw && k < cw) ? F[(cb + t) + (long long)(cb + k) * ld] : T(0);
    }
    __syncthreads();
    for (int q = wid; q < nc; q += blockDim.x >> 5) {  // the diagonal block, one warp per column
      T* x = xs + q * max_nf + cb;
      T v = lane < cw ? x[lane] : T(0);
      if (!transpose) {  // U11: x_k = x_k / U(k, k), then x_t -= U(t, k) x_k
        for (int k = cw - 1; k >= 0; --k) {
          const T xk = __shfl_sync(0xffffffffu, v, k) / B[k][k];
          if (lane == k) v = xk;
          if (lane < k) v -= B[lane][k] * xk;
        }
      } else {  // L11^T (unit upper): x_t -= L(k, t) x_k
        for (int k = cw - 1; k >= 0; --k) {
          const T xk = __shfl_sync(0xffffffffu, v, k);
          if (lane < k) v -= B[k][lane] * xk;
        }
      }
      if (lane < cw) x[lane] = v;
    }
    __syncthreads();
    if (!transpose) {  // rows above the block: x_r -= U(r, block) x_block
      for (int r = threadIdx.x; r < cb; r += blockDim.x) {
        T acc[BLK_NC];
#pragma unroll
        for (int q = 0; q < BLK_NC; ++q) acc[q] = T(0);
        for (int k = 0; k < cw; ++k) {
          const T u = F[r + (long long)(cb + k) * ld];
#pragma unroll
          for (int q = 0; q < BLK_NC; ++q)
            if (q < nc) acc[q] += u * xs[q * max_nf + cb + k];
        }
#pragma unroll
        for (int q = 0; q < BLK_NC; ++q)
          if (q < nc) xs[q * max_nf + r] -= acc[q];
      }
    } else {  // columns left of the block: x_c -= L(block, c)^T x_block
      for (int c = threadIdx.x; c < cb; c += blockDim.x) {
        T acc[BLK_NC];
#pragma unroll
        for (int q = 0; q < BLK_NC; ++q) acc[q] = T(0);
        const T* Fc = F + (long long)c * ld + cb;
        for (int k = 0; k < cw; ++k) {
          const T l = Fc[k];
#pragma unroll
          for (int q = 0; q < BLK_NC; ++q)
            if (q < nc) acc[q] += l * xs[q * max_nf + cb + k];
        }
#pragma unroll
        for (int q = 0; q < BLK_NC; ++q)
          if (q < nc) xs[q * max_nf + c] -= acc[q];
      }
    }
    __syncthreads();
  }
  if (transpose && threadIdx.x < nc) {  // P^T
    T* x = xs + threadIdx.x * max_nf;
    for (int i = ns - 1; i >= 0; --i) {
      const int p = pv[i];
      if (p != i) { const T t = x[i]; x[i] = x[p]; x[p] = t; }
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nc * ns; e += blockDim.x) {
    const int q = e / ns, r = e % ns;
    xp[f.sep_begin + r + (long long)(j0 + q) * n] = xs[q * max_nf + r];
  }
}

// right-hand sides per CTA of the blocked sweeps (0: the front does not fit)
template <typename T>
static int blk_cols(int max_nf, int nrhs) {
  if (max_nf <= 0 || sizeof(int) * (size_t)max_nf >= kBlkSolveSmem / 2) return 0;
  const size_t room = kBlkSolveSmem - sizeof(int) * (size_t)max_nf;  // the pivots' staging
  const int nc = (int)std::min<size_t>(BLK_NC, room / ((size_t)max_nf * sizeof(T)));
  return std::min(nc, std::max(nrhs, 1));
}

// threads of a blocked-sweep CTA: fewer for small fronts, whose blocks are short
static int blk_threads(int max_nf) { return max_nf <= 96 ? 64 : max_nf <= 192 ? 128 : 256; }

// dynamic shared memory of the blocked sweeps: nc staged columns and the pivots
template <typename T>
static size_t blk_smem(int nc, int max_nf) {
  return (size_t)nc * max_nf * sizeof(T) + sizeof(int) * (size_t)max_nf;
}

template <typename T>
void Kern<T>::solve_fwd_dense(const DevSym& ds, const T* arena, const int* piv, T* W,
                              const int* flist, int nfr, int max_nf, int nrhs, int transpose, cudaStream_t s) {
  if (nfr <= 0) return;
  const int nc = blk_cols<T>(max_nf, nrhs);
  if (nc > 0) {
    set_func_attr((const void*)k_solve_fwd_blk<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBlkSolveSmem);
    const size_t smem = blk_smem<T>(nc, max_nf);
    k_solve_fwd_blk<T><<<dim3(nfr, (nrhs + nc - 1) / nc), blk_threads(max_nf), smem, s>>>(ds.fronts, arena, piv, W, flist, nrhs, nc,
                                                                         max_nf, transpose);
  } else if (warp_cols_fit<T>(max_nf, nrhs)) {
    set_func_attr((const void*)k_solve_fwd_dense_wc<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWarpColSmem);
    const size_t smem = (size_t)WC_WARPS * max_nf * sizeof(T);
    k_solve_fwd_dense_wc<T><<<dim3(nfr, (nrhs + WC_WARPS - 1) / WC_WARPS), 256, smem, s>>>(
        ds.fronts, arena, piv, W, flist, nrhs, max_nf, transpose);
  } else {
    k_solve_fwd_dense<T><<<dim3(nfr, std::min(nrhs, 64)), 256, 0, s>>>(ds.fronts, arena, piv, W, flist, nrhs,
                                                                      transpose);
  }
  count_launch();
}

// Backward solve: W_f(ns + i) = x(I^upd(i)).  Grid (front, chunk).
template <typename T>
__global__ void k_solve_bwd_gather(const DFront* __restrict__ fr, const int* __restrict__ ints,
                                   T* __restrict__ W, const T* __restrict__ xp,
                                   const int* __restrict__ flist, int n, int nrhs) {
  const DFront f = fr[flist[blockIdx.x]];
  const int i = blockIdx.y * blockDim.x + threadIdx.x;
  if (i >= f.nu) return;
  const int g = ints[f.upd_off + i];
  for (int j = 0; j < nrhs; ++j) W[f.w_off + f.ns + i + (long long)j * f.nf] = xp[g + (long long)j * n];
}

template <typename T>
void Kern<T>::solve_bwd_gather(const DevSym& ds, T* W, const T* xp, const int* flist, int nfr,
                               int max_nu, int nrhs, cudaStream_t s) {
  if (nfr <= 0 || max_nu <= 0) return;
  dim3 g(nfr, (max_nu + 255) / 256);
  k_solve_bwd_gather<T><<<g, 256, 0, s>>>(ds.fronts, ds.ints, W, xp, flist, ds.n, nrhs);
  count_launch();
}

// ---------------------------------------------------------------------------
// Backward sweep of a dense front, one CTA per front; writes x(I^sep).
//   transpose = 0: y -= U12 x_u (column-oriented), then column-oriented
//     upper substitution with U11.
//   transpose = 1: y -= L21^T x_u (warp per column of L21), unit-upper
//     substitution with L11^T (dot-product form), then P^T.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_solve_bwd_dense(const DFront* __restrict__ fr,
                                                         const T* __restrict__ ar,
                                                         const int* __restrict__ piv,
                                                         T* __restrict__ W, T* __restrict__ xp,
                                                         const int* __restrict__ flist, int n,
                                                         int nrhs, int transpose) {
  const DFront f = fr[flist[blockIdx.x]];
  if (f.is_hss) return;
  const T* F = ar + f.off;
  const long long ld = f.nf;
  __shared__ T sh[33];
  for (int j = blockIdx.y; j < nrhs; j += gridDim.y) {  // columns are independent
    T* x = W + f.w_off + (long long)j * f.nf;
    if (!transpose) {
      for (int r = threadIdx.x; r < f.ns; r += blockDim.x) {
        T acc = T(0);
        for (int c = f.ns; c < f.nf; ++c) acc += F[r + c * ld] * x[c];
        x[r] -= acc;
      }
      __syncthreads();
      for (int c = f.ns - 1; c >= 0; --c) {
        const T xc = x[c] / F[c + c * ld];
        __syncthreads();
        if (threadIdx.x == 0) x[c] = xc;
        for (int r = threadIdx.x; r < c; r += blockDim.x) x[r] -= F[r + c * ld] * xc;
        __syncthreads();
      }
    } else {
      const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
      for (int r = wid; r < f.ns; r += nw) {
        T part = T(0);
        for (int c = f.ns + lane; c < f.nf; c += 32) part += F[c + r * ld] * x[c];
        for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
        if (lane == 0) x[r] -= part;
      }
      __syncthreads();
      for (int c = f.ns - 1; c >= 0; --c) {  // L11^T unit upper: x_c -= L(c+1:ns, c) . x(c+1:ns)
        T part = T(0);
        for (int r = c + 1 + threadIdx.x; r < f.ns; r += blockDim.x) part += F[r + c * ld] * x[r];
        T s = block_sum(part, sh);
        if (threadIdx.x == 0) x[c] -= s;
        __syncthreads();
      }
      if (threadIdx.x == 0) {
        for (int i = f.ns - 1; i >= 0; --i) {
          int p = piv[f.piv_off + i];
          if (p != i) { T t = x[i]; x[i] = x[p]; x[p] = t; }
        }
      }
      __syncthreads();
    }
    for (int r = threadIdx.x; r < f.ns; r += blockDim.x) xp[f.sep_begin + r + (long long)j * n] = x[r];
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_solve_bwd_dense_wc(const DFront* __restrict__ fr,
                                                            const T* __restrict__ ar,
                                                            const int* __restrict__ piv,
                                                            T* __restrict__ W, T* __restrict__ xp,
                                                            const int* __restrict__ flist, int n, int nrhs,
                                                            int max_nf, int transpose) {
  const DFront f = fr[flist[blockIdx.x]];
  if (f.is_hss) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int j = blockIdx.y * WC_WARPS + wid;
  if (j >= nrhs) return;
  extern __shared__ __align__(16) unsigned char wc_raw[];
  T* xw = reinterpret_cast<T*>(wc_raw) + (size_t)wid * max_nf;
  const T* F = ar + f.off;
  const long long ld = f.nf;
  const T* x = W + f.w_off + (long long)j * f.nf;
  for (int r = lane; r < f.nf; r += 32) xw[r] = x[r];
  __syncwarp();
  if (!transpose) {
    for (int r = lane; r < f.ns; r += 32) {  // y -= U12 x_u
      T acc = T(0);
      for (int c = f.ns; c < f.nf; ++c) acc += F[r + c * ld] * xw[c];
      xw[r] -= acc;
    }
    __syncwarp();
    for (int c = f.ns - 1; c >= 0; --c) {  // U11, column-oriented
      const T* Fc = F + c * ld;
      const T xc = xw[c] / Fc[c];
      __syncwarp();
      if (lane == 0) xw[c] = xc;
      for (int r = lane; r < c; r += 32) xw[r] -= Fc[r] * xc;
      __syncwarp();
    }
  } else {
    for (int r = 0; r < f.ns; ++r) {  // y -= L21^T x_u
      const T* Fr = F + r * ld;
      T part = T(0);
      for (int c = f.ns + lane; c < f.nf; c += 32) part += Fr[c] * xw[c];
      part = warp_allsum(part);
      if (lane == 0) xw[r] -= part;
    }
    __syncwarp();
    for (int c = f.ns - 1; c >= 0; --c) {  // L11^T unit upper: x_c -= L(c+1:ns, c) . x(c+1:ns)
      const T* Fc = F + c * ld;
      T part = T(0);
      for (int r = c + 1 + lane; r < f.ns; r += 32) part += Fc[r] * xw[r];
      part = warp_allsum(part);
      if (lane == 0) xw[c] -= part;
      __syncwarp();
    }
    if (lane == 0)
      for (int i = f.ns - 1; i >= 0; --i) {
        const int p = piv[f.piv_off + i];
        if (p != i) { const T t = xw[i]; xw[i] = xw[p]; xw[p] = t; }
      }
    __syncwarp();
  }
  for (int r = lane; r < f.ns; r += 32) xp[f.sep_begin + r + (long long)j * n] = xw[r];
}

template <typename T>
void Kern<T>::solve_bwd_dense(const DevSym& ds, const T* arena, const int* piv, T* W, T* xp,
                              const int* flist, int nfr, int max_nf, int nrhs, int transpose, cudaStream_t s) {
  if (nfr <= 0) return;
  const int nc = blk_cols<T>(max_nf, nrhs);
  if (nc > 0) {
    set_func_attr((const void*)k_solve_bwd_blk<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBlkSolveSmem);
    const size_t smem = blk_smem<T>(nc, max_nf);
    k_solve_bwd_blk<T><<<dim3(nfr, (nrhs + nc - 1) / nc), blk_threads(max_nf), smem, s>>>(ds.fronts, arena, piv, W, xp, flist, ds.n,
                                                                         nrhs, nc, max_nf, transpose);
  } else if (warp_cols_fit<T>(max_nf, nrhs)) {
    set_func_attr((const void*)k_solve_bwd_dense_wc<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWarpColSmem);
    const size_t smem = (size_t)WC_WARPS * max_nf * sizeof(T);
    k_solve_bwd_dense_wc<T><<<dim3(nfr, (nrhs + WC_WARPS - 1) / WC_WARPS), 256, smem, s>>>(
        ds.fronts, arena, piv, W, xp, flist, ds.n, nrhs, max_nf, transpose);
  } else {
    k_solve_bwd_dense<T><<<dim3(nfr, std::min(nrhs, 64)), 256, 0, s>>>(ds.fronts, arena, piv, W, xp, flist, ds.n,
                                                                      nrhs, transpose);
  }
  count_launch();
}

template struct Kern<double>;
template struct Kern<float>;

// ===========================================================================
// FP64 outer-iteration kernels
// ===========================================================================
__global__ void k_spmv(const int* __restrict__ rowptr, const int* __restrict__ colind,
                       const int* __restrict__ tpos, const double* __restrict__ val,
                       const double* __restrict__ x, long long ldx, double* __restrict__ y,
                       long long ldy, const double* __restrict__ b, long long ldb, int n, int nrhs,
                       int transpose) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long tot = (long long)n * nrhs;
  for (; t < tot; t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t % n), j = (int)(t / n);
    double s = 0.0;
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
      double a = transpose ? val[tpos[p]] : val[p];
      s += a * x[colind[p] + j * ldx];
    }
    y[i + j * ldy] = b ? b[i + j * ldb] - s : s;
  }
}

// out[p] = -sum_c lambda[row(p) + c ld] x[col(p) + c ld] over the natural
// CSR pattern: the gradient of L(x(A)) with respect to the stored entries of
// A, given x = A^-1 b and lambda = A^-T dL/dx.  One thread per row.
__global__ void k_pattern_grad(const int* __restrict__ rowptr, const int* __restrict__ colind,
                               const double* __restrict__ lam, const double* __restrict__ x, long long ld,
                               int n, int nrhs, double* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
      const int j = colind[p];
      double s = 0.0;
      for (int c = 0; c < nrhs; ++c) s += lam[i + c * ld] * x[j + c * ld];
      out[p] = -s;
    }
  }
}

void pattern_grad(const DevSym& ds, const double* lam, const double* x, long long ld, int nrhs, double* out,
                  cudaStream_t s) {
  k_pattern_grad<<<grid_for(ds.n), 256, 0, s>>>(ds.rowptr, ds.colind, lam, x, ld, ds.n, nrhs, out);
  count_launch();
}

void spmv(const DevSym& ds, const double* values, const double* x, double* y, int nrhs,
          int transpose, cudaStream_t s) {
  k_spmv<<<grid_for((long long)ds.n * nrhs), 256, 0, s>>>(ds.rowptr, ds.colind, ds.tpos, values, x,
                                                          ds.n, y, ds.n, nullptr, 0, ds.n, nrhs,
                                                          transpose);
  count_launch();
}

void residual(const DevSym& ds, const double* values, const double* b, long long ldb,
              const double* x, double* r, int nrhs, int transpose, cudaStream_t s) {
  k_spmv<<<grid_for((long long)ds.n * nrhs), 256, 0, s>>>(ds.rowptr, ds.colind, ds.tpos, values, x,
                                                          ds.n, r, ds.n, b, ldb, ds.n, nrhs,
                                                          transpose);
  count_launch();
}

// deterministic dots: grid (64, nrhs) partial sums, then one block per column
__global__ void k_dot_partial(const double* __restrict__ x, const double* __restrict__ y, int n,
                              double* __restrict__ partial) {
  __shared__ double sh[33];
  const int j = blockIdx.y;
  const double* xj = x + (long long)j * n;
  const double* yj = y + (long long)j * n;
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    s += xj[i] * yj[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) partial[blockIdx.x + j * gridDim.x] = s;
}

__global__ void k_dot_final(const double* __restrict__ partial, int np, double* __restrict__ out,
                            long long ostride) {
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < np; ++i) s += partial[i + blockIdx.x * np];
    out[blockIdx.x * ostride] = s;
  }
}

void dots(const double* x, const double* y, int n, int nrhs, double* partial, double* out,
          long long ostride, cudaStream_t s) {
  dim3 g(64, nrhs);
  k_dot_partial<<<g, 256, 0, s>>>(x, y, n, partial);
  k_dot_final<<<nrhs, 32, 0, s>>>(partial, 64, out, ostride);
  count_launch(2);
}

// Squared 2-norms of the row segments [off[g], off[g+1]) of every column:
// one CTA per (segment, column), deterministic block sums.
__global__ void k_seg_norm2(const double* __restrict__ x, int n, const int* __restrict__ off, int nseg,
                            double* __restrict__ out) {
  __shared__ double sh[33];
  const int g = blockIdx.x, j = blockIdx.y;
  const double* xj = x + (long long)j * n;
  double s = 0.0;
  for (int i = off[g] + threadIdx.x; i < off[g + 1]; i += blockDim.x) {
    const double v = xj[i];
    s += v * v;
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) out[g + (long long)nseg * j] = s;
}

void seg_norms2(const double* x, int n, int nrhs, const int* off, int nseg, double* out, cudaStream_t s) {
  if (nseg <= 0 || nrhs <= 0) return;
  k_seg_norm2<<<dim3(nseg, nrhs), 256, 0, s>>>(x, n, off, nseg, out);
  count_launch();
}

__global__ void k_sqrt_dev(double* a, long long astride, int nrhs) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < nrhs) a[c * astride] = sqrt(a[c * astride]);
}

void sqrt_dev(double* a, long long astride, int nrhs, cudaStream_t s) {
  k_sqrt_dev<<<(nrhs + 63) / 64, 64, 0, s>>>(a, astride, nrhs);
  count_launch();
}

__global__ void k_axpy_dev(double* __restrict__ y, const double* __restrict__ x,
                           const double* __restrict__ a, long long astride, double sgn, int n,
                           int nrhs, const int* __restrict__ active) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long tot = (long long)n * nrhs;
  for (; t < tot; t += (long long)gridDim.x * blockDim.x) {
    int j = (int)(t / n);
    if (active && !active[j]) continue;
    y[t] += sgn * a[j * astride] * x[t];
  }
}

void axpy_dev(double* y, const double* x, const double* a, long long astride, double alpha_sign,
              int n, int nrhs, const int* active, cudaStream_t s) {
  k_axpy_dev<<<grid_for((long long)n * nrhs), 256, 0, s>>>(y, x, a, astride, alpha_sign, n, nrhs,
                                                           active);
  count_launch();
}

__global__ void k_scale_dev(double* __restrict__ y, const double* __restrict__ x,
                            const double* __restrict__ a, long long astride, int n, int nrhs) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long tot = (long long)n * nrhs;
  for (; t < tot; t += (long long)gridDim.x * blockDim.x) {
    int j = (int)(t / n);
    double d = a[j * astride];
    y[t] = d != 0.0 ? x[t] / d : 0.0;
  }
}

void scale_dev(double* y, const double* x, const double* a, long long astride, int n, int nrhs,
               cudaStream_t s) {
  k_scale_dev<<<grid_for((long long)n * nrhs), 256, 0, s>>>(y, x, a, astride, n, nrhs);
  count_launch();
}

__global__ void k_copy_cols(double* __restrict__ y, long long ldy, const double* __restrict__ x,
                            long long ldx, int n, int nrhs) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long tot = (long long)n * nrhs;
  for (; t < tot; t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t % n), j = (int)(t / n);
    y[i + j * ldy] = x[i + j * ldx];
  }
}

void copy_cols(double* y, long long ldy, const double* x, long long ldx, int n, int nrhs,
               cudaStream_t s) {
  k_copy_cols<<<grid_for((long long)n * nrhs), 256, 0, s>>>(y, ldy, x, ldx, n, nrhs);
  count_launch();
}

__global__ void k_add_cols(double* __restrict__ y, const double* __restrict__ x, int n, int nrhs,
                           const int* __restrict__ active) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long tot = (long long)n * nrhs;
  for (; t < tot; t += (long long)gridDim.x * blockDim.x) {
    int j = (int)(t / n);
    if (active && !active[j]) continue;
    y[t] += x[t];
  }
}

void add_cols(double* y, const double* x, int n, int nrhs, const int* active, cudaStream_t s) {
  k_add_cols<<<grid_for((long long)n * nrhs), 256, 0, s>>>(y, x, n, nrhs, active);
  count_launch();
}

// H(i, j, c) at H[i + (m + 1) * (j + m * c)]
__global__ void k_givens(double* H, double* cs, double* sn, double* g, int m, int j, int nrhs,
                         const int* active) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nrhs || (active && !active[c])) return;
  double* h = H + (long long)(m + 1) * (j + (long long)m * c);
  double* csc = cs + (long long)m * c;
  double* snc = sn + (long long)m * c;
  double* gc = g + (long long)(m + 1) * c;
  for (int i = 0; i < j; ++i) {
    double t = csc[i] * h[i] + snc[i] * h[i + 1];
    h[i + 1] = -snc[i] * h[i] + csc[i] * h[i + 1];
    h[i] = t;
  }
  double den = hypot(h[j], h[j + 1]);
  double cj = den != 0.0 ? h[j] / den : 1.0;
  double sj = den != 0.0 ? h[j + 1] / den : 0.0;
  csc[j] = cj;
  snc[j] = sj;
  h[j] = den;
  h[j + 1] = 0.0;
  gc[j + 1] = -sj * gc[j];
  gc[j] = cj * gc[j];
}

void givens_step(double* H, double* cs, double* sn, double* g, int m, int j, int nrhs,
                 const int* active, cudaStream_t s) {
  k_givens<<<(nrhs + 63) / 64, 64, 0, s>>>(H, cs, sn, g, m, j, nrhs, active);
  count_launch();
}

__global__ void k_hess_solve(const double* H, const double* g, double* y, int m, int j, int nrhs,
                             const int* active) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nrhs || (active && !active[c])) return;
  const double* Hc = H + (long long)(m + 1) * m * c;
  const double* gc = g + (long long)(m + 1) * c;
  double* yc = y + (long long)m * c;
  for (int i = j - 1; i >= 0; --i) {
    double s = gc[i];
    for (int k = i + 1; k < j; ++k) s -= Hc[i + (m + 1) * k] * yc[k];
    double d = Hc[i + (m + 1) * i];
    yc[i] = d != 0.0 ? s / d : 0.0;
  }
}

void hess_solve(const double* H, const double* g, double* y, int m, int j, int nrhs,
                const int* active, cudaStream_t s) {
  k_hess_solve<<<(nrhs + 63) / 64, 64, 0, s>>>(H, g, y, m, j, nrhs, active);
  count_launch();
}

__global__ void k_update_x(double* __restrict__ X, const double* __restrict__ Z, long long zstride,
                           const double* __restrict__ y, int m, int j, int n, int nrhs,
                           const int* __restrict__ active) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long tot = (long long)n * nrhs;
  for (; t < tot; t += (long long)gridDim.x * blockDim.x) {
    int c = (int)(t / n);
    if (active && !active[c]) continue;
    double s = 0.0;
    for (int i = 0; i < j; ++i) s += Z[t + i * zstride] * y[i + (long long)m * c];
    X[t] += s;
  }
}

void update_x(double* X, const double* Z, long long zstride, const double* y, int m, int j, int n,
              int nrhs, const int* active, cudaStream_t s) {
  k_update_x<<<grid_for((long long)n * nrhs), 256, 0, s>>>(X, Z, zstride, y, m, j, n, nrhs, active);
  count_launch();
}

}  // namespace hssmf
