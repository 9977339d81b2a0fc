// Kernels of the HSS frontal matrices (Sections 2.2, 2.3, 4.3-4.5).
#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <type_traits>

#include "hss_kernels.h"
#include "id_common.cuh"

namespace hssmf {

namespace {

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_sumf(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T wsum(T v);
template <>
__device__ __forceinline__ double wsum<double>(double v) { return warp_sum(v); }
template <>
__device__ __forceinline__ float wsum<float>(float v) { return warp_sumf(v); }


// block-wide sum in T, result in every thread (sh: 32 T)
template <typename T>
__device__ T block_sum_t(T v, T* sh) {
  v = wsum<T>(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  T s = T(0);
  for (int w = 0; w < nw; ++w) s += sh[w];
  __syncthreads();
  return s;
}

// One warp applies H = I - tau v v^T (v[i] = 1) to nc <= 4 columns at once:
// the loads and the shuffle reductions of the columns are independent and
// interleave, which hides the latency of each.  nn[c] receives the squared
// norm of rows i+1..d-1 of column c after the update (all lanes).
// (All arithmetic is in T: FP64 runs at a small fraction of the FP32 rate on
// this GPU, so the FP32 form keeps FP64 for the per-step rank decision only.)
template <typename T>
__device__ __forceinline__ void warp_reflect4(T* w0, T* w1, T* w2, T* w3, int nc, const T* v,
                                              int i, int d, T tau, int lane, T* nn) {
  T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
  for (int r = i + lane; r < d; r += 32) {
    const T vr = v[r];
    s0 += vr * w0[r];
    s1 += vr * w1[r];
    s2 += vr * w2[r];
    s3 += vr * w3[r];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    s3 += __shfl_xor_sync(0xffffffffu, s3, o);
  }
  const T f0 = tau * s0, f1 = tau * s1, f2 = tau * s2, f3 = tau * s3;
  T p0 = T(0), p1 = T(0), p2 = T(0), p3 = T(0);
  for (int r = i + lane; r < d; r += 32) {
    const T vr = v[r];
    const T x0 = w0[r] - f0 * vr, x1 = w1[r] - f1 * vr, x2 = w2[r] - f2 * vr, x3 = w3[r] - f3 * vr;
    w0[r] = x0;
    if (nc > 1) w1[r] = x1;
    if (nc > 2) w2[r] = x2;
    if (nc > 3) w3[r] = x3;
    if (r > i) {
      p0 += x0 * x0;
      p1 += x1 * x1;
      p2 += x2 * x2;
      p3 += x3 * x3;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    p0 += __shfl_xor_sync(0xffffffffu, p0, o);
    p1 += __shfl_xor_sync(0xffffffffu, p1, o);
    p2 += __shfl_xor_sync(0xffffffffu, p2, o);
    p3 += __shfl_xor_sync(0xffffffffu, p3, o);
  }
  nn[0] = p0;
  nn[1] = p1;
  nn[2] = p2;
  nn[3] = p3;
}

// The same with the reflector unscaled: v holds the raw pivot column on rows
// > i, vi replaces row i, and tau is tau / vi^2 (H = I - tau v v^T is
// unchanged).  Row i of every column is updated as well.
template <typename T>
__device__ __forceinline__ void warp_reflect4v(T* w0, T* w1, T* w2, T* w3, int nc, const T* v, T vi,
                                               int i, int d, T tau, int lane, T* nn) {
  T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
  for (int r = i + lane; r < d; r += 32) {
    const T vr = r == i ? vi : v[r];
    s0 += vr * w0[r];
    s1 += vr * w1[r];
    s2 += vr * w2[r];
    s3 += vr * w3[r];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    s3 += __shfl_xor_sync(0xffffffffu, s3, o);
  }
  const T f0 = tau * s0, f1 = tau * s1, f2 = tau * s2, f3 = tau * s3;
  T p0 = T(0), p1 = T(0), p2 = T(0), p3 = T(0);
  for (int r = i + lane; r < d; r += 32) {
    const T vr = r == i ? vi : v[r];
    const T x0 = w0[r] - f0 * vr, x1 = w1[r] - f1 * vr, x2 = w2[r] - f2 * vr, x3 = w3[r] - f3 * vr;
    w0[r] = x0;
    if (nc > 1) w1[r] = x1;
    if (nc > 2) w2[r] = x2;
    if (nc > 3) w3[r] = x3;
    if (r > i) {
      p0 += x0 * x0;
      p1 += x1 * x1;
      p2 += x2 * x2;
      p3 += x3 * x3;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    p0 += __shfl_xor_sync(0xffffffffu, p0, o);
    p1 += __shfl_xor_sync(0xffffffffu, p1, o);
    p2 += __shfl_xor_sync(0xffffffffu, p2, o);
    p3 += __shfl_xor_sync(0xffffffffu, p3, o);
  }
  nn[0] = p0;
  nn[1] = p1;
  nn[2] = p2;
  nn[3] = p3;
}

// eps^2 |R_11|^2 in FP64, rounded down to T: for every T value b,
// b > id_threshold(eps, r11sq) iff b > eps^2 r11sq exactly.
template <typename T>
__device__ __forceinline__ T id_threshold(double eps, T r11sq);
template <>
__device__ __forceinline__ float id_threshold<float>(double eps, float r11sq) {
  return __double2float_rd(eps * eps * (double)fmaxf(r11sq, 0.f));
}
template <>
__device__ __forceinline__ double id_threshold<double>(double eps, double r11sq) {
  return eps * eps * fmax(r11sq, 0.0);
}

// The per-step decision of the column-pivoted QR, taken by one thread in
// FP64: pivot norm from the largest remaining squared norm, |R_11| at the
// first step, and the rank rule |R_{i+1,i+1}| <= eps |R_11| (stop also when
// R_11 = 0).  Returns 1 to stop.
__device__ __forceinline__ int id_decide(double best, int i, double eps, double* r11, double* nrm) {
  *nrm = sqrt(fmax(best, 0.0));
  if (i == 0) {
    *r11 = *nrm;
    return !(*nrm > 0.0);
  }
  return !(*nrm > eps * *r11);
}

// Philox4x32-10 (Salmon et al., SC'11): ten rounds, Weyl key schedule.
__device__ __forceinline__ void philox4x32_10(unsigned c[4], unsigned k0, unsigned k1) {
  const unsigned M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    unsigned hi0 = __umulhi(M0, c[0]), lo0 = M0 * c[0];
    unsigned hi1 = __umulhi(M1, c[2]), lo1 = M1 * c[2];
    unsigned n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

// G(seed, g, c) = sqrt(-2 ln u1) cos(2 pi u2), u = (x + 0.5) 2^-32, FP64.
__device__ __forceinline__ double gauss(unsigned long long seed, unsigned g, unsigned c) {
  unsigned ctr[4] = {g, c, 0u, 0u};
  philox4x32_10(ctr, (unsigned)(seed & 0xFFFFFFFFull), (unsigned)(seed >> 32));
  const double s = 2.3283064365386963e-10;  // 2^-32
  double u1 = ((double)ctr[0] + 0.5) * s;
  double u2 = ((double)ctr[1] + 0.5) * s;
  return sqrt(-2.0 * log(u1)) * cos(2.0 * 3.141592653589793 * u2);
}

// The FP32 form's sampling matrix: the same Gaussian, evaluated in FP32 from
// the top 24 bits of the two Philox words, rounded to the nearest BF16 value.
// Exactly-BF16 values make the products U R on the tensor cores exact in R;
// the whole FP32 factorization uses these values, so the random sketch stays
// consistent across fronts (eq. Rmerge).
__device__ __forceinline__ float gauss_bf16(unsigned long long seed, unsigned g, unsigned c) {
  unsigned ctr[4] = {g, c, 0u, 0u};
  philox4x32_10(ctr, (unsigned)(seed & 0xFFFFFFFFull), (unsigned)(seed >> 32));
  const float s = 5.9604644775390625e-8f;  // 2^-24
  const float u1 = ((float)(ctr[0] >> 8) + 0.5f) * s;
  const float u2 = ((float)(ctr[1] >> 8) + 0.5f) * s;
  const float v = sqrtf(-2.f * logf(u1)) * cospif(2.f * u2);
  return __bfloat162float(__float2bfloat16_rn(v));
}

template <typename T>
__device__ __forceinline__ T gauss_t(unsigned long long seed, unsigned g, unsigned c);
template <>
__device__ __forceinline__ double gauss_t<double>(unsigned long long seed, unsigned g, unsigned c) {
  return gauss(seed, g, c);
}
template <>
__device__ __forceinline__ float gauss_t<float>(unsigned long long seed, unsigned g, unsigned c) {
  return gauss_bf16(seed, g, c);
}

}  // namespace

// ---------------------------------------------------------------------------
// Gather/transposing copies over 32 x (32 COPY_TN) strips of the destination
// (tile list entries (job, tm, tn): rows 32 tm.., the COPY_TN 32-column tiles
// from tn); transposed sources go through a shared-memory tile
// so that both the reads and the writes are coalesced.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_copy(const CopyJob* __restrict__ jobs, const Tile* __restrict__ tiles) {
  const Tile tl = tiles[blockIdx.x];
  const CopyJob jb = jobs[tl.job];
  __shared__ T tile[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int i0 = tl.tm * 32;
  T* dst = (T*)jb.dst;
  // source element (si, sj) of the concatenated source: its address
  auto src_at = [&](int i, int j) -> const T* {
    const int si = jb.rmap ? jb.rmap[i] : i;
    int sj = jb.cmap ? jb.cmap[j] : j;
    const T* sp = (const T*)jb.src;
    long long lds = jb.lds;
    if (jb.src2 && sj >= jb.split) {
      sp = (const T*)jb.src2;
      lds = jb.lds2;
      sj -= jb.split;
    }
    return jb.src_trans ? sp + sj + (long long)si * lds : sp + si + (long long)sj * lds;
  };
  if (!jb.src_trans) {  // every load of the CTA's COPY_TN tiles issued before the first store
    const int i = i0 + tx;
    T v[COPY_TN][4];
#pragma unroll
    for (int q = 0; q < COPY_TN; ++q)
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int j = (tl.tn + q) * 32 + ty + 8 * u;
        v[q][u] = (i < jb.rows && j < jb.cols) ? *src_at(i, j) : T(0);
      }
#pragma unroll
    for (int q = 0; q < COPY_TN; ++q)
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int j = (tl.tn + q) * 32 + ty + 8 * u;
        if (i < jb.rows && j < jb.cols) dst[i + (long long)j * jb.ldd] = jb.scale_neg ? -v[q][u] : v[q][u];
      }
    return;
  }
  for (int q = 0; q < COPY_TN; ++q) {
    const int j0 = (tl.tn + q) * 32;
    if (j0 >= jb.cols) break;  // uniform in the CTA
    for (int ii = ty; ii < 32; ii += 8) {  // lanes along the source's contiguous index (j)
      const int i = i0 + ii, j = j0 + tx;
      if (i < jb.rows && j < jb.cols) tile[ii][tx] = *src_at(i, j);
    }
    __syncthreads();
    const int i = i0 + tx;
    for (int jj = ty; jj < 32; jj += 8) {
      const int j = j0 + jj;
      if (i < jb.rows && j < jb.cols) {
        const T v = tile[tx][jj];
        dst[i + (long long)j * jb.ldd] = jb.scale_neg ? -v : v;
      }
    }
    __syncthreads();
  }
}

template <typename T>
void HssKern<T>::copy(const CopyJob* jobs, const Tile* tiles, int ntiles, cudaStream_t s) {
  if (ntiles <= 0) return;
  k_copy<T><<<ntiles, 256, 0, s>>>(jobs, tiles);
  count_launch();
}

__global__ void k_int_gather(const IntGatherJob* __restrict__ jobs) {
  const IntGatherJob jb = jobs[blockIdx.x];
  for (int i = threadIdx.x; i < jb.n; i += blockDim.x) {
    int p = jb.idx[i];
    jb.out[i] = p < jb.split ? jb.a[p] : jb.b[p - jb.split];
  }
}

template <typename T>
void HssKern<T>::int_gather(const IntGatherJob* jobs, int njobs, cudaStream_t s) {
  if (njobs <= 0) return;
  k_int_gather<<<njobs, 128, 0, s>>>(jobs);
  count_launch();
}

// ---------------------------------------------------------------------------
// Columns of the random matrix R for a list of global rows (Section 2.2.2,
// Section 4.3: every entry depends only on its global row and column).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_philox(const PhiloxJob* __restrict__ jobs, unsigned long long seed) {
  const PhiloxJob jb = jobs[blockIdx.x];
  const int i = blockIdx.y * blockDim.x + threadIdx.x;
  if (i >= jb.rows) return;
  const unsigned g = (unsigned)jb.gidx[i];
  if constexpr (std::is_same<T, float>::value) {
    if (jb.bf16) {
      __nv_bfloat16* o16 = (__nv_bfloat16*)jb.out;
      for (int c = jb.c0; c < jb.c1; ++c)
        o16[i + (long long)c * jb.ld] = __float2bfloat16_rn(gauss_t<T>(seed, g, (unsigned)c));
      return;
    }
  }
  T* out = (T*)jb.out;
  for (int c = jb.c0; c < jb.c1; ++c) out[i + (long long)c * jb.ld] = gauss_t<T>(seed, g, (unsigned)c);
}

template <typename T>
void HssKern<T>::philox(const PhiloxJob* jobs, int njobs, int max_rows, unsigned long long seed,
                        cudaStream_t s) {
  if (njobs <= 0 || max_rows <= 0) return;
  k_philox<T><<<dim3(njobs, (max_rows + 127) / 128), 128, 0, s>>>(jobs, seed);
  count_launch();
}

// ---------------------------------------------------------------------------
// Original-entry part of the samples (eq. FtimesR): S^r = A_i R, S^c = A_i^T R
// over the local sparse rows of front i; A_i^T uses the transposed entries.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_sample_a(const DFront* __restrict__ fr, const int* __restrict__ ints,
                           const int* __restrict__ tpos, const double* __restrict__ values,
                           const SampleAJob* __restrict__ jobs) {
  const SampleAJob jb = jobs[blockIdx.x];
  const DFront f = fr[jb.front];
  const int r = blockIdx.y * blockDim.x + threadIdx.x;
  if (r >= f.nf) return;
  const int* arow = ints + f.arow_off;
  const int nnz_f = arow[f.nf];
  const int* acol = arow + f.nf + 1;
  const int* aval = acol + nnz_f;
  const T* R = (const T*)jb.R;
  T* Sr = (T*)jb.Sr;
  T* Sc = (T*)jb.Sc;
  const int p0 = arow[r], p1 = arow[r + 1];
  for (int c = jb.c0; c < jb.c1; ++c) {
    T sr = T(0), sc = T(0);
    for (int p = p0; p < p1; ++p) {
      T rv = R[acol[p] + (long long)c * jb.ld];
      sr += T(values[aval[p]]) * rv;
      sc += T(values[tpos[aval[p]]]) * rv;
    }
    Sr[r + (long long)c * jb.ld] = sr;
    Sc[r + (long long)c * jb.ld] = sc;
  }
}

template <typename T>
void HssKern<T>::sample_a(const DevSym& ds, const double* values, const SampleAJob* jobs, int njobs,
                          int max_rows, cudaStream_t s) {
  if (njobs <= 0) return;
  k_sample_a<T><<<dim3(njobs, (max_rows + 127) / 128), 128, 0, s>>>(ds.fronts, ds.ints, ds.tpos,
                                                                    values, jobs);
  count_launch();
}

// ---------------------------------------------------------------------------
// Element extraction from a front (Sections 4.3 and 4.5): entries of A_i plus
// the children's update matrices at their positions.  Grid (job, 16 chunks).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_extract(const DFront* __restrict__ fr, const int* __restrict__ ints,
                          const double* __restrict__ values, const T* __restrict__ ar,
                          const ExtractJob* __restrict__ jobs) {
  const ExtractJob jb = jobs[blockIdx.x];
  const DFront f = fr[jb.front];
  const int* arow = ints + f.arow_off;
  const int nnz_f = arow[f.nf];
  const int* acol = arow + f.nf + 1;
  const int* aval = acol + nnz_f;
  T* out = (T*)jb.out;
  const long long tot = (long long)jb.nr * jb.nc;
  for (long long e = blockIdx.y * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.y * blockDim.x) {
    int i = (int)(e % jb.nr), j = (int)(e / jb.nr);
    int r = jb.rows[i], c = jb.cols[j];
    T v = T(0);
    for (int p = arow[r]; p < arow[r + 1]; ++p)
      if (acol[p] == c) {
        v = T(values[aval[p]]);
        break;
      }
    for (int k = 0; k < f.nchild; ++k) {
      const int* inv = ints + f.inv_off + (long long)k * f.nf;
      int ir = inv[r], ic = inv[c];
      if (ir >= 0 && ic >= 0) {
        const DFront ch = fr[k == 0 ? f.child0 : f.child1];
        v += ar[ch.u_off + ir + (long long)ic * ch.u_ld];
      }
    }
    out[i + (long long)j * jb.ld] = v;
  }
}

template <typename T>
void HssKern<T>::extract(const DevSym& ds, const double* values, const T* arena,
                         const ExtractJob* jobs, int njobs, cudaStream_t s) {
  if (njobs <= 0) return;
  k_extract<T><<<dim3(njobs, 16), 256, 0, s>>>(ds.fronts, ds.ints, values, arena, jobs);
  count_launch();
}

// ---------------------------------------------------------------------------
// Interpolative decomposition by column-pivoted Householder QR (Section 2.2;
// rank rule of Section 5.3).  One CTA per job.  Y (d x m) is copied to W;
// column norms (sums in T: FP64 for the FP64 form, FP32 for the FP32 form)
// are recomputed from the trailing rows after every step; the pivot is the
// first column of largest norm; the rank is the first i with
// |R_{i+1,i+1}| <= eps |R_11| (in the FP32 form compared against a
// threshold formed in FP64, id_threshold).  Then X = R1^-1 R2 by back
// substitution, one warp per column.
// ---------------------------------------------------------------------------
// Threads per CTA (measured on GB300): 512 with two CTAs per SM for the
// one-CTA kernel (many small nodes), 1024 for the cluster kernel (few large
// nodes, whose per-step work is latency-bound and splits over more warps).
constexpr int ID_THREADS = 512;
constexpr int IDC_THREADS = 1024;

template <typename T>
__global__ void __launch_bounds__(ID_THREADS, 2) k_cpqr_id(const IdJob* __restrict__ jobs, double eps) {
  const IdJob jb = jobs[blockIdx.x];
  const int d = jb.d, m = jb.m;
  const long long ld = d;
  const T* Y = (const T*)jb.Y;
  T* W = (T*)jb.W;
  extern __shared__ double smem[];
  T* cn = (T*)smem;                  // m column norms^2
  T* vsh = (T*)(smem + m);           // d: Householder vector of the step
  int* perm = (int*)(smem + m + d);  // m
  __shared__ T s_bv[ID_THREADS / 32];
  __shared__ int s_bi[ID_THREADS / 32];
  __shared__ T s_nrm;
  __shared__ int s_bidx, s_stop;
  __shared__ double s_r11;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = wid; j < m; j += nw) {
    T sp = T(0);
    for (int r = lane; r < d; r += 32) {
      T v = Y[r + j * ld];
      W[r + j * ld] = v;
      sp += v * v;
    }
    sp = wsum<T>(sp);
    if (lane == 0) {
      cn[j] = sp;
      perm[j] = j;
    }
  }
  __syncthreads();
  const int kmax = min(d, m);
  int k = kmax;
  for (int i = 0; i < kmax; ++i) {
    T bv = T(-1);
    int bi = m;
    for (int j = i + threadIdx.x; j < m; j += blockDim.x) {
      const T v = cn[j];
      if (v > bv) { bv = v; bi = j; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const T ov = __shfl_down_sync(0xffffffffu, bv, o);
      const int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    if (lane == 0) { s_bv[wid] = bv; s_bi[wid] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {  // the only FP64 work of the step
      T b = s_bv[0];
      int ix = s_bi[0];
      for (int w = 1; w < nw; ++w)
        if (s_bv[w] > b || (s_bv[w] == b && s_bi[w] < ix)) { b = s_bv[w]; ix = s_bi[w]; }
      double r11 = s_r11, nrm;
      s_stop = id_decide((double)b, i, eps, &r11, &nrm);
      s_r11 = r11;
      s_nrm = T(nrm);
      s_bidx = ix;
    }
    __syncthreads();
    const int p = s_bidx;
    if (s_stop) {
      k = i;
      break;
    }
    if (p != i) {
      for (int r = threadIdx.x; r < d; r += blockDim.x) {
        T t = W[r + i * ld];
        W[r + i * ld] = W[r + p * ld];
        W[r + p * ld] = t;
      }
      if (threadIdx.x == 0) {
        T t = cn[i]; cn[i] = cn[p]; cn[p] = t;
        int q = perm[i]; perm[i] = perm[p]; perm[p] = q;
      }
    }
    __syncthreads();
    const T nrm = s_nrm;
    const T alpha = W[i + i * ld];
    const T beta = alpha >= T(0) ? T(-nrm) : T(nrm);
    const T tau = (beta - alpha) / beta;
    const T scl = T(1) / (alpha - beta);
    for (int r = i + 1 + threadIdx.x; r < d; r += blockDim.x) vsh[r] = W[r + i * ld] * scl;
    if (threadIdx.x == 0) vsh[i] = T(1);
    __syncthreads();
    for (int j0 = i + 1 + 4 * wid; j0 < m; j0 += 4 * nw) {  // 4 columns per warp
      const int nc = min(4, m - j0);
      T* w0 = W + j0 * ld;
      T* w1 = nc > 1 ? w0 + ld : w0;
      T* w2 = nc > 2 ? w0 + 2 * ld : w0;
      T* w3 = nc > 3 ? w0 + 3 * ld : w0;
      T nn[4];
      warp_reflect4<T>(w0, w1, w2, w3, nc, vsh, i, d, tau, lane, nn);
      if (lane < nc) cn[j0 + lane] = lane == 0 ? nn[0] : lane == 1 ? nn[1] : lane == 2 ? nn[2] : nn[3];
    }
    __syncthreads();
    if (threadIdx.x == 0) W[i + i * ld] = beta;
    __syncthreads();
  }
  // X = R1^-1 R2 (k x (m - k), ld k): back substitution in place on rows
  // 0..k-1 of the non-skeleton columns, 4 per warp, then copied out
  T* X = (T*)jb.X;
  for (int j0 = k + 4 * wid; j0 < m; j0 += 4 * nw) {
    const int nc = min(4, m - j0);
    T* b0 = W + j0 * ld;
    T* b1 = nc > 1 ? b0 + ld : b0;
    T* b2 = nc > 2 ? b0 + 2 * ld : b0;
    T* b3 = nc > 3 ? b0 + 3 * ld : b0;
    warp_backsub4<T>(b0, b1, b2, b3, nc, k, [&](int c) { return (const T*)(W + c * ld); },
                     [&](int c) { return W[c + c * ld]; }, lane);
    for (int q = 0; q < nc; ++q)
      for (int r = lane; r < k; r += 32) X[r + (long long)(j0 - k + q) * k] = W[r + (j0 + q) * ld];
  }
  for (int j = threadIdx.x; j < m; j += blockDim.x) jb.piv[j] = perm[j];
  if (threadIdx.x == 0) *jb.rank = k;
}

template <typename T>
int HssKern<T>::batched_id(const IdJob* jobs, int njobs, int max_m, int max_d, double eps,
                           cudaStream_t s) {
  if (njobs <= 0) return 0;
  // m norms (double), d vector entries (double), m pivots (int)
  const size_t smem = 12 * (size_t)std::max(max_m, 1) + 8 * (size_t)std::max(max_d, 1);
  if (smem > 200 * 1024) return -1;
  if (!set_func_attr((const void*)k_cpqr_id<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024)) return -1;
  k_cpqr_id<T><<<njobs, ID_THREADS, smem, s>>>(jobs, eps);
  count_launch();
  return 0;
}

// ---------------------------------------------------------------------------
// The same ID for large nodes on a thread-block cluster of ID_CL CTAs (one
// cluster per job).  CTA r of the cluster owns the columns j = r (mod ID_CL)
// of W (global memory, L2-resident).  Per step: every CTA proposes its
// largest remaining column norm; the cluster reduces the proposals through
// distributed shared memory (largest norm, then smallest column index);
// every CTA rebuilds the Householder vector from the pivot column and applies
// it to its own columns, recomputing their norms from the trailing rows.
// Columns are not moved: the pivot order is recorded, the skeleton columns
// come first in piv and the others follow in increasing index, and X = R1^-1
// R2 is laid out in that order (the basis Pi [I; X^T] does not depend on the
// order of the non-skeleton columns).
// ---------------------------------------------------------------------------
template <typename T, int ID_CL>
__global__ void __launch_bounds__(IDC_THREADS, 1) k_cpqr_id_cluster(const IdJob* __restrict__ jobs,
                                                                double eps, double* rdiag_all,
                                                                int* order_all, int max_m, int max_k) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int jid = blockIdx.x / ID_CL;
  const IdJob jb = jobs[jid];
  const int d = jb.d, m = jb.m;
  const long long ld = d;
  const T* Y = (const T*)jb.Y;
  T* W = (T*)jb.W;
  double* rdiag = rdiag_all + (long long)jid * max_k;  // |R| diagonal, by step
  int* order = order_all + (long long)jid * max_m;     // pivot column of each step
  extern __shared__ double smem[];
  const int mo = (m - rank + ID_CL - 1) / ID_CL;  // columns owned by this CTA: rank + ID_CL * l
  T* cn = (T*)smem;                                        // mo norms^2 (negative: pivoted)
  T* v = (T*)(smem + mo);                                  // d: Householder vector of the step
  unsigned char* skel = (unsigned char*)(smem + mo + d);   // m flags, replicated in every CTA
  __shared__ T s_bv[IDC_THREADS / 32];
  __shared__ int s_bi[IDC_THREADS / 32];
  __shared__ T s_cand_v;
  __shared__ int s_cand_i;
  __shared__ T s_nrm;
  __shared__ int s_p, s_stop;
  __shared__ double s_r11;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int l = wid; l < mo; l += nw) {
    const int j = rank + ID_CL * l;
    T sp = T(0);
    for (int r = lane; r < d; r += 32) {
      T x = Y[r + j * ld];
      W[r + j * ld] = x;
      sp += x * x;
    }
    sp = wsum<T>(sp);
    if (lane == 0) cn[l] = sp;
  }
  for (int j = threadIdx.x; j < m; j += blockDim.x) skel[j] = 0;
  __syncthreads();
  const int kmax = min(d, m);
  int k = kmax;
  for (int i = 0; i < kmax; ++i) {
    // local proposal: largest norm among the owned, unpivoted columns
    T bv = T(-1);
    int bi = m;
    for (int l = threadIdx.x; l < mo; l += blockDim.x) {
      const T x = cn[l];
      if (x > bv) { bv = x; bi = rank + ID_CL * l; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const T ov = __shfl_down_sync(0xffffffffu, bv, o);
      const int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    if (lane == 0) { s_bv[wid] = bv; s_bi[wid] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
      T b = s_bv[0];
      int ix = s_bi[0];
      for (int w = 1; w < nw; ++w)
        if (s_bv[w] > b || (s_bv[w] == b && s_bi[w] < ix)) { b = s_bv[w]; ix = s_bi[w]; }
      s_cand_v = b;
      s_cand_i = ix;
    }
    cluster.sync();
    if (wid == 0) {  // every CTA reduces the same proposals (lane r reads CTA r)
      T b = T(-1);
      int ix = m;
      if (lane < ID_CL) {
        b = *cluster.map_shared_rank(&s_cand_v, lane);
        ix = *cluster.map_shared_rank(&s_cand_i, lane);
      }
      for (int o = 16; o > 0; o >>= 1) {
        const T ov = __shfl_xor_sync(0xffffffffu, b, o);
        const int oi = __shfl_xor_sync(0xffffffffu, ix, o);
        if (ov > b || (ov == b && oi < ix)) { b = ov; ix = oi; }
      }
      if (lane == 0) {  // identical in every CTA: same inputs, same FP64 decision
        double r11 = s_r11, nrm;
        s_stop = id_decide((double)b, i, eps, &r11, &nrm) || ix >= m;
        s_r11 = r11;
        s_nrm = T(nrm);
        s_p = ix;
      }
    }
    __syncthreads();
    const int p = s_p;
    if (s_stop) {
      k = i;
      break;
    }
    const T nrm = s_nrm;
    // Householder vector of the pivot column, rows i..d-1
    const T alpha = W[i + p * ld];
    const T beta = alpha >= T(0) ? T(-nrm) : T(nrm);
    const T tau = (beta - alpha) / beta;
    const T scl = T(1) / (alpha - beta);
    for (int r = i + 1 + threadIdx.x; r < d; r += blockDim.x) v[r] = W[r + p * ld] * scl;
    if (threadIdx.x == 0) {
      v[i] = T(1);
      skel[p] = 1;
      if (rank == 0) {
        rdiag[i] = (double)beta;
        order[i] = p;
      }
    }
    if (p % ID_CL == rank && threadIdx.x == 0) cn[p / ID_CL] = T(-1);
    __syncthreads();
    // apply to the owned unpivoted columns; recompute their norms
    for (int g = wid; 4 * g < mo; g += nw) {  // up to 4 owned, unpivoted columns per warp
      int ls[4];
      int nc = 0;
      for (int q = 0; q < 4; ++q) {
        const int l = 4 * g + q;
        if (l < mo && !skel[rank + ID_CL * l]) ls[nc++] = l;
      }
      if (nc == 0) continue;
      for (int q = nc; q < 4; ++q) ls[q] = ls[0];
      T* w0 = W + (rank + ID_CL * ls[0]) * ld;
      T* w1 = W + (rank + ID_CL * ls[1]) * ld;
      T* w2 = W + (rank + ID_CL * ls[2]) * ld;
      T* w3 = W + (rank + ID_CL * ls[3]) * ld;
      T nn[4];
      warp_reflect4<T>(w0, w1, w2, w3, nc, v, i, d, tau, lane, nn);
      if (lane < nc) cn[ls[lane]] = lane == 0 ? nn[0] : lane == 1 ? nn[1] : lane == 2 ? nn[2] : nn[3];
    }
    cluster.sync();  // every column updated before the next proposals
  }
  // No CTA leaves while a peer may still read its proposal; also publishes
  // every column update and rdiag/order to the whole cluster.
  cluster.sync();
  // X = R1^-1 R2, one warp per owned non-skeleton column; R1(r, c) = W[r, order[c]],
  // R1(r, r) = rdiag[r] (written by CTA 0 before the last cluster barrier)
  const double* rd = rdiag;
  T* X = (T*)jb.X;
  for (int g = wid; 4 * g < mo; g += nw) {  // up to 4 owned non-skeleton columns per warp
    int ls[4];
    int nc = 0;
    for (int q = 0; q < 4; ++q) {
      const int l = 4 * g + q;
      if (l < mo && !skel[rank + ID_CL * l]) ls[nc++] = l;
    }
    if (nc == 0) continue;
    for (int q = nc; q < 4; ++q) ls[q] = ls[0];
    T* b0 = W + (rank + ID_CL * ls[0]) * ld;
    T* b1 = W + (rank + ID_CL * ls[1]) * ld;
    T* b2 = W + (rank + ID_CL * ls[2]) * ld;
    T* b3 = W + (rank + ID_CL * ls[3]) * ld;
    warp_backsub4<T>(b0, b1, b2, b3, nc, k, [&](int c) { return (const T*)(W + (long long)order[c] * ld); },
                     [&](int c) { return T(rd[c]); }, lane);
    for (int q = 0; q < nc; ++q) {
      const int j = rank + ID_CL * ls[q];
      int pos = 0;  // number of non-skeleton columns before j
      for (int c = lane; c < j; c += 32) pos += skel[c] ? 0 : 1;
      for (int o = 16; o > 0; o >>= 1) pos += __shfl_xor_sync(0xffffffffu, pos, o);
      for (int r = lane; r < k; r += 32) X[r + (long long)pos * k] = W[r + j * ld];
      if (lane == 0) jb.piv[k + pos] = j;
    }
  }
  if (rank == 0) {
    for (int i = threadIdx.x; i < k; i += blockDim.x) jb.piv[i] = order[i];
    if (threadIdx.x == 0) *jb.rank = k;
  }
}

template <typename T, int CL>
static int launch_id_cluster(const IdJob* jobs, int njobs, int max_m, int max_d, double eps,
                             double* rdiag, int* order, cudaStream_t s) {
  const size_t smem = sizeof(double) * ((size_t)max_m / CL + 1 + (size_t)max_d) + (size_t)max_m + 16;
  if (smem > 200 * 1024) return -1;
  if (!set_func_attr((const void*)k_cpqr_id_cluster<T, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024))
    return -1;
  if (CL > 8 && !set_func_attr((const void*)k_cpqr_id_cluster<T, CL>,
                               cudaFuncAttributeNonPortableClusterSizeAllowed, 1))
    return -1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(njobs * CL, 1, 1);
  cfg.blockDim = dim3(IDC_THREADS, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const int max_k = std::max(std::min(max_m, max_d), 1);
  if (cudaLaunchKernelEx(&cfg, k_cpqr_id_cluster<T, CL>, jobs, eps, rdiag, order, std::max(max_m, 1),
                         max_k) != cudaSuccess) {
    cudaGetLastError();
    return -1;  // cluster not schedulable: the caller falls back
  }
  count_launch();
  return 0;
}

template <typename T>
int HssKern<T>::batched_id_cluster(const IdJob* jobs, int njobs, int max_m, int max_d, double eps,
                                   double* rdiag, int* order, cudaStream_t s, int cl) {
  if (njobs <= 0) return 0;
  if (cl >= 16 && launch_id_cluster<T, 16>(jobs, njobs, max_m, max_d, eps, rdiag, order, s) == 0) return 0;
  return launch_id_cluster<T, 8>(jobs, njobs, max_m, max_d, eps, rdiag, order, s);
}

// ---------------------------------------------------------------------------
// The ID with the node's matrix resident in shared memory, spread over a
// cluster of CL CTAs (CL = 1 is a single CTA): CTA r keeps its columns
// j = r (mod CL) in its own shared memory for the whole factorization, so a
// step touches no global memory.  The pivot column is read from its owner
// through distributed shared memory into a local copy of the Householder
// vector.  Same pivot rule, rank rule, outputs and column order as
// k_cpqr_id_cluster.
// ---------------------------------------------------------------------------
constexpr int IDS_THREADS = 1024;
// dynamic shared memory of these kernels: the 227 KB a CTA can opt into,
// less 1 KB for their static shared memory (at most 816 bytes)
constexpr size_t kIdSmemBudget = 226 * 1024;

// column stride of the resident matrix: 16-byte aligned columns
__host__ __device__ inline int id_smem_ld(int d) { return (d + 3) & ~3; }

// shared memory of the ID kernels: the owned columns, the pivot-column
// buffers (one on a single CTA; two and a staging column on a cluster) and
// the skeleton flags
__host__ __device__ inline size_t id_smem_bytes(int d, int m, int cl, int esz) {
  const size_t mo = (size_t)(m + cl - 1) / cl;
  const size_t ld = (size_t)id_smem_ld(d);
  return (size_t)esz * mo * ld + (size_t)(cl > 1 ? 3 : 1) * esz * ld + (size_t)m + 64;
}

// Per step (every CTA of the cluster, 32 warps): the warps' proposals (the
// largest trailing norm among the columns each warp updated in the previous
// step) are reduced to a CTA proposal, exchanged through distributed shared
// memory, and every warp takes the same decision (rank rule compared in T
// against eps^2 |R_11|^2 computed once in FP64 and rounded down, which is
// exact for every T value); every CTA copies the raw pivot column from its
// owner with 16-byte loads, and the warps apply the reflector with the
// Householder scaling folded into tau, recomputing norms and proposals.
template <typename T, int CL, bool OVF>
__global__ void __launch_bounds__(IDS_THREADS, 1) k_cpqr_id_smem(const IdJob* __restrict__ jobs, double eps,
                                                                 double* rdiag_all, int* order_all, int max_m,
                                                                 int max_k, int ms, int fail_p) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = CL > 1 ? (int)cluster.block_rank() : 0;
  const int jid = blockIdx.x / CL;
  const IdJob jb = jobs[jid];
  const int d = jb.d, m = jb.m;
  const int ldw = id_smem_ld(d);
  const T* Y = (const T*)jb.Y;
  T* W = (T*)jb.W;  // owned columns beyond the shared-memory capacity stay here (ld d)
  double* rdiag = rdiag_all + (long long)jid * max_k;
  int* order = order_all + (long long)jid * max_m;
  extern __shared__ __align__(16) unsigned char sraw[];
  const int mo = (m - rank + CL - 1) / CL;  // owned columns rank + CL * l
  const int mo_max = (m + CL - 1) / CL;     // same layout in every CTA of the cluster
  const int msh = min(mo_max, ms);          // local columns 0..msh-1 in shared memory
  T* Wl = (T*)sraw;                          // ldw x msh
  T* v = Wl + (size_t)ldw * msh;             // ldw: raw pivot column of the step
  unsigned char* skel = (unsigned char*)(v + ldw);  // m
  // column l owned by this CTA: shared memory, or global memory past the capacity
  // (OVF: some owned columns live in global memory; otherwise all are shared)
  auto colp = [&](int l) -> T* {
    if (!OVF || l < ms) return Wl + (size_t)l * ldw;
    return W + (size_t)(rank + CL * l) * d;
  };
  __shared__ T s_bv[IDS_THREADS / 32];
  __shared__ int s_bi[IDS_THREADS / 32];
  __shared__ T s_cand_v[2];
  __shared__ int s_cand_i[2];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  {  // copy in, initial norms and proposals
    T bv = T(-1);
    int bi = m;
    for (int g = wid; 4 * g < mo; g += nw) {
      for (int q = 0; q < 4; ++q) {
        const int l = 4 * g + q;
        if (l >= mo) break;
        const int j = rank + CL * l;
        T sp = T(0);
        T* col = colp(l);
        for (int r = lane; r < d; r += 32) {
          const T x = Y[r + (long long)j * d];
          col[r] = x;
          sp += x * x;
        }
        sp = wsum<T>(sp);
        if (sp > bv) { bv = sp; bi = j; }
      }
    }
    if (lane == 0) { s_bv[wid] = bv; s_bi[wid] = bi; }
  }
  for (int j = threadIdx.x; j < m; j += blockDim.x) skel[j] = 0;
  // reduction of the warp proposals to the cluster's pivot (b, p), taken
  // identically by every warp
  auto pivot = [&](int par, T& b, int& p) {
    __syncthreads();
    if (CL == 1) {
      b = s_bv[lane];
      p = s_bi[lane];
    } else {
      if (wid == 0) {
        T c = s_bv[lane];
        int ci = s_bi[lane];
        for (int o = 16; o > 0; o >>= 1) {
          const T ov = __shfl_xor_sync(0xffffffffu, c, o);
          const int oi = __shfl_xor_sync(0xffffffffu, ci, o);
          if (ov > c || (ov == c && oi < ci)) { c = ov; ci = oi; }
        }
        if (lane == 0) { s_cand_v[par] = c; s_cand_i[par] = ci; }
      }
      cluster.sync();
      b = T(-1);
      p = m;
      if (lane < CL) {
        b = *cluster.map_shared_rank(&s_cand_v[par], lane);
        p = *cluster.map_shared_rank(&s_cand_i[par], lane);
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const T ov = __shfl_xor_sync(0xffffffffu, b, o);
      const int oi = __shfl_xor_sync(0xffffffffu, p, o);
      if (ov > b || (ov == b && oi < p)) { b = ov; p = oi; }
    }
  };
  T b;
  int p;
  pivot(0, b, p);
  const T thr = id_threshold<T>(eps, b);  // eps^2 |R_11|^2, rounded down to T
  const int kmax = min(d, m);
  int k = kmax;
  bool doomed = false;
  for (int i = 0; i < kmax; ++i) {
    if (i > 0) pivot(i & 1, b, p);
    const bool stop = (i == 0 ? !(b > T(0)) : !(b > thr)) || p >= m;
    if (stop) {
      k = i;
      break;
    }
    if (fail_p >= 0 && m > d && i >= d - fail_p) {  // the ID fails whatever follows (see k_cpqr_id_push)
      k = i + 1;
      doomed = true;
      break;
    }
    const T nrm = sqrt(b);
    // raw pivot column, rows from the 16-byte boundary at or below i
    const int owner = p % CL, lp = p / CL;
    if (!OVF || lp < ms) {
      const T* pc = Wl + (size_t)lp * ldw;
      if (CL > 1) pc = cluster.map_shared_rank(pc, owner);
      constexpr int E = 16 / sizeof(T);
      const int i0 = i - i % E;
      const int4* src = reinterpret_cast<const int4*>(pc + i0);
      int4* dst = reinterpret_cast<int4*>(v + i0);
      for (int q = threadIdx.x; q < (ldw - i0) / E; q += blockDim.x) dst[q] = src[q];
    } else {  // (global writes of the owner are ordered by the cluster barrier)
      const T* pc = W + (size_t)p * d;
      for (int r = i + threadIdx.x; r < d; r += blockDim.x) v[r] = pc[r];
    }
    if (threadIdx.x == 0) skel[p] = 1;
    __syncthreads();
    const T alpha = v[i];
    const T beta = alpha >= T(0) ? -nrm : nrm;
    const T vi = alpha - beta;           // row i of the unscaled reflector
    const T tau = T(-1) / (beta * vi);   // tau / vi^2
    if (rank == 0 && threadIdx.x == 0) {
      rdiag[i] = (double)beta;
      order[i] = p;
    }
    T bv = T(-1);
    int bi = m;
    for (int g = wid; 4 * g < mo; g += nw) {  // up to 4 owned, unpivoted columns per warp
      int ls[4];
      int nc = 0;
      for (int q = 0; q < 4; ++q) {
        const int l = 4 * g + q;
        if (l < mo && !skel[rank + CL * l]) ls[nc++] = l;
      }
      if (nc == 0) continue;
      for (int q = nc; q < 4; ++q) ls[q] = ls[0];
      T nn[4];
      if (!OVF || ls[nc - 1] < ms)  // all in shared memory: keep the shared-memory addressing visible
        warp_reflect4v<T>(Wl + ls[0] * (size_t)ldw, Wl + ls[1] * (size_t)ldw, Wl + ls[2] * (size_t)ldw,
                          Wl + ls[3] * (size_t)ldw, nc, v, vi, i, d, tau, lane, nn);
      else
        warp_reflect4v<T>(colp(ls[0]), colp(ls[1]), colp(ls[2]), colp(ls[3]), nc, v, vi, i, d, tau, lane, nn);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = rank + CL * ls[q];
        if (q < nc && (nn[q] > bv || (nn[q] == bv && j < bi))) { bv = nn[q]; bi = j; }
      }
    }
    if (lane == 0) { s_bv[wid] = bv; s_bi[wid] = bi; }
  }
  if (CL > 1) cluster.sync(); else __syncthreads();
  // X = R1^-1 R2 on the owned non-skeleton columns, R1 columns read from their owners
  const double* rd = rdiag;
  T* X = (T*)jb.X;
  for (int g = wid; !doomed && 4 * g < mo; g += nw) {
    int ls[4];
    int nc = 0;
    for (int q = 0; q < 4; ++q) {
      const int l = 4 * g + q;
      if (l < mo && !skel[rank + CL * l]) ls[nc++] = l;
    }
    if (nc == 0) continue;
    for (int q = nc; q < 4; ++q) ls[q] = ls[0];
    warp_backsub4<T>(colp(ls[0]), colp(ls[1]), colp(ls[2]), colp(ls[3]), nc, k,
                     [&](int c) {
                       const int pc2 = order[c], l2 = pc2 / CL;
                       if (OVF && l2 >= ms) return (const T*)(W + (size_t)pc2 * d);
                       T* col = Wl + (size_t)l2 * ldw;
                       return (const T*)(CL > 1 ? cluster.map_shared_rank(col, pc2 % CL) : col);
                     },
                     [&](int c) { return T(rd[c]); }, lane);
    for (int q = 0; q < nc; ++q) {
      const int j = rank + CL * ls[q];
      int pos = 0;
      for (int c = lane; c < j; c += 32) pos += skel[c] ? 0 : 1;
      for (int o = 16; o > 0; o >>= 1) pos += __shfl_xor_sync(0xffffffffu, pos, o);
      const T* col = colp(ls[q]);
      for (int r = lane; r < k; r += 32) X[r + (long long)pos * k] = col[r];
      if (lane == 0) jb.piv[k + pos] = j;
    }
  }
  if (rank == 0) {
    for (int i = threadIdx.x; !doomed && i < k; i += blockDim.x) jb.piv[i] = order[i];
    if (threadIdx.x == 0) *jb.rank = k;
  }
  // peers may still read this CTA's R1 columns
  if (CL > 1) cluster.sync();
}

// ---------------------------------------------------------------------------
// The shared-memory ID on a cluster (CL >= 2) without cluster-wide barriers
// in the step loop: every CTA pushes its proposal (norm, column) into a slot
// of every peer's shared memory and arrives on the peer's mbarrier (release
// at cluster scope); the owner of the pivot column broadcasts it with bulk
// asynchronous copies (shared::cta -> shared::cluster) that complete on each
// receiver's mbarrier through its transaction count.  Per step: one CTA
// barrier and two mbarrier waits.  Slots, vectors and barriers alternate by
// step parity; every wait is bounded, a wait that runs out makes the ID
// report rank -1.
// ---------------------------------------------------------------------------
namespace push {
__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint32_t mapa(uint32_t a, int cta) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(cta));
  return r;
}
__device__ __forceinline__ void init(uint32_t bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void arrive_expect(uint32_t bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void arrive_remote(uint32_t rbar) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(rbar) : "memory");
}
__device__ __forceinline__ bool wait(uint32_t bar, uint32_t parity) {
  for (int it = 0; it < (1 << 22); ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}
__device__ __forceinline__ void st(uint32_t a, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}
__device__ __forceinline__ void st(uint32_t a, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(a), "d"(v) : "memory");
}
__device__ __forceinline__ void st(uint32_t a, int v) {
  asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void copy(uint32_t dst, uint32_t src, unsigned bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "r"(src), "r"(bytes), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void fence_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
}  // namespace push

template <typename T, int CL, bool OVF>
__global__ void __launch_bounds__(IDS_THREADS, 1) k_cpqr_id_push(const IdJob* __restrict__ jobs, double eps,
                                                                 double* rdiag_all, int* order_all, int max_m,
                                                                 int max_k, int ms, int fail_p) {
  static_assert(CL >= 2 && CL <= 16, "cluster of 2..16 CTAs");
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int jid = blockIdx.x / CL;
  const IdJob jb = jobs[jid];
  const int d = jb.d, m = jb.m;
  const int ldw = id_smem_ld(d);
  const T* Y = (const T*)jb.Y;
  T* W = (T*)jb.W;
  double* rdiag = rdiag_all + (long long)jid * max_k;
  int* order = order_all + (long long)jid * max_m;
  extern __shared__ __align__(16) unsigned char sraw[];
  const int mo = (m - rank + CL - 1) / CL;
  const int mo_max = (m + CL - 1) / CL;
  const int msh = min(mo_max, ms);
  T* Wl = (T*)sraw;                      // ldw x msh
  T* vbuf = Wl + (size_t)ldw * msh;      // 2 x ldw: pivot column of the step, by parity
  T* vstage = vbuf + 2 * (size_t)ldw;    // ldw: staging of a pivot column kept in global memory
  unsigned char* skel = (unsigned char*)(vstage + ldw);
  __shared__ T s_bv[IDS_THREADS / 32];
  __shared__ int s_bi[IDS_THREADS / 32];
  __shared__ T s_cv[2][16];
  __shared__ int s_cj[2][16];
  __shared__ __align__(8) unsigned long long bar_c[2], bar_v[2];
  __shared__ int s_fail;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  auto colp = [&](int l) -> T* {
    if (!OVF || l < ms) return Wl + (size_t)l * ldw;
    return W + (size_t)(rank + CL * l) * d;
  };
  {
    T bv = T(-1);
    int bi = m;
    for (int g = wid; 4 * g < mo; g += nw) {
      for (int q = 0; q < 4; ++q) {
        const int l = 4 * g + q;
        if (l >= mo) break;
        const int j = rank + CL * l;
        T sp = T(0);
        T* col = colp(l);
        for (int r = lane; r < d; r += 32) {
          const T x = Y[r + (long long)j * d];
          col[r] = x;
          sp += x * x;
        }
        for (int r = d + lane; r < ldw; r += 32) col[r] = T(0);  // (rows past d travel with the column)
        sp = wsum<T>(sp);
        if (sp > bv) { bv = sp; bi = j; }
      }
    }
    if (lane == 0) { s_bv[wid] = bv; s_bi[wid] = bi; }
  }
  for (int j = threadIdx.x; j < m; j += blockDim.x) skel[j] = 0;
  if (threadIdx.x == 0) {
    for (int q = 0; q < 2; ++q) {
      push::init(push::saddr(&bar_c[q]), CL);
      push::init(push::saddr(&bar_v[q]), 1);
    }
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  push::fence_async();
  cluster.sync();  // every CTA's barriers exist before the first push
  constexpr int E = 16 / sizeof(T);
  auto vbytes = [&](int i) { return (unsigned)((ldw - (i - i % E)) * sizeof(T)); };
  // exchange of the proposals of step i; false if a wait ran out
  auto pivot = [&](int i, T& b, int& p) -> bool {
    const int par = i & 1;
    __syncthreads();
    if (s_fail) return false;
    if (wid == 0) {
      T c = s_bv[lane];
      int ci = s_bi[lane];
      for (int o = 16; o > 0; o >>= 1) {
        const T ov = __shfl_xor_sync(0xffffffffu, c, o);
        const int oi = __shfl_xor_sync(0xffffffffu, ci, o);
        if (ov > c || (ov == c && oi < ci)) { c = ov; ci = oi; }
      }
      if (lane == 0) push::arrive_expect(push::saddr(&bar_v[par]), vbytes(i));  // before any pivot column can come
      __syncwarp();
      if (lane < CL) {
        push::st(push::mapa(push::saddr(&s_cv[par][rank]), lane), c);
        push::st(push::mapa(push::saddr(&s_cj[par][rank]), lane), ci);
        push::arrive_remote(push::mapa(push::saddr(&bar_c[par]), lane));
      }
    }
    // a wait that ran out only marks the failure (every thread keeps the same
    // control flow); the CTA stops at the next step's barrier
    if (!push::wait(push::saddr(&bar_c[par]), (i >> 1) & 1)) s_fail = 1;
    b = lane < CL ? s_cv[par][lane] : T(-1);
    p = lane < CL ? s_cj[par][lane] : m;
    for (int o = 16; o > 0; o >>= 1) {
      const T ov = __shfl_xor_sync(0xffffffffu, b, o);
      const int oi = __shfl_xor_sync(0xffffffffu, p, o);
      if (ov > b || (ov == b && oi < p)) { b = ov; p = oi; }
    }
    return true;
  };
  T b;
  int p;
  bool ok = pivot(0, b, p);
  const T thr = id_threshold<T>(eps, b);
  const int kmax = min(d, m);
  int k = kmax;
  bool doomed = false;
  for (int i = 0; i < kmax; ++i) {
    const int par = i & 1;
    if (i > 0) ok = pivot(i, b, p);
    const bool stop = !ok || (i == 0 ? !(b > T(0)) : !(b > thr)) || p >= m;
    if (stop) {
      k = i;
      break;
    }
    // with fail_p >= 0: pivot i takes the rank past d - fail_p and the rank
    // cannot reach m (m > d), so the adaptive scheme rejects the ID whatever
    // follows: stop with rank i + 1 and no X (the same decision in every CTA;
    // the pivot column of step i has not been sent, the last copies landed)
    if (fail_p >= 0 && m > d && i >= d - fail_p) {
      k = i + 1;
      doomed = true;
      break;
    }
    const T nrm = sqrt(b);
    const int owner = p % CL, lp = p / CL;
    const int i0 = i - i % E;
    if (rank == owner) {  // broadcast the raw pivot column, rows from the 16-byte boundary at or below i
      const T* src = Wl + (size_t)lp * ldw + i0;
      if (OVF && lp >= ms) {
        for (int r = i0 + threadIdx.x; r < ldw; r += blockDim.x) vstage[r] = r < d ? W[(size_t)p * d + r] : T(0);
        push::fence_async();
        __syncthreads();
        src = vstage + i0;
      }
      if (threadIdx.x == 0) {
        const uint32_t s0 = push::saddr(src), dv = push::saddr(vbuf + (size_t)par * ldw + i0);
        const uint32_t bv = push::saddr(&bar_v[par]);
        for (int q = 0; q < CL; ++q) push::copy(push::mapa(dv, q), s0, vbytes(i), push::mapa(bv, q));
        if (OVF) {  // vstage is rewritten by a later step only after these reads
          asm volatile("cp.async.bulk.commit_group;" ::: "memory");
          asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
        }
      }
    }
    if (threadIdx.x == 0) skel[p] = 1;  // (seen by every warp after the next CTA barrier)
    if (!push::wait(push::saddr(&bar_v[par]), (i >> 1) & 1)) s_fail = 1;
    const T* v = vbuf + (size_t)par * ldw;
    const T alpha = v[i];
    const T beta = alpha >= T(0) ? -nrm : nrm;
    const T vi = alpha - beta;
    const T tau = T(-1) / (beta * vi);
    if (rank == 0 && threadIdx.x == 0) {
      rdiag[i] = (double)beta;
      order[i] = p;
    }
    T bv = T(-1);
    int bi = m;
    for (int g = wid; 4 * g < mo; g += nw) {
      int ls[4];
      int nc = 0;
      for (int q = 0; q < 4; ++q) {
        const int l = 4 * g + q;
        const int j = rank + CL * l;
        if (l < mo && j != p && !skel[j]) ls[nc++] = l;
      }
      if (nc == 0) continue;
      for (int q = nc; q < 4; ++q) ls[q] = ls[0];
      T nn[4];
      if (!OVF || ls[nc - 1] < ms)
        warp_reflect4v<T>(Wl + ls[0] * (size_t)ldw, Wl + ls[1] * (size_t)ldw, Wl + ls[2] * (size_t)ldw,
                          Wl + ls[3] * (size_t)ldw, nc, v, vi, i, d, tau, lane, nn);
      else
        warp_reflect4v<T>(colp(ls[0]), colp(ls[1]), colp(ls[2]), colp(ls[3]), nc, v, vi, i, d, tau, lane, nn);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = rank + CL * ls[q];
        if (q < nc && (nn[q] > bv || (nn[q] == bv && j < bi))) { bv = nn[q]; bi = j; }
      }
    }
    if (lane == 0) { s_bv[wid] = bv; s_bi[wid] = bi; }
    push::fence_async();  // the updated columns may be sent by a bulk copy next step
  }
  cluster.sync();
  const bool failed = s_fail != 0;
  const double* rd = rdiag;
  T* X = (T*)jb.X;
  for (int g = wid; !failed && !doomed && 4 * g < mo; g += nw) {
    int ls[4];
    int nc = 0;
    for (int q = 0; q < 4; ++q) {
      const int l = 4 * g + q;
      if (l < mo && !skel[rank + CL * l]) ls[nc++] = l;
    }
    if (nc == 0) continue;
    for (int q = nc; q < 4; ++q) ls[q] = ls[0];
    warp_backsub4<T>(colp(ls[0]), colp(ls[1]), colp(ls[2]), colp(ls[3]), nc, k,
                     [&](int c) {
                       const int pc2 = order[c], l2 = pc2 / CL;
                       if (OVF && l2 >= ms) return (const T*)(W + (size_t)pc2 * d);
                       return (const T*)cluster.map_shared_rank(Wl + (size_t)l2 * ldw, pc2 % CL);
                     },
                     [&](int c) { return T(rd[c]); }, lane);
    for (int q = 0; q < nc; ++q) {
      const int j = rank + CL * ls[q];
      int pos = 0;
      for (int c = lane; c < j; c += 32) pos += skel[c] ? 0 : 1;
      for (int o = 16; o > 0; o >>= 1) pos += __shfl_xor_sync(0xffffffffu, pos, o);
      const T* col = colp(ls[q]);
      for (int r = lane; r < k; r += 32) X[r + (long long)pos * k] = col[r];
      if (lane == 0) jb.piv[k + pos] = j;
    }
  }
  if (rank == 0) {
    for (int i = threadIdx.x; !doomed && i < k; i += blockDim.x) jb.piv[i] = order[i];
    if (threadIdx.x == 0) *jb.rank = failed ? -1 : k;
  }
  cluster.sync();  // peers may still read this CTA's R1 columns
}

template <typename T, int CL>
static int launch_id_smem(const IdJob* jobs, int njobs, int max_m, int max_d, double eps, double* rdiag,
                          int* order, int fail_p, cudaStream_t s) {
  // owned columns per CTA kept in shared memory; the rest stay in the job's W
  // (clusters: two pivot-column buffers and a staging column besides)
  const size_t col = sizeof(T) * (size_t)id_smem_ld(max_d);
  const size_t fixed = (CL > 1 ? 3 : 1) * col + (size_t)max_m + 64;
  if (fixed + col > kIdSmemBudget) return -1;
  const int mo_max = (std::max(max_m, 1) + CL - 1) / CL;
  const int ms = (int)std::min<size_t>((size_t)mo_max, (kIdSmemBudget - fixed) / col);
  const size_t smem = fixed + col * (size_t)ms;
  const bool ovf = ms < mo_max;
  void (*kern)(const IdJob*, double, double*, int*, int, int, int, int);
  if constexpr (CL > 1)
    kern = ovf ? k_cpqr_id_push<T, CL, true> : k_cpqr_id_push<T, CL, false>;
  else
    kern = ovf ? k_cpqr_id_smem<T, CL, true> : k_cpqr_id_smem<T, CL, false>;
  if (!set_func_attr((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kIdSmemBudget)) return -1;
  if (CL > 8 && !set_func_attr((const void*)kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) return -1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(njobs * CL, 1, 1);
  cfg.blockDim = dim3(IDS_THREADS, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const int max_k = std::max(std::min(max_m, max_d), 1);
  if (cudaLaunchKernelEx(&cfg, kern, jobs, eps, rdiag, order, std::max(max_m, 1), max_k, ms, fail_p) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  count_launch();
  return 0;
}

template <typename T>
int HssKern<T>::id_smem_cluster_size(int d, int m) {
  for (int cl = 1; cl <= 16; cl *= 2)
    if (id_smem_bytes(d, m, cl, sizeof(T)) <= kIdSmemBudget) return cl;
  return 0;
}

template <typename T>
int HssKern<T>::batched_id_smem(const IdJob* jobs, int njobs, int max_m, int max_d, double eps, double* rdiag,
                                int* order, int cl, cudaStream_t s, int fail_p) {
  if (njobs <= 0) return 0;
  switch (cl) {
    case 1: return launch_id_smem<T, 1>(jobs, njobs, max_m, max_d, eps, rdiag, order, fail_p, s);
    case 2: return launch_id_smem<T, 2>(jobs, njobs, max_m, max_d, eps, rdiag, order, fail_p, s);
    case 4: return launch_id_smem<T, 4>(jobs, njobs, max_m, max_d, eps, rdiag, order, fail_p, s);
    case 8: return launch_id_smem<T, 8>(jobs, njobs, max_m, max_d, eps, rdiag, order, fail_p, s);
    case 16: return launch_id_smem<T, 16>(jobs, njobs, max_m, max_d, eps, rdiag, order, fail_p, s);
    default: return -1;
  }
}

// ---------------------------------------------------------------------------
// The same ID (FP32) with the matrix held in registers, for nodes with
// d <= 32 RPL rows and m <= RR_NW CPW CL columns.  CTA r of a cluster of CL
// owns the columns j = r (mod CL); warp w owns local columns w + RR_NW c
// (c < CPW) and lane l holds rows l + 32 s (s < RPL) of each of them, so the
// per-step Householder update touches no shared memory.  Per step:
//   - every warp proposes its largest trailing norm (the norms sit in every
//     lane after the shuffle reductions), one barrier, then every warp
//     reduces the proposals itself (and, in a cluster, the CTA proposals
//     exchanged through distributed shared memory) and takes the same
//     decision: FP64 rank rule |R_ii|^2 <= eps^2 |R_11|^2 on the FP32 norms;
//   - the owner warp of the pivot column writes the Householder vector to
//     shared memory (peers in a cluster copy it with 16-byte DSMEM loads);
//   - every warp applies the reflector to its unpivoted columns and
//     recomputes their norms from the trailing rows.
// R stays in place (columns are never moved); at the end the owned columns
// go to the job's W array, and X = R1^-1 R2 is formed as in the cluster
// kernels.
// ---------------------------------------------------------------------------
constexpr int RR_THREADS = 512;
constexpr int RR_NW = RR_THREADS / 32;

// Column of the CPW held by a warp whose total lane l holds after rr_reduce,
// and the first lane holding the total of column c.
template <int CPW>
__device__ __forceinline__ int rr_col_of_lane(int lane) {
  static_assert(CPW == 4 || CPW == 8, "4 or 8 columns per warp");
  return CPW == 8 ? (((lane >> 4) & 1) << 2) | (((lane >> 3) & 1) << 1) | ((lane >> 2) & 1)
                  : (((lane >> 4) & 1) << 1) | ((lane >> 3) & 1);
}
template <int CPW>
__device__ __forceinline__ int rr_lane_of_col(int c) {
  return CPW == 8 ? (((c >> 2) & 1) << 4) | (((c >> 1) & 1) << 3) | ((c & 1) << 2)
                  : (((c >> 1) & 1) << 4) | ((c & 1) << 3);
}

// Warp sums of CPW per-lane values by a butterfly that hands half of the
// values to the partner at each of the first log2(CPW) levels: CPW - 1 +
// log2(32 / CPW) shuffles instead of 5 CPW.  Lane l returns the total of
// column rr_col_of_lane(l).
template <int CPW>
__device__ __forceinline__ float rr_reduce(float (&y)[CPW], int lane) {
#pragma unroll
  for (int h = CPW / 2, off = 16; h >= 1; h >>= 1, off >>= 1) {
    const bool up = (lane & off) != 0;
#pragma unroll
    for (int q = 0; q < h; ++q) {
      const float send = up ? y[q] : y[q + h];
      const float keep = up ? y[q + h] : y[q];
      y[q] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
  float t = y[0];
#pragma unroll
  for (int off = 16 / CPW; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
  return t;
}

// Largest value, then smallest index, over the lanes (offsets from 16 down to lo).
__device__ __forceinline__ void rr_argmax(float& b, int& p, int lo = 1) {
#pragma unroll
  for (int o = 16; o >= lo; o >>= 1) {
    const float ov = __shfl_xor_sync(0xffffffffu, b, o);
    const int op = __shfl_xor_sync(0xffffffffu, p, o);
    if (ov > b || (ov == b && op < p)) { b = ov; p = op; }
  }
}

template <int RPL, int CPW, int CL>
__global__ void __launch_bounds__(RR_THREADS, 1) k_cpqr_id_rr(const IdJob* __restrict__ jobs, double eps,
                                                            double* rdiag_all, int* order_all, int max_m,
                                                            int max_k) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  constexpr int DMAX = 32 * RPL;
  const int rank = CL > 1 ? (int)cluster.block_rank() : 0;
  const int jid = blockIdx.x / CL;
  const IdJob jb = jobs[jid];
  const int d = jb.d, m = jb.m;
  const long long ld = d;
  const float* Y = (const float*)jb.Y;
  float* W = (float*)jb.W;
  double* rdiag = rdiag_all + (long long)jid * max_k;
  int* order = order_all + (long long)jid * max_m;
  __shared__ __align__(16) float s_v[DMAX];   // Householder vector of the step (owner CTA)
  __shared__ __align__(16) float s_vl[DMAX];  // its copy in every CTA of a cluster
  __shared__ float s_wv[RR_NW];
  __shared__ int s_wj[RR_NW];
  __shared__ float s_cv, s_tau, s_taul;
  __shared__ int s_cj;
  extern __shared__ unsigned char skel[];  // m flags for the epilogue
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int mycol = rr_col_of_lane<CPW>(lane);
  const int myj = rank + CL * (wid + RR_NW * mycol);

  float a[CPW][RPL];
  unsigned act = 0;  // bit c: column c of this warp exists and is not pivoted
  float y[CPW];
#pragma unroll
  for (int c = 0; c < CPW; ++c) {
    const int j = rank + CL * (wid + RR_NW * c);
    if (j < m) act |= 1u << c;
    float s2 = 0.f;
#pragma unroll
    for (int s = 0; s < RPL; ++s) {
      const int r = lane + 32 * s;
      a[c][s] = (j < m && r < d) ? Y[r + (long long)j * ld] : 0.f;
      s2 += a[c][s] * a[c][s];
    }
    y[c] = s2;
  }
  float cnl = rr_reduce<CPW>(y, lane);  // trailing norm^2 of column mycol
  if (!((act >> mycol) & 1)) cnl = -1.f;
  // |R_11|^2 = the largest initial norm^2; thr = eps^2 |R_11|^2 computed in
  // FP64 and rounded down to FP32, so that for every FP32 b, b > thr iff
  // b > eps^2 |R_11|^2 exactly (no FP64 work inside the step loop)
  float thr;
  {
    float bv = cnl;
    int bj = cnl >= 0.f ? myj : m;
    rr_argmax(bv, bj, 32 / CPW);
    if (lane == 0) s_wv[wid] = bv;
    __syncthreads();
    float b = lane < RR_NW ? s_wv[lane] : -1.f;
    rr_argmax(b, bj);
    if (CL > 1) {
      if (threadIdx.x == 0) s_cv = b;
      cluster.sync();
      b = lane < CL ? *cluster.map_shared_rank(&s_cv, lane) : -1.f;
      rr_argmax(b, bj);
      cluster.sync();  // s_cv is rewritten in the first step
    } else {
      __syncthreads();
    }
    thr = __double2float_rd(eps * eps * (double)fmaxf(b, 0.f));
  }
  const int kmax = min(d, m);
  int k = kmax;
  for (int i = 0; i < kmax; ++i) {
    {  // proposal of this warp
      float bv = cnl;
      int bj = cnl >= 0.f ? myj : m;
      rr_argmax(bv, bj, 32 / CPW);
      if (lane == 0) { s_wv[wid] = bv; s_wj[wid] = bj; }
    }
    __syncthreads();
    float b = lane < RR_NW ? s_wv[lane] : -1.f;
    int p = lane < RR_NW ? s_wj[lane] : m;
    rr_argmax(b, p);
    if (CL > 1) {
      if (threadIdx.x == 0) { s_cv = b; s_cj = p; }
      cluster.sync();
      b = -1.f;
      p = m;
      if (lane < CL) {
        b = *cluster.map_shared_rank(&s_cv, lane);
        p = *cluster.map_shared_rank(&s_cj, lane);
      }
      rr_argmax(b, p);
    }
    // the decision, identical in every warp of every CTA (same inputs)
    const bool stop = (i == 0 ? !(b > 0.f) : !(b > thr)) || p >= m;
    if (stop) {
      k = i;
      break;
    }
    const float nrm = sqrtf(b);
    const int powner = p % CL, pl = p / CL, pw = pl % RR_NW, pc = pl / RR_NW;
    if (rank == powner && wid == pw) {
      float col[RPL];
#pragma unroll
      for (int s = 0; s < RPL; ++s) {
        float x = 0.f;
#pragma unroll
        for (int c = 0; c < CPW; ++c)
          if (c == pc) x = a[c][s];
        col[s] = x;
      }
      const int si = i >> 5;
      float xi = 0.f;
#pragma unroll
      for (int s = 0; s < RPL; ++s)
        if (s == si) xi = col[s];
      const float alpha = __shfl_sync(0xffffffffu, xi, i & 31);
      const float beta = alpha >= 0.f ? -nrm : nrm;
      const float scl = __frcp_rn(alpha - beta);
#pragma unroll
      for (int s = 0; s < RPL; ++s) {
        const int r = lane + 32 * s;
        s_v[r] = r > i ? col[s] * scl : (r == i ? 1.f : 0.f);
      }
      if (lane == 0) {
        s_tau = (beta - alpha) * __frcp_rn(beta);
        rdiag[i] = (double)beta;
        order[i] = p;
      }
      act &= ~(1u << pc);  // the pivot column leaves the active set
      if (mycol == pc) cnl = -1.f;
    }
    const float* vv = s_v;
    float tau;
    if (CL == 1) {
      __syncthreads();
      tau = s_tau;
    } else {
      cluster.sync();
      const float4* src = reinterpret_cast<const float4*>(cluster.map_shared_rank(s_v, powner));
      float4* dst = reinterpret_cast<float4*>(s_vl);
      for (int q = threadIdx.x; q < DMAX / 4; q += RR_THREADS) dst[q] = src[q];
      if (threadIdx.x == 0) s_taul = *cluster.map_shared_rank(&s_tau, powner);
      __syncthreads();
      vv = s_vl;
      tau = s_taul;
    }
    float vr[RPL];
#pragma unroll
    for (int s = 0; s < RPL; ++s) vr[s] = vv[lane + 32 * s];
#pragma unroll
    for (int c = 0; c < CPW; ++c) {
      float t = 0.f;
#pragma unroll
      for (int s = 0; s < RPL; ++s) t += vr[s] * a[c][s];
      y[c] = t;
    }
    const float dt = rr_reduce<CPW>(y, lane);
#pragma unroll
    for (int c = 0; c < CPW; ++c) {
      const float dc = __shfl_sync(0xffffffffu, dt, rr_lane_of_col<CPW>(c));
      const float f = ((act >> c) & 1) ? tau * dc : 0.f;
      float t = 0.f;
#pragma unroll
      for (int s = 0; s < RPL; ++s) {
        a[c][s] -= f * vr[s];
        if (lane + 32 * s > i) t += a[c][s] * a[c][s];
      }
      y[c] = t;
    }
    const float nt = rr_reduce<CPW>(y, lane);
    if ((act >> mycol) & 1) cnl = nt;
  }
  // publish the owned columns (R rows in place) for the back substitution
#pragma unroll
  for (int c = 0; c < CPW; ++c) {
    const int j = rank + CL * (wid + RR_NW * c);
    if (j < m) {
#pragma unroll
      for (int s = 0; s < RPL; ++s) {
        const int r = lane + 32 * s;
        if (r < d) W[r + (long long)j * ld] = a[c][s];
      }
    }
  }
  // every CTA has left the loop (no DSMEM reads remain) and every column,
  // rdiag and order entry is visible to the whole cluster
  if (CL > 1) cluster.sync(); else __syncthreads();
  for (int j = threadIdx.x; j < m; j += RR_THREADS) skel[j] = 0;
  __syncthreads();
  for (int t = threadIdx.x; t < k; t += RR_THREADS) skel[order[t]] = 1;
  __syncthreads();
  const double* rd = rdiag;
  float* X = (float*)jb.X;
  const int mo = (m - rank + CL - 1) / CL;
  for (int g = wid; 4 * g < mo; g += RR_NW) {  // up to 4 owned non-skeleton columns per warp
    int ls[4];
    int nc = 0;
    for (int q = 0; q < 4; ++q) {
      const int l = 4 * g + q;
      if (l < mo && !skel[rank + CL * l]) ls[nc++] = l;
    }
    if (nc == 0) continue;
    for (int q = nc; q < 4; ++q) ls[q] = ls[0];
    float* b0 = W + (rank + CL * ls[0]) * ld;
    float* b1 = W + (rank + CL * ls[1]) * ld;
    float* b2 = W + (rank + CL * ls[2]) * ld;
    float* b3 = W + (rank + CL * ls[3]) * ld;
    warp_backsub4<float>(b0, b1, b2, b3, nc, k, [&](int c) { return (const float*)(W + (long long)order[c] * ld); },
                         [&](int c) { return (float)rd[c]; }, lane);
    for (int q = 0; q < nc; ++q) {
      const int j = rank + CL * ls[q];
      int pos = 0;  // number of non-skeleton columns before j
      for (int c = lane; c < j; c += 32) pos += skel[c] ? 0 : 1;
      for (int o = 16; o > 0; o >>= 1) pos += __shfl_xor_sync(0xffffffffu, pos, o);
      for (int r = lane; r < k; r += 32) X[r + (long long)pos * k] = W[r + j * ld];
      if (lane == 0) jb.piv[k + pos] = j;
    }
  }
  if (rank == 0) {
    for (int t = threadIdx.x; t < k; t += RR_THREADS) jb.piv[t] = order[t];
    if (threadIdx.x == 0) *jb.rank = k;
  }
}

template <int RPL, int CPW, int CL>
static int launch_id_rr(const IdJob* jobs, int njobs, int max_m, int max_d, double eps, double* rdiag,
                        int* order, cudaStream_t s) {
  if (max_d > 32 * RPL || max_m > RR_NW * CPW * CL) return -1;
  if (CL > 8 && !set_func_attr((const void*)k_cpqr_id_rr<RPL, CPW, CL>,
                               cudaFuncAttributeNonPortableClusterSizeAllowed, 1))
    return -1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(njobs * CL, 1, 1);
  cfg.blockDim = dim3(RR_THREADS, 1, 1);
  cfg.dynamicSmemBytes = (size_t)std::max(max_m, 1);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const int max_k = std::max(std::min(max_m, max_d), 1);
  if (cudaLaunchKernelEx(&cfg, k_cpqr_id_rr<RPL, CPW, CL>, jobs, eps, rdiag, order, std::max(max_m, 1), max_k) !=
      cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  count_launch();
  return 0;
}

template <typename T>
int HssKern<T>::id_rr_config(int d, int m) {
  if constexpr (!std::is_same<T, float>::value) {
    return 0;
  } else {
    for (int cl = 1; cl <= 16; cl *= 2) {
      if (d <= 256 && m <= RR_NW * 8 * cl) return cl;        // 8 rows x 8 columns per lane
      if (d <= 512 && m <= RR_NW * 4 * cl) return 32 + cl;   // 16 rows x 4 columns per lane
    }
    return 0;
  }
}

template <typename T>
int HssKern<T>::batched_id_rr(const IdJob* jobs, int njobs, int max_m, int max_d, double eps, double* rdiag,
                              int* order, int cfg, cudaStream_t s) {
  if (njobs <= 0) return 0;
  if (!std::is_same<T, float>::value) return -1;
  switch (cfg) {
    case 1: return launch_id_rr<8, 8, 1>(jobs, njobs, max_m, max_d, eps, rdiag, order, s);
    case 2: return launch_id_rr<8, 8, 2>(jobs, njobs, max_m, max_d, eps, rdiag, order, s);
    case 4: return launch_id_rr<8, 8, 4>(jobs, njobs, max_m, max_d, eps, rdiag, order, s);
    case 8: return launch_id_rr<8, 8, 8>(jobs, njobs, max_m, max_d, eps, rdiag, order, s);
    case 16: return launch_id_rr<8, 8, 16>(jobs, njobs, max_m, max_d, eps, rdiag, order, s);
    case 33: return launch_id_rr<16, 4, 1>(jobs, njobs, max_m, max_d, eps, rdiag, order, s);
    case 34: return launch_id_rr<16, 4, 2>(jobs, njobs, max_m, max_d, eps, rdiag, order, s);
    case 36: return launch_id_rr<16, 4, 4>(jobs, njobs, max_m, max_d, eps, rdiag, order, s);
    case 40: return launch_id_rr<16, 4, 8>(jobs, njobs, max_m, max_d, eps, rdiag, order, s);
    case 48: return launch_id_rr<16, 4, 16>(jobs, njobs, max_m, max_d, eps, rdiag, order, s);
    default: return -1;
  }
}

// ---------------------------------------------------------------------------
// Explicit interpolative basis Pi [I; X^T] (eq. UVstructure).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_basis(const BasisJob* __restrict__ jobs) {
  const BasisJob jb = jobs[blockIdx.x];
  const T* X = (const T*)jb.X;
  T* out = (T*)jb.out;
  const long long tot = (long long)jb.m * jb.k;
  for (long long e = blockIdx.y * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.y * blockDim.x) {
    int j = (int)(e % jb.m), c = (int)(e / jb.m);  // j: position in pivoted order
    T v = j < jb.k ? T(j == c ? 1 : 0) : X[c + (long long)(j - jb.k) * jb.k];
    out[jb.piv[j] + (long long)c * jb.ldo] = v;
  }
}

template <typename T>
void HssKern<T>::basis(const BasisJob* jobs, int njobs, cudaStream_t s) {
  if (njobs <= 0) return;
  k_basis<T><<<dim3(njobs, 8), 256, 0, s>>>(jobs);
  count_launch();
}

// ---------------------------------------------------------------------------
// Blocked LQ, one panel of rows [j0, j1) per job (one CTA per job):
// Householder reflectors of the panel rows (LAPACK larfg convention, v
// stored in the zeroed part of its row, tau), applied to the panel rows
// below; then the block reflector H_j0 ... H_j1-1 = I - V^T T V with V
// (w x (m - j0), explicit unit diagonal and zeros, ld nb) and the upper
// triangular T (forward accumulation).  The rows below the panel and V_t
// are updated afterwards by batched GEMMs.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_lq_panel(const LqJob* __restrict__ jobs, int j0, int nb) {
  const LqJob jb = jobs[blockIdx.x];
  const int m = jb.m, nk = jb.m - jb.k;
  if (j0 >= nk) return;
  const int j1 = min(j0 + nb, nk), w = j1 - j0, n = m - j0;
  T* D = (T*)jb.Dt;
  T* tau = (T*)jb.tau;
  T* Vb = (T*)jb.Vb;
  T* Tb = (T*)jb.Tb + (long long)(j0 / nb) * nb * nb;  // T of this panel, kept for the solve
  __shared__ T sh[33];
  __shared__ T sT[32][33];
  __shared__ T sg[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = j0; i < j1; ++i) {
    T part = T(0);
    for (int c = i + 1 + threadIdx.x; c < m; c += blockDim.x) {
      const T v = D[i + (long long)c * m];
      part += v * v;
    }
    const T alpha = D[i + (long long)i * m];
    const T xn2 = block_sum_t<T>(part, sh);
    T t = T(0), beta = alpha, scl = T(0);
    if (xn2 > T(0)) {
      const T b = sqrt(alpha * alpha + xn2);
      beta = alpha >= T(0) ? -b : b;
      t = (beta - alpha) / beta;
      scl = T(1) / (alpha - beta);
    }
    for (int c = i + 1 + threadIdx.x; c < m; c += blockDim.x) D[i + (long long)c * m] *= scl;
    __syncthreads();
    if (threadIdx.x == 0) {
      D[i + (long long)i * m] = beta;
      tau[i] = t;
    }
    if (t != T(0)) {  // panel rows below i: row_r[i:m] -= t (row_r . v) v
      for (int r = i + 1 + wid; r < j1; r += nw) {
        T s = T(0);
        for (int c = i + 1 + lane; c < m; c += 32) s += D[r + (long long)c * m] * D[i + (long long)c * m];
        s = wsum<T>(s) + D[r + (long long)i * m];
        const T f = t * s;
        __syncwarp();
        if (lane == 0) D[r + (long long)i * m] -= f;
        for (int c = i + 1 + lane; c < m; c += 32) D[r + (long long)c * m] -= f * D[i + (long long)c * m];
      }
    }
    __syncthreads();
  }
  // V of the block reflector (rows beyond w are zero)
  for (long long e = threadIdx.x; e < (long long)nb * n; e += blockDim.x) {
    const int q = (int)(e % nb), c = (int)(e / nb);
    T val = T(0);
    if (q < w) val = c < q ? T(0) : c == q ? T(1) : D[(j0 + q) + (long long)(j0 + c) * m];
    Vb[q + (long long)c * nb] = val;
  }
  __syncthreads();
  // Gram entries G(p, q) = V(p, :) . V(q, :) for p < q (warp per pair)
  for (int pq = wid; pq < w * w; pq += nw) {
    const int p = pq % w, q = pq / w;
    if (p >= q) continue;
    T s = T(0);
    for (int c = q + lane; c < n; c += 32) s += Vb[p + (long long)c * nb] * Vb[q + (long long)c * nb];
    s = wsum<T>(s);
    if (lane == 0) sT[p][q] = s;  // holds G until T(:, q) replaces it below
  }
  __syncthreads();
  // T(q, q) = tau_q; T(0:q, q) = -tau_q T(0:q, 0:q) G(0:q, q)
  for (int q = 0; q < w; ++q) {
    if (threadIdx.x < q) sg[threadIdx.x] = sT[threadIdx.x][q];
    __syncthreads();
    const T tq = tau[j0 + q];
    if (threadIdx.x < q) {
      const int p = threadIdx.x;
      T s = T(0);
      for (int r = p; r < q; ++r) s += sT[p][r] * sg[r];
      sT[p][q] = -tq * s;
    }
    if (threadIdx.x == 0) sT[q][q] = tq;
    __syncthreads();
  }
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int p = e % nb, q = e / nb;
    Tb[e] = (p < w && q < w && p <= q) ? sT[p][q] : T(0);
  }
}

// The same panel with the panel rows staged in shared memory: the kernel
// above walks rows of the column-major Dt (one 32-byte sector per element);
// here the w x n panel is loaded once with coalesced column reads
// (P[c * 33 + q] = Dt(j0 + q, j0 + c)), factored in shared memory with the
// same thread assignment and operation order (the same results), and
// written back once.
constexpr size_t kPanelSmemMax = 212 * 1024;  // dynamic part; the static arrays take up to 9 KB
template <typename T>
__global__ void __launch_bounds__(256) k_lq_panel_s(const LqJob* __restrict__ jobs, int j0, int nb) {
  const LqJob jb = jobs[blockIdx.x];
  const int m = jb.m, nk = jb.m - jb.k;
  if (j0 >= nk) return;
  const int j1 = min(j0 + nb, nk), w = j1 - j0, n = m - j0;
  T* D = (T*)jb.Dt;
  T* tau = (T*)jb.tau;
  T* Vb = (T*)jb.Vb;
  T* Tb = (T*)jb.Tb + (long long)(j0 / nb) * nb * nb;  // T of this panel, kept for the solve
  extern __shared__ __align__(16) unsigned char lq_raw[];
  T* P = (T*)lq_raw;
  __shared__ T sh[33];
  __shared__ T sT[32][33];
  __shared__ T sg[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (long long e = threadIdx.x; e < 32LL * n; e += blockDim.x) {
    const int q = (int)(e & 31), c = (int)(e >> 5);
    if (q < w) P[c * 33 + q] = D[(j0 + q) + (long long)(j0 + c) * m];
  }
  __syncthreads();
  for (int i = 0; i < w; ++i) {  // panel row i: row j0 + i of Dt, its diagonal at panel column i
    T part = T(0);
    for (int c = i + 1 + threadIdx.x; c < n; c += blockDim.x) {
      const T v = P[c * 33 + i];
      part += v * v;
    }
    const T alpha = P[i * 33 + i];
    const T xn2 = block_sum_t<T>(part, sh);
    T t = T(0), beta = alpha, scl = T(0);
    if (xn2 > T(0)) {
      const T b = sqrt(alpha * alpha + xn2);
      beta = alpha >= T(0) ? -b : b;
      t = (beta - alpha) / beta;
      scl = T(1) / (alpha - beta);
    }
    for (int c = i + 1 + threadIdx.x; c < n; c += blockDim.x) P[c * 33 + i] *= scl;
    __syncthreads();
    if (threadIdx.x == 0) {
      P[i * 33 + i] = beta;
      tau[j0 + i] = t;
    }
    if (t != T(0)) {  // panel rows below i: row_r[i:] -= t (row_r . v) v
      for (int r = i + 1 + wid; r < w; r += nw) {
        T sacc = T(0);
        for (int c = i + 1 + lane; c < n; c += 32) sacc += P[c * 33 + r] * P[c * 33 + i];
        sacc = wsum<T>(sacc) + P[i * 33 + r];
        const T f = t * sacc;
        __syncwarp();
        if (lane == 0) P[i * 33 + r] -= f;
        for (int c = i + 1 + lane; c < n; c += 32) P[c * 33 + r] -= f * P[c * 33 + i];
      }
    }
    __syncthreads();
  }
  for (long long e = threadIdx.x; e < 32LL * n; e += blockDim.x) {
    const int q = (int)(e & 31), c = (int)(e >> 5);
    if (q < w) D[(j0 + q) + (long long)(j0 + c) * m] = P[c * 33 + q];
  }
  // V of the block reflector (rows beyond w are zero)
  auto V = [&](int q, int c) -> T { return q >= w ? T(0) : c < q ? T(0) : c == q ? T(1) : P[c * 33 + q]; };
  for (long long e = threadIdx.x; e < (long long)nb * n; e += blockDim.x) {
    const int q = (int)(e % nb), c = (int)(e / nb);
    Vb[q + (long long)c * nb] = V(q, c);
  }
  // Gram entries G(p, q) = V(p, :) . V(q, :) for p < q (warp per pair)
  for (int pq = wid; pq < w * w; pq += nw) {
    const int p = pq % w, q = pq / w;
    if (p >= q) continue;
    T sacc = T(0);
    for (int c = q + lane; c < n; c += 32) sacc += V(p, c) * V(q, c);
    sacc = wsum<T>(sacc);
    if (lane == 0) sT[p][q] = sacc;  // holds G until T(:, q) replaces it below
  }
  __syncthreads();
  // T(q, q) = tau_q; T(0:q, q) = -tau_q T(0:q, 0:q) G(0:q, q)
  for (int q = 0; q < w; ++q) {
    if (threadIdx.x < q) sg[threadIdx.x] = sT[threadIdx.x][q];
    __syncthreads();
    const T tq = tau[j0 + q];
    if (threadIdx.x < q) {
      const int pp = threadIdx.x;
      T sacc = T(0);
      for (int r = pp; r < q; ++r) sacc += sT[pp][r] * sg[r];
      sT[pp][q] = -tq * sacc;
    }
    if (threadIdx.x == 0) sT[q][q] = tq;
    __syncthreads();
  }
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int pp = e % nb, q = e / nb;
    Tb[e] = (pp < w && q < w && pp <= q) ? sT[pp][q] : T(0);
  }
}

template <typename T>
void HssKern<T>::lq_panel(const LqJob* jobs, int njobs, int j0, int nb, int max_n, cudaStream_t s) {
  if (njobs <= 0) return;
  const size_t smem = sizeof(T) * 33 * (size_t)std::max(max_n, 1);
  if (nb <= 32 && smem <= kPanelSmemMax &&
      set_func_attr((const void*)k_lq_panel_s<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPanelSmemMax)) {
    k_lq_panel_s<T><<<njobs, 256, smem, s>>>(jobs, j0, nb);
  } else {
    k_lq_panel<T><<<njobs, 256, 0, s>>>(jobs, j0, nb);
  }
  count_launch();
}

// ---------------------------------------------------------------------------
// Blocked LU with partial pivoting over all rows: panel columns [k0, k1)
// (first maximum wins, full-row swaps), one CTA per job.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_lu_panel(const LuJob* __restrict__ jobs, int k0, int nb,
                                                  unsigned* status) {
  const LuJob jb = jobs[blockIdx.x];
  const int m = jb.m;
  if (k0 >= m) return;
  const int k1 = min(k0 + nb, m);
  T* A = (T*)jb.A;
  const long long ld = m;
  __shared__ T s_v[8];  // (comparisons of |a| are exact in T: same pivots as in FP64)
  __shared__ int s_i[8];
  __shared__ int s_p;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int j = k0; j < k1; ++j) {
    T bv = T(-1);
    int bi = m;
    for (int r = j + threadIdx.x; r < m; r += blockDim.x) {
      const T a = tabs(A[r + j * ld]);
      if (a > bv) { bv = a; bi = r; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      T ov = __shfl_down_sync(0xffffffffu, bv, o);
      int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    if (lane == 0) { s_v[wid] = bv; s_i[wid] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
      T b = s_v[0];
      int ix = s_i[0];
      for (int w2 = 1; w2 < (int)(blockDim.x >> 5); ++w2)
        if (s_v[w2] > b || (s_v[w2] == b && s_i[w2] < ix)) { b = s_v[w2]; ix = s_i[w2]; }
      if (!(b > T(0)) || !isfinite(b)) {
        atomicOr(status, b == T(0) ? ST_ZERO_PIVOT : ST_NONFINITE);
        ix = j;
      }
      s_p = ix;
      jb.piv[j] = ix;
    }
    __syncthreads();
    const int p = s_p;
    if (p != j)  // the panel columns now; the others in k_lu_trsm after the panel
      for (int c = k0 + threadIdx.x; c < k1; c += blockDim.x) {
        T t = A[j + c * ld];
        A[j + c * ld] = A[p + c * ld];
        A[p + c * ld] = t;
      }
    __syncthreads();
    const T dj = A[j + j * ld];
    const T inv = dj != T(0) ? T(1) / dj : T(0);
    for (int r = j + 1 + threadIdx.x; r < m; r += blockDim.x) {
      T l = A[r + j * ld] * inv;
      A[r + j * ld] = l;
      for (int c = j + 1; c < k1; ++c) A[r + c * ld] -= l * A[j + c * ld];
    }
    __syncthreads();
  }
}

// The same panel staged in shared memory: rows [k0, m) of the panel
// columns, L[c * n + r] = A(k0 + r, k0 + c), loaded and written back once
// with coalesced column accesses; the same thread assignment and operation
// order as above (the same pivots and factors).
template <typename T>
__global__ void __launch_bounds__(256) k_lu_panel_s(const LuJob* __restrict__ jobs, int k0, int nb,
                                                    unsigned* status) {
  const LuJob jb = jobs[blockIdx.x];
  const int m = jb.m;
  if (k0 >= m) return;
  const int k1 = min(k0 + nb, m), w = k1 - k0, n = m - k0;
  T* A = (T*)jb.A;
  const long long ld = m;
  extern __shared__ __align__(16) unsigned char lu_raw[];
  T* L = (T*)lu_raw;
  __shared__ T s_v[8];
  __shared__ int s_i[8];
  __shared__ int s_p;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (long long e = threadIdx.x; e < (long long)w * n; e += blockDim.x) {
    const int c = (int)(e / n), r = (int)(e % n);
    L[e] = A[(k0 + r) + (long long)(k0 + c) * ld];
  }
  __syncthreads();
  for (int j = k0; j < k1; ++j) {
    const int jj = j - k0;
    const T* Lj = L + (long long)jj * n - k0;  // Lj[r] = A(r, j) for r >= k0
    T bv = T(-1);
    int bi = m;
    for (int r = j + threadIdx.x; r < m; r += blockDim.x) {
      const T a = tabs(Lj[r]);
      if (a > bv) { bv = a; bi = r; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      T ov = __shfl_down_sync(0xffffffffu, bv, o);
      int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    if (lane == 0) { s_v[wid] = bv; s_i[wid] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
      T b = s_v[0];
      int ix = s_i[0];
      for (int w2 = 1; w2 < (int)(blockDim.x >> 5); ++w2)
        if (s_v[w2] > b || (s_v[w2] == b && s_i[w2] < ix)) { b = s_v[w2]; ix = s_i[w2]; }
      if (!(b > T(0)) || !isfinite(b)) {
        atomicOr(status, b == T(0) ? ST_ZERO_PIVOT : ST_NONFINITE);
        ix = j;
      }
      s_p = ix;
      jb.piv[j] = ix;
    }
    __syncthreads();
    const int p = s_p;
    if (p != j)  // the panel columns now; the others in k_lu_trsm after the panel
      for (int c = threadIdx.x; c < w; c += blockDim.x) {
        T* Lc = L + (long long)c * n - k0;
        const T t = Lc[j];
        Lc[j] = Lc[p];
        Lc[p] = t;
      }
    __syncthreads();
    const T dj = Lj[j];
    const T inv = dj != T(0) ? T(1) / dj : T(0);
    for (int r = j + 1 + threadIdx.x; r < m; r += blockDim.x) {
      T* Lr = L + r - k0;
      const T l = Lr[(long long)jj * n] * inv;
      Lr[(long long)jj * n] = l;
      for (int c = jj + 1; c < w; ++c) Lr[(long long)c * n] -= l * Lj[j + (long long)(c - jj) * n];
    }
    __syncthreads();
  }
  for (long long e = threadIdx.x; e < (long long)w * n; e += blockDim.x) {
    const int c = (int)(e / n), r = (int)(e % n);
    A[(k0 + r) + (long long)(k0 + c) * ld] = L[e];
  }
}

template <typename T>
void HssKern<T>::lu_panel(const LuJob* jobs, int njobs, int k0, int nb, unsigned* status, int max_n,
                          cudaStream_t s) {
  if (njobs <= 0) return;
  const size_t smem = sizeof(T) * (size_t)nb * (size_t)std::max(max_n, 1);
  if (smem <= kPanelSmemMax &&
      set_func_attr((const void*)k_lu_panel_s<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPanelSmemMax)) {
    k_lu_panel_s<T><<<njobs, 256, smem, s>>>(jobs, k0, nb, status);
  } else {
    k_lu_panel<T><<<njobs, 256, 0, s>>>(jobs, k0, nb, status);
  }
  count_launch();
}

// After a panel: the panel's row interchanges on every column outside it
// (one thread per column, in order), then the U row block right of the panel:
// rows [k0, k1), columns [k1, m) <- L_panel^-1 (unit lower, nb <= 32).
template <typename T>
__global__ void __launch_bounds__(128) k_lu_trsm(const LuJob* __restrict__ jobs, int k0, int nb) {
  const LuJob jb = jobs[blockIdx.x];
  const int m = jb.m;
  if (k0 >= m) return;
  const int k1 = min(k0 + nb, m), w = k1 - k0;
  T* A = (T*)jb.A;
  const long long ld = m;
  __shared__ T L[32][33];
  __shared__ int pv[32];
  for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
    int i = e & 31, j = e >> 5;
    L[i][j] = (i < w && j < w) ? A[(k0 + i) + (k0 + j) * ld] : T(0);
  }
  if (threadIdx.x < w) pv[threadIdx.x] = jb.piv[k0 + threadIdx.x];
  __syncthreads();
  int c = blockIdx.y * 128 + threadIdx.x;  // columns outside [k0, k1)
  if (c >= k0) c += w;
  if (c >= m) return;
  for (int i = 0; i < w; ++i) {
    const int p = pv[i];
    if (p != k0 + i) {
      const T t = A[(k0 + i) + c * ld];
      A[(k0 + i) + c * ld] = A[p + c * ld];
      A[p + c * ld] = t;
    }
  }
  if (c < k1) return;
  T x[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) x[i] = (i < w) ? A[(k0 + i) + c * ld] : T(0);
#pragma unroll
  for (int i = 0; i < 32; ++i) {
#pragma unroll
    for (int r = i + 1; r < 32; ++r) x[r] -= L[r][i] * x[i];
  }
#pragma unroll
  for (int i = 0; i < 32; ++i)
    if (i < w) A[(k0 + i) + c * ld] = x[i];
}

template <typename T>
void HssKern<T>::lu_trsm(const LuJob* jobs, int njobs, int k0, int nb, int max_m, cudaStream_t s) {
  // (every panel, the last included: the interchanges reach the columns on its left)
  if (njobs <= 0 || k0 >= max_m || max_m - std::min(nb, max_m - k0) <= 0) return;
  k_lu_trsm<T><<<dim3(njobs, (max_m - std::min(nb, max_m - k0) + 127) / 128), 128, 0, s>>>(jobs, k0, nb);
  count_launch();
}

// ---------------------------------------------------------------------------
// Blocked triangular sweeps on a shared-memory vector (one CTA), used by the
// ULV solve: warp 0 solves each 32 x 32 diagonal block with the block's rows
// in registers, then every thread updates the rows past the block with
// coalesced column reads; two barriers per 32 columns.
// ---------------------------------------------------------------------------
// x[0:n] <- L^-1 x[0:n] (L = A(0:n, 0:n) lower, unit diagonal if unit), then
// x[n:mt] -= A(n:mt, 0:n) x[0:n].
template <typename T>
__device__ void blk_lower_solve(const T* __restrict__ A, long long lda, T* x, int n, int mt, bool unit) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int c0 = 0; c0 < n; c0 += 32) {
    const int nb = min(32, n - c0);
    if (wid == 0) {
      T Lr[32];
#pragma unroll
      for (int c = 0; c < 32; ++c)
        Lr[c] = (lane < nb && c < nb) ? A[(c0 + lane) + (long long)(c0 + c) * lda] : T(0);
      T v = lane < nb ? x[c0 + lane] : T(0);
      const T inv = (!unit && lane < nb) ? T(1) / A[(c0 + lane) + (long long)(c0 + lane) * lda] : T(1);
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        if (c < nb) {
          const T xc = __shfl_sync(0xffffffffu, v, c) * __shfl_sync(0xffffffffu, inv, c);
          if (lane == c) v = xc;
          else if (lane > c) v -= Lr[c] * xc;
        }
      }
      if (lane < nb) x[c0 + lane] = v;
    }
    __syncthreads();
    for (int r = c0 + nb + threadIdx.x; r < mt; r += blockDim.x) {
      T s = T(0);
      for (int c = 0; c < nb; ++c) s += A[r + (long long)(c0 + c) * lda] * x[c0 + c];
      x[r] -= s;
    }
    __syncthreads();
  }
}

// x[0:n] <- U^-1 x[0:n], U = A(0:n, 0:n) upper with its diagonal.
template <typename T>
__device__ void blk_upper_solve(const T* __restrict__ A, long long lda, T* x, int n) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int b = (n + 31) / 32 - 1; b >= 0; --b) {
    const int c0 = 32 * b, nb = min(32, n - c0);
    if (wid == 0) {
      T Ur[32];
#pragma unroll
      for (int c = 0; c < 32; ++c)
        Ur[c] = (lane < nb && c < nb) ? A[(c0 + lane) + (long long)(c0 + c) * lda] : T(0);
      T v = lane < nb ? x[c0 + lane] : T(0);
      const T inv = lane < nb ? T(1) / A[(c0 + lane) + (long long)(c0 + lane) * lda] : T(1);
#pragma unroll
      for (int c = 31; c >= 0; --c) {
        if (c < nb) {
          const T xc = __shfl_sync(0xffffffffu, v, c) * __shfl_sync(0xffffffffu, inv, c);
          if (lane == c) v = xc;
          else if (lane < c) v -= Ur[c] * xc;
        }
      }
      if (lane < nb) x[c0 + lane] = v;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < c0; r += blockDim.x) {
      T s = T(0);
      for (int c = 0; c < nb; ++c) s += A[r + (long long)(c0 + c) * lda] * x[c0 + c];
      x[r] -= s;
    }
    __syncthreads();
  }
}

constexpr int ULV_THREADS = 512;  // one CTA per (node, column): more loads in flight per node
constexpr size_t kUlvSmemMax = 200 * 1024;

// ---------------------------------------------------------------------------
// ULV forward step of one node (see UlvFwdJob), one CTA per (node, column):
//   b_t = leaf rows of b, or [bhat_1 - B12 w_2; bhat_2 - B21 w_1];
//   root: x = U^-1 L^-1 P b_t;
//   else: bo = Omega b_t, x1 = L^-1 bo[0:m-k], bhat = bo[m-k:] - D21 x1,
//         w = V_t^T [w_1; w_2] + Vt(0:m-k, :)^T x1.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(ULV_THREADS) k_ulv_fwd(const UlvFwdJob* __restrict__ jobs) {
  const UlvFwdJob jb = jobs[blockIdx.x];
  const int nrhs = jb.nrhs;
  const int m = jb.m, k = jb.k, nk = jb.m - jb.k;
  const T* Dt = (const T*)jb.Dt;
  const T* X = (const T*)jb.X;
  const T* Vt = (const T*)jb.Vt;
  const T* Vloc = (const T*)jb.Vloc;
  const T* B12 = (const T*)jb.B12;
  const T* B21 = (const T*)jb.B21;
  const T* bsrc = (const T*)jb.bsrc;
  const T* bh1 = (const T*)jb.bh1;
  const T* bh2 = (const T*)jb.bh2;
  const T* wc1 = (const T*)jb.wc1;
  const T* wc2 = (const T*)jb.wc2;
  extern __shared__ __align__(16) unsigned char ulv_sm[];
  T* bt = (T*)ulv_sm;  // m
  T* pb = bt + m;      // m
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = blockIdx.y; j < nrhs; j += gridDim.y) {  // columns are independent
    if (jb.leaf) {
      for (int i = threadIdx.x; i < m; i += blockDim.x) bt[i] = bsrc[i + j * jb.ldbsrc];
    } else {
      const T* w2 = wc2 + (long long)j * jb.kc2;
      const T* w1 = wc1 + (long long)j * jb.kc1;
      // thread per row, four partial sums over the columns (independent loads in flight)
      for (int i = threadIdx.x; i < jb.k1; i += blockDim.x) {
        T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
        int c = 0;
        for (; c + 3 < jb.kc2; c += 4) {
          s0 += B12[i + (long long)c * jb.k1] * w2[c];
          s1 += B12[i + (long long)(c + 1) * jb.k1] * w2[c + 1];
          s2 += B12[i + (long long)(c + 2) * jb.k1] * w2[c + 2];
          s3 += B12[i + (long long)(c + 3) * jb.k1] * w2[c + 3];
        }
        for (; c < jb.kc2; ++c) s0 += B12[i + (long long)c * jb.k1] * w2[c];
        bt[i] = bh1[i + (long long)j * jb.ldbh1] - ((s0 + s1) + (s2 + s3));
      }
      for (int i = threadIdx.x; i < jb.k2; i += blockDim.x) {
        T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
        int c = 0;
        for (; c + 3 < jb.kc1; c += 4) {
          s0 += B21[i + (long long)c * jb.k2] * w1[c];
          s1 += B21[i + (long long)(c + 1) * jb.k2] * w1[c + 1];
          s2 += B21[i + (long long)(c + 2) * jb.k2] * w1[c + 2];
          s3 += B21[i + (long long)(c + 3) * jb.k2] * w1[c + 3];
        }
        for (; c < jb.kc1; ++c) s0 += B21[i + (long long)c * jb.k2] * w1[c];
        bt[jb.k1 + i] = bh2[i + (long long)j * jb.ldbh2] - ((s0 + s1) + (s2 + s3));
      }
    }
    __syncthreads();
    // pb = P b_t: the LU row permutation at the root, Pi^T otherwise
    for (int i = threadIdx.x; i < m; i += blockDim.x) pb[i] = bt[jb.piv[i]];
    __syncthreads();
    T* bo = (T*)jb.bo + (long long)j * m;
    if (jb.is_root) {
      blk_lower_solve<T>(Dt, m, pb, m, m, true);
      blk_upper_solve<T>(Dt, m, pb, m);
      for (int i = threadIdx.x; i < m; i += blockDim.x) bo[i] = pb[i];
      __syncthreads();
      continue;
    }
    // Omega: bt[0:nk] = pb[k + i] - E(i, :) pb[0:k]; bt[nk:] = pb[0:k]
    for (int i = wid; i < nk; i += nw) {
      T s = T(0);
      for (int c = lane; c < k; c += 32) s += X[c + (long long)i * k] * pb[c];
      s = wsum<T>(s);
      if (lane == 0) bt[i] = pb[k + i] - s;
    }
    for (int i = threadIdx.x; i < k; i += blockDim.x) bt[nk + i] = pb[i];
    __syncthreads();
    // x1 = L^-1 bt[0:nk]; bhat = bt[nk:] - D21 x1
    blk_lower_solve<T>(Dt, m, bt, nk, m, false);
    for (int i = threadIdx.x; i < m; i += blockDim.x) bo[i] = bt[i];
    // w = V_t^T [wc1; wc2] + Vt(0:nk, :)^T x1, one warp per entry
    T* w = (T*)jb.w + (long long)j * jb.kc;
    for (int c = wid; c < jb.kc; c += nw) {
      T s = T(0);
      if (!jb.leaf) {
        for (int r = lane; r < jb.kc1; r += 32) s += Vloc[r + (long long)c * jb.mc] * wc1[r + (long long)j * jb.kc1];
        for (int r = lane; r < jb.kc2; r += 32)
          s += Vloc[jb.kc1 + r + (long long)c * jb.mc] * wc2[r + (long long)j * jb.kc2];
      }
      for (int r = lane; r < nk; r += 32) s += Vt[r + (long long)c * m] * bt[r];
      s = wsum<T>(s);
      if (lane == 0) w[c] = s;
    }
    __syncthreads();
  }
}

template <typename T>
int HssKern<T>::ulv_fwd(const UlvFwdJob* jobs, int njobs, int max_nrhs, int max_m, cudaStream_t s) {
  if (njobs <= 0) return 0;
  const size_t smem = 2 * sizeof(T) * (size_t)std::max(max_m, 1);
  if (smem > kUlvSmemMax) return -1;
  if (!set_func_attr((const void*)k_ulv_fwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kUlvSmemMax))
    return -1;
  k_ulv_fwd<T><<<dim3(njobs, std::min(std::max(max_nrhs, 1), 256)), ULV_THREADS, smem, s>>>(jobs);
  count_launch();
  return 0;
}

// ---------------------------------------------------------------------------
// ULV backward step of one node: x = H_0 ... H_{m-k-1} [x1; xhat2], applied
// one 32-reflector panel at a time from the last: with V_b the panel's
// reflector rows (unit at their own column, Dt to the right) and T_b its
// upper-triangular factor, x <- x - V_b^T (T_b (V_b x)).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(ULV_THREADS) k_ulv_bwd(const UlvBwdJob* __restrict__ jobs) {
  const UlvBwdJob jb = jobs[blockIdx.x];
  const int nrhs = jb.nrhs;
  const int m = jb.m, nk = jb.m - jb.k;
  const T* Dt = (const T*)jb.Dt;
  const T* Tq = (const T*)jb.Tq;
  const T* x1 = (const T*)jb.x1;
  const T* xh2 = (const T*)jb.xh2;
  extern __shared__ __align__(16) unsigned char ulv_sm[];
  T* x = (T*)ulv_sm;  // m
  __shared__ T part[ULV_THREADS / 32][32];
  __shared__ T zq[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = blockIdx.y; j < nrhs; j += gridDim.y) {  // columns are independent
    for (int i = threadIdx.x; i < nk; i += blockDim.x) x[i] = x1[i + (long long)j * m];
    for (int i = threadIdx.x; i < jb.k; i += blockDim.x) x[nk + i] = xh2[i + (long long)j * jb.ldxh2];
    __syncthreads();
    for (int b = (nk + 31) / 32 - 1; b >= 0; --b) {
      const int i0 = 32 * b, w = min(32, nk - i0);
      // y_q = v_{i0+q} . x, lanes = reflectors, warps split the columns
      T y = T(0);
      if (lane < w) {
        const int iq = i0 + lane;
        for (int c = i0 + wid; c < m; c += nw) {
          const T xc = x[c];
          if (c > iq) y += Dt[iq + (long long)c * m] * xc;
          else if (c == iq) y += xc;
        }
      }
      part[wid][lane] = y;
      __syncthreads();
      if (wid == 0) {
        T yq = T(0);
        for (int q = 0; q < nw; ++q) yq += part[q][lane];
        // z = T_b y (upper triangular)
        const T* Tb = Tq + (long long)b * 1024;
        T z = T(0);
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          const T yc = __shfl_sync(0xffffffffu, yq, c);
          if (c < w && lane <= c) z += Tb[lane + 32 * c] * yc;
        }
        zq[lane] = lane < w ? z : T(0);
      }
      __syncthreads();
      // x[c] -= sum_q V_b(q, c) z_q for c >= i0
      for (int c = i0 + threadIdx.x; c < m; c += blockDim.x) {
        T s = T(0);
        const int qmax = min(w, c - i0 + 1);
        for (int q = 0; q < qmax; ++q) {
          const int iq = i0 + q;
          s += (c == iq ? T(1) : Dt[iq + (long long)c * m]) * zq[q];
        }
        x[c] -= s;
      }
      __syncthreads();
    }
    T* out = (T*)jb.out + (long long)j * jb.ldout;
    for (int i = threadIdx.x; i < m; i += blockDim.x) out[i] = x[i];
    __syncthreads();
  }
}

template <typename T>
int HssKern<T>::ulv_bwd(const UlvBwdJob* jobs, int njobs, int max_nrhs, int max_m, cudaStream_t s) {
  if (njobs <= 0) return 0;
  const size_t smem = sizeof(T) * (size_t)std::max(max_m, 1);
  if (smem > kUlvSmemMax) return -1;
  if (!set_func_attr((const void*)k_ulv_bwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kUlvSmemMax))
    return -1;
  k_ulv_bwd<T><<<dim3(njobs, std::min(std::max(max_nrhs, 1), 256)), ULV_THREADS, smem, s>>>(jobs);
  count_launch();
  return 0;
}

// Row permutation of a finished LU from its sequential interchanges.
__global__ void k_lu_perm(const LuJob* __restrict__ jobs) {
  const LuJob jb = jobs[blockIdx.x];
  if (threadIdx.x != 0) return;
  for (int i = 0; i < jb.m; ++i) jb.perm[i] = i;
  for (int i = 0; i < jb.m; ++i) {
    const int p = jb.piv[i];
    if (p != i && p >= 0 && p < jb.m) {
      const int t = jb.perm[i];
      jb.perm[i] = jb.perm[p];
      jb.perm[p] = t;
    }
  }
}

template <typename T>
void HssKern<T>::lu_perm(const LuJob* jobs, int njobs, cudaStream_t s) {
  if (njobs <= 0) return;
  k_lu_perm<<<njobs, 32, 0, s>>>(jobs);
  count_launch();
}

template struct HssKern<double>;
template struct HssKern<float>;

}  // namespace hssmf
