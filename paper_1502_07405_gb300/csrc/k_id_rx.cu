// Interpolative decomposition of FP32 nodes (Section 2.2; rank rule of
// Section 5.3) with the node's matrix held in registers across a
// thread-block cluster and one exchange round per pivot step.
//
// Y (d x m) is factored by column-pivoted Householder QR: the pivot is the
// first column of largest trailing norm, the norms are recomputed from the
// trailing rows after every step, the rank k is the first i with
// |R_{i+1,i+1}| <= eps |R_11| (FP64 threshold, rounded down to FP32, which
// decides every FP32 norm exactly as FP64 would), and X = R1^-1 R2.
//
// Layout: CTA r of a cluster of CL owns the columns j = r (mod CL); its warp
// w owns the local columns l = w + NW c (c < CPW) and lane t holds rows
// t + 32 s (s < RPL) of each, so the Householder updates touch no memory.
// One pivot step:
//   1. every warp stages its best candidate column (largest trailing norm)
//      in shared memory and posts its proposal;        -- CTA barrier
//   2. every warp reduces the CTA's proposals; on a cluster, one thread
//      writes the proposal (norm, column) behind the CTA's candidate and
//      sends both to every CTA of the cluster with bulk asynchronous copies
//      (shared::cta -> shared::cluster) that complete on the receiver's
//      mbarrier through its transaction count;
//   3. every thread waits (bounded) on its own mbarrier, reduces the CL
//      proposals to the same decision and finds the pivot column already
//      in its own shared memory;                         -- CTA barrier
//   4. every warp applies the reflector to its columns in registers and
//      recomputes their trailing norms.
// One CTA runs the same steps without the copies (one barrier per step).
// Staging and landing areas alternate with the step's parity: a CTA
// rewrites its staging area two steps later, after its next wait, which
// completes only when every peer has sent the next step's copy, which a
// peer does only after this step's copy has landed in it.
// A wait that runs out makes the whole CTA stop (the barrier after the wait
// reduces the outcome); the kernel still meets every cluster barrier (no
// CTA leaves while a peer may read its shared memory) and reports rank -1.
// Then X = R1^-1 R2 by a blocked back substitution (32-row blocks of R1
// read from W, 16 right-hand sides at a time in shared memory).
#include <cooperative_groups.h>

#include <algorithm>
#include <cstdint>

#include "hss_kernels.h"
#include "id_common.cuh"

namespace hssmf {
namespace {

constexpr int RX_SPIN = 1 << 22;  // polls of a bounded wait

__device__ __forceinline__ uint32_t rx_saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint32_t rx_mapa(uint32_t a, int cta) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(cta));
  return r;
}
__device__ __forceinline__ bool rx_wait(uint32_t bar, uint32_t parity, int spin) {
  for (int it = 0; it < spin; ++it) {
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

template <int N>
struct Pow2Ceil {
  static constexpr int value = N <= 1 ? 1 : 2 * Pow2Ceil<(N + 1) / 2>::value;
};
template <>
struct Pow2Ceil<1> {
  static constexpr int value = 1;
};
template <int P>
struct Log2 {
  static constexpr int value = 1 + Log2<P / 2>::value;
};
template <>
struct Log2<1> {
  static constexpr int value = 0;
};

// Warp sums of P per-lane values (P a power of two <= 32) by a butterfly
// that hands half of the values to the partner at each of the first log2 P
// levels (P - 1 + log2(32 / P) shuffles).  Lane t returns the total of value
// t >> (5 - log2 P).
template <int P>
__device__ __forceinline__ float rx_reduce(float (&y)[P], int lane) {
#pragma unroll
  for (int h = P / 2, off = 16; h >= 1; h >>= 1, off >>= 1) {
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
  for (int off = 16 / P; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
  return t;
}

constexpr int RX_SEG = 8;  // row blocks per segment of the Householder passes

template <int RPL, int CPW, int NW>
__global__ void __launch_bounds__(32 * NW, 1) k_cpqr_id_rx(const IdJob* __restrict__ jobs, double eps,
                                                            double* __restrict__ rdiag_all,
                                                            int* __restrict__ order_all, int max_m, int max_k,
                                                            int spin, int hang_rank, int fail_p, int ncl) {
  constexpr int P = Pow2Ceil<CPW>::value;
  constexpr int LP = Log2<P>::value;
  constexpr int LDV = 32 * RPL;  // rows of a staged column
  constexpr int LDS = LDV + 4;   // + a 16-byte header: proposal norm and column
  namespace cg = cooperative_groups;
  const int rank = ncl > 1 ? (int)cg::this_cluster().block_rank() : 0;
  const int jid = blockIdx.x / ncl;
  // x / ncl for 0 <= x < 8192 (columns: m <= 16 x 256) by a 32-bit
  // multiply and a shift (exact: rounding 2^19 / ncl up adds less than
  // x / 2^19 < 1 / ncl, and x (2^19 / ncl + 1) < 2^32)
  const unsigned cl_mul = ((1u << 19) + ncl - 1) / ncl;
  auto cdiv = [cl_mul](int x) { return (int)(((unsigned)x * cl_mul) >> 19); };
  const IdJob jb = jobs[jid];
  const int d = jb.d, m = jb.m;
  const float* Y = (const float*)jb.Y;
  float* W = (float*)jb.W;
  double* rdiag = rdiag_all + (long long)jid * max_k;
  int* order = order_all + (long long)jid * max_m;
  extern __shared__ __align__(16) float rx_smem[];
  float* stage = rx_smem;                       // [2][NW][LDS]: each warp's candidate, by step parity
  float* land = stage + 2 * NW * LDS;        // [2][ncl][LDS]: the ncl CTAs' candidates (ncl > 1)
  float* vm = land + (ncl > 1 ? 2 * ncl * LDS : 0);  // [LDV]: the step's reflector, masked
  float* rdb = vm + LDV;                            // [32][33]: diagonal block (epilogue)
  unsigned char* skel = (unsigned char*)(rdb + 32 * 33);  // [m]: skeleton flags (epilogue)
  __shared__ float s_wv[NW];
  __shared__ int s_wj[NW];
  __shared__ __align__(8) unsigned long long bar_c[2];
  __shared__ int s_fail, s_nl;
  __shared__ int s_list[NW * CPW];  // epilogue: this CTA's non-skeleton columns
  __shared__ float s_rd[32];           // epilogue: R1 diagonal of a block
  __shared__ int s_ord[32];            // epilogue: pivot columns of a block
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int mycol = lane >> (5 - LP);  // column whose norm this lane holds after rx_reduce
  const int myj = mycol < CPW ? rank + ncl * (wid + NW * mycol) : m;

  float a[CPW][RPL];
  unsigned act = 0;  // bit c: column c of this warp exists and is not pivoted
  float y[P];
#pragma unroll
  for (int c = 0; c < P; ++c) y[c] = 0.f;
#pragma unroll
  for (int c = 0; c < CPW; ++c) {
    const int j = rank + ncl * (wid + NW * c);
    if (j < m) act |= 1u << c;
#pragma unroll
    for (int s = 0; s < RPL; ++s) {
      const int r = lane + 32 * s;
      a[c][s] = (j < m && r < d) ? Y[r + (long long)j * d] : 0.f;
      y[c] = fmaf(a[c][s], a[c][s], y[c]);
    }
  }
  float cn = rx_reduce<P>(y, lane);  // trailing norm^2 of column mycol
  if (!(mycol < CPW && ((act >> mycol) & 1))) cn = -1.f;
  if (threadIdx.x == 0) {
    s_fail = 0;
    if (ncl > 1) {
      for (int q = 0; q < 2; ++q)
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(rx_saddr(&bar_c[q])) : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
  }
  if (ncl > 1)
    cg::this_cluster().sync();  // every CTA's barriers exist before the first copy
  else
    __syncthreads();

  const int kmax = min(d, m);
  int k = kmax;
  bool failed = false, doomed = false;
  float thr = 0.f;
  for (int i = 0; i < kmax; ++i) {
    const int par = i & 1;
    const int i0 = i & ~3;  // copies start at the 16-byte boundary at or below row i
    // 1. each warp stages its best candidate column
    {
      float bv = cn;
      int bj = cn >= 0.f ? myj : m;
      id_argmax(bv, bj, 32 >> LP);
      if (bj < m) {
        const int cs = (cdiv(bj - rank) - wid) / NW;  // the candidate's slot in this warp
        float* st = stage + ((size_t)par * NW + wid) * LDS;
#pragma unroll
        for (int c = 0; c < CPW; ++c)
          if (c == cs) {
#pragma unroll
            for (int g = 0; g < RPL; g += RX_SEG) {  // rows from the segment holding row i
              if (32 * (g + RX_SEG) <= i) continue;
#pragma unroll
              for (int s = g; s < g + RX_SEG && s < RPL; ++s) st[lane + 32 * s] = a[c][s];
            }
          }
      }
      if (lane == 0) {
        s_wv[wid] = bv;
        s_wj[wid] = bj;
      }
      if (ncl > 1) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // read next by bulk copies
    }
    __syncthreads();
    // 2. the CTA's proposal; in a cluster, its candidate goes to every CTA
    float b = lane < NW ? s_wv[lane] : -1.f;
    int p = lane < NW ? s_wj[lane] : m;
    id_argmax(b, p);
    bool ok = true;
    const float* vsrc;
    if (ncl == 1) {
      vsrc = stage + ((size_t)par * NW + (p < m ? p % NW : 0)) * LDS;
    } else {
      const unsigned bytes = (unsigned)(LDS - i0) * 4u;
      if (threadIdx.x == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(rx_saddr(&bar_c[par])),
                     "r"(bytes * ncl)
                     : "memory");
        if (p < m && !(i == 0 && rank == hang_rank)) {
          float* st = stage + ((size_t)par * NW + cdiv(p) % NW) * LDS;
          st[LDV] = b;
          st[LDV + 1] = __int_as_float(p);
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          const uint32_t src = rx_saddr(st + i0);
          const uint32_t dst = rx_saddr(land + ((size_t)par * ncl + rank) * LDS + i0);
          const uint32_t bar = rx_saddr(&bar_c[par]);
          for (int q = 0; q < ncl; ++q)
            asm volatile(
                "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    rx_mapa(dst, q)),
                "r"(src), "r"(bytes), "r"(rx_mapa(bar, q))
                : "memory");
        } else if (!(i == 0 && rank == hang_rank)) {  // no candidate left: an empty proposal
          float* st = stage + (size_t)par * NW * LDS;
          st[LDV] = -1.f;
          st[LDV + 1] = __int_as_float(m);
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          const uint32_t src = rx_saddr(st + i0);
          const uint32_t dst = rx_saddr(land + ((size_t)par * ncl + rank) * LDS + i0);
          const uint32_t bar = rx_saddr(&bar_c[par]);
          for (int q = 0; q < ncl; ++q)
            asm volatile(
                "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    rx_mapa(dst, q)),
                "r"(src), "r"(bytes), "r"(rx_mapa(bar, q))
                : "memory");
        }
        // (the stage these copies read is rewritten two steps later, after
        // this CTA's next wait: every peer sends its next copy only after
        // its own copy of this step has landed)
      }
      ok = rx_wait(rx_saddr(&bar_c[par]), (i >> 1) & 1, spin);
      b = -1.f;
      p = m;
      if (ok && lane < ncl) {
        const float* h = land + ((size_t)par * ncl + lane) * LDS + LDV;
        b = h[0];
        p = __float_as_int(h[1]);
      }
      id_argmax(b, p);
      if (p < 0 || p > m) p = m;
      vsrc = land + ((size_t)par * ncl + (p < m ? p - ncl * cdiv(p) : 0)) * LDS;
    }
    if (i == 0) thr = __double2float_rd(eps * eps * (double)fmaxf(b, 0.f));
    const bool stop = !ok || (i == 0 ? !(b > 0.f) : !(b > thr)) || p >= m;
    // 3. the reflector H = I - tau w w^T with w = x - beta e_i (x the pivot
    // column's trailing part): w is kept unscaled, row i replaced by vi; the
    // CTA writes it masked (zero above row i) from the first active segment
    const float nrm = sqrtf(b);
    const float alpha = stop ? 1.f : vsrc[i];
    const float beta = alpha >= 0.f ? -nrm : nrm;
    const float vi = alpha - beta;
    const float tau = -1.f / (beta * vi);
    if (!stop)
      for (int r = (i / (32 * RX_SEG)) * (32 * RX_SEG) + threadIdx.x; r < LDV; r += 32 * NW)
        vm[r] = r > i ? vsrc[r] : (r == i ? vi : 0.f);
    if (__syncthreads_or(!ok)) {  // a wait ran out somewhere in the CTA
      failed = true;
      k = i;
      break;
    }
    if (stop) {
      k = i;
      break;
    }
    // with fail_p >= 0: pivot i takes the rank past d - fail_p and the rank
    // cannot reach m (m > d), so the ID fails whatever follows; stop with the
    // rank i + 1 and no X (the adaptive scheme retries the node with more
    // samples)
    if (fail_p >= 0 && m > d && i >= d - fail_p) {
      k = i + 1;
      doomed = true;
      break;
    }
    if (rank == 0 && threadIdx.x == 0) {
      rdiag[i] = (double)beta;
      order[i] = p;
    }
    {
      const int lp = cdiv(p);  // the pivot's local column in its owner CTA
      if (rank == p - ncl * lp && wid == lp % NW) act &= ~(1u << (lp / NW));
    }
#pragma unroll
    for (int c = 0; c < P; ++c) y[c] = 0.f;
    // segments of RX_SEG row blocks: skipped when they lie wholly above row i
    // or below row d, computed without branches otherwise
#pragma unroll
    for (int g = 0; g < RPL; g += RX_SEG) {
      if (32 * (g + RX_SEG) <= i || 32 * g >= d) continue;
#pragma unroll
      for (int s = g; s < g + RX_SEG && s < RPL; ++s) {
        const float vr = vm[lane + 32 * s];
#pragma unroll
        for (int c = 0; c < CPW; ++c) y[c] = fmaf(vr, a[c][s], y[c]);
      }
    }
    const float dt = rx_reduce<P>(y, lane);
    float f[CPW];
#pragma unroll
    for (int c = 0; c < CPW; ++c) {
      const float dc = __shfl_sync(0xffffffffu, dt, c << (5 - LP));
      f[c] = ((act >> c) & 1) ? tau * dc : 0.f;
    }
#pragma unroll
    for (int c = 0; c < P; ++c) y[c] = 0.f;
#pragma unroll
    for (int g = 0; g < RPL; g += RX_SEG) {
      if (32 * (g + RX_SEG) <= i || 32 * g >= d) continue;
#pragma unroll
      for (int s = g; s < g + RX_SEG && s < RPL; ++s) {
        const int r = lane + 32 * s;
        const float vr = vm[r];
#pragma unroll
        for (int c = 0; c < CPW; ++c) {
          a[c][s] = fmaf(-f[c], vr, a[c][s]);
          const float t = r > i ? a[c][s] : 0.f;
          y[c] = fmaf(t, t, y[c]);
        }
      }
    }
    cn = rx_reduce<P>(y, lane);
    if (!(mycol < CPW && ((act >> mycol) & 1))) cn = -1.f;
  }
  // the owned columns (R in place) go to W for the back substitution
#pragma unroll
  for (int c = 0; c < CPW; ++c) {
    const int j = rank + ncl * (wid + NW * c);
    if (j < m) {
#pragma unroll
      for (int s = 0; s < RPL; ++s) {
        const int r = lane + 32 * s;
        if (r < d) W[r + (long long)j * d] = a[c][s];
      }
    }
  }
  if (failed && threadIdx.x == 0) s_fail = 1;
  // every CTA has left the step loop (its copies have landed: each CTA
  // waited for all of them), and W, rdiag and order are visible
  if (ncl > 1)
    cg::this_cluster().sync();
  else
    __syncthreads();
  bool any_fail = s_fail != 0;
  if (ncl > 1)
    for (int q = 0; q < ncl; ++q) any_fail = any_fail || *cg::this_cluster().map_shared_rank(&s_fail, q) != 0;
  if (!any_fail && !doomed) {
    // X = R1^-1 R2 for this CTA's non-skeleton columns: a blocked back
    // substitution over 32-row blocks from the bottom, 16 columns at a time
    // in shared memory (the staging area), R1 read from W
    for (int j = threadIdx.x; j < m; j += (32 * NW)) skel[j] = 0;
    __syncthreads();
    for (int t = threadIdx.x; t < k; t += (32 * NW)) skel[order[t]] = 1;
    __syncthreads();
    if (threadIdx.x == 0) {
      int n = 0;
      for (int j = rank; j < m; j += ncl)
        if (!skel[j]) s_list[n++] = j;
      s_nl = n;
    }
    __syncthreads();
    float* X = (float*)jb.X;
    float* Bs = stage;  // k x 16, ld k
    const int nl = s_nl;
    for (int cb = 0; cb < nl && k > 0; cb += 16) {
      const int nc = min(16, nl - cb);
      for (int e = threadIdx.x; e < 16 * k; e += (32 * NW)) {
        const int q = e / k, r = e - q * k;
        Bs[e] = q < nc ? W[r + (long long)s_list[cb + q] * d] : 0.f;
      }
      for (int r1 = k; r1 > 0; r1 -= 32) {
        const int r0 = max(r1 - 32, 0), nb = r1 - r0;
        if (threadIdx.x < 32) {
          s_ord[threadIdx.x] = threadIdx.x < nb ? order[r0 + threadIdx.x] : 0;
          s_rd[threadIdx.x] = threadIdx.x < nb ? (float)rdiag[r0 + threadIdx.x] : 1.f;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < 32 * 32; e += (32 * NW)) {  // R1(r0:r1, r0:r1), upper part
          const int t = e & 31, c = e >> 5;
          rdb[t * 33 + c] = (t < nb && c < nb && t < c) ? W[(r0 + t) + (long long)s_ord[c] * d] : 0.f;
        }
        __syncthreads();
        for (int q = wid; q < nc; q += NW) {  // the diagonal block, one warp per column
          float x = lane < nb ? Bs[r0 + lane + q * k] : 0.f;
          for (int c = nb - 1; c >= 0; --c) {
            const float xc = __shfl_sync(0xffffffffu, x, c) / s_rd[c];
            if (lane == c) x = xc;
            if (lane < c) x = fmaf(-rdb[lane * 33 + c], xc, x);
          }
          if (lane < nb) Bs[r0 + lane + q * k] = x;
        }
        __syncthreads();
        for (int r = threadIdx.x; r < r0; r += (32 * NW)) {  // rows above the block
          float acc[16];
#pragma unroll
          for (int q = 0; q < 16; ++q) acc[q] = 0.f;
          for (int c = 0; c < nb; ++c) {
            const float rc = W[r + (long long)s_ord[c] * d];
#pragma unroll
            for (int q = 0; q < 16; ++q) acc[q] = fmaf(rc, Bs[r0 + c + q * k], acc[q]);
          }
#pragma unroll
          for (int q = 0; q < 16; ++q) Bs[r + q * k] -= acc[q];
        }
        __syncthreads();
      }
      for (int q = wid; q < nc; q += NW) {  // X column and its place among the non-skeleton columns
        const int j = s_list[cb + q];
        int pos = 0;
        for (int c = lane; c < j; c += 32) pos += skel[c] ? 0 : 1;
        for (int o = 16; o > 0; o >>= 1) pos += __shfl_xor_sync(0xffffffffu, pos, o);
        for (int r = lane; r < k; r += 32) X[r + (long long)pos * k] = Bs[r + q * k];
        if (lane == 0) jb.piv[k + pos] = j;
      }
      __syncthreads();
    }
    if (k == 0)  // nothing to solve: every column keeps its place
      for (int q = threadIdx.x; q < nl; q += (32 * NW)) {
        const int j = s_list[q];
        jb.piv[j] = j;
      }
  }
  if (rank == 0) {
    if (!any_fail && !doomed)
      for (int t = threadIdx.x; t < k; t += (32 * NW)) jb.piv[t] = order[t];
    if (threadIdx.x == 0) *jb.rank = any_fail ? -1 : k;
  }
  if (ncl > 1) cg::this_cluster().sync();  // peers may still read this CTA's failure flag
}

// shared memory of a configuration (bytes)
inline size_t rx_smem_bytes(int rpl, int nw, int cl, int max_m) {
  const size_t lds = 32 * (size_t)rpl + 4;
  return sizeof(float) * ((2 * nw + (cl > 1 ? 2 * cl : 0)) * lds + 32 * rpl + 32 * 33) + (size_t)std::max(max_m, 1);
}

template <int RPL, int CPW, int NW>
int launch_rx(int cl, const IdJob* jobs, int njobs, int max_m, int max_d, double eps, double* rdiag, int* order,
              cudaStream_t s, int spin, int hang_rank, int fail_p) {
  if (cl < 1 || cl > 16 || max_d > 32 * RPL || max_m > cl * NW * CPW) return -1;
  auto kern = k_cpqr_id_rx<RPL, CPW, NW>;
  const size_t smem = rx_smem_bytes(RPL, NW, cl, max_m);
  // one limit per kernel (the largest cluster and m it takes), so that the
  // attribute set on a device never needs lowering or raising
  if (!set_func_attr((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                     (int)rx_smem_bytes(RPL, NW, 16, 16 * NW * CPW)))
    return -1;
  if (cl > 8 && !set_func_attr((const void*)kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) return -1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(njobs * cl, 1, 1);
  cfg.blockDim = dim3(32 * NW, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cl;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = cl > 1 ? 1 : 0;
  const int max_k = std::max(std::min(max_m, max_d), 1);
  if (cudaLaunchKernelEx(&cfg, kern, jobs, eps, rdiag, order, std::max(max_m, 1), max_k,
                         spin > 0 ? spin : RX_SPIN, hang_rank, fail_p, cl) != cudaSuccess) {
    cudaGetLastError();
    return -1;  // not schedulable: the caller falls back
  }
  count_launch();
  return 0;
}

// Configurations (rows per lane RPL: d <= 32 RPL; columns per warp CPW; warps
// per CTA NW).  Family 0 (256-thread CTAs, up to 255 registers a thread):
// one shape per multiple of 64 in d, so that no lane holds rows beyond d,
// with CPW * RPL data registers near 180; family 1 (512-thread CTAs, 128
// registers a thread): three shapes.  A node of m columns takes the first
// shape of its family with d <= 32 RPL and the smallest cluster holding its
// columns (m <= cluster x NW x CPW): clusters of any size from 1 to 16 (the
// GPU co-schedules 15 clusters of 7 to 9 CTAs but only 7 of 13 to 16).
struct RxShape {
  int rpl, cpw, nw;
};
constexpr int RX_FAMILY0 = 12;
constexpr RxShape RX_SHAPES[RX_FAMILY0 + 3] = {
    {4, 32, 8},  {6, 24, 8},  {8, 16, 8},  {10, 16, 8}, {12, 14, 8}, {14, 12, 8}, {16, 10, 8}, {18, 9, 8},
    {20, 8, 8},  {22, 8, 8},  {24, 7, 8},  {26, 7, 8},  {8, 8, 16},  {16, 4, 16}, {26, 3, 16}};

}  // namespace

int id_rx_config(int d, int m, int family) {
  const int t0 = family == 0 ? 0 : RX_FAMILY0, t1 = family == 0 ? RX_FAMILY0 : RX_FAMILY0 + 3;
  for (int t = t0; t < t1; ++t) {
    const RxShape& c = RX_SHAPES[t];
    if (d > 32 * c.rpl) continue;
    const int cap = c.nw * c.cpw;
    const int cl = std::max(1, (m + cap - 1) / cap);
    return cl <= 16 ? 32 * t + cl : 0;
  }
  return 0;
}

int batched_id_rx(const IdJob* jobs, int njobs, int max_m, int max_d, double eps, double* rdiag, int* order,
                  int cfg, cudaStream_t s, int spin, int hang_rank, int fail_p) {
  if (njobs <= 0) return 0;
  const int t = cfg / 32, cl = cfg % 32;
#define RX_CASE(T, R, C, N) \
  case T: return launch_rx<R, C, N>(cl, jobs, njobs, max_m, max_d, eps, rdiag, order, s, spin, hang_rank, fail_p)
  switch (t) {
    RX_CASE(0, 4, 32, 8);
    RX_CASE(1, 6, 24, 8);
    RX_CASE(2, 8, 16, 8);
    RX_CASE(3, 10, 16, 8);
    RX_CASE(4, 12, 14, 8);
    RX_CASE(5, 14, 12, 8);
    RX_CASE(6, 16, 10, 8);
    RX_CASE(7, 18, 9, 8);
    RX_CASE(8, 20, 8, 8);
    RX_CASE(9, 22, 8, 8);
    RX_CASE(10, 24, 7, 8);
    RX_CASE(11, 26, 7, 8);
    RX_CASE(12, 8, 8, 16);
    RX_CASE(13, 16, 4, 16);
    RX_CASE(14, 26, 3, 16);
    default: return -1;
  }
#undef RX_CASE
}

}  // namespace hssmf
