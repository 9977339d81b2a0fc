// FP32 products of the FP32 factorization on the tensor cores, fed by TMA:
//
//  1. k_split3: every FP32 operand op(X) (rows x K) is split once into nt
//     BF16 terms (x = x0 + x1 + x2, x0 = bf16(x), x1 = bf16(x - x0),
//     x2 = bf16(x - x0 - x1); nt = 1 for an operand whose values are exactly
//     BF16) and stored K-major, term t at out + t rows Kp (Kp = K rounded up
//     to 8 elements, the extra columns zero).
//  2. k_gemm_tma: one CTA per 128 x bn tile of C (and K split).  Warp 0
//     (one thread) loads 128 x 64 tiles of every term of A and bn x 64 tiles
//     of every term of B with cp.async.bulk.tensor (128-byte swizzle, zero
//     fill outside the matrices) into a ring of stages guarded by "full"
//     mbarriers (transaction counts); warp 1 (one thread) issues the
//     tcgen05.mma products of the term pairs of order >= 2^-16 (i + j <= 2)
//     into an FP32 accumulator in tensor memory and releases each stage
//     through its "empty" mbarrier (tcgen05.commit); the four warps read the
//     accumulator back with tcgen05.ld and write C (rows crow(i), alpha, beta)
//     or, for a K split, the partial tile.
//
// The same products as k_gemm_tc (sampling S = U R of eq. FtimesR, sample
// updates of Algorithm 1, Schur complements of Sections 3.2 and 4.4), without
// the per-element split inside the GEMM loop.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

#include "gemm_tma.h"

namespace hssmf {

namespace {

constexpr int TT_M = 128, TT_K = 64;  // tile rows; K per stage (128 bytes of BF16: one swizzle row)
constexpr int TT_THREADS = 128;
constexpr int TT_TERM_A = TT_M * TT_K * 2;  // 16 KB
constexpr int TT_SMEM_BUDGET = 200 * 1024;
constexpr long long TT_SPIN = 1LL << 24;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint32_t b, unsigned n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(b), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_expect(uint32_t b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool bar_wait(uint32_t b, uint32_t parity) {
  for (long long it = 0; it < TT_SPIN; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(b), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// TMA: box (64 K, rows, 1 term) of a 3D BF16 tensor (K, rows, terms) to shared memory
__device__ __forceinline__ void tma_load3(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

// Shared-memory descriptor of a K-major BF16 tile written by TMA with the
// 128-byte swizzle: 8-row groups 1024 bytes apart, descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) |
         (2ull << 61);
}

// kind::f16, FP32 accumulator, BF16 A and B, K-major, M = 128, N = n.
__device__ __forceinline__ uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TT_M >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
        "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
        "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ---------------------------------------------------------------------------
// Split of op(X) into BF16 terms, K-major: 32 x 32 tiles (rows r0.., k0..)
// through shared memory so that reads and writes are coalesced whichever
// direction of X is contiguous.  Tile list (job, tm = row block, tn = k block).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_split3(const SplitJob* __restrict__ jobs, const Tile* __restrict__ tiles) {
  const Tile tl = tiles[blockIdx.x];
  const SplitJob jb = jobs[tl.job];
  __shared__ float t[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int r0 = tl.tm * 32, k0 = tl.tn * 32;
  // load: t[rr][kk] = op(X)(r0 + rr, k0 + kk), lanes along X's contiguous direction
  for (int a = ty; a < 32; a += 8) {
    int rr, kk;
    if (jb.krow) { rr = a; kk = tx; } else { rr = tx; kk = a; }
    const int r = r0 + rr, k = k0 + kk;
    float v = 0.f;
    if (r < jb.rows && k < jb.K) v = jb.krow ? jb.X[k + (long long)r * jb.ldx] : jb.X[r + (long long)k * jb.ldx];
    t[rr][kk] = v;
  }
  __syncthreads();
  // store: lanes along k (K-major output rows)
  for (int rr = ty; rr < 32; rr += 8) {
    const int r = r0 + rr, k = k0 + tx;
    if (r >= jb.rows || k >= jb.Kp) continue;
    const float x = t[rr][tx];
    const long long o = (long long)r * jb.Kp + k;
    const __nv_bfloat16 h0 = __float2bfloat16_rn(x);
    jb.out[o] = h0;
    if (jb.nt > 1) {
      const float r1 = x - __bfloat162float(h0);
      const __nv_bfloat16 h1 = __float2bfloat16_rn(r1);
      const float r2 = r1 - __bfloat162float(h1);
      jb.out[o + jb.term] = h1;
      jb.out[o + 2 * jb.term] = __float2bfloat16_rn(r2);
    }
  }
}

// ---------------------------------------------------------------------------
// The TMA-fed tcgen05 GEMM over a tile list (job, tm, tn, ks).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(TT_THREADS, 1) k_gemm_tma(const TmaJob* __restrict__ jobs,
                                                           const Tile* __restrict__ tiles, int stages,
                                                           unsigned* __restrict__ status) {
  extern __shared__ char smem_raw[];
  __shared__ __align__(8) unsigned long long s_full[TT_MAX_STAGES], s_empty[TT_MAX_STAGES], s_done;
  __shared__ uint32_t s_tmem;
  char* smem = (char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const Tile tl = tiles[blockIdx.x];
  const TmaJob* jp = jobs + tl.job;
  const int M = jp->M, N = jp->N, na = jp->na, nb = jp->nb, bn = jp->bn;
  const int m0 = tl.tm * TT_M, n0 = tl.tn * bn;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tb_bytes = bn * TT_K * 2;
  const int stage_bytes = na * TT_TERM_A + nb * tb_bytes;  // multiple of 1024
  // K tiles of this split
  const int ktiles = (jp->K + TT_K - 1) / TT_K;
  const int S = jp->ksplit > 1 ? jp->ksplit : 1;
  const int per = (ktiles + S - 1) / S;
  const int kt0 = min(ktiles, tl.ks * per), kt1 = min(ktiles, kt0 + per);
  const int nk = kt1 - kt0;

  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&s_tmem)),
                 "r"(128)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      bar_init(su32(&s_full[s]), 1);
      bar_init(su32(&s_empty[s]), 1);
    }
    bar_init(su32(&s_done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&jp->ta) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&jp->tb) : "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;
  bool ok = true;

  // Drain rule for bounded waits: the producer and the MMA issuer stop at
  // their first wait that runs out and issue nothing more; the producer then
  // waits (bounded) until its last load into every stage has landed, so no
  // bulk copy is in flight when the CTA exits; the final commit covers only
  // the MMAs that were issued.  A timeout is reported as ST_TIMEOUT and the
  // accumulator is not read.
  if (threadIdx.x == 0) {  // producer
    int loaded = 0;
    for (int t = 0; t < nk; ++t) {
      const int s = t % stages, round = t / stages;
      if (round > 0 && !bar_wait(su32(&s_empty[s]), (round - 1) & 1)) {
        ok = false;
        break;
      }
      const uint32_t fb = su32(&s_full[s]);
      bar_expect(fb, (unsigned)stage_bytes);
      const uint32_t base = su32(smem + (size_t)s * stage_bytes);
      const int k0 = (kt0 + t) * TT_K;
      for (int a = 0; a < na; ++a) tma_load3(base + a * TT_TERM_A, &jp->ta, k0, m0, a, fb);
      for (int b = 0; b < nb; ++b) tma_load3(base + na * TT_TERM_A + b * tb_bytes, &jp->tb, k0, n0, b, fb);
      loaded = t + 1;
    }
    if (!ok)  // the most recent load into each stage (consumed or not) has landed
      for (int t = max(0, loaded - stages); t < loaded; ++t)
        if (!bar_wait(su32(&s_full[t % stages]), (t / stages) & 1)) break;
  } else if (threadIdx.x == 32) {  // MMA issuer
    const uint32_t idesc = idesc_bf16(bn);
    for (int t = 0; t < nk; ++t) {
      const int s = t % stages, round = t / stages;
      if (!bar_wait(su32(&s_full[s]), round & 1)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t base = su32(smem + (size_t)s * stage_bytes);
#pragma unroll
      for (int kk = 0; kk < TT_K / 16; ++kk)
        for (int i = 0; i < na; ++i)
          for (int j = 0; j < nb && i + j <= 2; ++j) {
            const uint64_t ad = sw128_desc(base + i * TT_TERM_A + kk * 32);
            const uint64_t bd = sw128_desc(base + na * TT_TERM_A + j * tb_bytes + kk * 32);
            mma(tmem, ad, bd, idesc, (t > 0 || kk > 0 || i > 0 || j > 0) ? 1u : 0u);
          }
      commit(su32(&s_empty[s]));
    }
    commit(su32(&s_done));  // covers every MMA issued before it (possibly none)
  }
  __syncwarp();
  if (nk > 0) ok = bar_wait(su32(&s_done), 0) && ok;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  ok = __syncthreads_and(ok);
  if (!ok && threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);

  // epilogue: warp w holds rows 32 w .. 32 w + 31 of the tile
  const int i = 32 * warp + lane, gi = m0 + i;
  const float alpha = (float)jp->alpha, beta = (float)jp->beta;
  const long long crow = gi < M ? (jp->crow ? jp->crow[gi] : gi) : 0;
  float* C = (float*)jp->C;
  for (int c0 = 0; c0 < bn; c0 += 32) {
    float v[32];
    if (nk > 0 && ok) {
      tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
    } else {
#pragma unroll
      for (int e = 0; e < 32; ++e) v[e] = 0.f;
    }
    if (S > 1) {
      float* wp = jp->ws + ((size_t)(tl.tm + tl.tn * jp->tiles_m) * S + tl.ks) * (TT_M * 128) + i;
#pragma unroll
      for (int e = 0; e < 32; ++e)
        if (c0 + e < bn) wp[(size_t)(c0 + e) * TT_M] = v[e];
    } else if (gi < M) {
#pragma unroll
      for (int e = 0; e < 32; ++e) {
        const int gj = n0 + c0 + e;
        if (c0 + e < bn && gj < N) {
          float* cp = C + crow + (long long)gj * jp->ldc;
          *cp = (jp->beta == 0.0) ? alpha * v[e] : alpha * v[e] + beta * *cp;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 2) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128) : "memory");
  }
}

// split-K partials of the TMA GEMM (128 x 128 stride per partial tile):
// CTA (x, y) sums columns 16 y .. 16 y + 15 of output tile x, 8 outputs a
// thread, every load issued before the first sum is used
constexpr int TT_RED_COLS = 16;
__global__ void __launch_bounds__(256) k_gemm_tma_reduce(const TmaJob* __restrict__ jobs,
                                                         const Tile* __restrict__ tiles) {
  const Tile tl = tiles[blockIdx.x];
  const TmaJob* jp = jobs + tl.job;
  const int S = jp->ksplit, bn = jp->bn;
  const int c0 = blockIdx.y * TT_RED_COLS;
  if (c0 >= bn) return;
  const int m0 = tl.tm * TT_M, n0 = tl.tn * bn;
  const float* wp = jp->ws + (size_t)(tl.tm + tl.tn * jp->tiles_m) * S * (TT_M * 128);
  float* C = (float*)jp->C;
  const float alpha = (float)jp->alpha, beta = (float)jp->beta;
  constexpr int PER = TT_M * TT_RED_COLS / 256;
  float sum[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) sum[q] = 0.f;
  for (int ks = 0; ks < S; ++ks)
#pragma unroll
    for (int q = 0; q < PER; ++q) sum[q] += wp[(size_t)ks * (TT_M * 128) + c0 * TT_M + threadIdx.x + 256 * q];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int e = c0 * TT_M + threadIdx.x + 256 * q;
    const int i = e % TT_M, c = e / TT_M;
    const int gi = m0 + i, gj = n0 + c;
    if (c >= bn || gi >= jp->M || gj >= jp->N) continue;
    const long long row = jp->crow ? jp->crow[gi] : gi;
    float* cp = C + row + (long long)gj * jp->ldc;
    *cp = (jp->beta == 0.0) ? alpha * sum[q] : alpha * sum[q] + beta * *cp;
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    cudaGetLastError();
  }
  return fn;
}

// 3D map (Kp, rows, nt) over K-major BF16 terms, box (64, box_rows, 1), 128-byte swizzle
bool encode3(CUtensorMap* m, const void* base, int Kp, int rows, int nt, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)nt};
  cuuint64_t strides[2] = {(cuuint64_t)Kp * 2, (cuuint64_t)rows * Kp * 2};
  cuuint32_t box[3] = {(cuuint32_t)TT_K, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool gemm_tma_available() { return encode_fn() != nullptr; }

int gemm_tma_batch(const std::vector<GemmJob>& gj, TmaScratch& mem, unsigned* status, cudaStream_t s) {
  if (gj.empty()) return 0;
  if (!gemm_tma_available()) return -1;
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) nsm = 148;
  }
  // split each distinct operand once
  std::vector<SplitJob> sj;
  std::vector<Tile> st;
  std::map<std::tuple<const void*, long long, int, int, int, int>, __nv_bfloat16*> done;
  auto split = [&](const void* X, long long ldx, int krow, int rows, int K, int nt) -> __nv_bfloat16* {
    const auto key = std::make_tuple(X, ldx, krow, rows, K, nt);
    auto it = done.find(key);
    if (it != done.end()) return it->second;
    const int Kp = (K + 7) & ~7;
    __nv_bfloat16* out = (__nv_bfloat16*)mem.alloc(sizeof(__nv_bfloat16) * (size_t)nt * rows * Kp);
    if (!out) return nullptr;
    SplitJob j;
    j.X = (const float*)X;
    j.ldx = ldx;
    j.krow = krow;
    j.rows = rows;
    j.K = K;
    j.Kp = Kp;
    j.nt = nt;
    j.term = (long long)rows * Kp;
    j.out = out;
    const int id = (int)sj.size();
    sj.push_back(j);
    for (int b = 0; b < (Kp + 31) / 32; ++b)
      for (int a = 0; a < (rows + 31) / 32; ++a) st.push_back(Tile{id, a, b, 0});
    done[key] = out;
    return out;
  };
  std::vector<TmaJob> tj(gj.size());
  long long t0 = 0;
  for (size_t i = 0; i < gj.size(); ++i) {
    const GemmJob& g = gj[i];
    TmaJob& t = tj[i];
    std::memset(&t, 0, sizeof(t));
    const int na = g.a_exact ? 1 : 3, nb = g.b_exact ? 1 : 3;
    const int Kp = (std::max(g.K, 1) + 7) & ~7;
    // op(A)(m, k): ta = 0 -> A[m + k lda] (rows contiguous); ta = 1 -> A[k + m lda]
    __nv_bfloat16* a = split(g.A, g.lda, g.ta ? 1 : 0, g.M, std::max(g.K, 1), na);
    // op(B)^T(n, k) = op(B)(k, n): tb = 0 -> B[k + n ldb] (k contiguous); tb = 1 -> B[n + k ldb]
    __nv_bfloat16* b = split(g.B, g.ldb, g.tb ? 0 : 1, g.N, std::max(g.K, 1), nb);
    if (!a || !b) return -1;
    t.bn = std::min(128, (g.N + 15) & ~15);
    if (!encode3(&t.ta, a, Kp, g.M, na, TT_M) || !encode3(&t.tb, b, Kp, g.N, nb, t.bn)) return -1;
    t.C = g.C;
    t.crow = g.crow;
    t.ldc = g.ldc;
    t.M = g.M;
    t.N = g.N;
    t.K = std::max(g.K, 0);
    t.na = na;
    t.nb = nb;
    t.alpha = g.alpha;
    t.beta = g.beta;
    t0 += (long long)((g.M + TT_M - 1) / TT_M) * ((g.N + t.bn - 1) / t.bn);
  }
  // split K for launches with fewer tiles than one CTA per SM
  const int S = t0 < nsm ? (int)std::min<long long>(8, (nsm + t0 - 1) / t0) : 1;
  std::vector<Tile> tiles, rtiles;
  int max_stage = 0;
  for (size_t i = 0; i < tj.size(); ++i) {
    TmaJob& t = tj[i];
    const int tm = (t.M + TT_M - 1) / TT_M, tn = (t.N + t.bn - 1) / t.bn;
    const int ktiles = (t.K + TT_K - 1) / TT_K;
    int sk = std::min(S, ktiles / 4);  // at least 4 K tiles per split
    if (sk > 1) {
      t.ws = (float*)mem.alloc(sizeof(float) * (size_t)tm * tn * sk * TT_M * 128);
      if (!t.ws) sk = 1;
    }
    if (sk > 1) {
      t.ksplit = sk;
      t.tiles_m = tm;
      for (int b = 0; b < tn; ++b)
        for (int a = 0; a < tm; ++a) rtiles.push_back(Tile{(int)i, a, b, 0});
    }
    for (int q = 0; q < std::max(sk, 1); ++q)
      for (int b = 0; b < tn; ++b)
        for (int a = 0; a < tm; ++a) tiles.push_back(Tile{(int)i, a, b, q});
    max_stage = std::max(max_stage, t.na * TT_TERM_A + t.nb * t.bn * TT_K * 2);
  }
  int stages = std::min(TT_MAX_STAGES, TT_SMEM_BUDGET / std::max(max_stage, 1));
  if (stages < 2) return -1;
  const size_t smem = (size_t)stages * max_stage + 1024;
  const SplitJob* dsj = (const SplitJob*)mem.put(sj.data(), sizeof(SplitJob) * sj.size());
  const Tile* dst = (const Tile*)mem.put(st.data(), sizeof(Tile) * st.size());
  const TmaJob* dtj = (const TmaJob*)mem.put(tj.data(), sizeof(TmaJob) * tj.size());
  const Tile* dt = (const Tile*)mem.put(tiles.data(), sizeof(Tile) * tiles.size());
  const Tile* dr = rtiles.empty() ? nullptr : (const Tile*)mem.put(rtiles.data(), sizeof(Tile) * rtiles.size());
  if (!dsj || !dst || !dtj || !dt || (!rtiles.empty() && !dr)) return -1;
  if (!set_func_attr((const void*)k_gemm_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, TT_SMEM_BUDGET + 1024))
    return -1;
  k_split3<<<(int)st.size(), 256, 0, s>>>(dsj, dst);
  count_launch();
  k_gemm_tma<<<(int)tiles.size(), TT_THREADS, smem, s>>>(dtj, dt, stages, status);
  count_launch();
  if (dr) {
    k_gemm_tma_reduce<<<dim3((int)rtiles.size(), 128 / TT_RED_COLS), 256, 0, s>>>(dtj, dr);
    count_launch();
  }
  return 0;
}

}  // namespace hssmf
