// FP32 GEMM on the 5th-generation tensor cores (tcgen05, accumulators in
// tensor memory) for the dense contractions of the FP32 factorization: the
// sampling products U_child R of eq. FtimesR (Section 4.3), the sample
// updates of Algorithm 1 and the Schur-complement products (Sections 3.2,
// 4.4).
//
// FP32 accuracy from BF16 multiplies: every FP32 operand value x is split
// into three BF16 terms x = x0 + x1 + x2 (x0 = bf16(x), x1 = bf16(x - x0),
// x2 = bf16(x - x0 - x1)), which represent x to about 2^-24 |x|; the product
// keeps the six term products of order >= 2^-16 (i + j <= 2), accumulated in
// FP32 in tensor memory.  An operand whose values are exactly BF16 (the
// sampling matrix R of the FP32 form) uses one term, and its products drop to
// three.
//
// One CTA computes one 128 x 128 tile of C over its K range, 16 K per stage
// (two CTAs per SM).  The FP32 operand tiles of the stages ahead stream into
// a ring of three shared-memory staging slots with 4-byte asynchronous copies
// (cp.async, zero fill outside the matrices; any leading dimension, no
// alignment needed), two stages in flight while the current one is split:
// all 256 threads split a staged stage into its BF16 terms, stored in the
// canonical K-major layout (8 x 8 core matrices, no swizzle) of one of two
// term stages; one thread issues the tcgen05.mma instructions of the stage
// and commits them to the stage's mbarrier, which the threads wait on before
// refilling that term stage.  A B operand stored as BF16 (b_exact = 2: the
// FP32 form's sampling matrix) is copied 16 bytes at a time straight into
// the canonical layout of its staging slot and moved to the term stage
// without a split.  The accumulator (128 lanes x 128 FP32 columns) is read
// back with tcgen05.ld and scattered to the rows crow(i) of C.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/hssmf.h"
#include "gemm_tma.h"
#include "kernels.h"

namespace hssmf {

namespace {

constexpr int TC_M = 128, TC_N = 128, TC_K = 16;
constexpr int TC_THREADS = 256;
constexpr int TC_TERM_BYTES = TC_M * TC_K * 2;          // one BF16 term of one operand tile
constexpr int TC_STAGE_BYTES = 6 * TC_TERM_BYTES;       // 3 terms of A, 3 terms of B
constexpr int TC_STAGES = 2;
// FP32 staging: TC_ST slots of [A | B] tiles, each TC_K rows of TC_SLD
// floats (element (r, k) of op(X) at k TC_SLD + r: lanes along r read and
// write without bank conflicts whichever direction of X is contiguous)
constexpr int TC_ST = 3;
constexpr int TC_SLD = TC_M + 1;
constexpr int TC_STG = TC_K * TC_SLD;  // floats of one operand tile
constexpr int TC_SMEM = TC_STAGES * TC_STAGE_BYTES + TC_ST * 2 * TC_STG * 4 + 1024;  // + alignment slack
constexpr unsigned TC_TMEM_COLS = 128;
constexpr long long TC_SPIN = 1LL << 26;  // bound on every mbarrier wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Byte offset of element (r, k) of a 128 x TC_K K-major BF16 tile: core
// matrices of 8 rows x 16 bytes stored contiguously (128 B), the TC_K / 8
// core matrices along K of a row group adjacent (leading byte offset 128 B),
// row groups TC_SBO bytes apart (stride byte offset).
constexpr int TC_SBO = TC_K / 8 * 128;
__device__ __forceinline__ int tile_off(int r, int k) {
  return (r >> 3) * TC_SBO + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// tcgen05 shared-memory matrix descriptor, no swizzle: start address,
// leading byte offset 128, stride byte offset TC_SBO, descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(128 >> 4) << 16) |
         ((uint64_t)(TC_SBO >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, M = 128, N = n (multiple of 16).
__device__ __forceinline__ uint32_t instr_desc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// Waits for the completion of the phase with the given parity; false if the
// bound ran out.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (long long it = 0; it < TC_SPIN; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
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

// Splits 8 FP32 values into nt BF16 terms (packed 8 per uint4).
__device__ __forceinline__ void split8(const float* x, int nt, uint4* t0, uint4* t1, uint4* t2) {
  uint32_t w0[4], w1[4], w2[4];
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const float a = x[2 * p], b = x[2 * p + 1];
    __nv_bfloat162 h0 = __floats2bfloat162_rn(a, b);
    w0[p] = *reinterpret_cast<uint32_t*>(&h0);
    if (nt > 1) {
      const float ra = a - __low2float(h0), rb = b - __high2float(h0);
      __nv_bfloat162 h1 = __floats2bfloat162_rn(ra, rb);
      w1[p] = *reinterpret_cast<uint32_t*>(&h1);
      const float sa = ra - __low2float(h1), sb = rb - __high2float(h1);
      __nv_bfloat162 h2 = __floats2bfloat162_rn(sa, sb);
      w2[p] = *reinterpret_cast<uint32_t*>(&h2);
    }
  }
  *t0 = make_uint4(w0[0], w0[1], w0[2], w0[3]);
  if (nt > 1) {
    *t1 = make_uint4(w1[0], w1[1], w1[2], w1[3]);
    *t2 = make_uint4(w2[0], w2[1], w2[2], w2[3]);
  }
}

__device__ __forceinline__ void cp_async4(uint32_t dst, const float* src, int bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// One thread's share of the staging copies of an operand: element (r, k)
// of op(X) sits at P[r * sr + k * sk]; rc: rows contiguous (sr = 1), else k
// contiguous (sk = 1).  Per K step the thread copies 8 elements:
//   rc:  row tid % 128, k = tid / 128 + 2 e (a warp: 32 rows of one k);
//   !rc: k = tid % 16, rows rb + off(e), off(e) = 8 (e % 2) + 32 (e / 2),
//        rb = tid / 32 + 16 ((tid / 16) % 2) (a warp: 16 k of two rows 16
//        apart).
// Both write distinct banks of the [k][r] staging layout (row length
// TC_SLD).  Elements in rows outside the operand are not copied (their
// products land in rows or columns of C that are never stored); k past K is
// zero-filled.  Addresses are formed once per tile and advanced per step.
struct Feed {
  const float* p;    // element 0 of the current K step
  const float* base; // the operand's first element (the source of zero fills)
  long long sk16;    // advance per K step
  long long de;      // rc: advance between elements (2 sk)
  long long sr8;     // !rc: 8 sr
  uint32_t sdst;     // byte offset of element 0 in a staging tile
  unsigned rmask;    // bit e: element e's row lies inside the operand
  int kt;            // k of element 0 within the step
};
constexpr int TC_PER = TC_M * TC_K / TC_THREADS;  // elements per thread per operand tile
static_assert(TC_K == 16 && TC_M == 128 && TC_THREADS == 256 && TC_PER == 8, "staging map");

__device__ __forceinline__ Feed feed_init(const float* P, long long sr, long long sk, bool rc, int r0, int R,
                                          int kbeg) {
  Feed f;
  const int t = threadIdx.x;
  f.base = P;
  f.sk16 = 16 * sk;
  f.de = 2 * sk;
  f.sr8 = 8 * sr;
  if (rc) {
    const int r = t & 127;
    f.kt = t >> 7;
    f.p = P + (long long)(r0 + r) * sr + (long long)(kbeg + f.kt) * sk;
    f.rmask = r0 + r < R ? 0xFFu : 0u;
    f.sdst = 4u * (uint32_t)(f.kt * TC_SLD + r);
  } else {
    const int rb = (t >> 5) + 16 * ((t >> 4) & 1);
    f.kt = t & 15;
    f.p = P + (long long)(r0 + rb) * sr + (long long)(kbeg + f.kt) * sk;
    f.rmask = 0u;
#pragma unroll
    for (int e = 0; e < TC_PER; ++e)
      if (r0 + rb + 8 * (e & 1) + 32 * (e >> 1) < R) f.rmask |= 1u << e;
    f.sdst = 4u * (uint32_t)(f.kt * TC_SLD + rb);
  }
  return f;
}

// The copies of one K step (kleft: K values left from the step's start)
// into the staging tile at shared address tile.
template <bool RC>
__device__ __forceinline__ void feed_issue(const Feed& f, int kleft, uint32_t tile) {
  const uint32_t d0 = tile + f.sdst;
#pragma unroll
  for (int e = 0; e < TC_PER; ++e) {
    if (!((f.rmask >> e) & 1)) continue;
    const bool kv = RC ? f.kt + 2 * e < kleft : f.kt < kleft;
    const float* src = RC ? f.p + e * f.de : f.p + (e & 1) * f.sr8 + (e >> 1) * 4 * f.sr8;
    const uint32_t dst = d0 + 4u * (uint32_t)(RC ? 2 * e * TC_SLD : 8 * (e & 1) + 32 * (e >> 1));
    cp_async4(dst, kv ? src : f.base, kv ? 4 : 0);
  }
}

// Splits a staged 128 x TC_K tile into nt BF16 terms (canonical K-major
// layout): thread t takes row t % 128, k chunk t / 128 (8 values).
__device__ __forceinline__ void tile_split(const float* stg, int nt, char* dst, bool row_in) {
  static_assert(TC_M * TC_K / 8 == TC_THREADS, "one chunk per thread");
  if (!row_in) return;  // rows outside the operand: not staged, not needed
  const int r = threadIdx.x & 127, kc = threadIdx.x >> 7;
  float x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = stg[(8 * kc + j) * TC_SLD + r];
  uint4 t0, t1, t2;
  split8(x, nt, &t0, &t1, &t2);
  const int o = tile_off(r, 8 * kc);
  *reinterpret_cast<uint4*>(dst + o) = t0;
  if (nt > 1) {
    *reinterpret_cast<uint4*>(dst + TC_TERM_BYTES + o) = t1;
    *reinterpret_cast<uint4*>(dst + 2 * TC_TERM_BYTES + o) = t2;
  }
}

__global__ void __launch_bounds__(TC_THREADS, 2) k_gemm_tc(const GemmJob* __restrict__ jobs,
                                                           const Tile* __restrict__ tiles,
                                                           unsigned* __restrict__ status) {
  extern __shared__ char smem_raw[];
  __shared__ __align__(8) unsigned long long s_bar[TC_STAGES];
  __shared__ uint32_t s_tmem;
  char* smem = (char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const Tile tl = tiles[blockIdx.x];
  const GemmJob jb = jobs[tl.job];
  const int m0 = tl.tm * TC_M, n0 = tl.tn * TC_N;
  const int M = jb.M, N = jb.N, K = jb.K;
  const int na = jb.a_exact ? 1 : 3, nb = jb.b_exact ? 1 : 3;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // op(A)(i, k) = A[i + k lda] or A[k + i lda]; op(B)(k, j) = B[k + j ldb] or B[j + k ldb]
  const float* A = (const float*)jb.A;
  const float* B = (const float*)jb.B;
  const long long a_sr = jb.ta ? jb.lda : 1, a_sk = jb.ta ? 1 : jb.lda;
  const long long b_sr = jb.tb ? 1 : jb.ldb, b_sk = jb.tb ? jb.ldb : 1;
  const int nmma = min(TC_N, (N - n0 + 15) & ~15);
  const uint32_t idesc = instr_desc(nmma);
  // K range of this tile's split
  const int S = jb.ksplit > 1 ? jb.ksplit : 1;
  int kbeg = 0, kend = K;
  if (S > 1) {
    const int kc = ((K + S - 1) / S + TC_K - 1) / TC_K * TC_K;
    kbeg = min(K, tl.ks * kc);
    kend = min(K, kbeg + kc);
  }

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 32) {
    for (int s = 0; s < TC_STAGES; ++s) mbar_init(smem_u32(&s_bar[s]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;

  const int nk = (kend - kbeg + TC_K - 1) / TC_K;
  bool ok = true;
  int issued = 0;  // K steps whose MMAs were issued and committed
  float* stg = (float*)(smem + TC_STAGES * TC_STAGE_BYTES);
  const bool a_rc = jb.ta == 0, b_rc = jb.tb != 0;
  // b_exact 2: B is BF16 with k contiguous (ldb a multiple of 8, 16-byte
  // aligned): thread t copies the 16 bytes of row t % 128, k chunk t / 128
  // straight into the canonical term layout of the staging slot
  const bool b16 = jb.b_exact == 2;
  const bool a_row = m0 + (int)(threadIdx.x & 127) < M, b_row = n0 + (int)(threadIdx.x & 127) < N;
  const int b16_off = tile_off(threadIdx.x & 127, 8 * (threadIdx.x >> 7));
  const __nv_bfloat16* B16 = (const __nv_bfloat16*)jb.B;
  const __nv_bfloat16* b16_row = B16 + (long long)(n0 + (int)(threadIdx.x & 127)) * jb.ldb + 8 * (threadIdx.x >> 7);
  Feed fa = feed_init(A, a_sr, a_sk, a_rc, m0, M, kbeg);
  Feed fb = feed_init(B, b_sr, b_sk, b_rc, n0, N, kbeg);
  auto issue = [&](int u) {  // the copies of K step u into staging slot u % TC_ST (steps in order)
    const uint32_t d = smem_u32(stg + (size_t)(u % TC_ST) * 2 * TC_STG);
    const int k = kbeg + u * TC_K;
    const int kleft = kend - k;
    if (a_rc) feed_issue<true>(fa, kleft, d); else feed_issue<false>(fa, kleft, d);
    if (b16) {
      const int nv = min(max(kleft - 8 * (int)(threadIdx.x >> 7), 0), 8);  // valid k of the chunk
      if (b_row) cp_async16(d + 4 * TC_STG + b16_off, nv > 0 ? (const void*)(b16_row + k) : (const void*)B16, 2 * nv);
    } else if (b_rc) {
      feed_issue<true>(fb, kleft, d + 4 * TC_STG);
    } else {
      feed_issue<false>(fb, kleft, d + 4 * TC_STG);
    }
    fa.p += fa.sk16;
    fb.p += fb.sk16;
  };
  // one commit group per K step (empty past the end), so that waiting for
  // all but the last TC_ST - 1 groups means step t has landed
#pragma unroll
  for (int u = 0; u < TC_ST - 1; ++u) {
    if (u < nk) issue(u);
    cp_commit();
  }
  for (int t = 0; t < nk; ++t) {
    const int st = t & 1;
    char* sa = smem + st * TC_STAGE_BYTES;
    char* sb = sa + 3 * TC_TERM_BYTES;
    // slot (t - 1) % TC_ST was split in step t - 1, before its closing barrier
    if (t + TC_ST - 1 < nk) issue(t + TC_ST - 1);
    cp_commit();
    cp_wait<TC_ST - 1>();
    __syncthreads();  // every thread's copies of step t are visible
    // term stage st is free once the MMAs of step t - 2 completed; after a
    // wait that ran out nothing more is stored or issued (drain rule below)
    const bool free_ok = t < TC_STAGES || mbar_wait(smem_u32(&s_bar[st]), ((t - TC_STAGES) >> 1) & 1);
    if (free_ok) {
      const float* src = stg + (size_t)(t % TC_ST) * 2 * TC_STG;
      tile_split(src, na, sa, a_row);
      if (b16) {
        if (b_row)
          *reinterpret_cast<uint4*>(sb + b16_off) =
              *reinterpret_cast<const uint4*>(reinterpret_cast<const char*>(src + TC_STG) + b16_off);
      } else {
        tile_split(src + TC_STG, nb, sb, b_row);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (!__syncthreads_and(free_ok)) {  // the same decision in every thread
      ok = false;
      break;
    }
    issued = t + 1;
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_u32(sa), b0 = smem_u32(sb);
#pragma unroll
      for (int kk = 0; kk < TC_K / 16; ++kk) {
        for (int i = 0; i < na; ++i)
          for (int j = 0; j < nb && i + j <= 2; ++j) {
            const uint64_t ad = smem_desc(a0 + i * TC_TERM_BYTES + kk * 256);
            const uint64_t bd = smem_desc(b0 + j * TC_TERM_BYTES + kk * 256);
            mma_bf16(tmem, ad, bd, idesc, (t > 0 || kk > 0 || i > 0 || j > 0) ? 1u : 0u);
          }
      }
      mma_commit(smem_u32(&s_bar[st]));
    }
  }
  cp_wait<0>();  // no copy in flight past this point (also after a stop)
  // Drain rule: the last commit covers every MMA issued before it, so one
  // wait on it (bounded) covers exactly the work that was issued; after a
  // wait that ran out the loop stopped before storing or issuing more, the
  // accumulator is not read, and ST_TIMEOUT is reported.
  if (issued > 0 && !mbar_wait(smem_u32(&s_bar[(issued - 1) & 1]), ((issued - 1) >> 1) & 1)) ok = false;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  ok = __syncthreads_and(ok);
  if (!ok && threadIdx.x == 0) set_status(status, ST_TIMEOUT);

  // epilogue: warp w reads lanes 32 (w % 4) .. +31 (rows), columns 64 (w / 4) .. +63
  const int q = warp & 3, h = warp >> 2;
  const int i = 32 * q + lane, gi = m0 + i;
  const float alpha = (float)jb.alpha, beta = (float)jb.beta;
  const long long crow = gi < M ? (jb.crow ? jb.crow[gi] : gi) : 0;
  float* C = (float*)jb.C;
#pragma unroll 1
  for (int cb = 0; cb < 2; ++cb) {
    const int c0 = 64 * h + 32 * cb;
    if (c0 >= nmma) break;  // warp-uniform
    float v[32];
    if (nk > 0 && ok) {
      tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, v);
    } else {
#pragma unroll
      for (int e = 0; e < 32; ++e) v[e] = 0.f;
    }
    if (S > 1) {  // raw partial sums, column-major 128 x 128 per split
      float* wp = jb.ws + ((size_t)(tl.tm + tl.tn * jb.tiles_m) * S + tl.ks) * (TC_M * TC_N) + i;
#pragma unroll
      for (int e = 0; e < 32; ++e) wp[(size_t)(c0 + e) * TC_M] = v[e];
    } else if (gi < M) {
#pragma unroll
      for (int e = 0; e < 32; ++e) {
        const int gj = n0 + c0 + e;
        if (gj < N) {
          float* c = C + crow + (long long)gj * jb.ldc;
          *c = (jb.beta == 0.0) ? alpha * v[e] : alpha * v[e] + beta * *c;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS)
                 : "memory");
  }
}

}  // namespace

void gemm_tc(const GemmJob* jobs, const Tile* tiles, int ntiles, unsigned* status, cudaStream_t s) {
  if (ntiles <= 0) return;
  set_func_attr((const void*)k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
  k_gemm_tc<<<ntiles, TC_THREADS, TC_SMEM, s>>>(jobs, tiles, status);
  count_launch();
}

// Sum of the K-split partial tiles in split order (deterministic), then
// C[crow(i), j] = alpha sum + beta C.  CTA (x, y) takes output tile x
// (ks = 0), columns 16 y .. 16 y + 15: 2048 outputs, 8 a thread, whose loads
// are all issued before the first sum is used.
constexpr int TC_RED_COLS = 16;
__global__ void __launch_bounds__(256) k_gemm_tc_reduce(const GemmJob* __restrict__ jobs,
                                                        const Tile* __restrict__ tiles) {
  const Tile tl = tiles[blockIdx.x];
  const GemmJob jb = jobs[tl.job];
  const int S = jb.ksplit;
  const int m0 = tl.tm * TC_M, n0 = tl.tn * TC_N, c0 = blockIdx.y * TC_RED_COLS;
  const float* wp = jb.ws + (size_t)(tl.tm + tl.tn * jb.tiles_m) * S * (TC_M * TC_N);
  float* C = (float*)jb.C;
  const float alpha = (float)jb.alpha, beta = (float)jb.beta;
  constexpr int PER = TC_M * TC_RED_COLS / 256;
  float sum[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) sum[q] = 0.f;
  for (int ks = 0; ks < S; ++ks)
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int e = c0 * TC_M + threadIdx.x + 256 * q;  // column-major within the tile
      sum[q] += wp[(size_t)ks * (TC_M * TC_N) + e];
    }
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int e = c0 * TC_M + threadIdx.x + 256 * q;
    const int i = e % TC_M, c = e / TC_M;
    const int gi = m0 + i, gj = n0 + c;
    if (gi >= jb.M || gj >= jb.N) continue;
    const long long row = jb.crow ? jb.crow[gi] : gi;
    float* cp = C + row + (long long)gj * jb.ldc;
    *cp = (jb.beta == 0.0) ? alpha * sum[q] : alpha * sum[q] + beta * *cp;
  }
}

void gemm_tc_reduce(const GemmJob* jobs, const Tile* tiles, int ntiles, cudaStream_t s) {
  if (ntiles <= 0) return;
  k_gemm_tc_reduce<<<dim3(ntiles, TC_N / TC_RED_COLS), 256, 0, s>>>(jobs, tiles);
  count_launch();
}

}  // namespace hssmf

namespace {
// device scratch of hssmf_gemm_f32 calls: blocks kept across calls (every call
// synchronizes its stream before returning, so the next call may reuse them);
// a request takes the smallest free block that holds it, else a new block
std::mutex g_scratch_mu;
std::vector<std::pair<void*, size_t>> g_scratch;
struct CallScratch : hssmf::TmaScratch {
  std::vector<bool> used;
  std::vector<std::pair<void*, size_t>> pinned;  // host staging of the job arrays
  cudaStream_t s;
  explicit CallScratch(cudaStream_t st) : used(g_scratch.size(), false), s(st) {}
  void* alloc(size_t bytes) override {
    bytes = std::max<size_t>((bytes + 255) & ~(size_t)255, 256);
    int best = -1;
    for (size_t i = 0; i < g_scratch.size(); ++i)
      if (!used[i] && g_scratch[i].second >= bytes && (best < 0 || g_scratch[i].second < g_scratch[best].second))
        best = (int)i;
    if (best < 0) {
      void* p = nullptr;
      if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
      }
      g_scratch.push_back({p, bytes});
      used.push_back(false);
      best = (int)g_scratch.size() - 1;
    }
    used[best] = true;
    return g_scratch[best].first;
  }
  const void* put(const void* host, size_t bytes) override {
    void* p = alloc(bytes);
    if (p && bytes && cudaMemcpyAsync(p, host, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return nullptr;
    return p;
  }
};
}  // namespace

extern "C" hssmf_status hssmf_gemm_f32(int transa, int transb, int m, int n, int k, float alpha,
                                       const float* A, long long lda, const float* B, long long ldb,
                                       float beta, float* C, long long ldc, int b_exact, void* cuda_stream) {
  using namespace hssmf;
  if (m < 0 || n < 0 || k < 0) return HSSMF_ERR_ARG;
  if (m == 0 || n == 0) return HSSMF_OK;
  if (!C || ldc < m) return HSSMF_ERR_ARG;
  if (k > 0 && (!A || !B || lda < (transa ? k : m) || ldb < (transb ? n : k))) return HSSMF_ERR_ARG;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  GemmJob j;
  std::memset(&j, 0, sizeof(j));
  j.A = A; j.B = B; j.C = C;
  j.lda = lda; j.ldb = ldb; j.ldc = ldc;
  j.M = m; j.N = n; j.K = k;
  j.ta = transa != 0; j.tb = transb != 0;
  j.b_exact = (b_exact & 1) != 0;
  j.alpha = alpha; j.beta = beta;
  if (k > 0 && !(b_exact & 2) && gemm_tma_available()) {  // split operands + TMA/tcgen05 pipeline
    unsigned* st = nullptr;
    if (cudaMalloc(&st, sizeof(unsigned)) != cudaSuccess) return HSSMF_ERR_CUDA;
    unsigned hs = 0;
    hssmf_status r = HSSMF_OK;
    {
      std::lock_guard<std::mutex> lock(g_scratch_mu);
      CallScratch mem(s);
      if (cudaMemsetAsync(st, 0, sizeof(unsigned), s) != cudaSuccess) r = HSSMF_ERR_CUDA;
      if (!r && gemm_tma_batch(std::vector<GemmJob>{j}, mem, st, s) < 0) r = HSSMF_ERR_CUDA;
      if (!r && (cudaGetLastError() != cudaSuccess ||
                 cudaMemcpyAsync(&hs, st, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess))
        r = HSSMF_ERR_CUDA;
      if (cudaStreamSynchronize(s) != cudaSuccess) r = HSSMF_ERR_CUDA;
    }
    cudaFree(st);
    if (!r && (hs & ST_TIMEOUT)) r = HSSMF_ERR_TIMEOUT;
    return r;
  }
  // split K when the output has fewer tiles than about two CTAs per SM
  int nsm = 148, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int tm = ceil_div(m, GEMM_TILE_TC), tn = ceil_div(n, GEMM_TILE_TC);
  int S = 1;
  if (k >= 512 && (long long)tm * tn < 2LL * nsm)
    S = std::max(1, std::min({8, (int)((2LL * nsm + tm * tn - 1) / ((long long)tm * tn)), k / 256}));
  std::vector<Tile> tiles, rtiles;
  for (int q = 0; q < S; ++q)
    for (int b = 0; b < tn; ++b)
      for (int a = 0; a < tm; ++a) tiles.push_back(Tile{0, a, b, q});
  if (S > 1)
    for (int b = 0; b < tn; ++b)
      for (int a = 0; a < tm; ++a) rtiles.push_back(Tile{0, a, b, 0});
  const size_t ws_bytes = S > 1 ? sizeof(float) * (size_t)tm * tn * S * GEMM_TILE_TC * GEMM_TILE_TC : 0;
  const size_t bytes = 256 + sizeof(GemmJob) + sizeof(Tile) * (tiles.size() + rtiles.size()) + 256 + ws_bytes;
  char* d = nullptr;
  if (cudaMalloc(&d, bytes) != cudaSuccess) return HSSMF_ERR_CUDA;
  unsigned* st = (unsigned*)d;
  GemmJob* dj = (GemmJob*)(d + 256);
  Tile* dt = (Tile*)(d + 256 + sizeof(GemmJob));
  Tile* dr = dt + tiles.size();
  if (S > 1) {
    j.ws = (float*)(((uintptr_t)(dr + rtiles.size()) + 255) & ~(uintptr_t)255);
    j.ksplit = S;
    j.tiles_m = tm;
  }
  hssmf_status r = HSSMF_OK;
  unsigned hs = 0;
  if (cudaMemsetAsync(st, 0, sizeof(unsigned), s) != cudaSuccess ||
      cudaMemcpyAsync(dj, &j, sizeof(j), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(dt, tiles.data(), sizeof(Tile) * tiles.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      (S > 1 && cudaMemcpyAsync(dr, rtiles.data(), sizeof(Tile) * rtiles.size(), cudaMemcpyHostToDevice, s) !=
                    cudaSuccess))
    r = HSSMF_ERR_CUDA;
  if (r == HSSMF_OK) {
    gemm_tc(dj, dt, (int)tiles.size(), st, s);
    if (S > 1) gemm_tc_reduce(dj, dr, (int)rtiles.size(), s);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&hs, st, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      r = HSSMF_ERR_CUDA;
    else if (hs & ST_TIMEOUT)
      r = HSSMF_ERR_TIMEOUT;
  }
  cudaFree(d);
  return r;
}
