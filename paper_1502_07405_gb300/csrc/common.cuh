// Shared device-side definitions of the sm_103a kernels.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace hssmf {

// Bits of the device status word (sticky, OR-ed by kernels, read by the host
// at the end of every phase).  Kernels never trap: they record and return.
enum : unsigned {
  ST_ZERO_PIVOT = 1u,    // zero pivot in a partial LU / root LU
  ST_NONFINITE = 2u,     // non-finite pivot or norm
  ST_TIMEOUT = 4u,       // a bounded wait ran out
  ST_BAD_INDEX = 8u,     // an index map entry out of range (skipped)
};

struct GemmJob {
  // C[crow(i), j] = alpha * sum_k op(A)(i, k) op(B)(k, j) + beta * C[crow(i), j]
  // op(A) is M x K, op(B) is K x N; column-major with leading dimensions.
  const void* A;
  const void* B;
  void* C;
  const int* crow;  // optional row map of C (nullptr = identity)
  long long lda, ldb, ldc;
  int M, N, K;
  int ta, tb;  // 1 = use the transpose
  // FP32 tensor-core path: operand values exactly representable in BF16
  // (one split term instead of three); b_exact = 2: B is stored as BF16
  // (op(B)(k, j) at B[k + j ldb]: ldb a multiple of 8, B 16-byte aligned;
  // tensor-core tiles only)
  int a_exact, b_exact;
  double alpha, beta;
  // tensor-core split-K (ksplit > 1): tile (tm, tn) of split ks writes its
  // partial sums to ws + ((tm + tn tiles_m) ksplit + ks) 128^2, reduced in
  // split order by gemm_tc_reduce
  float* ws;
  int ksplit, tiles_m;
};

struct Tile {  // one output tile of one job (64 x 64 SIMT, 128 x 128 tensor cores); ks: K split
  int job, tm, tn, ks;
};

constexpr int GEMM_TILE = 64;
constexpr size_t kFrontLuSmemMax = 200 * 1024;  // shared memory of the persistent front kernel
constexpr int GEMM_TILE_TC = 128;
constexpr int GEMV_MAX_N = 4;  // products with N <= this use the GEMV kernel
// rows per GEMV tile: op(A) = A / op(A) = A^T
constexpr int GEMV_ROWS_N = 32, GEMV_ROWS_T = 8;

inline int ceil_div(long long a, int b) { return (int)((a + b - 1) / b); }

__device__ __forceinline__ void set_status(unsigned* st, unsigned bit) { atomicOr(st, bit); }

template <typename T>
__device__ __forceinline__ T tabs(T x) { return x < T(0) ? -x : x; }

}  // namespace hssmf
