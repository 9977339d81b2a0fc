// FP32 products on the tensor cores through BF16 term arrays and TMA
// (k_gemm_tma.cu).
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <vector>

#include "kernels.h"

namespace hssmf {

constexpr int TT_MAX_STAGES = 8;

struct SplitJob {  // op(X) (rows x K) -> nt BF16 terms, K-major (ld Kp), term t at out + t term
  const float* X;
  long long ldx;
  int krow;  // 1: op(X)(r, k) = X[k + r ldx]; 0: X[r + k ldx]
  int rows, K, Kp, nt, pad;
  long long term;
  __nv_bfloat16* out;
};

struct TmaJob {  // (aligned as CUtensorMap: the maps are read by TMA from global memory)
  CUtensorMap ta;  // (Kp, M, na) terms of op(A), box (64, 128, 1), 128-byte swizzle
  CUtensorMap tb;  // (Kp, N, nb) terms of op(B)^T, box (64, bn, 1)
  void* C;
  const int* crow;
  long long ldc;
  int M, N, K, na, nb, bn;  // bn: tile columns, multiple of 16, <= 128
  double alpha, beta;
  float* ws;  // K split: partial tiles (128 x 128 stride) of split ks
  int ksplit, tiles_m;
};

// Device scratch for one batch (valid until its launches have run, in stream
// order): alloc() returns device memory, put() stages a host array on the device.
struct TmaScratch {
  virtual void* alloc(size_t bytes) = 0;
  virtual const void* put(const void* host, size_t bytes) = 0;
  virtual ~TmaScratch() = default;
};

// True when the driver's tensor-map encoder is available.
bool gemm_tma_available();
// Splits the operands and runs the FP32 jobs (N > GEMV_MAX_N) on the
// TMA/tcgen05 pipeline; status gets ST_TIMEOUT if a bounded wait ran out.
// Returns -1 (nothing launched) if a tensor map cannot be built or the
// scratch is exhausted.
int gemm_tma_batch(const std::vector<GemmJob>& jobs, TmaScratch& mem, unsigned* status, cudaStream_t s);

}  // namespace hssmf
