// Device helpers shared by the interpolative-decomposition kernels
// (Section 2.2): the back substitution X = R1^-1 R2 and the pivot argmax.
#pragma once
#include <cuda_runtime.h>

namespace hssmf {

// One warp solves R1 x = b by column-oriented back substitution for nc <= 4
// right-hand sides b0..b3 (rows 0..k-1, overwritten by x): x_c = b_c /
// R1(c, c), then b[0:c] -= R1(0:c, c) x_c, reading column c of R1
// (rcol(c), rows 0..c-1) once for all right-hand sides; diag(c) = R1(c, c).
template <typename T, typename ColF, typename DiagF>
__device__ __forceinline__ void warp_backsub4(T* b0, T* b1, T* b2, T* b3, int nc, int k, ColF rcol,
                                              DiagF diag, int lane) {
  for (int c = k - 1; c >= 0; --c) {
    const T dc = diag(c);
    const T x0 = b0[c] / dc, x1 = b1[c] / dc, x2 = b2[c] / dc, x3 = b3[c] / dc;
    __syncwarp();
    if (lane == 0) {
      b0[c] = x0;
      if (nc > 1) b1[c] = x1;
      if (nc > 2) b2[c] = x2;
      if (nc > 3) b3[c] = x3;
    }
    const T* rc = rcol(c);
    for (int r = lane; r < c; r += 32) {
      const T a = rc[r];
      b0[r] -= a * x0;
      if (nc > 1) b1[r] -= a * x1;
      if (nc > 2) b2[r] -= a * x2;
      if (nc > 3) b3[r] -= a * x3;
    }
    __syncwarp();
  }
}

// Largest value, then smallest index, over the lanes whose index differs in
// the bits of the offsets 16 .. lo (lo = 1: the whole warp).
__device__ __forceinline__ void id_argmax(float& b, int& p, int lo = 1) {
#pragma unroll
  for (int o = 16; o >= lo; o >>= 1) {
    const float ov = __shfl_xor_sync(0xffffffffu, b, o);
    const int op = __shfl_xor_sync(0xffffffffu, p, o);
    if (ov > b || (ov == b && op < p)) {
      b = ov;
      p = op;
    }
  }
}

}  // namespace hssmf
