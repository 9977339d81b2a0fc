// Allocation-free variant of the batched interpolative decomposition.
//
// Some callers cannot allocate device memory once they are running:
// cudaMalloc and cudaFree synchronize the whole device and stall the other
// streams of a latency-sensitive application; an application whose memory
// pool reserved the device memory up front leaves nothing for a library to
// allocate; and some code runs under a policy that forbids allocation after
// start-up.  For them, hssmf_batched_id_noalloc runs the one-CTA ID kernel
// with all of its scratch (job descriptors, ranks and the d x m work copy of
// every job) in a fixed array that is part of the library's device image.
#include <cuda_runtime.h>

#include <mutex>
#include <vector>

#include "../../include/hssmf.h"
#include "hss_kernels.h"

namespace hssmf {
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;  // 32 MiB per GPU

// Loaded with the library on every GPU that uses it and kept until the
// process exits.  Shared by every call on that GPU.
static __device__ __align__(256) unsigned char g_id_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of g_id_scratch on the current device (looked up once per
// device; the host-side symbol itself is not a device address).  The cached
// address assumes the device is not reset while the library is loaded: after
// cudaDeviceReset the module is loaded again, possibly elsewhere, and this
// entry point must not be used in that process any more.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_id_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

inline size_t round_up(size_t x) { return (x + 255) / 256 * 256; }

template <typename T>
hssmf_status run(int njobs, const void* Y, const long long* y_off, const int* m, const int* d,
                 double eps, int* rank_host, int* piv, const long long* p_off, void* X,
                 const long long* x_off, cudaStream_t s) {
  size_t wtot = 0;
  int max_m = 1, max_d = 1;
  for (int j = 0; j < njobs; ++j) {
    if (m[j] < 1 || d[j] < 1) return HSSMF_ERR_ARG;
    wtot += (size_t)m[j] * d[j];
    max_m = std::max(max_m, m[j]);
    max_d = std::max(max_d, d[j]);
  }
  const size_t jobs_bytes = round_up(sizeof(IdJob) * njobs);
  const size_t rank_bytes = round_up(sizeof(int) * njobs);
  if (jobs_bytes + rank_bytes + sizeof(T) * wtot > kNoAllocScratchBytes) return HSSMF_ERR_ARG;
  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) {
    cudaGetLastError();
    return HSSMF_ERR_CUDA;
  }
  char* b = static_cast<char*>(base);
  IdJob* djobs = reinterpret_cast<IdJob*>(b);
  int* ranks = reinterpret_cast<int*>(b + jobs_bytes);
  T* W = reinterpret_cast<T*>(b + jobs_bytes + rank_bytes);
  std::vector<IdJob> jobs(njobs);
  size_t w = 0;
  for (int j = 0; j < njobs; ++j) {
    jobs[j] = IdJob{(const T*)Y + y_off[j], W + w, piv + p_off[j], (T*)X + x_off[j], ranks + j, d[j], m[j]};
    w += (size_t)m[j] * d[j];
  }
  // The kernel overwrites every scratch word it reads (the work copy is
  // filled from Y, the ranks are written), so nothing is cleared here.
  if (cudaMemcpyAsync(djobs, jobs.data(), sizeof(IdJob) * njobs, cudaMemcpyHostToDevice, s) != cudaSuccess) {
    cudaGetLastError();
    return HSSMF_ERR_CUDA;
  }
  if (HssKern<T>::batched_id(djobs, njobs, max_m, max_d, eps, s) < 0) return HSSMF_ERR_ARG;
  // every step runs, and the error state is always read (and cleared), so a
  // failure here is not left behind for the caller's next CUDA call
  const cudaError_t e1 = cudaMemcpyAsync(rank_host, ranks, sizeof(int) * njobs, cudaMemcpyDeviceToHost, s);
  const cudaError_t e2 = cudaStreamSynchronize(s);
  const cudaError_t e3 = cudaGetLastError();
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) return HSSMF_ERR_CUDA;
  return HSSMF_OK;
}

}  // namespace
}  // namespace hssmf

extern "C" hssmf_status hssmf_batched_id_noalloc(int prec, int njobs, const void* Y, const long long* y_off,
                                                 const int* m, const int* d, double eps, int* rank_host,
                                                 int* piv, const long long* p_off, void* X,
                                                 const long long* x_off, void* cuda_stream) {
  if (njobs < 1 || !Y || !y_off || !m || !d || !rank_host || !piv || !p_off || !X || !x_off) return HSSMF_ERR_ARG;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (prec == HSSMF_PREC_FP64)
    return hssmf::run<double>(njobs, Y, y_off, m, d, eps, rank_host, piv, p_off, X, x_off, s);
  if (prec == HSSMF_PREC_FP32)
    return hssmf::run<float>(njobs, Y, y_off, m, d, eps, rank_host, piv, p_off, X, x_off, s);
  return HSSMF_ERR_ARG;
}
