// The solver context behind the opaque hssmf_ctx handle.
#pragma once
#include <cuda_runtime.h>

#include <memory>
#include <string>
#include <vector>

#include "../../include/hssmf.h"
#include "analyze.h"
#include "kernels.h"

namespace hssmf {

struct StepPlan {  // one panel step of the dense partial LU of a level
  int k0 = 0, trsm_chunks = 0, tile_off = 0, ntiles = 0;
  std::vector<int> prefix;  // GEMM tiles of the first i dense fronts of the level
};

struct LevelPlan {
  std::vector<int> dense, hss;  // dense fronts largest first
  int all_off = 0, nall = 0, dense_off = 0, ndense = 0, hss_off = 0;
  int max_nf = 0, max_nu = 0, max_nf_dense = 0;
  int asm_off = 0, asm_n = 0;
  std::vector<int> asm_prefix;  // assembly tiles of the first i dense fronts
  std::vector<StepPlan> steps;
  // split of the dense fronts: the first nlarge take the blocked panel path,
  // the others the persistent shared-memory kernel with `threads` threads
  // (chosen by the autotuner from timed trials, else the default bound)
  int nlarge = 0, nfmax = 0, threads = 256, tuned = 0;
  float tuned_ms = 0.f;
};

struct HssState;  // HSS-front factor data (hss.cu)

constexpr int kIdTraceFields = 11;  // ints per record of hssmf_get_id_trace

enum Phase {
  PH_DENSE = 0, PH_SAMPLE, PH_EXTRACT, PH_PREID, PH_ID, PH_POSTID, PH_ULV, PH_SCHUR, PH_SOLVE,
  PH_OUTER, PH_IDK, PH_COUNT  // PH_IDK: the ID kernels alone (PH_ID keeps the rest of that step)
};

// Phase timeline: an event is recorded at every phase change; the time
// between two consecutive events is charged to the earlier phase.  Events
// are resolved after stream synchronizations, so profiling adds no syncs.
struct PhaseProf {
  bool on = false;
  double ms[PH_COUNT] = {0};
  std::vector<std::pair<int, cudaEvent_t>> pending;
  std::vector<cudaEvent_t> spare;
  int cur = -2;
  void mark(int p, cudaStream_t s) {
    if (!on || p == cur) return;
    cudaEvent_t e;
    if (spare.empty()) {
      if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return; }
    } else {
      e = spare.back();
      spare.pop_back();
    }
    cudaEventRecord(e, s);
    pending.push_back({p, e});
    cur = p;
  }
  void resolve() {  // call only after the stream has been synchronized
    if (pending.size() < 2) return;
    for (size_t i = 0; i + 1 < pending.size(); ++i) {
      float t = 0.f;
      if (pending[i].first >= 0 && cudaEventElapsedTime(&t, pending[i].second, pending[i + 1].second) == cudaSuccess)
        ms[pending[i].first] += t;
      else
        cudaGetLastError();
      spare.push_back(pending[i].second);
    }
    pending.erase(pending.begin(), pending.end() - 1);
  }
  void finish(cudaStream_t s) {  // after a synchronization: close and drop the open interval
    mark(-1, s);
    cudaStreamSynchronize(s);
    resolve();
    for (auto& p : pending) spare.push_back(p.second);
    pending.clear();
    cur = -2;
  }
  void reset() {
    for (double& v : ms) v = 0.0;
  }
  void release() {
    for (auto& p : pending) cudaEventDestroy(p.second);
    for (auto e : spare) cudaEventDestroy(e);
    pending.clear();
    spare.clear();
  }
};

}  // namespace hssmf

struct hssmf_ctx {
  hssmf_opts opts{};
  bool fp32 = false;
  int num_sms = 148;  // streaming multiprocessors of the context's device
  cudaStream_t stream = nullptr;
  std::string err;
  bool analyzed = false, factored = false;
  hssmf::Symbolic sym;
  std::vector<hssmf::LevelPlan> plan;
  std::vector<int> is_hss;
  int n_hss = 0;
  hssmf::DevSym ds{};
  std::vector<hssmf::DFront> fronts_host;
  std::vector<hssmf::GemmJob> dense_jobs_host;
  std::vector<int> ints_host, flist_host, rowptr_host, colind_host;
  std::vector<hssmf::Tile> tiles_host;
  long long piv_total_host = 0;
  bool on_device = false;
  // device memory owned by the context
  std::vector<void*> owned, owned_host;
  unsigned* d_status = nullptr;
  int* d_counter = nullptr;  // work queue of the persistent front kernel
  bool autotune = true;       // time the dense-front splits at the first factorization
  int *d_perm = nullptr, *d_rowptr = nullptr, *d_colind = nullptr, *d_tpos = nullptr;
  double* d_values = nullptr;
  hssmf::DFront* d_fronts = nullptr;
  int* d_ints = nullptr;
  int* d_flist = nullptr;
  hssmf::Tile* d_tiles = nullptr;
  hssmf::GemmJob* d_jobs = nullptr;
  int* d_piv = nullptr;
  void* d_arena = nullptr;
  long long arena_elems = 0;
  // solve workspace
  void* d_W = nullptr;
  size_t w_bytes = 0;
  int w_nrhs = -1;
  double* d_io = nullptr;
  size_t io_bytes = 0;
  // Krylov workspace: kry_bytes / kry_nrhs describe the current layout inside
  // kry_base (kry_cap bytes); k_active holds act_cap ints
  size_t kry_bytes = 0, kry_cap = 0;
  int kry_nrhs = -1, act_cap = 0;
  double* kry_base = nullptr;
  double *k_V = nullptr, *k_Z = nullptr, *k_x = nullptr, *k_r = nullptr, *k_w = nullptr,
         *k_b = nullptr, *k_t = nullptr, *k_H = nullptr, *k_cs = nullptr, *k_sn = nullptr,
         *k_g = nullptr, *k_y = nullptr, *k_part = nullptr, *k_s = nullptr;
  int* k_active = nullptr;
  void* h_pin = nullptr;
  // per-system residual norms of a batch of independent grids
  int* d_sysoff = nullptr;
  double* k_seg = nullptr;
  size_t seg_cap = 0;
  // statistics
  hssmf_stats stats{};
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  double dense_flops = 0.0, hss_flops = 0.0, factor_bytes_dense = 0.0, hss_bytes = 0.0;
  int hss_max_rank = 0, hss_max_d = 0, hss_rounds = 0, hss_first_level = -1;
  int id_launches = 0;
  double id_bytes = 0.0, id_flops = 0.0;
  int factor_launches = 0;
  int last_iters = 0;
  double last_relres = 0.0;
  // HSS-front state
  hssmf::HssState* hss = nullptr;
  hssmf::PhaseProf prof;
  // per-node ID records of the last factor (profiling on): front, node, round,
  // d, m, mc, kr, kc, accepted, kernel of the row ID, kernel of the column ID
  std::vector<int> id_trace;
  // per-launch records of the ID kernels of the last profiled factor: kernel
  // code, CTAs per job, jobs, largest d, largest m, device ms
  std::vector<double> id_launch_trace;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> id_ev;  // pending, with their descriptors
  std::vector<double> id_ev_desc;

  hssmf_status fail(hssmf_status st, const std::string& msg);
  hssmf_status cuda_check(cudaError_t e, const char* what);
  void* dalloc(size_t bytes);
  void dfree(void* p);  // frees one allocation of dalloc (no-op for others)
  void free_all();
  void reset_device_pointers() {
    d_status = nullptr;
    d_counter = nullptr;
    d_perm = d_rowptr = d_colind = d_tpos = nullptr;
    d_values = nullptr;
    d_fronts = nullptr;
    d_ints = d_flist = d_piv = nullptr;
    d_tiles = nullptr;
    d_jobs = nullptr;
    d_arena = nullptr;
    d_W = nullptr;
    w_bytes = 0;
    w_nrhs = -1;
    d_io = nullptr;
    io_bytes = 0;
    kry_bytes = 0;
    kry_nrhs = -1;
    kry_cap = 0;
    act_cap = 0;
    kry_base = nullptr;
    k_active = nullptr;
    h_pin = nullptr;
    d_sysoff = nullptr;
    k_seg = nullptr;
    seg_cap = 0;
  }
  hssmf_status upload(void* dst, const void* src, size_t bytes);
  hssmf_status read_status();
  hssmf_status build_plan();
  hssmf_status ensure_device();
  template <typename T>
  hssmf_status factor_impl();
  template <typename T>
  int dense_level(const hssmf::LevelPlan& L, int nlarge, int nfmax, int threads);  // -1: refused
  template <typename T>
  hssmf_status tune_level(hssmf::LevelPlan& L);
  template <typename T>
  hssmf_status apply_impl(const double* b, double* x, int nrhs, int transpose);
  hssmf_status apply(const double* b, double* x, int nrhs, int transpose);
  hssmf_status ensure_krylov(int nrhs);
  hssmf_status read_cols(const double* dev, long long stride, int nrhs, std::vector<double>& out);
  hssmf_status outer_solve(const double* B, long long ldb, double* X, long long ldx, int nrhs,
                           int transpose);
  hssmf_status batched_refine(int nrhs, int transpose);
};
