// C ABI of the solver: context, symbolic upload, level-batched numerical
// factorization, multifrontal solve and the FP64 outer iteration.
//
// The host walks the elimination-tree levels bottom-up and enqueues batched
// launches on one stream: every kernel of a level covers all fronts of that
// level (Section 5's tree parallelism becomes level batching).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <set>
#include <string>
#include <tuple>
#include <type_traits>
#include <vector>

#include "../../include/hssmf.h"
#include "analyze.h"
#include "hss.h"
#include "hss_kernels.h"
#include "kernels.h"
#include "solver_ctx.h"

namespace hssmf {
std::atomic<long long> g_launches{0};
std::atomic<int> g_launch_error{0};

bool set_func_attr(const void* func, cudaFuncAttribute attr, int value) {
  static std::mutex mu;
  static std::set<std::tuple<int, const void*, int, int>> done;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const auto key = std::make_tuple(dev, func, (int)attr, value);
  std::lock_guard<std::mutex> lock(mu);
  if (done.count(key)) return true;
  if (cudaFuncSetAttribute(func, attr, value) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  done.insert(key);
  return true;
}
}

using namespace hssmf;

namespace {

constexpr int NB = 32;  // panel width of the dense partial LU

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

hssmf_status hssmf_ctx::fail(hssmf_status st, const std::string& msg) {
  err = msg;
  return st;
}

hssmf_status hssmf_ctx::cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return HSSMF_OK;
  err = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? HSSMF_ERR_OOM : HSSMF_ERR_CUDA;
}

void* hssmf_ctx::dalloc(size_t bytes) {
  if (bytes == 0) bytes = 16;
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  owned.push_back(p);
  return p;
}

void hssmf_ctx::dfree(void* p) {
  if (!p) return;
  auto it = std::find(owned.begin(), owned.end(), p);
  if (it == owned.end()) return;
  cudaFree(p);
  owned.erase(it);
}

void hssmf_ctx::free_all() {
  for (void* p : owned) cudaFree(p);
  owned.clear();
  for (void* p : owned_host) cudaFreeHost(p);
  owned_host.clear();
}

hssmf_status hssmf_ctx::upload(void* dst, const void* src, size_t bytes) {
  if (bytes == 0) return HSSMF_OK;
  return cuda_check(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, stream), "upload");
}

hssmf_status hssmf_ctx::read_status() {
  if (g_launch_error.exchange(0)) {
    cudaGetLastError();
    return fail(HSSMF_ERR_CUDA, "a kernel launch was rejected");
  }
  unsigned st = 0;
  hssmf_status s = cuda_check(cudaMemcpyAsync(&st, d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, stream), "status");
  if (s) return s;
  s = cuda_check(cudaStreamSynchronize(stream), "synchronize");
  if (s) return s;
  if (st & ST_ZERO_PIVOT) return fail(HSSMF_ERR_SINGULAR, "zero pivot in a frontal factorization");
  if (st & ST_NONFINITE) return fail(HSSMF_ERR_SINGULAR, "non-finite value in a frontal factorization");
  if (st & ST_TIMEOUT) return fail(HSSMF_ERR_TIMEOUT, "a bounded device-side wait ran out");
  if (st & ST_BAD_INDEX) return fail(HSSMF_ERR_CUDA, "index map entry out of range");
  return HSSMF_OK;
}

// ---------------------------------------------------------------------------
// Structure upload and the static launch plan of the dense fronts
// ---------------------------------------------------------------------------
hssmf_status hssmf_ctx::build_plan() {
  const Symbolic& S = sym;
  const int nfr = (int)S.fronts.size();
  const size_t esz = fp32 ? sizeof(float) : sizeof(double);
  std::vector<DFront> fr(nfr);
  std::vector<int> ints;
  long long dense_elems = 0, piv_total = 0;
  is_hss.assign(nfr, 0);
  n_hss = 0;
  for (int i = 0; i < nfr; ++i) {
    const FrontSym& f = S.fronts[i];
    if (f.nf() >= opts.hss_min_front) {
      is_hss[i] = 1;
      ++n_hss;
    }
  }
  for (int i = 0; i < nfr; ++i) {
    const FrontSym& f = S.fronts[i];
    DFront& d = fr[i];
    std::memset(&d, 0, sizeof(DFront));
    d.nf = f.nf();
    d.ns = f.ns();
    d.nu = f.nu();
    d.sep_begin = f.sep_begin;
    d.nchild = f.nchild;
    d.child0 = f.child[0];
    d.child1 = f.child[1];
    d.is_hss = is_hss[i];
    if (!is_hss[i]) {
      d.off = dense_elems;
      dense_elems += (long long)d.nf * d.nf;
      d.u_off = d.off + d.ns + (long long)d.ns * d.nf;
      d.u_ld = d.nf;
      d.piv_off = piv_total;
      piv_total += d.ns;
    } else {
      d.off = -1;
      d.u_ld = std::max(d.nu, 1);
      d.piv_off = -1;
    }
    // inverse maps parent-local -> child I^upd index
    d.inv_off = (long long)ints.size();
    for (int c = 0; c < f.nchild; ++c) {
      size_t base = ints.size();
      ints.resize(base + d.nf, -1);
      const FrontSym& ch = S.fronts[f.child[c]];
      for (int j = 0; j < ch.nu(); ++j) ints[base + ch.pos_in_parent[j]] = j;
    }
    d.arow_off = (long long)ints.size();
    ints.insert(ints.end(), f.a_rowptr.begin(), f.a_rowptr.end());
    ints.insert(ints.end(), f.a_col.begin(), f.a_col.end());
    ints.insert(ints.end(), f.a_val.begin(), f.a_val.end());
    d.upd_off = (long long)ints.size();
    ints.insert(ints.end(), f.upd.begin(), f.upd.end());
  }
  // update matrices of HSS fronts live after the dense fronts
  for (int i = 0; i < nfr; ++i)
    if (is_hss[i]) {
      fr[i].u_off = dense_elems;
      dense_elems += (long long)fr[i].nu * fr[i].nu;
    }
  arena_elems = dense_elems;

  // level plans
  plan.assign(S.levels.size(), LevelPlan());
  std::vector<int> flist;
  std::vector<Tile> tiles;
  std::vector<GemmJob> jobs;
  for (size_t h = 0; h < S.levels.size(); ++h) {
    LevelPlan& L = plan[h];
    for (int f : S.levels[h]) (is_hss[f] ? L.hss : L.dense).push_back(f);
    std::stable_sort(L.dense.begin(), L.dense.end(), [&](int a, int b) { return fr[a].nf > fr[b].nf; });
    L.all_off = (int)flist.size();
    L.nall = (int)S.levels[h].size();
    for (int f : S.levels[h]) {
      flist.push_back(f);
      L.max_nf = std::max(L.max_nf, fr[f].nf);
      L.max_nu = std::max(L.max_nu, fr[f].nu);
      if (!is_hss[f]) L.max_nf_dense = std::max(L.max_nf_dense, fr[f].nf);
    }
    L.dense_off = (int)flist.size();
    L.ndense = (int)L.dense.size();
    int max_ns = 0;
    for (int f : L.dense) {
      flist.push_back(f);
      max_ns = std::max(max_ns, fr[f].ns);
    }
    L.hss_off = (int)flist.size();
    for (int f : L.hss) flist.push_back(f);
    // assembly tiles (32 x 32)
    L.asm_off = (int)tiles.size();
    L.asm_prefix.assign(1, 0);
    for (int f : L.dense) {
      int t = ceil_div(fr[f].nf, 32);
      for (int tn = 0; tn < t; ++tn)
        for (int tm = 0; tm < t; ++tm) tiles.push_back(Tile{f, tm, tn});
      L.asm_prefix.push_back((int)tiles.size() - L.asm_off);
    }
    L.asm_n = (int)tiles.size() - L.asm_off;
    // default split: every dense front whose matrix fits the persistent
    // kernel's shared memory goes to it (the autotuner may move the bound)
    L.nfmax = (int)std::sqrt((double)kFrontLuSmemMax / (double)esz);
    L.nlarge = 0;
    while (L.nlarge < (int)L.dense.size() && fr[L.dense[L.nlarge]].nf > L.nfmax) ++L.nlarge;
    // panel steps
    for (int k0 = 0; k0 < max_ns; k0 += NB) {
      StepPlan sp;
      sp.k0 = k0;
      sp.trsm_chunks = 0;
      sp.tile_off = (int)tiles.size();
      sp.prefix.assign(1, 0);
      for (int f : L.dense) {
        const DFront& d = fr[f];
        struct PrefixPush {  // the prefix grows by this front's tiles, however the loop body exits
          StepPlan& sp;
          std::vector<Tile>& t;
          ~PrefixPush() { sp.prefix.push_back((int)t.size() - sp.tile_off); }
        } pp{sp, tiles};
        if (k0 >= d.ns) continue;
        int k1 = std::min(k0 + NB, d.ns);
        sp.trsm_chunks = std::max(sp.trsm_chunks, ceil_div(d.nf - k1, 128));
        int M = d.nf - k1;
        if (M <= 0) continue;
        GemmJob j;
        std::memset(&j, 0, sizeof(j));
        j.A = (const void*)(uintptr_t)((d.off + k1 + (long long)k0 * d.nf) * esz);
        j.B = (const void*)(uintptr_t)((d.off + k0 + (long long)k1 * d.nf) * esz);
        j.C = (void*)(uintptr_t)((d.off + k1 + (long long)k1 * d.nf) * esz);
        j.lda = j.ldb = j.ldc = d.nf;
        j.M = M;
        j.N = M;
        j.K = k1 - k0;
        j.alpha = -1.0;
        j.beta = 1.0;
        int jid = (int)jobs.size();
        jobs.push_back(j);
        int t = ceil_div(M, GEMM_TILE);
        for (int tn = 0; tn < t; ++tn)
          for (int tm = 0; tm < t; ++tm) tiles.push_back(Tile{jid, tm, tn});
      }
      sp.ntiles = (int)tiles.size() - sp.tile_off;
      L.steps.push_back(sp);
    }
  }
  dense_jobs_host = jobs;  // A/B/C hold byte offsets into the arena until upload
  fronts_host = fr;
  ints_host = std::move(ints);
  flist_host = std::move(flist);
  tiles_host = std::move(tiles);
  piv_total_host = piv_total;
  factor_bytes_dense = 0;
  for (int i = 0; i < nfr; ++i)
    if (!is_hss[i]) factor_bytes_dense += (double)esz * ((double)fr[i].ns * fr[i].ns + 2.0 * fr[i].ns * fr[i].nu);
  return HSSMF_OK;
}

// First device use after analyze: allocate the factor storage and upload the
// structure and the static launch plan once.
hssmf_status hssmf_ctx::ensure_device() {
  if (on_device) return HSSMF_OK;
  const Symbolic& S = sym;
  const int n = S.n, nfr = (int)S.fronts.size();
  const size_t esz = fp32 ? sizeof(float) : sizeof(double);
  hssmf_status st;
  {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) ==
                                                   cudaSuccess && nsm > 0)
      num_sms = nsm;
    cudaGetLastError();
  }
  if (!ev0 && (st = cuda_check(cudaEventCreate(&ev0), "event"))) return st;
  if (!ev1 && (st = cuda_check(cudaEventCreate(&ev1), "event"))) return st;
  d_status = (unsigned*)dalloc(sizeof(unsigned) * 4);
  d_counter = (int*)dalloc(sizeof(int) * 4);
  d_perm = (int*)dalloc(sizeof(int) * n);
  d_rowptr = (int*)dalloc(sizeof(int) * (n + 1));
  d_colind = (int*)dalloc(sizeof(int) * std::max(S.nnz, 1));
  d_tpos = (int*)dalloc(sizeof(int) * std::max(S.nnz, 1));
  d_values = (double*)dalloc(sizeof(double) * std::max(S.nnz, 1));
  d_fronts = (DFront*)dalloc(sizeof(DFront) * std::max(nfr, 1));
  d_ints = (int*)dalloc(sizeof(int) * std::max<size_t>(ints_host.size(), 1));
  d_flist = (int*)dalloc(sizeof(int) * std::max<size_t>(flist_host.size(), 1));
  d_tiles = (Tile*)dalloc(sizeof(Tile) * std::max<size_t>(tiles_host.size(), 1));
  d_piv = (int*)dalloc(sizeof(int) * std::max<long long>(piv_total_host, 1));
  d_arena = dalloc(esz * std::max<long long>(arena_elems, 1));
  d_jobs = (GemmJob*)dalloc(sizeof(GemmJob) * std::max<size_t>(dense_jobs_host.size(), 1));
  d_sysoff = (int*)dalloc(sizeof(int) * (S.sys_off.size() + 1));
  if (!d_status || !d_counter || !d_perm || !d_rowptr || !d_colind || !d_tpos || !d_values || !d_fronts ||
      !d_ints || !d_flist || !d_tiles || !d_piv || !d_arena || !d_jobs || !d_sysoff)
    return fail(HSSMF_ERR_OOM, "device allocation of the factor storage failed");
  std::vector<GemmJob> jobs = dense_jobs_host;
  const uintptr_t base = (uintptr_t)d_arena;
  for (auto& j : jobs) {
    j.A = (const void*)(base + (uintptr_t)j.A);
    j.B = (const void*)(base + (uintptr_t)j.B);
    j.C = (void*)(base + (uintptr_t)j.C);
  }
  if ((st = cuda_check(cudaMemsetAsync(d_status, 0, sizeof(unsigned) * 4, stream), "memset"))) return st;
  if ((st = upload(d_perm, S.perm.data(), sizeof(int) * n))) return st;
  if ((st = upload(d_rowptr, rowptr_host.data(), sizeof(int) * (n + 1)))) return st;
  if ((st = upload(d_colind, colind_host.data(), sizeof(int) * S.nnz))) return st;
  if ((st = upload(d_tpos, S.tpos.data(), sizeof(int) * S.nnz))) return st;
  if ((st = upload(d_fronts, fronts_host.data(), sizeof(DFront) * nfr))) return st;
  if ((st = upload(d_ints, ints_host.data(), sizeof(int) * ints_host.size()))) return st;
  if ((st = upload(d_flist, flist_host.data(), sizeof(int) * flist_host.size()))) return st;
  if ((st = upload(d_tiles, tiles_host.data(), sizeof(Tile) * tiles_host.size()))) return st;
  if ((st = upload(d_jobs, jobs.data(), sizeof(GemmJob) * jobs.size()))) return st;
  if ((st = upload(d_sysoff, S.sys_off.data(), sizeof(int) * S.sys_off.size()))) return st;
  ds.fronts = d_fronts;
  ds.ints = d_ints;
  ds.perm = d_perm;
  ds.rowptr = d_rowptr;
  ds.colind = d_colind;
  ds.tpos = d_tpos;
  ds.n = n;
  ds.nnz = S.nnz;
  if ((st = hss_device_init(*this))) return st;
  if ((st = cuda_check(cudaStreamSynchronize(stream), "structure upload"))) return st;
  on_device = true;
  return HSSMF_OK;
}

// ---------------------------------------------------------------------------
// Numerical factorization
// ---------------------------------------------------------------------------
template <typename T>
int hssmf_ctx::dense_level(const LevelPlan& L, int nlarge, int nfmax, int threads) {
  T* ar = static_cast<T*>(d_arena);
  if (nlarge > 0) {
    Kern<T>::assemble(ds, ar, d_values, d_tiles + L.asm_off, L.asm_prefix[nlarge], stream);
    int max_ns = 0;
    for (int i = 0; i < nlarge; ++i) max_ns = std::max(max_ns, fronts_host[L.dense[i]].ns);
    for (const StepPlan& sp : L.steps) {
      if (sp.k0 >= max_ns) break;
      Kern<T>::panel_lu(ds, ar, d_piv, d_flist + L.dense_off, nlarge, sp.k0, NB, d_status, stream);
      Kern<T>::panel_trsm(ds, ar, d_flist + L.dense_off, nlarge, sp.k0, NB, sp.trsm_chunks, stream);
      Kern<T>::gemm(d_jobs, d_tiles + sp.tile_off, sp.prefix[nlarge], stream);  // K = NB: CUDA cores
    }
  }
  if (nlarge < L.ndense) {
    const int max_nf = fronts_host[L.dense[nlarge]].nf;  // largest first
    if (max_nf > nfmax) return -1;
    return Kern<T>::front_lu(ds, ar, d_values, d_piv, d_flist + L.dense_off + nlarge, L.ndense - nlarge, max_nf,
                             threads, num_sms, d_counter, d_status, stream);
  }
  return 0;
}

// Autotuner of a level's dense fronts (timed trials, once per analysis): the
// size bound below which fronts take the persistent shared-memory kernel
// (every distinct split of the level among the candidate bounds, including
// none) and its threads per CTA (128 or 256).  A level's dense work can be
// repeated: assembly rebuilds every front from A and the children's update
// matrices, which it does not modify.
template <typename T>
hssmf_status hssmf_ctx::tune_level(LevelPlan& L) {
  const size_t esz = sizeof(T);
  const int cap = (int)std::sqrt((double)kFrontLuSmemMax / (double)esz);
  const int bounds[] = {0, 48, 64, 96, 128, 160, 192, cap};
  float best = -1.f;
  int best_nl = L.ndense, best_b = 0, best_t = 256;
  int last_nl = -1;
  hssmf_status st;
  cudaEvent_t t0 = nullptr, t1 = nullptr;  // (the context's events time the whole factorization)
  if ((st = cuda_check(cudaEventCreate(&t0), "tuning"))) return st;
  if ((st = cuda_check(cudaEventCreate(&t1), "tuning"))) {
    cudaEventDestroy(t0);
    return st;
  }
  struct Ev {
    cudaEvent_t a, b;
    ~Ev() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } ev_guard{t0, t1};
  for (int b : bounds) {
    if (b > cap) continue;
    int nl = 0;
    while (nl < L.ndense && fronts_host[L.dense[nl]].nf > b) ++nl;
    if (nl == last_nl) continue;
    last_nl = nl;
    for (int t : {128, 256}) {
      if (nl == L.ndense && t == 128) continue;  // no persistent launch
      if ((st = cuda_check(cudaEventRecord(t0, stream), "tuning"))) return st;
      const int r = dense_level<T>(L, nl, b, t);
      if ((st = cuda_check(cudaEventRecord(t1, stream), "tuning"))) return st;
      if ((st = cuda_check(cudaEventSynchronize(t1), "tuning"))) return st;
      float ms = 0.f;
      if ((st = cuda_check(cudaEventElapsedTime(&ms, t0, t1), "tuning"))) return st;
      if (r < 0) continue;  // refused configuration
      if (best < 0.f || ms < best) {
        best = ms;
        best_nl = nl;
        best_b = b;
        best_t = t;
      }
    }
  }
  if (best >= 0.f) {
    L.nlarge = best_nl;
    L.nfmax = best_b;
    L.threads = best_t;
    L.tuned_ms = best;
  }
  L.tuned = 1;
  return HSSMF_OK;
}

template <typename T>
hssmf_status hssmf_ctx::factor_impl() {
  T* ar = static_cast<T*>(d_arena);
  hssmf_status st;
  dense_flops = 0.0;
  hss_begin_factor(*this);
  for (size_t h = 0; h < plan.size(); ++h) {
    const LevelPlan& L = plan[h];
    // dense fronts: the large ones by assembly and the blocked partial LU,
    // the others by the persistent shared-memory kernel (split tuned once)
    prof.mark(PH_DENSE, stream);
    if (autotune && !L.tuned && L.ndense > 0)
      if ((st = tune_level<T>(plan[h]))) return st;
    if (dense_level<T>(L, L.nlarge, L.nfmax, L.threads) < 0)
      return fail(HSSMF_ERR_CUDA, "the persistent dense-front kernel could not be launched");
    for (int f : L.dense) {
      double ns = fronts_host[f].ns, nu = fronts_host[f].nu;
      dense_flops += 2.0 / 3.0 * ns * ns * ns + 2.0 * ns * ns * nu + 2.0 * ns * nu * nu;
    }
    // HSS fronts of this level
    if (!L.hss.empty()) {
      if ((st = hss_factor_level<T>(*this, (int)h))) return st;
    }
  }
  return HSSMF_OK;
}

// ---------------------------------------------------------------------------
// Application of the factorization: x = M^-1 b (or M^-T b), FP64 in and out
// (n x nrhs, leading dimension n), arithmetic T inside.
// ---------------------------------------------------------------------------
template <typename T>
hssmf_status hssmf_ctx::apply_impl(const double* b, double* x, int nrhs, int transpose) {
  const int n = sym.n;
  const size_t esz = sizeof(T);
  // per-solve workspace sizes
  long long wtot = 0;
  for (auto& d : fronts_host) wtot += (long long)d.nf * nrhs;
  if (nrhs != w_nrhs) {
    long long off = 0;
    for (auto& d : fronts_host) {
      d.w_off = off;
      off += (long long)d.nf * nrhs;
    }
    hssmf_status st = upload(d_fronts, fronts_host.data(), sizeof(DFront) * fronts_host.size());
    if (st) return st;
    w_nrhs = nrhs;
  }
  if ((size_t)(wtot + 2LL * n * nrhs) * esz > w_bytes) {
    w_bytes = (size_t)(wtot + 2LL * n * nrhs) * esz;
    d_W = dalloc(w_bytes);
    if (!d_W) return fail(HSSMF_ERR_OOM, "solve workspace allocation failed");
  }
  T* W = static_cast<T*>(d_W);
  T* bp = W + wtot;
  T* xp = bp + (long long)n * nrhs;
  const T* ar = static_cast<const T*>(d_arena);
  prof.mark(PH_SOLVE, stream);
  Kern<T>::permute_in(b, n, bp, d_perm, n, nrhs, stream);
  for (size_t h = 0; h < plan.size(); ++h) {  // forward, bottom-up
    const LevelPlan& L = plan[h];
    Kern<T>::solve_gather(ds, W, bp, d_flist + L.all_off, L.nall, L.max_nf, nrhs, stream);
    Kern<T>::solve_fwd_dense(ds, ar, d_piv, W, d_flist + L.dense_off, L.ndense, L.max_nf_dense, nrhs, transpose,
                             stream);
    if (!L.hss.empty()) {
      hssmf_status st = hss_solve_fwd_level<T>(*this, (int)h, W, nrhs, transpose);
      if (st) return st;
    }
  }
  for (int h = (int)plan.size() - 1; h >= 0; --h) {  // backward, top-down
    const LevelPlan& L = plan[h];
    Kern<T>::solve_bwd_gather(ds, W, xp, d_flist + L.all_off, L.nall, L.max_nu, nrhs, stream);
    Kern<T>::solve_bwd_dense(ds, ar, d_piv, W, xp, d_flist + L.dense_off, L.ndense, L.max_nf_dense, nrhs,
                             transpose, stream);
    if (!L.hss.empty()) {
      hssmf_status st = hss_solve_bwd_level<T>(*this, h, W, xp, nrhs, transpose);
      if (st) return st;
    }
  }
  Kern<T>::permute_out(xp, x, n, d_perm, n, nrhs, stream);
  prof.mark(PH_OUTER, stream);
  return HSSMF_OK;
}

hssmf_status hssmf_ctx::apply(const double* b, double* x, int nrhs, int transpose) {
  return fp32 ? apply_impl<float>(b, x, nrhs, transpose) : apply_impl<double>(b, x, nrhs, transpose);
}

// ---------------------------------------------------------------------------
// Outer iteration (FP64): iterative refinement without HSS fronts,
// right-preconditioned GMRES(m) with modified Gram-Schmidt otherwise.
// ---------------------------------------------------------------------------
hssmf_status hssmf_ctx::ensure_krylov(int nrhs) {
  const int n = sym.n, m = std::max(opts.gmres_restart, 1);
  const size_t nn = (size_t)n * nrhs;
  // refinement (no HSS front, or a batch of grids) keeps no Krylov basis
  const bool basis = n_hss > 0 && sym.nsys == 1 && opts.maxit > 0;
  // layout (in doubles); the allocation is the exact sum of these sizes
  const size_t sizes[] = {basis ? nn * (m + 1) : 0, basis ? nn * m : 0, nn, nn, nn, nn, nn,
                          (size_t)(m + 1) * m * nrhs, (size_t)m * nrhs, (size_t)m * nrhs,
                          (size_t)(m + 1) * nrhs, (size_t)m * nrhs, 64 * (size_t)nrhs,
                          8 * (size_t)nrhs};
  double** ptrs[] = {&k_V, &k_Z, &k_x, &k_r, &k_w, &k_b, &k_t, &k_H, &k_cs, &k_sn, &k_g, &k_y,
                     &k_part, &k_s};
  size_t total = 0;
  for (size_t s : sizes) total += s;
  const size_t need = sizeof(double) * total;
  if (need <= kry_bytes && nrhs == kry_nrhs) return HSSMF_OK;
  // a smaller or equal workspace is laid out again inside the current one;
  // a larger one replaces it (queued work may still read the old one)
  if (need > kry_cap || nrhs > act_cap) {
    cudaStreamSynchronize(stream);
    dfree(kry_base);
    dfree(k_active);
    kry_base = nullptr;
    k_active = nullptr;
    kry_cap = 0;
    act_cap = 0;
    kry_bytes = 0;
    kry_nrhs = -1;
    double* p = (double*)dalloc(need);
    int* a = (int*)dalloc(sizeof(int) * (size_t)nrhs);
    if (!p || !a) return fail(HSSMF_ERR_OOM, "Krylov workspace allocation failed");
    kry_base = p;
    kry_cap = need;
    k_active = a;
    act_cap = nrhs;
  }
  double* p = kry_base;
  for (size_t i = 0; i < sizeof(sizes) / sizeof(sizes[0]); ++i) {
    *ptrs[i] = p;
    p += sizes[i];
  }
  kry_bytes = need;
  kry_nrhs = nrhs;
  if (!h_pin) {
    if (cudaMallocHost(&h_pin, 1 << 20) != cudaSuccess) {
      cudaGetLastError();
      return fail(HSSMF_ERR_OOM, "pinned host allocation failed");
    }
    owned_host.push_back(h_pin);
  }
  return HSSMF_OK;
}

hssmf_status hssmf_ctx::read_cols(const double* dev, long long stride, int nrhs, std::vector<double>& out) {
  double* hp = (double*)h_pin;
  out.resize(nrhs);
  if (stride == 1) {
    hssmf_status st = cuda_check(cudaMemcpyAsync(hp, dev, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, stream), "read");
    if (st) return st;
  } else {
    for (int c = 0; c < nrhs; ++c) {
      hssmf_status st = cuda_check(cudaMemcpyAsync(hp + c, dev + c * stride, sizeof(double), cudaMemcpyDeviceToHost, stream), "read");
      if (st) return st;
    }
  }
  hssmf_status st = cuda_check(cudaStreamSynchronize(stream), "read sync");
  if (st) return st;
  for (int c = 0; c < nrhs; ++c) out[c] = hp[c];
  return HSSMF_OK;
}

hssmf_status hssmf_ctx::outer_solve(const double* B, long long ldb, double* X, long long ldx, int nrhs, int transpose) {
  const int n = sym.n;
  hssmf_status st;
  last_iters = 0;
  last_relres = 0.0;
  if (opts.maxit <= 0) {  // apply the factorization once
    if ((st = ensure_krylov(nrhs))) return st;
    copy_cols(k_b, n, B, ldb, n, nrhs, stream);
    count_launch();
    if ((st = apply(k_b, k_x, nrhs, transpose))) return st;
    copy_cols(X, ldx, k_x, n, n, nrhs, stream);
    count_launch();
    last_iters = 1;
    return HSSMF_OK;
  }
  if ((st = ensure_krylov(nrhs))) return st;
  copy_cols(k_b, n, B, ldb, n, nrhs, stream);
  count_launch();
  if (sym.nsys > 1) {
    if ((st = batched_refine(nrhs, transpose))) {
      copy_cols(X, ldx, k_x, n, n, nrhs, stream);
      return st;
    }
    copy_cols(X, ldx, k_x, n, n, nrhs, stream);
    count_launch();
    return HSSMF_OK;
  }
  std::vector<double> bn, rn;
  dots(k_b, k_b, n, nrhs, k_part, k_s, 1, stream);
  if ((st = read_cols(k_s, 1, nrhs, bn))) return st;
  for (auto& v : bn) v = std::sqrt(v);
  const double rtol = opts.rtol;
  std::vector<int> act(nrhs, 1), its(nrhs, 0);
  auto upload_active = [&]() { return upload(k_active, act.data(), sizeof(int) * nrhs); };
  if (n_hss == 0) {
    // iterative refinement: x = M^-1 b; x += M^-1 (b - A x)
    if ((st = apply(k_b, k_x, nrhs, transpose))) return st;
    for (int c = 0; c < nrhs; ++c) its[c] = 1;
    for (int it = 0;; ++it) {
      residual(ds, d_values, k_b, n, k_x, k_r, nrhs, transpose, stream);
      dots(k_r, k_r, n, nrhs, k_part, k_s, 1, stream);
      if ((st = read_cols(k_s, 1, nrhs, rn))) return st;
      bool all = true;
      for (int c = 0; c < nrhs; ++c) {
        double rel = bn[c] > 0 ? std::sqrt(rn[c]) / bn[c] : 0.0;
        last_relres = std::max(last_relres, rel);
        if (rel <= rtol || !act[c]) act[c] = 0; else all = false;
      }
      if (all) break;
      if (*std::max_element(its.begin(), its.end()) >= opts.maxit) {
        copy_cols(X, ldx, k_x, n, n, nrhs, stream);
        last_iters = *std::max_element(its.begin(), its.end());
        return fail(HSSMF_ERR_NOCONV, "iterative refinement did not reach rtol");
      }
      last_relres = 0.0;
      if ((st = upload_active())) return st;
      if ((st = apply(k_r, k_w, nrhs, transpose))) return st;
      add_cols(k_x, k_w, n, nrhs, k_active, stream);
      for (int c = 0; c < nrhs; ++c) its[c] += act[c];
    }
    copy_cols(X, ldx, k_x, n, n, nrhs, stream);
    last_iters = *std::max_element(its.begin(), its.end());
    return HSSMF_OK;
  }
  // GMRES(m), right preconditioned, x0 = 0
  const int m = std::max(opts.gmres_restart, 1);
  const long long nn = (long long)n * nrhs;
  const long long hs = (long long)(m + 1) * m;  // H stride per rhs
  cudaMemsetAsync(k_x, 0, sizeof(double) * nn, stream);
  copy_cols(k_r, n, k_b, n, n, nrhs, stream);
  count_launch();
  std::vector<double> beta = bn;
  for (int c = 0; c < nrhs; ++c) act[c] = bn[c] > 0 ? 1 : 0;
  while (true) {
    if ((st = upload_active())) return st;
    cudaMemsetAsync(k_g, 0, sizeof(double) * (m + 1) * nrhs, stream);
    cudaMemsetAsync(k_H, 0, sizeof(double) * hs * nrhs, stream);
    // g(0) = beta, V0 = r / beta
    for (int c = 0; c < nrhs; ++c) ((double*)h_pin)[c] = beta[c];
    for (int c = 0; c < nrhs; ++c)
      cudaMemcpyAsync(k_g + (long long)(m + 1) * c, (double*)h_pin + c, sizeof(double), cudaMemcpyHostToDevice, stream);
    scale_dev(k_V, k_r, k_g, m + 1, n, nrhs, stream);
    std::vector<int> jend(nrhs, 0);
    std::vector<int> inner = act;  // columns still iterating in this cycle
    for (int j = 0; j < m; ++j) {
      bool any = false;
      for (int c = 0; c < nrhs; ++c) any |= inner[c] != 0;
      if (!any) break;
      double* Vj = k_V + nn * j;
      double* Zj = k_Z + nn * j;
      if ((st = apply(Vj, Zj, nrhs, transpose))) return st;
      spmv(ds, d_values, Zj, k_w, nrhs, transpose, stream);
      for (int i = 0; i <= j; ++i) {  // modified Gram-Schmidt
        double* hij = k_H + i + (long long)(m + 1) * j;
        dots(k_w, k_V + nn * i, n, nrhs, k_part, hij, hs, stream);
        axpy_dev(k_w, k_V + nn * i, hij, hs, -1.0, n, nrhs, k_active, stream);
      }
      double* hj1 = k_H + (j + 1) + (long long)(m + 1) * j;
      dots(k_w, k_w, n, nrhs, k_part, hj1, hs, stream);
      sqrt_dev(hj1, hs, nrhs, stream);
      scale_dev(k_V + nn * (j + 1), k_w, hj1, hs, n, nrhs, stream);
      givens_step(k_H, k_cs, k_sn, k_g, m, j, nrhs, k_active, stream);
      for (int c = 0; c < nrhs; ++c) its[c] += inner[c];
      std::vector<double> gj;
      if ((st = read_cols(k_g + (j + 1), m + 1, nrhs, gj))) return st;
      bool changed = false;
      for (int c = 0; c < nrhs; ++c) {
        if (!inner[c]) continue;
        jend[c] = j + 1;
        bool stop = std::fabs(gj[c]) <= rtol * bn[c] || its[c] >= opts.maxit || j + 1 == m;
        if (stop) {
          // finalize this column: y = H^-1 g, x += Z y
          std::vector<int> one(nrhs, 0);
          one[c] = 1;
          if ((st = upload(k_active, one.data(), sizeof(int) * nrhs))) return st;
          hess_solve(k_H, k_g, k_y, m, j + 1, nrhs, k_active, stream);
          update_x(k_x, k_Z, nn, k_y, m, j + 1, n, nrhs, k_active, stream);
          inner[c] = 0;
          changed = true;
        }
      }
      if (changed) {
        if ((st = upload(k_active, inner.data(), sizeof(int) * nrhs))) return st;
      }
    }
    // true residual
    residual(ds, d_values, k_b, n, k_x, k_r, nrhs, transpose, stream);
    dots(k_r, k_r, n, nrhs, k_part, k_s, 1, stream);
    if ((st = read_cols(k_s, 1, nrhs, rn))) return st;
    bool all = true, out_of_its = false;
    last_relres = 0.0;
    for (int c = 0; c < nrhs; ++c) {
      beta[c] = std::sqrt(rn[c]);
      double rel = bn[c] > 0 ? beta[c] / bn[c] : 0.0;
      last_relres = std::max(last_relres, rel);
      if (rel <= rtol || bn[c] == 0) act[c] = 0;
      else {
        act[c] = 1;
        all = false;
        if (its[c] >= opts.maxit) out_of_its = true;
      }
    }
    if (all) break;
    if (out_of_its) {
      copy_cols(X, ldx, k_x, n, n, nrhs, stream);
      last_iters = *std::max_element(its.begin(), its.end());
      return fail(HSSMF_ERR_NOCONV, "GMRES did not reach rtol within maxit");
    }
  }
  copy_cols(X, ldx, k_x, n, n, nrhs, stream);
  count_launch();
  last_iters = *std::max_element(its.begin(), its.end());
  return HSSMF_OK;
}

// Independent grids (a block-diagonal system): iterative refinement
// x <- x + M^-1 (b - A x) on all of them at once, stopped when the relative
// residual of every grid and right-hand side is <= rtol.  A Krylov method
// over the stacked vector would couple the grids through shared
// coefficients; refinement needs only the per-grid norms.  b is in k_b, the
// solution is left in k_x.
hssmf_status hssmf_ctx::batched_refine(int nrhs, int transpose) {
  const int n = sym.n, ns = sym.nsys;
  const size_t nv = (size_t)ns * nrhs;
  if (nv > ((size_t)1 << 20) / sizeof(double) || nrhs > 65535)
    return fail(HSSMF_ERR_ARG, "grids x right-hand sides above 131072 (or nrhs above 65535) in one refinement");
  if (nv > seg_cap) {
    k_seg = (double*)dalloc(sizeof(double) * nv);
    if (!k_seg) return fail(HSSMF_ERR_OOM, "refinement norm buffer");
    seg_cap = nv;
  }
  hssmf_status st;
  std::vector<double> bn, rn;
  seg_norms2(k_b, n, nrhs, d_sysoff, ns, k_seg, stream);
  if ((st = read_cols(k_seg, 1, (int)nv, bn))) return st;
  std::vector<int> act(nrhs, 1);
  if ((st = apply(k_b, k_x, nrhs, transpose))) return st;
  int it = 1;
  for (;;) {
    residual(ds, d_values, k_b, n, k_x, k_r, nrhs, transpose, stream);
    seg_norms2(k_r, n, nrhs, d_sysoff, ns, k_seg, stream);
    if ((st = read_cols(k_seg, 1, (int)nv, rn))) return st;
    last_relres = 0.0;
    bool all = true;
    for (int c = 0; c < nrhs; ++c) {
      act[c] = 0;
      for (int g = 0; g < ns; ++g) {
        const size_t v = (size_t)g + (size_t)ns * c;
        const double rel = bn[v] > 0 ? std::sqrt(rn[v] / bn[v]) : (rn[v] > 0 ? INFINITY : 0.0);
        last_relres = std::max(last_relres, rel);
        if (!(rel <= opts.rtol)) act[c] = 1;
      }
      all = all && !act[c];
    }
    if (all) break;
    if (it >= opts.maxit) {
      last_iters = it;
      return fail(HSSMF_ERR_NOCONV, "iterative refinement did not reach rtol in every grid");
    }
    if ((st = upload(k_active, act.data(), sizeof(int) * nrhs))) return st;
    if ((st = apply(k_r, k_w, nrhs, transpose))) return st;
    add_cols(k_x, k_w, n, nrhs, k_active, stream);
    ++it;
  }
  last_iters = it;
  return HSSMF_OK;
}

// Symbolic phase common to every analysis entry point: run the ordering,
// keep the pattern, build the launch plans and the HSS structure.
template <class F>
static hssmf_status analyze_common(hssmf_ctx* c, int n, const int* rowptr, const int* colind, F order) {
  if (!c) return HSSMF_ERR_ARG;
  auto t0 = std::chrono::steady_clock::now();
  if (c->on_device) cudaStreamSynchronize(c->stream);
  c->free_all();
  hss_release(*c);
  c->reset_device_pointers();
  c->on_device = false;
  c->analyzed = c->factored = false;
  std::string e = order();
  if (!e.empty()) return c->fail(HSSMF_ERR_ARG, e);
  hssmf_status st;
  const Symbolic& S = c->sym;
  c->rowptr_host.assign(rowptr, rowptr + n + 1);
  c->colind_host.assign(colind, colind + S.nnz);
  if ((st = c->build_plan())) return st;
  if ((st = hss_prepare(*c))) return st;
  c->analyzed = true;
  c->stats = hssmf_stats();
  c->stats.n = n;
  c->stats.n_fronts = (int)S.fronts.size();
  c->stats.n_levels = (int)S.levels.size();
  c->stats.n_hss_fronts = c->n_hss;
  for (auto& f : S.fronts) c->stats.max_front = std::max(c->stats.max_front, f.nf());
  c->stats.t_analyze_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return HSSMF_OK;
}

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void hssmf_default_opts(hssmf_opts* o) {
  if (!o) return;
  o->hss_tol = 1e-4;
  o->d0 = 128;
  o->dd = 64;
  o->oversample_p = 10;
  o->hss_min_front = 1024;
  o->hss_leaf = 128;
  o->nd_leaf = 8;
  o->seed = 0;
  o->precision = HSSMF_PREC_FP64;
  o->gmres_restart = 30;
  o->maxit = 300;
  o->rtol = 1e-10;
}

hssmf_status hssmf_create(hssmf_ctx** out, const hssmf_opts* opts, void* stream) {
  if (!out) return HSSMF_ERR_ARG;
  *out = nullptr;
  hssmf_ctx* c = new (std::nothrow) hssmf_ctx();
  if (!c) return HSSMF_ERR_OOM;
  if (opts) c->opts = *opts; else hssmf_default_opts(&c->opts);
  const hssmf_opts& o = c->opts;
  if (o.d0 < 1 || o.dd < 1 || o.oversample_p < 0 || o.hss_leaf < 1 || o.nd_leaf < 1 ||
      o.gmres_restart < 1 || !(o.hss_tol >= 0) || o.maxit < 0 ||
      (o.precision != HSSMF_PREC_FP64 && o.precision != HSSMF_PREC_FP32)) {
    delete c;
    return HSSMF_ERR_ARG;
  }
  c->fp32 = o.precision == HSSMF_PREC_FP32;
  c->stream = (cudaStream_t)stream;
  *out = c;
  return HSSMF_OK;
}

hssmf_status hssmf_analyze_grid(hssmf_ctx* c, int nx, int ny, int nz, int n, const int* rowptr,
                                const int* colind) {
  const int dims[3] = {nx, ny, nz};
  return hssmf_analyze_grids(c, 1, dims, n, rowptr, colind);
}

hssmf_status hssmf_analyze_grids(hssmf_ctx* c, int nsys, const int* dims, int n, const int* rowptr,
                                 const int* colind) {
  if (!c) return HSSMF_ERR_ARG;
  return analyze_common(c, n, rowptr, colind, [&] {
    return analyze_grids(nsys, dims, n, rowptr, colind, c->opts.nd_leaf, c->opts.hss_leaf, c->sym);
  });
}

hssmf_status hssmf_analyze_csr(hssmf_ctx* c, int n, const int* rowptr, const int* colind, int nfronts,
                               const int* perm, const int* sep_ptr, const int* parent) {
  if (!c) return HSSMF_ERR_ARG;
  if (n < 1 || !rowptr || !colind) return c->fail(HSSMF_ERR_ARG, "empty or null pattern");
  return analyze_common(c, n, rowptr, colind, [&] {
    return analyze_csr(n, rowptr, colind, nfronts, perm, sep_ptr, parent, c->opts.nd_leaf, c->opts.hss_leaf,
                       c->sym);
  });
}

hssmf_status hssmf_factor(hssmf_ctx* c, const double* values) {
  if (!c || !values) return HSSMF_ERR_ARG;
  if (!c->analyzed) return c->fail(HSSMF_ERR_ARG, "factor called before analyze");
  hssmf_status st;
  if ((st = c->ensure_device())) return st;
  const size_t vb = sizeof(double) * c->sym.nnz;
  long long l0 = g_launches.load();
  c->prof.reset();
  cudaEventRecord(c->ev0, c->stream);
  c->prof.mark(PH_DENSE, c->stream);
  if (is_device_ptr(values)) {
    if ((st = c->cuda_check(cudaMemcpyAsync(c->d_values, values, vb, cudaMemcpyDeviceToDevice, c->stream), "values"))) return st;
  } else {
    if ((st = c->cuda_check(cudaMemcpyAsync(c->d_values, values, vb, cudaMemcpyHostToDevice, c->stream), "values"))) return st;
  }
  cudaMemsetAsync(c->d_status, 0, sizeof(unsigned) * 4, c->stream);
  c->factored = false;
  st = c->fp32 ? c->factor_impl<float>() : c->factor_impl<double>();
  if (st) return st;
  cudaEventRecord(c->ev1, c->stream);
  if ((st = c->cuda_check(cudaGetLastError(), "factor launch"))) return st;
  if ((st = c->read_status())) return st;
  c->prof.finish(c->stream);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  c->stats.t_factor_ms = ms;
  c->stats.factor_flops = c->dense_flops + c->hss_flops;
  c->stats.factor_bytes = c->factor_bytes_dense + c->hss_bytes;
  c->factor_launches = (int)(g_launches.load() - l0);
  c->factored = true;
  return HSSMF_OK;
}

static hssmf_status solve_common(hssmf_ctx* c, const double* B, double* X, int nrhs, int ldb, int transpose) {
  if (!c || !B || !X || nrhs < 1) return HSSMF_ERR_ARG;
  if (!c->factored) return c->fail(HSSMF_ERR_ARG, "solve called before a successful factor");
  const int n = c->sym.n;
  if (ldb < n) return c->fail(HSSMF_ERR_ARG, "ldb < n");
  hssmf_status st;
  long long l0 = g_launches.load();
  const bool bdev = is_device_ptr(B), xdev = is_device_ptr(X);
  const size_t bytes = sizeof(double) * (size_t)n * nrhs;
  if ((!bdev || !xdev) && c->io_bytes < 2 * bytes) {
    c->io_bytes = 2 * bytes;
    c->d_io = (double*)c->dalloc(c->io_bytes);
    if (!c->d_io) return c->fail(HSSMF_ERR_OOM, "staging allocation failed");
  }
  cudaEventRecord(c->ev0, c->stream);
  const double* Bd = B;
  long long ldbd = ldb;
  if (!bdev) {
    if ((st = c->cuda_check(cudaMemcpy2DAsync(c->d_io, sizeof(double) * n, B, sizeof(double) * ldb,
                                              sizeof(double) * n, nrhs, cudaMemcpyHostToDevice, c->stream), "B upload")))
      return st;
    Bd = c->d_io;
    ldbd = n;
  }
  double* Xd = xdev ? X : c->d_io + (size_t)n * nrhs;
  long long ldxd = xdev ? ldb : n;
  cudaMemsetAsync(c->d_status, 0, sizeof(unsigned) * 4, c->stream);
  c->prof.mark(PH_OUTER, c->stream);
  st = c->outer_solve(Bd, ldbd, Xd, ldxd, nrhs, transpose);
  hssmf_status st2 = HSSMF_OK;
  if (!xdev && (st == HSSMF_OK || st == HSSMF_ERR_NOCONV))
    st2 = c->cuda_check(cudaMemcpy2DAsync(X, sizeof(double) * ldb, Xd, sizeof(double) * n, sizeof(double) * n,
                                          nrhs, cudaMemcpyDeviceToHost, c->stream), "X download");
  cudaEventRecord(c->ev1, c->stream);
  hssmf_status st3 = c->read_status();
  c->prof.finish(c->stream);
  if (st3 == HSSMF_ERR_CUDA) return st3;  // a rejected launch explains any other failure
  if (st) return st;
  if (st2) return st2;
  if (st3) return st3;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  c->stats.t_solve_ms = ms;
  c->stats.iterations = c->last_iters;
  c->stats.relres = c->last_relres;
  c->stats.gpu_launches = c->factor_launches + (int)(g_launches.load() - l0);
  return HSSMF_OK;
}

hssmf_status hssmf_solve(hssmf_ctx* c, const double* B, double* X, int nrhs, int ldb) {
  return solve_common(c, B, X, nrhs, ldb, 0);
}

hssmf_status hssmf_solve_T(hssmf_ctx* c, const double* B, double* X, int nrhs, int ldb) {
  return solve_common(c, B, X, nrhs, ldb, 1);
}

hssmf_status hssmf_get_stats(const hssmf_ctx* c, hssmf_stats* out) {
  if (!c || !out) return HSSMF_ERR_ARG;
  *out = c->stats;
  out->max_rank = c->hss_max_rank;
  out->max_d = c->hss_max_d;
  out->adaptive_rounds = c->hss_rounds;
  out->id_launches = c->id_launches;
  out->id_bytes = c->id_bytes;
  out->id_flops = c->id_flops;
  return HSSMF_OK;
}

hssmf_status hssmf_get_symbolic(const hssmf_ctx* c, int* perm, int* sep_begin, int* sep_end,
                                int* parent, int* n_upd) {
  if (!c) return HSSMF_ERR_ARG;
  if (!c->analyzed) return HSSMF_ERR_ARG;
  const Symbolic& S = c->sym;
  if (perm) std::copy(S.perm.begin(), S.perm.end(), perm);
  for (size_t i = 0; i < S.fronts.size(); ++i) {
    if (sep_begin) sep_begin[i] = S.fronts[i].sep_begin;
    if (sep_end) sep_end[i] = S.fronts[i].sep_end;
    if (parent) parent[i] = S.fronts[i].parent;
    if (n_upd) n_upd[i] = S.fronts[i].nu();
  }
  return HSSMF_OK;
}

hssmf_status hssmf_get_upd(const hssmf_ctx* c, int f, int* upd) {
  if (!c || !c->analyzed || !upd || f < 0 || f >= (int)c->sym.fronts.size()) return HSSMF_ERR_ARG;
  std::copy(c->sym.fronts[f].upd.begin(), c->sym.fronts[f].upd.end(), upd);
  return HSSMF_OK;
}

}  // extern "C"

template <typename T>
static hssmf_status batched_id_impl(int njobs, const void* Y, const long long* y_off, const int* m,
                                    const int* d, double eps, int* rank_host, int* piv,
                                    const long long* p_off, void* X, const long long* x_off,
                                    int use_cluster, cudaStream_t s) {
  std::vector<IdJob> jobs(njobs);
  long long wtot = 0;
  int max_m = 1, max_d = 1;
  for (int j = 0; j < njobs; ++j) {
    if (m[j] < 1 || d[j] < 1) return HSSMF_ERR_ARG;
    wtot += (long long)m[j] * d[j];
    max_m = std::max(max_m, m[j]);
    max_d = std::max(max_d, d[j]);
  }
  char* buf = nullptr;
  const size_t bytes = sizeof(T) * wtot + sizeof(int) * njobs + sizeof(double) * (size_t)njobs * max_m +
                       sizeof(int) * (size_t)njobs * max_m + 1024;
  if (cudaMalloc(&buf, bytes) != cudaSuccess) {
    cudaGetLastError();
    return HSSMF_ERR_OOM;
  }
  T* W = (T*)buf;
  int* rk = (int*)(W + wtot);
  double* rdiag = (double*)(((uintptr_t)(rk + njobs) + 255) & ~(uintptr_t)255);
  int* order = (int*)(rdiag + (size_t)njobs * max_m);
  long long w = 0;
  for (int j = 0; j < njobs; ++j) {
    jobs[j] = IdJob{(const T*)Y + y_off[j], W + w, piv + p_off[j], (T*)X + x_off[j], rk + j, d[j], m[j]};
    w += (long long)m[j] * d[j];
  }
  IdJob* dj = nullptr;
  hssmf_status st = HSSMF_OK;
  if (cudaMalloc(&dj, sizeof(IdJob) * njobs) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(buf);
    return HSSMF_ERR_OOM;
  }
  cudaMemcpyAsync(dj, jobs.data(), sizeof(IdJob) * njobs, cudaMemcpyHostToDevice, s);
  int r;
  if (use_cluster == -3 || use_cluster == -4) {  // register-resident matrices, one exchange per step (FP32)
    const int cfg = std::is_same<T, float>::value ? id_rx_config(max_d, max_m, -3 - use_cluster) : 0;
    r = cfg > 0 ? batched_id_rx(dj, njobs, max_m, max_d, eps, rdiag, order, cfg, s) : -1;
  } else if (use_cluster == -2) {  // register-resident matrices (FP32) on a cluster sized for the largest job
    const int cfg = HssKern<T>::id_rr_config(max_d, max_m);
    r = cfg > 0 ? HssKern<T>::batched_id_rr(dj, njobs, max_m, max_d, eps, rdiag, order, cfg, s) : -1;
  } else if (use_cluster <= -102 && use_cluster >= -116) {  // shared-memory kernel on a given cluster size
    r = HssKern<T>::batched_id_smem(dj, njobs, max_m, max_d, eps, rdiag, order, -use_cluster - 100, s);
  } else if (use_cluster < 0) {  // shared-memory-resident matrices on a cluster sized for the largest job
    const int cl = HssKern<T>::id_smem_cluster_size(max_d, max_m);
    r = HssKern<T>::batched_id_smem(dj, njobs, max_m, max_d, eps, rdiag, order, cl > 0 ? cl : 16, s);
  } else if (use_cluster > 0) {
    r = HssKern<T>::batched_id_cluster(dj, njobs, max_m, max_d, eps, rdiag, order, s, use_cluster >= 16 ? 16 : 8);
  } else {
    r = HssKern<T>::batched_id(dj, njobs, max_m, max_d, eps, s);
  }
  if (r < 0) st = HSSMF_ERR_ARG;
  if (!st) cudaMemcpyAsync(rank_host, rk, sizeof(int) * njobs, cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) st = HSSMF_ERR_CUDA;
  for (int j = 0; !st && j < njobs; ++j)
    if (rank_host[j] < 0) st = HSSMF_ERR_TIMEOUT;
  cudaFree(dj);
  cudaFree(buf);
  return st;
}

extern "C" {

hssmf_status hssmf_id_timeout_test(int cl, int spin) {
  if (cl < 2 || cl > 16 || spin < 1) return HSSMF_ERR_ARG;
  const int d = 64, m = 8 * cl;
  char* buf = nullptr;
  const size_t bytes = 2 * sizeof(float) * d * m + sizeof(float) * m * m + sizeof(int) * (2 * m + 1) +
                       sizeof(double) * m + sizeof(IdJob) + 1024;
  if (cudaMalloc(&buf, bytes) != cudaSuccess) {
    cudaGetLastError();
    return HSSMF_ERR_OOM;
  }
  hssmf_status st = HSSMF_OK;
  if (cudaMemset(buf, 0, bytes) != cudaSuccess) st = HSSMF_ERR_CUDA;
  float* Y = (float*)buf;
  float* W = Y + d * m;
  float* X = W + d * m;
  int* piv = (int*)(X + m * m);
  int* order = piv + m;
  int* rank = order + m;
  double* rdiag = (double*)(((uintptr_t)(rank + 1) + 255) & ~(uintptr_t)255);
  IdJob* dj = (IdJob*)(((uintptr_t)(rdiag + m) + 255) & ~(uintptr_t)255);
  const IdJob job{Y, W, piv, X, rank, d, m};
  if (!st && cudaMemcpy(dj, &job, sizeof(IdJob), cudaMemcpyHostToDevice) != cudaSuccess) st = HSSMF_ERR_CUDA;
  if (!st && batched_id_rx(dj, 1, m, d, 1e-4, rdiag, order, cl, 0, spin, 0) < 0) st = HSSMF_ERR_CUDA;
  int rk = 0;
  if (!st && (cudaMemcpy(&rk, rank, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)) st = HSSMF_ERR_CUDA;
  if (cudaGetLastError() != cudaSuccess && !st) st = HSSMF_ERR_CUDA;
  cudaFree(buf);
  if (st) return st;
  return rk < 0 ? HSSMF_ERR_TIMEOUT : HSSMF_OK;
}

hssmf_status hssmf_batched_id(int prec, int njobs, const void* Y, const long long* y_off, const int* m,
                              const int* d, double eps, int* rank_host, int* piv, const long long* p_off,
                              void* X, const long long* x_off, int use_cluster, void* cuda_stream) {
  if (njobs < 1 || !Y || !y_off || !m || !d || !rank_host || !piv || !p_off || !X || !x_off) return HSSMF_ERR_ARG;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (prec == HSSMF_PREC_FP64)
    return batched_id_impl<double>(njobs, Y, y_off, m, d, eps, rank_host, piv, p_off, X, x_off, use_cluster, s);
  if (prec == HSSMF_PREC_FP32)
    return batched_id_impl<float>(njobs, Y, y_off, m, d, eps, rank_host, piv, p_off, X, x_off, use_cluster, s);
  return HSSMF_ERR_ARG;
}

hssmf_status hssmf_get_phase_times(const hssmf_ctx* c, double* ms, int n) {
  if (!c || !ms || n < 0) return HSSMF_ERR_ARG;
  for (int i = 0; i < n && i < PH_COUNT; ++i) ms[i] = c->prof.ms[i];
  return HSSMF_OK;
}

hssmf_status hssmf_pattern_grad(hssmf_ctx* c, const double* lambda, const double* x, int nrhs, int ld,
                                double* out) {
  if (!c) return HSSMF_ERR_ARG;
  if (!c->on_device) return c->fail(HSSMF_ERR_ARG, "pattern_grad needs a factorization (device structure)");
  if (!lambda || !x || !out || nrhs < 1 || ld < c->sym.n) return c->fail(HSSMF_ERR_ARG, "bad pattern_grad arguments");
  cudaPointerAttributes a[3];
  const void* ptr[3] = {lambda, x, out};
  for (int q = 0; q < 3; ++q)
    if (cudaPointerGetAttributes(&a[q], ptr[q]) != cudaSuccess || a[q].type != cudaMemoryTypeDevice) {
      cudaGetLastError();
      return c->fail(HSSMF_ERR_ARG, "pattern_grad takes device arrays");
    }
  pattern_grad(c->ds, lambda, x, ld, nrhs, out, c->stream);
  return c->cuda_check(cudaStreamSynchronize(c->stream), "pattern_grad");
}

int hssmf_get_id_trace(const hssmf_ctx* c, int* rec, int max_records) {
  if (!c) return -1;
  const int n = (int)(c->id_trace.size() / kIdTraceFields);
  if (rec)
    for (int i = 0; i < std::min(n, max_records) * kIdTraceFields; ++i) rec[i] = c->id_trace[i];
  return n;
}

int hssmf_get_id_launch_trace(const hssmf_ctx* c, double* rec, int max_records) {
  if (!c) return -1;
  const int n = (int)(c->id_launch_trace.size() / 6);
  if (rec)
    for (int i = 0; i < std::min(n, max_records) * 6; ++i) rec[i] = c->id_launch_trace[i];
  return n;
}

hssmf_status hssmf_set_autotune(hssmf_ctx* c, int on) {
  if (!c) return HSSMF_ERR_ARG;
  c->autotune = on != 0;
  return HSSMF_OK;
}

int hssmf_get_tuning(const hssmf_ctx* c, int* rec, int max_levels) {
  if (!c) return -1;
  const int n = (int)c->plan.size();
  if (rec)
    for (int h = 0; h < std::min(n, max_levels); ++h) {
      const LevelPlan& L = c->plan[h];
      const int r[6] = {L.ndense, L.nlarge, L.nfmax, L.threads, L.tuned, (int)(L.tuned_ms * 1000.f)};
      for (int q = 0; q < 6; ++q) rec[6 * h + q] = r[q];
    }
  return n;
}

hssmf_status hssmf_set_profiling(hssmf_ctx* c, int on) {
  if (!c) return HSSMF_ERR_ARG;
  c->prof.on = on != 0;
  return HSSMF_OK;
}

const char* hssmf_last_error(const hssmf_ctx* c) { return c ? c->err.c_str() : "null context"; }

void hssmf_destroy(hssmf_ctx* c) {
  if (!c) return;
  if (c->on_device) cudaStreamSynchronize(c->stream);
  c->free_all();
  hss_release(*c);
  c->prof.release();
  for (auto& e : c->id_ev) {  // launch timers left by a failed factorization
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  delete c;
}

}  // extern "C"
