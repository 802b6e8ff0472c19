// sched.cu -- scheduler of many independent solve jobs (scatterer configurations of uneven size,
// each with its own wavenumber list) on one GPU.
// Jobs are queued with their host inputs, ordered by estimated cost (largest first: the LU's
// (8/3) N^3 plus the assembly's N E Q per wavenumber), and pulled by worker threads, each owning
// a context on its own CUDA stream, so that small configurations run next to large ones instead
// of after them.  A worker sizes its batches to its share of device memory and, when a tuning
// cache is given, applies (or first measures) the tuned launch parameters of the job's N bucket.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <mutex>
#include <thread>

#include "bie_common.cuh"

struct bie_sched {
  int device = 0;
  int workers = 1;
  std::string cache;
  struct Job {
    std::vector<double> nodes, normals;
    std::vector<int32_t> elems;
    std::vector<uint8_t> bc;
    double dir[3];
    std::vector<double> k;
    int mode;
    void* surf;
    bie_report* rep;
    double cost;
    double ms = 0.0;
    int worker = -1;
  };
  std::vector<Job> jobs;
};

namespace bie {
int autotune(bie_ctx* c, const double* k, int64_t nk, const char* cache_path, bie_tune_result* out);
}

extern "C" {

int bie_sched_create(bie_sched** out, int cuda_device, int workers, const char* tune_cache) {
  if (!out) return bie::fail(BIE_ERR_INVALID_ARG, "NULL out");
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || cuda_device < 0 || cuda_device >= n)
    return bie::fail(BIE_ERR_INVALID_ARG, "bad device index");
  if (workers < 1 || workers > 64) return bie::fail(BIE_ERR_INVALID_ARG, "workers must be in [1, 64]");
  bie_sched* s = new (std::nothrow) bie_sched();
  if (!s) return bie::fail(BIE_ERR_OOM, "host allocation failed");
  s->device = cuda_device;
  s->workers = workers;
  if (tune_cache) s->cache = tune_cache;
  *out = s;
  return BIE_OK;
}

int bie_sched_destroy(bie_sched* s) {
  delete s;
  return BIE_OK;
}

int bie_sched_add(bie_sched* s, const double* nodes, int64_t N, const int32_t* elems, int64_t E, const double* normals,
                  const uint8_t* bc, const double* dir, const double* k, int64_t Nk, int mode, void* surf_out,
                  bie_report* rep, int32_t* job_id) {
  if (!s) return bie::fail(BIE_ERR_INVALID_ARG, "NULL scheduler");
  if (!nodes || !elems || !bc || !k || !surf_out || N < 3 || E < 1 || Nk < 1)
    return bie::fail(BIE_ERR_INVALID_ARG, "job needs nodes, elems, bc, k, surf_out, N >= 3, E >= 1, Nk >= 1");
  if (mode != BIE_MODE_FP64 && mode != BIE_MODE_MIXED && mode != BIE_MODE_LEARNED)
    return bie::fail(BIE_ERR_INVALID_ARG, "unknown mode");
  bie_sched::Job j;
  j.nodes.assign(nodes, nodes + 3 * N);
  j.elems.assign(elems, elems + 6 * E);
  if (normals) j.normals.assign(normals, normals + 3 * N);
  j.bc.assign(bc, bc + N);
  const double d0[3] = {0.0, 0.0, 1.0};
  for (int a = 0; a < 3; ++a) j.dir[a] = dir ? dir[a] : d0[a];
  j.k.assign(k, k + Nk);
  j.mode = mode;
  j.surf = surf_out;
  j.rep = rep;
  j.cost = (double)Nk * ((8.0 / 3.0) * (double)N * N * N + 16.0 * 40.0 * (double)N * E);
  if (job_id) *job_id = (int32_t)s->jobs.size();
  s->jobs.push_back(std::move(j));
  return BIE_OK;
}

int bie_sched_run(bie_sched* s, bie_sched_stats* stats) {
  if (!s) return bie::fail(BIE_ERR_INVALID_ARG, "NULL scheduler");
  const int nj = (int)s->jobs.size();
  std::vector<int> order(nj);
  for (int i = 0; i < nj; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return s->jobs[a].cost > s->jobs[b].cost; });
  if (cudaSetDevice(s->device) != cudaSuccess) return bie::fail(BIE_ERR_CUDA, "cudaSetDevice");
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return bie::fail(BIE_ERR_CUDA, "cudaMemGetInfo");
  const int W = std::min(s->workers, std::max(1, nj));
  const size_t share = (size_t)(0.8 * (double)free_b) / (size_t)W;
  std::atomic<int> next{0};
  std::atomic<int> first_err{BIE_OK};
  std::mutex err_mu;
  std::string err_msg;
  std::vector<double> busy((size_t)W, 0.0);
  const auto t0 = std::chrono::steady_clock::now();
  auto worker = [&](int w) {
    cudaSetDevice(s->device);
    cudaStream_t st = nullptr;
    bie_ctx* c = nullptr;
    auto record = [&](int rc) {
      int expected = BIE_OK;
      if (first_err.compare_exchange_strong(expected, rc)) {
        std::lock_guard<std::mutex> g(err_mu);
        err_msg = bie_last_error();
      }
    };
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      record(bie::fail(BIE_ERR_CUDA, "stream creation"));
      return;
    }
    int rc = bie_create(&c, s->device, st);
    if (rc != BIE_OK) {
      record(rc);
      cudaStreamDestroy(st);
      return;
    }
    for (;;) {
      if (first_err.load() != BIE_OK) break;
      const int i = next.fetch_add(1);
      if (i >= nj) break;
      bie_sched::Job& j = s->jobs[order[i]];
      const auto a = std::chrono::steady_clock::now();
      const int64_t N = (int64_t)j.bc.size();
      rc = bie_set_geometry(c, j.nodes.data(), N, j.elems.data(), (int64_t)j.elems.size() / 6,
                            j.normals.empty() ? nullptr : j.normals.data(), j.bc.data());
      if (rc == BIE_OK) rc = bie_set_incident_plane_wave(c, j.dir);
      if (rc == BIE_OK && !s->cache.empty() && j.mode != BIE_MODE_FP64) {
        bie_tune_result tr;
        rc = bie::autotune(c, j.k.data(), (int64_t)std::min<size_t>(j.k.size(), 8), s->cache.c_str(), &tr);
      }
      if (rc == BIE_OK) {  // this worker's share of device memory bounds its workspaces
        c->mem_budget = share;
        rc = bie_solve_frequencies(c, j.k.data(), (int64_t)j.k.size(), j.mode, j.surf, j.rep);
      }
      if (rc != BIE_OK) {
        record(rc);
        break;
      }
      j.ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - a).count();
      j.worker = w;
      busy[w] += j.ms;
    }
    bie_destroy(c);
    cudaStreamDestroy(st);
  };
  std::vector<std::thread> th;
  for (int w = 0; w < W; ++w) th.emplace_back(worker, w);
  for (auto& t : th) t.join();
  const double wall = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (stats) {
    stats->jobs = nj;
    stats->workers = W;
    stats->wall_ms = wall;
    double b = 0.0;
    for (double x : busy) b += x;
    stats->busy_ms = b;
  }
  if (first_err.load() != BIE_OK) return bie::fail(first_err.load(), "scheduler job failed: " + err_msg);
  s->jobs.clear();
  return BIE_OK;
}

}  // extern "C"
