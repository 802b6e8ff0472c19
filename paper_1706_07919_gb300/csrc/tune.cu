// tune.cu -- autotuner of the mixed path's launch parameters per problem size.
// For a geometry of N nodes the tuner times one batch of mixed-precision frequency solves for
// every candidate (wavenumbers per batch x LU trailing-update kernel) and keeps the fastest per
// wavenumber, then for the deferred update (tcgen05 = 3) the block over which it is deferred
// (128, 256, 512 columns), the panel width (64, 32) and the update's tile width (256, 128 real
// columns) at the chosen batch.  Results are cached per N bucket (N rounded up to a multiple of
// 64) in a small JSON file:
//   {"bie_autotune": 1, "entries": {"2944": {"batch": 128, "tcgen05": 3, "lu_block": 256,
//                                            "us_per_k": ..., "lu_panel": 64, "lu_tile": 256}}}
// (entries written without "lu_panel" / "lu_tile" read as 64 / 256).
#include <algorithm>
#include <cstdio>
#include <fstream>
#include <atomic>
#include <map>
#include <mutex>
#include <sstream>
#include <thread>

#include <unistd.h>

#include "bie_common.cuh"

namespace bie {

int solve_mixed(bie_ctx* c, const double* k, int64_t Nk, cd* surf_out, bie_report* rep, cf* lu_keep,
                int32_t* perm_keep, cf* d_keep, const double* dirs, int ndir);

struct TuneEntry {
  int batch = 0, tc = 0, block = 256;
  double us_per_k = 0.0;
  int panel = 64, tile = 256;
};

static std::map<int, TuneEntry> load_cache(const char* path) {
  std::map<int, TuneEntry> m;
  if (!path) return m;
  std::ifstream f(path);
  if (!f) return m;
  std::stringstream ss;
  ss << f.rdbuf();
  const std::string s = ss.str();
  for (size_t i = 0; i + 1 < s.size(); ++i) {
    if (s[i] != '"' || !(s[i + 1] >= '0' && s[i + 1] <= '9')) continue;
    int key = 0, b = 0, t = 0, blk = 0, pan = 64, til = 256;
    double us = 0.0;
    const int got = std::sscanf(
        s.c_str() + i,
        "\"%d\": {\"batch\": %d, \"tcgen05\": %d, \"lu_block\": %d, \"us_per_k\": %lf, \"lu_panel\": %d, \"lu_tile\": %d}",
        &key, &b, &t, &blk, &us, &pan, &til);
    if (got < 6) pan = 64;
    if (got < 7) til = 256;
    if (got >= 5 && b >= 1 && t >= 0 && t <= 3 && (blk == 128 || blk == 256 || blk == 512) &&
        (pan == 32 || pan == 64) && (til == 128 || til == 256))
      m[key] = TuneEntry{b, t, blk, us, pan, til};
  }
  return m;
}

static std::mutex g_cache_mu;  // read-modify-write of cache files within this process

static bool save_cache(const char* path, const std::map<int, TuneEntry>& m) {
  static std::atomic<uint64_t> seq{0};
  const std::string tmp = std::string(path) + "." + std::to_string((long)getpid()) + "." +
                          std::to_string((uint64_t)std::hash<std::thread::id>()(
                              std::this_thread::get_id())) + "." + std::to_string(seq.fetch_add(1)) + ".tmp";
  std::ofstream f(tmp);
  if (!f) return false;
  f << "{\"bie_autotune\": 1, \"entries\": {\n";
  size_t i = 0;
  for (const auto& kv : m) {
    char line[256];
    std::snprintf(line, sizeof(line),
                  "  \"%d\": {\"batch\": %d, \"tcgen05\": %d, \"lu_block\": %d, \"us_per_k\": %.3f, \"lu_panel\": %d, "
                  "\"lu_tile\": %d}%s\n",
                  kv.first, kv.second.batch, kv.second.tc, kv.second.block, kv.second.us_per_k, kv.second.panel,
                  kv.second.tile, (++i < m.size()) ? "," : "");
    f << line;
  }
  f << "}}\n";
  f.close();
  return std::rename(tmp.c_str(), path) == 0;
}

int autotune(bie_ctx* c, const double* k, int64_t nk, const char* cache_path, bie_tune_result* out) {
  const int64_t N = c->N;
  const int key = (int)((N + 63) / 64 * 64);
  auto cache = load_cache(cache_path);
  auto it = cache.find(key);
  if (it != cache.end()) {
    c->mixed_batch = it->second.batch;
    c->tc_version = it->second.tc;
    c->lu_block = it->second.block;
    c->lu_panel = it->second.panel;
    c->lu_tile = it->second.tile;
    if (out)
      *out = bie_tune_result{key, it->second.batch, it->second.tc, 1, it->second.us_per_k, it->second.block,
                             it->second.panel, it->second.tile};
    return BIE_OK;
  }
  if (nk < 1) return fail(BIE_ERR_INVALID_ARG, "autotune needs at least one sample wavenumber");
  const int64_t ld = (N + 63) / 64 * 64;
  const size_t perk = 2 * (size_t)N * ld * sizeof(cf) + 64 * (size_t)N;
  size_t free_b = 0;
  BIE_TRY(device_free(c, &free_b));
  const int saved_batch = c->mixed_batch, saved_tc = c->tc_version, saved_graph = c->mixed_graph,
            saved_block = c->lu_block, saved_panel = c->lu_panel, saved_tile = c->lu_tile;
  TuneEntry best;
  best.us_per_k = 1e300;
  std::vector<double> kk;
  cd* surf = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = BIE_OK;
  const int batches[] = {8, 16, 32, 64, 128, 256};
  const int tcs[] = {3, 2};
  size_t surf_bytes = (size_t)256 * 2 * N * sizeof(cd);
  if (dev_alloc(c, (void**)&surf, surf_bytes) != BIE_OK || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess)
    rc = fail(BIE_ERR_OOM, "autotune scratch");
  // one timed batch (after an untimed one that sizes the workspace and builds the tables)
  auto measure = [&](int b, int tc, int block, double* us, int panel = 64, int tile = 256) -> int {
    kk.resize((size_t)b);
    for (int i = 0; i < b; ++i) kk[i] = k[i % nk];
    c->mixed_batch = b;
    c->tc_version = tc;
    c->lu_block = block;
    c->lu_panel = panel;
    c->lu_tile = tile;
    c->mixed_graph = 0;
    BIE_TRY(solve_mixed(c, kk.data(), b, surf, nullptr, nullptr, nullptr, nullptr, nullptr, 1));
    cudaEventRecord(e0, c->stream);
    BIE_TRY(solve_mixed(c, kk.data(), b, surf, nullptr, nullptr, nullptr, nullptr, nullptr, 1));
    cudaEventRecord(e1, c->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    *us = 1e3 * ms / b;
    return BIE_OK;
  };
  for (int tc : tcs) {
    for (int b : batches) {
      if (rc != BIE_OK) break;
      if ((size_t)b * perk > free_b / 3) continue;
      double us = 0.0;
      rc = measure(b, tc, 256, &us);
      if (rc == BIE_OK && us < best.us_per_k) best = TuneEntry{b, tc, 256, us, 64, 256};
    }
  }
  if (rc == BIE_OK && best.tc == 3)  // then the block of the deferred update at the chosen batch
    for (int block : {128, 512}) {
      double us = 0.0;
      rc = measure(best.batch, 3, block, &us);
      if (rc != BIE_OK) break;
      if (us < best.us_per_k) best = TuneEntry{best.batch, 3, block, us, 64, 256};
    }
  if (rc == BIE_OK && best.tc == 3) {  // then the panel width at the chosen batch and block
    double us = 0.0;
    rc = measure(best.batch, 3, best.block, &us, 32);
    if (rc == BIE_OK && us < best.us_per_k) best = TuneEntry{best.batch, 3, best.block, us, 32, 256};
  }
  if (rc == BIE_OK && best.tc >= 2) {  // then the update's tile width
    double us = 0.0;
    rc = measure(best.batch, best.tc, best.block, &us, best.panel, 128);
    if (rc == BIE_OK && us < best.us_per_k) best = TuneEntry{best.batch, best.tc, best.block, us, best.panel, 128};
  }
  dev_free(c, surf);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  c->mixed_graph = saved_graph;
  if (rc != BIE_OK || best.batch == 0) {
    c->mixed_batch = saved_batch;
    c->tc_version = saved_tc;
    c->lu_block = saved_block;
    c->lu_panel = saved_panel;
    c->lu_tile = saved_tile;
    return rc != BIE_OK ? rc : fail(BIE_ERR_OOM, "autotune: no candidate fits in device memory");
  }
  c->mixed_batch = best.batch;
  c->tc_version = best.tc;
  c->lu_block = best.block;
  c->lu_panel = best.panel;
  c->lu_tile = best.tile;
  if (cache_path) {
    std::lock_guard<std::mutex> g(g_cache_mu);
    cache = load_cache(cache_path);  // another thread or process may have added entries meanwhile
    cache[key] = best;
    if (!save_cache(cache_path, cache)) return fail(BIE_ERR_INVALID_ARG, std::string("cannot write ") + cache_path);
  }
  if (out) *out = bie_tune_result{key, best.batch, best.tc, 0, best.us_per_k, best.block, best.panel, best.tile};
  return BIE_OK;
}

}  // namespace bie
