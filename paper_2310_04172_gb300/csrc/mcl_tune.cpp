// Autotuner of the sensor-update launch shape (C ABI in include/mcl.h).
//
// Times candidate shapes with CUDA events on the caller's particles and scan
// (a leading subset of the particles), by coordinate descent over the knobs:
// particles per work item, look-ups in flight per lane, pipelining, particle
// order, work-item order, and, if allowed, points per chunk and lanes per particle (these two
// fix the FP32 summation order, so a tuned pair must stay fixed for a
// session). Winners are cached per (GPU, map kind, layout, storage type, score
// mode, P bucket, N bucket) in a JSON-lines file.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <mutex>
#include <string>
#include <vector>

#include "runtime.h"

using namespace mcl;

namespace {

std::mutex g_tune_mu;

struct Knobs {
  int chunk, lanes, ppi, unroll, pipeline, order, items;
};

int log2_bucket(int64_t v) {
  int b = 0;
  while ((1LL << (b + 1)) <= v) ++b;
  return b;
}

// Cache key: GPU, kernel kind, brick layout, storage type, kernel mode (the
// score map's own), read and neglect flags, whether the scan is staged in
// patches, and the power-of-two buckets of P and N.
std::string tune_key(const mcl_map_s* m, const mcl_sensor_params* p, int64_t P, int64_t N, bool summation) {
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, m->device);
  char buf[320];
  snprintf(buf, sizeof buf, "%s|k%d|l%d|d%d|m%d|f%u|r%d|P%d|N%d|s%d", prop.name, kernel_kind(m),
           m->view.layout, m->dtype, kernel_mode(m, p->mode), (unsigned)p->flags,
           patch_rings(N, p->scan_rings) ? 1 : 0, log2_bucket(P), log2_bucket(N), summation ? 1 : 0);
  std::string s(buf);
  for (char& c : s)
    if (c == '"' || c == ' ') c = '_';
  return s;
}

bool cache_lookup(const char* path, const std::string& key, Knobs* k, double* ms) {
  FILE* f = path ? fopen(path, "r") : nullptr;
  if (!f) return false;
  char line[1024];
  bool found = false;
  while (fgets(line, sizeof line, f)) {
    char kbuf[512];
    Knobs t;
    double tms;
    if (sscanf(line,
               "{\"key\": \"%511[^\"]\", \"points_per_chunk\": %d, \"lanes_per_particle\": %d, "
               "\"particles_per_item\": %d, \"unroll\": %d, \"pipeline\": %d, \"particle_order\": %d, "
               "\"item_order\": %d, \"ms\": %lf}",
               kbuf, &t.chunk, &t.lanes, &t.ppi, &t.unroll, &t.pipeline, &t.order, &t.items, &tms) == 9 &&
        key == kbuf) {
      *k = t;  // the last entry for a key wins
      *ms = tms;
      found = true;
    }
  }
  fclose(f);
  return found;
}

void cache_store(const char* path, const std::string& key, const Knobs& k, double ms) {
  FILE* f = path ? fopen(path, "a") : nullptr;
  if (!f) return;
  fprintf(f,
          "{\"key\": \"%s\", \"points_per_chunk\": %d, \"lanes_per_particle\": %d, "
          "\"particles_per_item\": %d, \"unroll\": %d, \"pipeline\": %d, \"particle_order\": %d, "
          "\"item_order\": %d, \"ms\": %.6f}\n",
          key.c_str(), k.chunk, k.lanes, k.ppi, k.unroll, k.pipeline, k.order, k.items, ms);
  fclose(f);
}

mcl_sensor_params to_params(const mcl_sensor_params& base, const Knobs& k) {
  mcl_sensor_params p = base;
  p.points_per_chunk = k.chunk;
  p.lanes_per_particle = k.lanes;
  p.particles_per_item = k.ppi;
  p.unroll = k.unroll;
  p.pipeline = k.pipeline;
  p.particle_order = k.order;
  p.item_order = k.items;
  return p;
}

}  // namespace

extern "C" {

mcl_status mcl_autotune(mcl_map_t m, const float* particles, int64_t P, const float* scan, int64_t N,
                        const mcl_sensor_params* base, const mcl_tune_params* tp,
                        mcl_tune_result* out, mcl_stream_t stream) {
  if (!m || !particles || !scan || !base || !tp || !out)
    return fail(MCL_EINVAL, "autotune: NULL argument");
  if (tp->struct_size < sizeof(mcl_tune_params) || out->struct_size < sizeof(mcl_tune_result))
    return fail(MCL_EINVAL, "autotune: struct_size");
  if (P < 1 || P > kMaxCount || N < 1 || N > kMaxCount) return fail(MCL_EINVAL, "autotune: sizes");
  if (mcl_status rc = check_params(base)) return rc;
  if (mcl_status rc = check_device(m)) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t Pt = std::min<int64_t>(P, tp->max_particles > 0 ? tp->max_particles : 65536);
  const int reps = tp->repeats > 0 ? tp->repeats : 3;
  const bool summation = tp->tune_summation != 0;
  const char* path = tp->cache_path ? tp->cache_path : getenv("MCL_TUNE_CACHE");
  if (!tp->use_cache) path = nullptr;
  const std::string key = tune_key(m, base, P, N, summation);

  // the base shape as given (a 0 keeps the library's default for that field)
  Knobs best{base->points_per_chunk, base->lanes_per_particle, base->particles_per_item, base->unroll,
             base->pipeline,         base->particle_order,     base->item_order};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    double ms = 0;
    Knobs k;
    if (path && cache_lookup(path, key, &k, &ms)) {
      out->best = to_params(*base, k);
      out->best_ms = ms;
      out->default_ms = 0;
      out->candidates = 0;
      out->from_cache = 1;
      return MCL_OK;
    }
  }

  float* logw = nullptr;
  MCL_CUDA(cudaMalloc(&logw, (size_t)Pt * sizeof(float)));
  cudaEvent_t a = nullptr, b = nullptr;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  int evaluated = 0;
  auto time_knobs = [&](const Knobs& k, double* ms) -> mcl_status {
    mcl_sensor_params p = to_params(*base, k);
    if (mcl_status rc = mcl_sensor_update(m, particles, Pt, scan, N, &p, logw, nullptr, stream)) return rc;
    double best_t = 1e300;
    for (int r = 0; r < reps; ++r) {
      cudaEventRecord(a, s);
      if (mcl_status rc = mcl_sensor_update(m, particles, Pt, scan, N, &p, logw, nullptr, stream)) return rc;
      cudaEventRecord(b, s);
      MCL_CUDA(cudaEventSynchronize(b));
      float t = 0;
      cudaEventElapsedTime(&t, a, b);
      best_t = std::min(best_t, (double)t);
    }
    ++evaluated;
    *ms = best_t;
    return MCL_OK;
  };
  mcl_status rc = MCL_OK;
  double best_ms = 0, default_ms = 0;
  rc = time_knobs(best, &best_ms);
  default_ms = best_ms;
  // coordinate descent: each knob in turn over its candidate values, twice
  const std::vector<int> chunks = {1024, 2048, 4096}, lanes = {32, 16}, ppis = {32, 64, 128, 256},
                         unrolls = {2, 4, 8}, pipes = {1, 2}, orders = {1, 2}, items = {1, 2, 3};
  for (int round = 0; round < 2 && rc == MCL_OK; ++round) {
    auto sweep = [&](int Knobs::*field, const std::vector<int>& vals) {
      for (int v : vals) {
        if (rc != MCL_OK || best.*field == v) continue;
        Knobs k = best;
        k.*field = v;
        const int g = k.lanes ? k.lanes : 32;
        if ((base->flags & MCL_TRILINEAR) && g != 32) continue;  // the trilinear read takes 32 lanes
        // narrower lane groups run the plain 4-deep loop: other unrolls and
        // pipelining would time the same kernel again
        if (g < 32 && ((k.unroll != 0 && k.unroll != 4) || k.pipeline == 2)) continue;
        if (k.unroll == 8 && k.pipeline == 2) continue;
        double t = 0;
        rc = time_knobs(k, &t);
        if (rc == MCL_OK && t < best_ms) {
          best_ms = t;
          best = k;
        }
      }
    };
    if (summation) {
      sweep(&Knobs::chunk, chunks);
      sweep(&Knobs::lanes, lanes);
    }
    sweep(&Knobs::unroll, unrolls);
    sweep(&Knobs::pipeline, pipes);
    sweep(&Knobs::ppi, ppis);
    sweep(&Knobs::order, orders);
    sweep(&Knobs::items, items);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(logw);
  if (rc != MCL_OK) return rc;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    cache_store(path, key, best, best_ms);
  }
  out->best = to_params(*base, best);
  out->best_ms = best_ms;
  out->default_ms = default_ms;
  out->candidates = evaluated;
  out->from_cache = 0;
  return MCL_OK;
}

}  // extern "C"
