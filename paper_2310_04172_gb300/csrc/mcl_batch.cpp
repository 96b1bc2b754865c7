// Batched sensor update over many robot sessions (C ABI in include/mcl.h).
//
// A plan fixes the sessions' device buffers, groups the sessions by map and
// score constants, and lays out one device workspace for the whole step. A
// run enqueues, per session, the spatial order, pose matrices and scan
// packing; per group, one persistent sensor kernel over the (session, point
// chunk, particle block) work items of all its sessions; per session, the
// log-weights, normalisation and (optionally) systematic resampling. With
// use_graph the step is captured once into a CUDA graph and replayed.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "runtime.h"

using namespace mcl;

namespace {

struct SessionPlan {
  mcl_session_update u;
  mcl_sensor_params prm;
  Plan pl;
  size_t base;                        // this session's block in the workspace
  size_t off_cum, off_tot, off_last;  // resample scratch inside the block
  int group;
};

struct Group {
  mcl_map_t map;
  int mode, neglect;
  uint32_t flags;
  float sigma;
  std::vector<int> sessions;
  SensorShape sh;
  BatchArgs args;
};

inline float sensor_c(float sigma) { return (float)(-0.5 / ((double)sigma * sigma)); }

// Score constants of a session, as the single-session update sets them.
void score_constants(const mcl_map_s* m, float sigma, int mode, SensorArgs* a) {
  const double sig = (double)sigma;
  const bool q16 = m->dtype == MCL_I16;
  const double scale = (double)m->view.scale;
  a->cs = q16 ? (float)(-0.5 / (sig * sig) * scale * scale) : sensor_c(sigma);
  a->store_scale = (q16 && mode == MCL_LOGPROD) ? (float)(scale * scale) : 1.0f;
}

}  // namespace

struct mcl_batch_s {
  int device = 0;
  std::vector<SessionPlan> s;
  std::vector<Group> g;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  double* d_r = nullptr;
  unsigned* status = nullptr;
  bool use_graph = false;
  cudaStream_t cap = nullptr;  // plan-owned stream the step is captured on
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int kernels_per_run = 0;
  long long n_items = 0, total_evals = 0;
};

namespace {

mcl_status enqueue(mcl_batch_s* b, cudaStream_t st, bool profile) {
  for (auto& sp : b->s) {
    const Plan& pl = sp.pl;
    char* ws = b->ws + sp.base;
    int* rank = pl.spatial ? (int*)(ws + pl.off_rank) : nullptr;
    if (pl.spatial)
      MCL_CUDA(launch_particle_order(sp.u.particles, (int)sp.u.P, sp.u.map->view,
                                     (uint32_t*)(ws + pl.off_key), (uint32_t*)(ws + pl.off_hist),
                                     rank, st));
    MCL_CUDA(launch_pose_and_pack(sp.u.particles, (int)sp.u.P, (float4*)(ws + pl.off_mats), rank,
                                  sp.u.scan, (int)sp.u.N, scan_layout(pl.sh), ws + pl.off_scan, st));
  }
  for (auto& g : b->g) {
    if (profile) {
      PhaseScope ps(MCL_PHASE_SENSOR, st);
      MCL_CUDA(launch_sensor_batch(kernel_kind(g.map), g.map->view.layout, g.map->dtype, g.args, g.sh, st));
    } else {
      MCL_CUDA(launch_sensor_batch(kernel_kind(g.map), g.map->view.layout, g.map->dtype, g.args, g.sh, st));
    }
  }
  for (size_t i = 0; i < b->s.size(); ++i) {
    auto& sp = b->s[i];
    const Plan& pl = sp.pl;
    char* ws = b->ws + sp.base;
    const int P = (int)sp.u.P;
    int* rank = pl.spatial ? (int*)(ws + pl.off_rank) : nullptr;
    float* L = sp.u.logw ? sp.u.logw : (float*)(ws + pl.off_logw);
    const double sig = (double)sp.u.sigma_hit;
    const float k = (float)(1.0 / std::sqrt(2.0 * 3.141592653589793 * sig * sig));
    const int nb = normalise_blocks(P);
    MCL_CUDA(launch_finish_and_normalise((float*)(ws + pl.off_partial), rank, P, pl.K, sp.u.mode,
                                         sensor_c(sp.u.sigma_hit), k, L,
                                         sp.u.estimate ? nullptr : sp.u.w,
                                         (float2*)(ws + pl.off_stats), nb, (float*)(ws + pl.off_ostats),
                                         st));
    if (sp.u.estimate)
      MCL_CUDA(launch_normalise_from_stats(L, P, sp.u.w, (float2*)(ws + pl.off_stats), nb,
                                           (float*)(ws + pl.off_ostats), sp.u.particles,
                                           (EstPartial*)(ws + pl.off_est), sp.u.estimate, st));
    if (sp.u.resample_idx)
      MCL_CUDA(launch_resample(sp.u.w, P, 0.0, sp.u.resample_idx,
                               sp.u.particles_out ? sp.u.particles : nullptr, sp.u.particles_out,
                               (double*)(ws + sp.off_cum), (double*)(ws + sp.off_tot),
                               (long long*)(ws + sp.off_last), st, b->d_r + i));
  }
  return MCL_OK;
}

}  // namespace

extern "C" {

mcl_status mcl_batch_create(const mcl_session_update* sessions, int32_t n,
                            const mcl_batch_params* bp, mcl_batch_t* out) {
  if (!out) return fail(MCL_EINVAL, "batch_create: NULL out");
  *out = nullptr;
  if (!sessions || n < 1) return fail(MCL_EINVAL, "batch_create: no sessions");
  if (!bp || bp->struct_size < sizeof(mcl_batch_params))
    return fail(MCL_EINVAL, "batch_create: params NULL or struct_size too small");
  if (bp->use_graph != 0 && bp->use_graph != 1) return fail(MCL_EINVAL, "batch_create: use_graph");
  DeviceState st;
  int dev = 0;
  if (mcl_status rc = device_state(&dev, &st)) return rc;

  auto* b = new mcl_batch_s();
  b->device = dev;
  b->status = st.status;
  b->use_graph = bp->use_graph == 1;
  auto bail = [&](mcl_status rc) {
    if (b->ws) cudaFree(b->ws);
    delete b;
    return rc;
  };
  size_t off = 0;
  for (int i = 0; i < n; ++i) {
    const mcl_session_update& u = sessions[i];
    if (u.struct_size < sizeof(mcl_session_update)) return bail(fail(MCL_EINVAL, "session %d: struct_size", i));
    if (!u.map || !u.particles || !u.scan) return bail(fail(MCL_EINVAL, "session %d: NULL map, particles or scan", i));
    if (u.P < 1 || u.P > kMaxCount || u.N < 1 || u.N > kMaxCount)
      return bail(fail(MCL_EINVAL, "session %d: P or N out of range", i));
    if (!u.logw && !u.w) return bail(fail(MCL_EINVAL, "session %d: both outputs NULL", i));
    if (u.resample_idx && !u.w) return bail(fail(MCL_EINVAL, "session %d: resampling needs w", i));
    if (u.estimate && !u.w) return bail(fail(MCL_EINVAL, "session %d: the estimate needs w", i));
    if (!aligned(u.estimate, 8)) return bail(fail(MCL_EINVAL, "session %d: estimate needs 8-byte alignment", i));
    if (u.particles_out && (!u.resample_idx || u.particles_out == u.particles))
      return bail(fail(MCL_EINVAL, "session %d: particles_out needs resample_idx and must not alias", i));
    for (const void* p : {(const void*)u.particles, (const void*)u.scan, (const void*)u.logw,
                          (const void*)u.w, (const void*)u.resample_idx, (const void*)u.particles_out})
      if (!aligned(p, 4)) return bail(fail(MCL_EINVAL, "session %d: pointers need 4-byte alignment", i));
    if (mcl_status rc = check_device(u.map)) return bail(rc);
    SessionPlan sp{};
    sp.u = u;
    sp.prm = mcl_sensor_params{sizeof(mcl_sensor_params), u.sigma_hit, u.mode, u.flags,
                               bp->points_per_chunk, bp->lanes_per_particle, bp->particles_per_item,
                               bp->unroll, bp->pipeline, bp->particle_order, bp->item_order};
    if (mcl_status rc = check_params(&sp.prm)) return bail(rc);
    if (mcl_status rc = make_plan(u.map, u.P, u.N, &sp.prm, &sp.pl)) return bail(rc);
    const int nt = resample_tiles((int)u.P);
    sp.base = off;
    size_t o = sp.pl.total;
    sp.off_cum = o;
    o = align256(o + (u.resample_idx ? (size_t)u.P * 8 : 0));
    sp.off_tot = o;
    o = align256(o + (u.resample_idx ? (size_t)(nt + 1) * 8 : 0));
    sp.off_last = o;
    o = align256(o + (u.resample_idx ? (size_t)(nt + 1) * 8 : 0));
    off = align256(off + o);
    // group by map, score constants and read rule
    const int neglect = (u.flags & MCL_NEGLECT_OUTSIDE) ? 1 : 0;
    int gi = -1;
    for (size_t k = 0; k < b->g.size(); ++k)
      if (b->g[k].map == u.map && b->g[k].mode == u.mode && b->g[k].flags == u.flags &&
          b->g[k].sigma == u.sigma_hit)
        gi = (int)k;
    if (gi < 0) {
      Group g{};
      g.map = u.map;
      g.mode = u.mode;
      g.neglect = neglect;
      g.flags = u.flags;
      g.sigma = u.sigma_hit;
      g.sh = sp.pl.sh;
      b->g.push_back(g);
      gi = (int)b->g.size() - 1;
    }
    sp.group = gi;
    b->g[gi].sessions.push_back(i);
    b->s.push_back(sp);
    b->total_evals += u.P * u.N;
  }
  // group tables and offsets follow the session blocks
  std::vector<size_t> off_tab(b->g.size()), off_beg(b->g.size());
  for (size_t k = 0; k < b->g.size(); ++k) {
    off_tab[k] = off;
    off = align256(off + b->g[k].sessions.size() * sizeof(BatchSession));
    off_beg[k] = off;
    off = align256(off + (b->g[k].sessions.size() + 1) * sizeof(long long));
  }
  const size_t off_r = off;
  off = align256(off + (size_t)n * sizeof(double));
  b->ws_bytes = off;
  cudaError_t e = cudaMalloc(&b->ws, b->ws_bytes);
  if (e != cudaSuccess) return bail(cuda_fail(e, "batch_create workspace"));
  b->d_r = (double*)(b->ws + off_r);
  e = cudaMemset(b->d_r, 0, (size_t)n * sizeof(double));
  if (e != cudaSuccess) return bail(cuda_fail(e, "batch_create offsets"));
  for (size_t k = 0; k < b->g.size(); ++k) {
    Group& g = b->g[k];
    std::vector<BatchSession> tab;
    std::vector<long long> beg{0};
    for (int i : g.sessions) {
      const SessionPlan& sp = b->s[i];
      char* ws = b->ws + sp.base;
      tab.push_back(BatchSession{(const float4*)(ws + sp.pl.off_mats), (const float4*)(ws + sp.pl.off_scan),
                                 (float*)(ws + sp.pl.off_partial), (int)sp.u.P, (int)sp.u.N, sp.pl.nblk,
                                 sp.pl.K, sp.pl.sweep, sp.pl.sh.ppi});
      beg.push_back(beg.back() + sp.pl.n_items);
    }
    e = cudaMemcpy(b->ws + off_tab[k], tab.data(), tab.size() * sizeof(BatchSession), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(b->ws + off_beg[k], beg.data(), beg.size() * sizeof(long long), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bail(cuda_fail(e, "batch_create tables"));
    int bps = 0;
    e = sensor_batch_occupancy(kernel_kind(g.map), g.map->view.layout, g.map->dtype, kernel_mode(g.map, g.mode),
                               g.sh, &bps);
    if (e != cudaSuccess || bps < 1) return bail(cuda_fail(e, "batch_create occupancy"));
    g.sh.grid = (int)std::min<long long>(beg.back(), (long long)st.sms * bps);
    SensorArgs& a = g.args.base;
    a = SensorArgs{};
    a.map = g.map->view;
    a.status = st.status;
    a.chunk = g.sh.chunk;
    a.ppi = g.sh.ppi;
    a.layout = scan_layout(g.sh);
    a.mode = kernel_mode(g.map, g.mode);
    a.neglect = g.neglect;
    score_constants(g.map, g.sigma, g.mode, &a);
    set_fills(g.map, &a);
    g.args.sessions = (const BatchSession*)(b->ws + off_tab[k]);
    g.args.item_begin = (const long long*)(b->ws + off_beg[k]);
    g.args.n_sessions = (int)g.sessions.size();
    g.args.n_items = beg.back();
    b->n_items += beg.back();
  }
  int kern = (int)b->g.size();
  for (auto& sp : b->s)
    kern += (sp.pl.spatial ? 4 : 0) + 1 + 1 + (sp.u.w ? 1 : 0) + (sp.u.estimate ? 1 : 0) +
            (sp.u.resample_idx ? resample_kernels((int)sp.u.P) : 0);
  b->kernels_per_run = kern;
  *out = b;
  return MCL_OK;
}

mcl_status mcl_batch_set_offsets(mcl_batch_t b, const double* r, mcl_stream_t stream) {
  if (!b || !r) return fail(MCL_EINVAL, "batch_set_offsets: NULL argument");
  for (size_t i = 0; i < b->s.size(); ++i)
    if (!(r[i] >= 0.0 && r[i] < 1.0)) return fail(MCL_EINVAL, "batch_set_offsets: r[%zu] outside [0, 1)", i);
  MCL_CUDA(cudaMemcpyAsync(b->d_r, r, b->s.size() * sizeof(double), cudaMemcpyHostToDevice,
                           (cudaStream_t)stream));
  return MCL_OK;
}

mcl_status mcl_batch_run(mcl_batch_t b, mcl_stream_t stream) {
  if (!b) return fail(MCL_EINVAL, "batch_run: NULL batch");
  int dev = 0;
  MCL_CUDA(cudaGetDevice(&dev));
  if (dev != b->device) return fail(MCL_EINVAL, "batch_run: batch lives on device %d", b->device);
  cudaStream_t st = (cudaStream_t)stream;
  if (!b->use_graph) return enqueue(b, st, true);
  if (!b->exec) {
    // capture on the plan's own stream (the caller's may be the legacy default
    // stream, which cannot be captured); the graph then runs on the caller's
    if (!b->cap) MCL_CUDA(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
    MCL_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    mcl_status rc = enqueue(b, b->cap, false);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->cap, &g);
    if (rc != MCL_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "batch_run capture");
    e = cudaGraphInstantiate(&b->exec, g, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(g);
      return cuda_fail(e, "batch_run instantiate");
    }
    b->graph = g;
  }
  PhaseScope ps(MCL_PHASE_SENSOR, st, b->kernels_per_run);
  MCL_CUDA(cudaGraphLaunch(b->exec, st));
  return MCL_OK;
}

mcl_status mcl_batch_get_info(mcl_batch_t b, mcl_batch_info* out) {
  if (!b || !out || out->struct_size < sizeof(mcl_batch_info))
    return fail(MCL_EINVAL, "batch_get_info: bad argument");
  out->n_sessions = (int32_t)b->s.size();
  out->n_groups = (int32_t)b->g.size();
  out->n_items = b->n_items;
  out->total_evals = b->total_evals;
  out->workspace_bytes = (int64_t)b->ws_bytes;
  out->kernels_per_run = b->kernels_per_run;
  out->graph_captured = b->exec ? 1 : 0;
  return MCL_OK;
}

mcl_status mcl_batch_destroy(mcl_batch_t b) {
  if (!b) return MCL_OK;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(b->device);
  cudaDeviceSynchronize();
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->ws) cudaFree(b->ws);
  cudaSetDevice(cur);
  delete b;
  return MCL_OK;
}

}  // extern "C"
