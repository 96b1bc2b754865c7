// Batched sensor update over many robot sessions (C ABI in include/mcl.h).
//
// A plan fixes the sessions' device buffers, groups the sessions whose maps
// share kernel kind, storage type, geometry and score constants (each
// session keeps its own map values and brick index, read from the group's
// device table), and lays out one device workspace for the whole step. A run
// enqueues one launch per side step for all sessions at once (spatial order,
// pose rows and scan packing; log-weights, normalisation with the optional
// estimate, systematic resampling; see SideSeg) and one persistent sensor
// kernel per group over the (session, point chunk, particle block) items of
// its sessions, handed out in order by a device counter for brick maps read
// nearest. The number of launches does not grow with the number of
// sessions. With use_graph the step is captured once into a CUDA graph and
// replayed.
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
  mcl_map_t map;  // the first session's map: geometry and score constants
  int mode, neglect;
  uint32_t flags;
  float sigma;
  bool dynamic;
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
  a->cs = sum_exponent_constant(sig, q16, scale);
  a->store_scale = (q16 && mode == MCL_LOGPROD) ? (float)(scale * scale) : 1.0f;
}

}  // namespace

namespace mcl {

// Maps whose sessions can share a batched sensor launch: the same kernel kind,
// brick layout, storage type, grid geometry, truncation and int16 scale, and
// the same kind of values (TSDF, or scores of one sigma). Values and brick
// index may differ.
bool same_geometry(const mcl_map_s* a, const mcl_map_s* b) {
  const MapView &x = a->view, &y = b->view;
  return kernel_kind(a) == kernel_kind(b) && a->dtype == b->dtype && x.layout == y.layout &&
         x.ox == y.ox && x.oy == y.oy && x.oz == y.oz && x.inv == y.inv && x.nx == y.nx &&
         x.ny == y.ny && x.nz == y.nz && x.nbx == y.nbx && x.nby == y.nby && x.tau == y.tau &&
         x.scale == y.scale && a->score_sigma == b->score_sigma &&
         a->score_outside == b->score_outside;
}

// The per-session fields of BatchSession that name its map.
void session_map(const mcl_map_s* m, BatchSession* t) {
  t->values = m->view.values;
  t->table = m->view.table;
  t->grid = m->view.grid;
  t->n_slots = m->view.n_slots;
  t->hash_mask = m->view.hash_mask;
  t->hash_shift = m->view.hash_shift;
  t->max_probe = m->view.max_probe;
}

}  // namespace mcl

struct mcl_batch_s {
  int device = 0;
  std::vector<SessionPlan> s;
  std::vector<Group> g;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  double* d_r = nullptr;
  unsigned long long* d_queue = nullptr;  // one item counter per group
  unsigned* status = nullptr;
  SideTables side;
  bool use_graph = false;
  cudaStream_t cap = nullptr;  // plan-owned stream the step is captured on
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int kernels_per_run = 0;
  long long n_items = 0, total_evals = 0;
};

namespace {

mcl_status enqueue(mcl_batch_s* b, cudaStream_t st, bool profile) {
  auto side = [&](std::initializer_list<int> kinds) -> mcl_status {
    for (int k : kinds)
      if (mcl_status rc = enqueue_side(b->side, k, st)) return rc;
    return MCL_OK;
  };
  auto count = [&](std::initializer_list<int> kinds) {
    int n = 0;
    for (int k : kinds) n += b->side.b[k].blocks > 0 ? 1 : 0;
    return n;
  };
  const auto pre = {(int)kSideOrderZero, (int)kSideOrderKeys, (int)kSideOrderTiles,
                    (int)kSideOrderTotals, (int)kSideOrderScatter, (int)kSidePosePack};
  const auto norm = {(int)kSideNormalise, (int)kSideEstimate};
  const auto res = {(int)kSideTileScan, (int)kSideTileOffsets, (int)kSideSystematic};
  {
    PhaseScope ps(MCL_PHASE_POSE, st, profile ? count(pre) : 0);
    if (mcl_status rc = side(pre)) return rc;
  }
  {
    PhaseScope ps(MCL_PHASE_SENSOR, st, profile ? (int)b->g.size() : 0);
    if (b->d_queue) MCL_CUDA(cudaMemsetAsync(b->d_queue, 0, b->g.size() * sizeof(unsigned long long), st));
    for (auto& g : b->g)
      MCL_CUDA(launch_sensor_batch(kernel_kind(g.map), g.map->view.layout, g.map->dtype, g.args, g.sh, st));
  }
  {
    PhaseScope ps(MCL_PHASE_REDUCE, st, profile ? count({(int)kSideStats}) : 0);
    if (mcl_status rc = side({(int)kSideStats})) return rc;
  }
  {
    PhaseScope ps(MCL_PHASE_NORMALISE, st, profile ? count(norm) : 0);
    if (mcl_status rc = side(norm)) return rc;
  }
  {
    PhaseScope ps(MCL_PHASE_RESAMPLE, st, profile ? count(res) : 0);
    if (mcl_status rc = side(res)) return rc;
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
                               bp->unroll, bp->pipeline, bp->particle_order, bp->item_order,
                               u.scan_rings};
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
    // group by map geometry, score constants and read rule
    const int neglect = (u.flags & MCL_NEGLECT_OUTSIDE) ? 1 : 0;
    int gi = -1;
    for (size_t k = 0; k < b->g.size(); ++k)
      if (same_geometry(b->g[k].map, u.map) && b->g[k].mode == u.mode && b->g[k].flags == u.flags &&
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
      // items handed out by a counter for brick maps (as the
      // single-session update does for large sets)
      g.dynamic = u.map->kind == MCL_MAP_BRICK && (bp->item_order == 0 || bp->item_order == 3);
      b->g.push_back(g);
      gi = (int)b->g.size() - 1;
    }
    sp.group = gi;
    b->g[gi].sessions.push_back(i);
    b->s.push_back(sp);
    b->total_evals += u.P * u.N;
  }
  // per group: resident CTAs and the item order (segments of one session's
  // items, sessions on one map interleaved sweep by sweep)
  const size_t ng = b->g.size();
  std::vector<std::vector<ItemSeg>> gsegs(ng);
  std::vector<std::vector<int>> gsweeps(ng);
  std::vector<long long> gitems(ng);
  for (size_t k = 0; k < ng; ++k) {
    Group& g = b->g[k];
    int bps = 0;
    cudaError_t e = sensor_batch_occupancy(kernel_kind(g.map), g.map->view.layout, g.map->dtype,
                                           kernel_mode(g.map, g.mode), g.sh, &bps);
    if (e != cudaSuccess || bps < 1) return bail(cuda_fail(e, "batch_create occupancy"));
    const long long slots = (long long)st.sms * bps;
    std::vector<SegSession> ss;
    for (int i : g.sessions) {
      const SessionPlan& sp = b->s[i];
      ss.push_back(SegSession{sp.u.map->view.values, sp.pl.nblk, sp.pl.K, sp.pl.sweep});
    }
    gitems[k] = item_segments(ss, slots, g.dynamic, kBatchMaxRounds, &gsweeps[k], &gsegs[k]);
    g.sh.grid = (int)std::min<long long>(gitems[k], slots);
  }
  // group tables, item counters, offsets and the side tables follow the session blocks
  std::vector<size_t> off_tab(ng), off_seg(ng);
  for (size_t k = 0; k < ng; ++k) {
    off_tab[k] = off;
    off = align256(off + b->g[k].sessions.size() * sizeof(BatchSession));
    off_seg[k] = off;
    off = align256(off + gsegs[k].size() * sizeof(ItemSeg));
  }
  const size_t off_queue = off;
  off = align256(off + b->g.size() * sizeof(unsigned long long));
  const size_t off_r = off;
  off = align256(off + (size_t)n * sizeof(double));
  const size_t off_side = off;
  off = align256(off + side_table_bytes(n));
  b->ws_bytes = off;
  cudaError_t e = cudaMalloc(&b->ws, b->ws_bytes);
  if (e != cudaSuccess) return bail(cuda_fail(e, "batch_create workspace"));
  b->d_r = (double*)(b->ws + off_r);
  e = cudaMemset(b->d_r, 0, (size_t)n * sizeof(double));
  if (e != cudaSuccess) return bail(cuda_fail(e, "batch_create offsets"));
  bool any_dynamic = false;
  for (size_t k = 0; k < b->g.size(); ++k) {
    Group& g = b->g[k];
    std::vector<BatchSession> tab;
    for (int i : g.sessions) {
      const SessionPlan& sp = b->s[i];
      char* ws = b->ws + sp.base;
      BatchSession t{};
      t.mats = (const float4*)(ws + sp.pl.off_mats);
      t.scan = (const float4*)(ws + sp.pl.off_scan);
      t.partial = (float*)(ws + sp.pl.off_partial);
      t.P = (int)sp.u.P;
      t.N = (int)sp.u.N;
      t.nblk = sp.pl.nblk;
      t.K = sp.pl.K;
      t.sweep = gsweeps[k][tab.size()];
      t.ppi = sp.pl.sh.ppi;
      session_map(sp.u.map, &t);
      tab.push_back(t);
    }
    e = cudaMemcpy(b->ws + off_tab[k], tab.data(), tab.size() * sizeof(BatchSession), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(b->ws + off_seg[k], gsegs[k].data(), gsegs[k].size() * sizeof(ItemSeg),
                     cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bail(cuda_fail(e, "batch_create tables"));
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
    if (g.dynamic) {
      a.queue = (unsigned long long*)(b->ws + off_queue) + k;
      any_dynamic = true;
    }
    g.args.sessions = (const BatchSession*)(b->ws + off_tab[k]);
    g.args.segs = (const ItemSeg*)(b->ws + off_seg[k]);
    g.args.n_segs = (int)gsegs[k].size() - 1;
    g.args.n_items = gitems[k];
    b->n_items += gitems[k];
  }
  if (any_dynamic) b->d_queue = (unsigned long long*)(b->ws + off_queue);
  // side tables of all sessions
  std::vector<SideSeg> segs(n);
  for (int i = 0; i < n; ++i) {
    const SessionPlan& sp = b->s[i];
    const Plan& pl = sp.pl;
    char* ws = b->ws + sp.base;
    SideSeg& q = segs[i];
    q = SideSeg{};
    q.particles = sp.u.particles;
    q.scan = sp.u.scan;
    q.P = (int)sp.u.P;
    q.N = (int)sp.u.N;
    if (pl.spatial) {
      q.key = (uint32_t*)(ws + pl.off_key);
      q.hist = (uint32_t*)(ws + pl.off_hist);
      q.rank = (int*)(ws + pl.off_rank);
      order_grid(sp.u.map->view, &q.order_o, &q.order_s);
    }
    q.mats = (float4*)(ws + pl.off_mats);
    q.frame = sensor_frame(sp.u.map->view, pl.sh.interp != 0);
    q.packed = ws + pl.off_scan;
    q.layout = scan_layout(pl.sh);
    q.partial = (const float*)(ws + pl.off_partial);
    q.K = pl.K;
    q.mode = sp.u.mode;
    const double sig = (double)sp.u.sigma_hit;
    q.c = sensor_c(sp.u.sigma_hit);
    q.k = (float)(1.0 / std::sqrt(2.0 * 3.141592653589793 * sig * sig));
    q.logw = sp.u.logw ? sp.u.logw : (float*)(ws + pl.off_logw);
    q.w = sp.u.w;
    q.stats = (float2*)(ws + pl.off_stats);
    q.nb = normalise_blocks(q.P);
    q.ostats = (float*)(ws + pl.off_ostats);
    if (sp.u.estimate) {
      q.est_part = (EstPartial*)(ws + pl.off_est);
      q.est = sp.u.estimate;
    }
    if (sp.u.resample_idx) {
      q.idx = sp.u.resample_idx;
      q.pin = sp.u.particles_out ? sp.u.particles : nullptr;
      q.pout = sp.u.particles_out;
      q.cum = (double*)(ws + sp.off_cum);
      q.tile_total = (double*)(ws + sp.off_tot);
      q.tile_last = (long long*)(ws + sp.off_last);
      q.r = b->d_r + i;
    }
  }
  std::vector<char> h(side_table_bytes(n));
  side_tables(segs, h.data(), b->ws + off_side, &b->side);
  e = cudaMemcpy(b->ws + off_side, h.data(), h.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return bail(cuda_fail(e, "batch_create side tables"));
  b->kernels_per_run = (int)b->g.size() + side_launch_count(b->side);
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
    mcl_status rc;
    {
      NoProfileScope np;  // no profiling events inside the graph
      rc = enqueue(b, b->cap, false);
    }
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
