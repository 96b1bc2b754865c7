// Serving loop (C ABI in include/mcl.h): device-resident robot sessions,
// admission by device-memory budget, latest-scan-wins queues and continuous
// batching of pending scans into batched filter steps on max_in_flight slots.
//
// Threads: client calls take the server mutex to queue scans and collect
// tickets; one scheduler thread forms batches and enqueues their work; a host
// function at the end of each slot's stream marks the slot done (it makes no
// CUDA call) and wakes the scheduler, which completes the slot's tickets.
#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "runtime.h"

using namespace mcl;

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Ticket {
  int status = -1;  // -1 pending, else MCL_RESULT_*
  double t_submit = 0, latency_ms = 0;
  int64_t evals = 0, step = 0;
  mcl_estimate est{};
};

struct Slot;

// Body-frame increment a followed by b (each relative to the body at its
// start), in FP64: t = t_a + R_a t_b, R = R_a R_b, angles read back as in the
// motion update (R = Rz(yaw) Ry(pitch) Rx(roll), yaw in [-pi, pi)).
void compose_increment(const float a[6], const float b[6], float out[6]) {
  auto rot = [](double r, double p, double y, double R[9]) {
    const double cr = std::cos(r), sr = std::sin(r), cp = std::cos(p), sp = std::sin(p),
                 cy = std::cos(y), sy = std::sin(y);
    R[0] = cy * cp; R[1] = cy * sp * sr - sy * cr; R[2] = cy * sp * cr + sy * sr;
    R[3] = sy * cp; R[4] = sy * sp * sr + cy * cr; R[5] = sy * sp * cr - cy * sr;
    R[6] = -sp;     R[7] = cp * sr;                R[8] = cp * cr;
  };
  double A[9], B[9], C[9];
  rot(a[3], a[4], a[5], A);
  rot(b[3], b[4], b[5], B);
  for (int r = 0; r < 3; ++r) {
    out[r] = (float)((double)a[r] + A[3 * r] * b[0] + A[3 * r + 1] * b[1] + A[3 * r + 2] * b[2]);
    for (int c = 0; c < 3; ++c) C[3 * r + c] = A[3 * r] * B[c] + A[3 * r + 1] * B[3 + c] + A[3 * r + 2] * B[6 + c];
  }
  out[3] = (float)std::atan2(C[7], C[8]);
  out[4] = (float)std::asin(std::fmin(1.0, std::fmax(-1.0, -C[6])));
  double yaw = std::atan2(C[3], C[0]);
  if (yaw >= 3.141592653589793) yaw = -3.141592653589793;
  out[5] = (float)yaw;
}

}  // namespace

struct mcl_session_s {
  mcl_server_s* srv = nullptr;
  mcl_map_t map = nullptr;
  int64_t P = 0, max_N = 0;
  float sigma = 0.1f;
  int mode = 0;
  uint32_t flags = 0;
  int scan_rings = 0;
  float msig[6] = {0, 0, 0, 0, 0, 0};
  uint64_t seed = 0;
  int64_t step = 0;
  int cur = 0;
  float* d_part[2] = {nullptr, nullptr};
  float *d_scan = nullptr, *d_logw = nullptr, *d_w = nullptr;
  int32_t* d_idx = nullptr;
  char* d_ws = nullptr;
  Plan pl{};
  size_t off_cum = 0, off_tot = 0, off_last = 0;
  float* h_stage[2] = {nullptr, nullptr};  // pinned scan staging: queued / running
  int stage_next = 0;
  // queued scan
  bool pending = false;
  int64_t pending_N = 0;
  bool pending_delta = false;
  float delta[6] = {0, 0, 0, 0, 0, 0};
  mcl_ticket_t pending_ticket = 0;
  double pending_since = 0;  // when the session last became pending (kept on supersede)
  // running step
  bool in_flight = false;
  bool closing = false;
  int64_t bytes = 0;
};

namespace {

struct Slot {
  cudaStream_t st = nullptr;
  char* d_tab = nullptr;  // device tables of the step (side launches, groups, counters, offsets)
  char* h_tab = nullptr;  // pinned staging of the same
  size_t tab_bytes = 0;
  mcl_estimate* d_est = nullptr;  // the step's estimates, one per session
  mcl_estimate* h_est = nullptr;  // pinned copy, read when the step completed
  bool busy = false;
  std::atomic<bool> done{false};
  mcl_server_s* srv = nullptr;
  std::vector<mcl_session_s*> sessions;
  std::vector<mcl_ticket_t> tickets;
};

}  // namespace

struct mcl_server_s {
  int device = 0;
  mcl_server_desc desc{};
  DeviceState dev{};
  std::mutex mu;
  std::condition_variable cv;       // wakes the scheduler
  std::condition_variable cv_done;  // wakes clients
  std::vector<mcl_session_s*> sessions;
  std::map<mcl_ticket_t, Ticket> tickets;
  mcl_ticket_t next_ticket = 1;
  std::vector<Slot*> slots;
  std::thread th;
  bool stop = false, paused = false;
  int64_t bytes_in_use = 0;
  // statistics since creation or reset
  std::vector<double> lat;
  int64_t completed = 0, superseded = 0, batches = 0, evals = 0, batch_sessions = 0;
  double t0 = 0;
  std::string sched_error;
};

namespace {

// Runs on a CUDA driver thread when the slot's stream reaches it: no CUDA
// call and no lock here (the scheduler also polls every 2 ms).
void CUDART_CB on_slot_done(void* p) {
  Slot* sl = static_cast<Slot*>(p);
  sl->done.store(true);
  sl->srv->cv.notify_all();
}

void free_session(mcl_session_s* ss) {
  cudaFree(ss->d_part[0]);
  cudaFree(ss->d_part[1]);
  cudaFree(ss->d_scan);
  cudaFree(ss->d_logw);
  cudaFree(ss->d_w);
  cudaFree(ss->d_idx);
  cudaFree(ss->d_ws);
  cudaFreeHost(ss->h_stage[0]);
  cudaFreeHost(ss->h_stage[1]);
  delete ss;
}

// Bytes of a slot's step tables for up to cap sessions (and as many groups).
size_t slot_table_bytes(int cap) {
  return side_table_bytes(cap) + (size_t)cap * (align256(sizeof(BatchSession)) + 256 + 256) +
         (size_t)cap * ((kServerMaxRounds + 1) * sizeof(ItemSeg) + 256) + 3 * align256((size_t)cap * 8) + 4096;
}

// Enqueues one batched filter step for the slot's sessions on its stream:
// per session the host-to-device copy of its scan, then one launch per step
// for all sessions (motion, spatial order, pose rows and scan packing), one
// sensor kernel per group of sessions whose maps share geometry, one launch
// per step again (log-weights, normalisation with the estimate, resampling)
// and one copy of all estimates back. The number of launches does not grow
// with the number of sessions.
mcl_status enqueue_step(mcl_server_s* S, Slot* sl, const std::vector<int64_t>& Ns,
                        const std::vector<int>& stages, const std::vector<bool>& deltas,
                        const std::vector<std::array<float, 6>>& dvals) {
  cudaStream_t st = sl->st;
  const size_t n = sl->sessions.size();
  for (size_t i = 0; i < n; ++i) {
    mcl_session_s* ss = sl->sessions[i];
    MCL_CUDA(cudaMemcpyAsync(ss->d_scan, ss->h_stage[stages[i]], (size_t)Ns[i] * 3 * sizeof(float),
                             cudaMemcpyHostToDevice, st));
  }
  // slot buffer: side tables | resampling offsets | item counters | group tables
  size_t off = side_table_bytes((int)n);
  const size_t off_r = off;
  off = align256(off + n * sizeof(double));
  const size_t off_queue = off;
  off = align256(off + n * sizeof(unsigned long long));
  double* h_r = (double*)(sl->h_tab + off_r);
  std::memset(sl->h_tab + off_queue, 0, n * sizeof(unsigned long long));  // counters start at 0
  std::vector<SideSeg> segs(n);
  for (size_t i = 0; i < n; ++i) {
    mcl_session_s* ss = sl->sessions[i];
    const Plan& pl = ss->pl;
    char* ws = ss->d_ws;
    float* part = ss->d_part[ss->cur];
    SideSeg& q = segs[i];
    q = SideSeg{};
    if (deltas[i]) {
      q.mpart = part;
      for (int k = 0; k < 6; ++k) {
        q.mdelta[k] = dvals[i][k];
        q.msig[k] = ss->msig[k];
      }
      q.mseed = ss->seed;
      q.mstep = (unsigned long long)ss->step;
    }
    q.particles = part;
    q.scan = ss->d_scan;
    q.P = (int)ss->P;
    q.N = (int)Ns[i];
    if (pl.spatial) {
      q.key = (uint32_t*)(ws + pl.off_key);
      q.hist = (uint32_t*)(ws + pl.off_hist);
      q.rank = (int*)(ws + pl.off_rank);
      order_grid(ss->map->view, &q.order_o, &q.order_s);
    }
    q.mats = (float4*)(ws + pl.off_mats);
    q.frame = sensor_frame(ss->map->view, pl.sh.interp != 0);
    q.packed = ws + pl.off_scan;
    q.layout = scan_layout(pl.sh);  // staging order by this scan's own N
    q.layout.rings = patch_rings(Ns[i], ss->scan_rings);
    q.layout.az = q.layout.rings ? (int)(Ns[i] / q.layout.rings) : 0;
    q.partial = (const float*)(ws + pl.off_partial);
    q.K = (int)((Ns[i] + pl.sh.chunk - 1) / pl.sh.chunk);
    q.mode = ss->mode;
    const double sig = (double)ss->sigma;
    q.c = (float)(-0.5 / (sig * sig));
    q.k = (float)(1.0 / std::sqrt(2.0 * 3.141592653589793 * sig * sig));
    q.logw = ss->d_logw;
    q.w = ss->d_w;
    q.stats = (float2*)(ws + pl.off_stats);
    q.nb = normalise_blocks(q.P);
    q.ostats = (float*)(ws + pl.off_ostats);
    q.est_part = (EstPartial*)(ws + pl.off_est);
    q.est = sl->d_est + i;
    q.idx = ss->d_idx;
    q.pin = part;
    q.pout = ss->d_part[1 - ss->cur];
    q.cum = (double*)(ws + ss->off_cum);
    q.tile_total = (double*)(ws + ss->off_tot);
    q.tile_last = (long long*)(ws + ss->off_last);
    q.r = (const double*)(sl->d_tab + off_r) + i;
    h_r[i] = resample_offset(ss->seed, (uint64_t)ss->step);
  }
  SideTables side;
  side_tables(segs, sl->h_tab, sl->d_tab, &side);
  // group the slot's sessions by map geometry and score constants
  struct G {
    mcl_map_t map;
    int mode, neglect;
    uint32_t flags;
    float sigma;
    std::vector<size_t> idx;
  };
  std::vector<G> groups;
  for (size_t i = 0; i < n; ++i) {
    mcl_session_s* ss = sl->sessions[i];
    const int neglect = (ss->flags & MCL_NEGLECT_OUTSIDE) ? 1 : 0;
    G* g = nullptr;
    for (auto& x : groups)
      if (same_geometry(x.map, ss->map) && x.mode == ss->mode && x.flags == ss->flags && x.sigma == ss->sigma)
        g = &x;
    if (!g) {
      groups.push_back(G{ss->map, ss->mode, neglect, ss->flags, ss->sigma, {}});
      g = &groups.back();
    }
    g->idx.push_back(i);
  }
  std::vector<BatchArgs> args(groups.size());
  std::vector<SensorShape> shapes(groups.size());
  for (size_t k = 0; k < groups.size(); ++k) {
    const G& g = groups[k];
    SensorShape sh = sl->sessions[g.idx.back()]->pl.sh;
    int bps = 0;
    MCL_CUDA(sensor_batch_occupancy(kernel_kind(g.map), g.map->view.layout, g.map->dtype,
                                    kernel_mode(g.map, g.mode), sh, &bps));
    const long long slots = (long long)S->dev.sms * std::max(bps, 1);
    // brick maps: items handed out in order by a counter, sessions on one map interleaved
    const bool dynamic =
        g.map->kind == MCL_MAP_BRICK && (S->desc.shape.item_order == 0 || S->desc.shape.item_order == 3);
    std::vector<SegSession> segin;
    for (size_t q = 0; q < g.idx.size(); ++q) {
      mcl_session_s* ss = sl->sessions[g.idx[q]];
      const int K = (int)((Ns[g.idx[q]] + ss->pl.sh.chunk - 1) / ss->pl.sh.chunk);
      segin.push_back(SegSession{ss->map->view.values, ss->pl.nblk, K, ss->pl.sweep});
    }
    std::vector<int> sweeps;
    std::vector<ItemSeg> segv;
    const long long n_items = item_segments(segin, slots, dynamic, kServerMaxRounds, &sweeps, &segv);
    BatchSession* tab = (BatchSession*)(sl->h_tab + off);
    const size_t off_tab = off;
    off = align256(off + g.idx.size() * sizeof(BatchSession));
    const size_t off_seg = off;
    off = align256(off + segv.size() * sizeof(ItemSeg));
    if (off > sl->tab_bytes) return fail(MCL_EINTERNAL, "server: step tables exceed the slot buffer");
    std::memcpy(sl->h_tab + off_seg, segv.data(), segv.size() * sizeof(ItemSeg));
    for (size_t q = 0; q < g.idx.size(); ++q) {
      mcl_session_s* ss = sl->sessions[g.idx[q]];
      const int64_t N = Ns[g.idx[q]];
      sh = ss->pl.sh;
      const int K = (int)((N + sh.chunk - 1) / sh.chunk);
      BatchSession t{};
      t.mats = (const float4*)(ss->d_ws + ss->pl.off_mats);
      t.scan = (const float4*)(ss->d_ws + ss->pl.off_scan);
      t.partial = (float*)(ss->d_ws + ss->pl.off_partial);
      t.P = (int)ss->P;
      t.N = (int)N;
      t.nblk = ss->pl.nblk;
      t.K = K;
      t.sweep = sweeps[q];
      t.ppi = ss->pl.sh.ppi;
      session_map(ss->map, &t);
      tab[q] = t;
    }
    sh.grid = (int)std::min<long long>(n_items, slots);
    shapes[k] = sh;
    BatchArgs& b = args[k];
    b = BatchArgs{};
    SensorArgs& a = b.base;
    a.map = g.map->view;
    a.status = S->dev.status;
    a.chunk = sh.chunk;
    a.ppi = sh.ppi;
    a.layout = scan_layout(sh);
    a.mode = kernel_mode(g.map, g.mode);
    a.neglect = g.neglect;
    const double sig = (double)g.sigma, scale = (double)g.map->view.scale;
    const bool q16 = g.map->dtype == MCL_I16;
    set_fills(g.map, &a);
    a.cs = sum_exponent_constant(sig, q16, scale);
    a.store_scale = (q16 && g.mode == MCL_LOGPROD) ? (float)(scale * scale) : 1.0f;
    if (dynamic) a.queue = (unsigned long long*)(sl->d_tab + off_queue) + k;
    b.sessions = (const BatchSession*)(sl->d_tab + off_tab);
    b.segs = (const ItemSeg*)(sl->d_tab + off_seg);
    b.n_segs = (int)segv.size() - 1;
    b.n_items = n_items;
  }
  MCL_CUDA(cudaMemcpyAsync(sl->d_tab, sl->h_tab, off, cudaMemcpyHostToDevice, st));
  for (int k : {(int)kSideMotion, (int)kSideOrderZero, (int)kSideOrderKeys, (int)kSideOrderTiles,
                (int)kSideOrderTotals, (int)kSideOrderScatter, (int)kSidePosePack})
    if (mcl_status rc = enqueue_side(side, k, st)) return rc;
  for (size_t k = 0; k < groups.size(); ++k)
    MCL_CUDA(launch_sensor_batch(kernel_kind(groups[k].map), groups[k].map->view.layout, groups[k].map->dtype,
                                 args[k], shapes[k], st));
  for (int k : {(int)kSideStats, (int)kSideNormalise, (int)kSideEstimate})
    if (mcl_status rc = enqueue_side(side, k, st)) return rc;
  MCL_CUDA(cudaMemcpyAsync(sl->h_est, sl->d_est, n * sizeof(mcl_estimate), cudaMemcpyDeviceToHost, st));
  for (int k : {(int)kSideTileScan, (int)kSideTileOffsets, (int)kSideSystematic})
    if (mcl_status rc = enqueue_side(side, k, st)) return rc;
  MCL_CUDA(cudaLaunchHostFunc(st, on_slot_done, sl));
  return MCL_OK;
}

// Completes a finished slot's tickets (server mutex held).
void finalize(mcl_server_s* S, Slot* sl) {
  const double t = now_s();
  for (size_t i = 0; i < sl->sessions.size(); ++i) {
    mcl_session_s* ss = sl->sessions[i];
    ss->in_flight = false;
    auto it = S->tickets.find(sl->tickets[i]);
    if (it != S->tickets.end()) {
      it->second.status = MCL_RESULT_DONE;
      it->second.est = sl->h_est[i];  // the slot's stream has completed
      it->second.latency_ms = 1e3 * (t - it->second.t_submit);
      S->lat.push_back(it->second.latency_ms);
      S->evals += it->second.evals;
    }
    ++S->completed;
  }
  S->batch_sessions += (int64_t)sl->sessions.size();
  ++S->batches;
  sl->sessions.clear();
  sl->tickets.clear();
  sl->busy = false;
  sl->done.store(false);
  S->cv_done.notify_all();
}

void scheduler(mcl_server_s* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    bool any_busy = false;
    for (Slot* sl : S->slots) {
      if (sl->busy && sl->done.load()) finalize(S, sl);
      any_busy = any_busy || sl->busy;
    }
    if (S->stop && !any_busy) break;
    Slot* free_slot = nullptr;
    for (Slot* sl : S->slots)
      if (!sl->busy) free_slot = sl;
    std::vector<mcl_session_s*> take;
    if (!S->stop && !S->paused && free_slot) {
      // the sessions that have waited longest first (since their first queued
      // scan, whatever superseded it), up to max_batch of them
      const int cap = S->desc.max_batch > 0 ? S->desc.max_batch : S->desc.max_sessions;
      std::vector<std::pair<double, mcl_session_s*>> ready;
      for (mcl_session_s* ss : S->sessions)
        if (ss->pending && !ss->in_flight && !ss->closing) ready.emplace_back(ss->pending_since, ss);
      std::stable_sort(ready.begin(), ready.end(),
                       [](const auto& a, const auto& b) { return a.first < b.first; });
      for (size_t i = 0; i < ready.size() && (int)take.size() < cap; ++i) take.push_back(ready[i].second);
    }
    if (take.empty()) {
      S->cv.wait_for(lk, std::chrono::milliseconds(2));
      continue;
    }
    // move the queued scans into the slot
    Slot* sl = free_slot;
    sl->busy = true;
    std::vector<int64_t> Ns;
    std::vector<int> stages;
    std::vector<bool> deltas;
    std::vector<std::array<float, 6>> dvals;
    for (mcl_session_s* ss : take) {
      ss->pending = false;
      ss->in_flight = true;
      Ns.push_back(ss->pending_N);
      stages.push_back(1 - ss->stage_next);  // the buffer the queued scan was written to
      deltas.push_back(ss->pending_delta);
      std::array<float, 6> d;
      std::copy(ss->delta, ss->delta + 6, d.begin());
      dvals.push_back(d);
      sl->sessions.push_back(ss);
      sl->tickets.push_back(ss->pending_ticket);
      auto it = S->tickets.find(ss->pending_ticket);
      if (it != S->tickets.end()) {
        it->second.evals = ss->P * ss->pending_N;
        it->second.step = ss->step + 1;
      }
    }
    mcl_status rc = enqueue_step(S, sl, Ns, stages, deltas, dvals);
    for (mcl_session_s* ss : take) {
      ++ss->step;
      ss->cur = 1 - ss->cur;  // the resampled set is the next step's input
    }
    if (rc != MCL_OK) {
      S->sched_error = mcl_last_error();
      sl->done.store(true);  // complete the tickets so no client waits forever
    }
  }
}

}  // namespace

extern "C" {

mcl_status mcl_server_create(const mcl_server_desc* d, mcl_server_t* out) {
  if (!d || !out || d->struct_size < sizeof(mcl_server_desc)) return fail(MCL_EINVAL, "server_create: bad desc");
  *out = nullptr;
  if (d->max_sessions < 1 || d->max_in_flight < 1 || d->max_in_flight > 8 || d->hbm_budget_bytes <= 0 ||
      d->max_batch < 0)
    return fail(MCL_EINVAL, "server_create: max_sessions, max_in_flight (1..8), budget must be positive");
  if (d->shape.use_graph) return fail(MCL_EINVAL, "server_create: steps are not graph-captured");
  auto* S = new mcl_server_s();
  S->desc = *d;
  if (mcl_status rc = device_state(&S->device, &S->dev)) {
    delete S;
    return rc;
  }
  const int cap = d->max_batch > 0 ? d->max_batch : d->max_sessions;
  for (int i = 0; i < d->max_in_flight; ++i) {
    Slot* sl = new Slot();
    sl->srv = S;
    sl->tab_bytes = slot_table_bytes(cap);
    cudaError_t e = cudaStreamCreateWithFlags(&sl->st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&sl->d_tab, sl->tab_bytes);
    if (e == cudaSuccess) e = cudaMallocHost(&sl->h_tab, sl->tab_bytes);
    if (e == cudaSuccess) e = cudaMalloc((void**)&sl->d_est, (size_t)cap * sizeof(mcl_estimate));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&sl->h_est, (size_t)cap * sizeof(mcl_estimate));
    S->slots.push_back(sl);
    if (e != cudaSuccess) {
      mcl_server_destroy(S);
      return cuda_fail(e, "server_create slots");
    }
  }
  S->t0 = now_s();
  S->th = std::thread(scheduler, S);
  *out = S;
  return MCL_OK;
}

mcl_status mcl_session_open(mcl_server_t S, const mcl_session_desc* d, mcl_session_t* out) {
  if (!S || !d || !out || d->struct_size < sizeof(mcl_session_desc)) return fail(MCL_EINVAL, "session_open: bad argument");
  *out = nullptr;
  if (!d->map || !d->particles || d->P < 1 || d->P > kMaxCount || d->max_N < 1 || d->max_N > kMaxCount)
    return fail(MCL_EINVAL, "session_open: map, particles, P or max_N");
  if (d->first_step < 0) return fail(MCL_EINVAL, "session_open: first_step < 0");
  for (int k = 0; k < 6; ++k)
    if (!(d->motion_sigma[k] >= 0.f && d->motion_sigma[k] < 1e30f)) return fail(MCL_EINVAL, "session_open: motion_sigma");
  mcl_sensor_params prm{sizeof(mcl_sensor_params), d->sigma_hit, d->mode, d->flags,
                        S->desc.shape.points_per_chunk, S->desc.shape.lanes_per_particle,
                        S->desc.shape.particles_per_item, S->desc.shape.unroll, S->desc.shape.pipeline,
                        S->desc.shape.particle_order, S->desc.shape.item_order, d->scan_rings};
  if (mcl_status rc = check_params(&prm)) return rc;
  int dev = 0;
  MCL_CUDA(cudaGetDevice(&dev));
  if (dev != S->device || d->map->device != S->device) return fail(MCL_EINVAL, "session_open: map on another device");
  auto* ss = new mcl_session_s();
  ss->srv = S;
  ss->map = d->map;
  ss->P = d->P;
  ss->max_N = d->max_N;
  ss->sigma = d->sigma_hit;
  ss->mode = d->mode;
  ss->flags = d->flags;
  ss->scan_rings = d->scan_rings;
  std::copy(d->motion_sigma, d->motion_sigma + 6, ss->msig);
  ss->seed = d->seed;
  ss->step = d->first_step;
  if (mcl_status rc = make_plan(d->map, d->P, d->max_N, &prm, &ss->pl)) {
    delete ss;
    return rc;
  }
  const int nt = resample_tiles((int)d->P);
  size_t o = ss->pl.total;
  ss->off_cum = o;
  o = align256(o + (size_t)d->P * 8);
  ss->off_tot = o;
  o = align256(o + (size_t)(nt + 1) * 8);
  ss->off_last = o;
  o = align256(o + (size_t)(nt + 1) * 8);
  const int64_t P = d->P;
  ss->bytes = (int64_t)o + 2 * P * 24 + d->max_N * 12 + P * 12 + (int64_t)sizeof(mcl_estimate);
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if ((int)S->sessions.size() >= S->desc.max_sessions) {
      delete ss;
      return fail(MCL_EBUSY, "session_open: %d sessions open (max_sessions)", S->desc.max_sessions);
    }
    if (S->bytes_in_use + ss->bytes > S->desc.hbm_budget_bytes) {
      const long long need = (long long)ss->bytes, used = (long long)S->bytes_in_use;
      delete ss;
      return fail(MCL_ENOMEM, "session_open: needs %lld bytes, %lld of %lld in use", need, used,
                  (long long)S->desc.hbm_budget_bytes);
    }
    S->bytes_in_use += ss->bytes;  // reserved before allocating
  }
  cudaError_t e = cudaMalloc(&ss->d_part[0], (size_t)P * 24);
  if (e == cudaSuccess) e = cudaMalloc(&ss->d_part[1], (size_t)P * 24);
  if (e == cudaSuccess) e = cudaMalloc(&ss->d_scan, (size_t)d->max_N * 12);
  if (e == cudaSuccess) e = cudaMalloc(&ss->d_logw, (size_t)P * 4);
  if (e == cudaSuccess) e = cudaMalloc(&ss->d_w, (size_t)P * 4);
  if (e == cudaSuccess) e = cudaMalloc(&ss->d_idx, (size_t)P * 4);
  if (e == cudaSuccess) e = cudaMalloc(&ss->d_ws, o);
  if (e == cudaSuccess) e = cudaMallocHost(&ss->h_stage[0], (size_t)d->max_N * 12);
  if (e == cudaSuccess) e = cudaMallocHost(&ss->h_stage[1], (size_t)d->max_N * 12);
  if (e == cudaSuccess) e = cudaMemcpy(ss->d_part[0], d->particles, (size_t)P * 24, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->bytes_in_use -= ss->bytes;
    }
    free_session(ss);
    return cuda_fail(e, "session_open");
  }
  std::lock_guard<std::mutex> lk(S->mu);
  S->sessions.push_back(ss);
  *out = ss;
  return MCL_OK;
}

mcl_status mcl_submit_scan(mcl_session_t ss, const float* scan, int64_t N, const float* delta,
                           mcl_ticket_t* out) {
  if (!ss || !scan || !out) return fail(MCL_EINVAL, "submit_scan: NULL argument");
  if (N < 1 || N > ss->max_N) return fail(MCL_EINVAL, "submit_scan: N = %lld outside [1, max_N]", (long long)N);
  if (delta)
    for (int k = 0; k < 6; ++k)
      if (!(delta[k] == delta[k]) || std::fabs(delta[k]) > 1e30f) return fail(MCL_EINVAL, "submit_scan: delta");
  mcl_server_s* S = ss->srv;
  std::lock_guard<std::mutex> lk(S->mu);
  if (ss->closing) return fail(MCL_EINVAL, "submit_scan: session is closing");
  const double now = now_s();
  if (ss->pending) {  // latest scan wins: the queued, unstarted one is superseded
    auto it = S->tickets.find(ss->pending_ticket);
    if (it != S->tickets.end()) it->second.status = MCL_RESULT_SUPERSEDED;
    ++S->superseded;
    // the robot still moved: the superseded scan's increment is kept, composed
    // with the new one
    if (ss->pending_delta && delta) {
      float c[6];
      compose_increment(ss->delta, delta, c);
      std::copy(c, c + 6, ss->delta);
    } else if (delta) {
      std::copy(delta, delta + 6, ss->delta);
    }
    ss->pending_delta = ss->pending_delta || delta != nullptr;
  } else {
    ss->stage_next = 1 - ss->stage_next;  // the other buffer may be in use by the running step
    ss->pending_since = now;
    ss->pending_delta = delta != nullptr;
    if (delta) std::copy(delta, delta + 6, ss->delta);
  }
  // the queued scan lives in h_stage[1 - stage_next]
  std::memcpy(ss->h_stage[1 - ss->stage_next], scan, (size_t)N * 12);
  ss->pending = true;
  ss->pending_N = N;
  const mcl_ticket_t t = S->next_ticket++;
  Ticket tk;
  tk.t_submit = now;
  S->tickets[t] = tk;
  ss->pending_ticket = t;
  *out = t;
  S->cv.notify_all();
  S->cv_done.notify_all();
  return MCL_OK;
}

mcl_status mcl_wait(mcl_server_t S, mcl_ticket_t t, int32_t timeout_ms, mcl_result* out) {
  if (!S || !out || out->struct_size < sizeof(mcl_result)) return fail(MCL_EINVAL, "wait: bad argument");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->tickets.find(t);
  if (it == S->tickets.end()) return fail(MCL_EINVAL, "wait: unknown ticket %llu", (unsigned long long)t);
  auto ready = [&] {
    auto i2 = S->tickets.find(t);
    return i2 == S->tickets.end() || i2->second.status >= 0;
  };
  if (timeout_ms < 0) S->cv_done.wait(lk, ready);
  else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
    return fail(MCL_ETIMEDOUT, "wait: ticket %llu not done after %d ms", (unsigned long long)t, timeout_ms);
  it = S->tickets.find(t);
  if (it == S->tickets.end()) return fail(MCL_EINVAL, "wait: ticket %llu vanished", (unsigned long long)t);
  out->status = it->second.status;
  out->latency_ms = it->second.latency_ms;
  out->evals = it->second.evals;
  out->step = it->second.step;
  out->estimate = it->second.est;
  S->tickets.erase(it);
  if (!S->sched_error.empty()) return fail(MCL_ECUDA, "server step failed: %s", S->sched_error.c_str());
  return MCL_OK;
}

mcl_status mcl_session_get_info(mcl_session_t ss, mcl_session_info* out, int32_t timeout_ms) {
  if (!ss || !out || out->struct_size < sizeof(mcl_session_info))
    return fail(MCL_EINVAL, "session_get_info: bad argument");
  mcl_server_s* S = ss->srv;
  std::unique_lock<std::mutex> lk(S->mu);
  auto idle = [&] { return !ss->pending && !ss->in_flight; };
  if (timeout_ms < 0) S->cv_done.wait(lk, idle);
  else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), idle))
    return fail(MCL_ETIMEDOUT, "session_get_info: session busy after %d ms", timeout_ms);
  out->P = ss->P;
  out->max_N = ss->max_N;
  out->step = ss->step;
  out->seed = ss->seed;
  out->device_bytes = ss->bytes;
  return MCL_OK;
}

mcl_status mcl_session_read(mcl_session_t ss, float* particles, float* w, int32_t timeout_ms) {
  if (!ss) return fail(MCL_EINVAL, "session_read: NULL session");
  mcl_server_s* S = ss->srv;
  std::unique_lock<std::mutex> lk(S->mu);
  auto idle = [&] { return !ss->pending && !ss->in_flight; };
  if (timeout_ms < 0) S->cv_done.wait(lk, idle);
  else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), idle))
    return fail(MCL_ETIMEDOUT, "session_read: session busy after %d ms", timeout_ms);
  if (particles) MCL_CUDA(cudaMemcpy(particles, ss->d_part[ss->cur], (size_t)ss->P * 24, cudaMemcpyDeviceToHost));
  if (w) MCL_CUDA(cudaMemcpy(w, ss->d_w, (size_t)ss->P * 4, cudaMemcpyDeviceToHost));
  return MCL_OK;
}

mcl_status mcl_session_close(mcl_session_t ss) {
  if (!ss) return MCL_OK;
  mcl_server_s* S = ss->srv;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    ss->closing = true;
    if (ss->pending) {
      auto it = S->tickets.find(ss->pending_ticket);
      if (it != S->tickets.end()) it->second.status = MCL_RESULT_CLOSED;
      ss->pending = false;
    }
    S->cv_done.notify_all();
    S->cv_done.wait(lk, [&] { return !ss->in_flight; });
    S->sessions.erase(std::remove(S->sessions.begin(), S->sessions.end(), ss), S->sessions.end());
    S->bytes_in_use -= ss->bytes;
  }
  free_session(ss);
  return MCL_OK;
}

mcl_status mcl_server_get_stats(mcl_server_t S, int32_t reset, mcl_server_stats* out) {
  if (!S || !out || out->struct_size < sizeof(mcl_server_stats)) return fail(MCL_EINVAL, "server_get_stats: bad argument");
  std::lock_guard<std::mutex> lk(S->mu);
  std::vector<double> l = S->lat;
  auto pct = [&](double q) {
    if (l.empty()) return 0.0;
    size_t k = (size_t)std::min<double>((double)l.size() - 1, std::floor(q * (double)(l.size() - 1) + 0.5));
    std::nth_element(l.begin(), l.begin() + k, l.end());
    return l[k];
  };
  out->completed = S->completed;
  out->superseded = S->superseded;
  out->batches = S->batches;
  out->evals = S->evals;
  out->p50_ms = pct(0.5);
  out->p99_ms = pct(0.99);
  out->max_ms = l.empty() ? 0.0 : *std::max_element(l.begin(), l.end());
  out->mean_batch_sessions = S->batches ? (double)S->batch_sessions / (double)S->batches : 0.0;
  out->wall_s = now_s() - S->t0;
  out->evals_per_s = out->wall_s > 0 ? (double)S->evals / out->wall_s : 0.0;
  out->bytes_in_use = S->bytes_in_use;
  out->sessions = (int32_t)S->sessions.size();
  int busy = 0;
  for (Slot* sl : S->slots) busy += sl->busy ? 1 : 0;
  out->in_flight = busy;
  if (reset) {
    S->lat.clear();
    S->completed = S->superseded = S->batches = S->evals = S->batch_sessions = 0;
    S->t0 = now_s();
  }
  return MCL_OK;
}

mcl_status mcl_server_pause(mcl_server_t S, int32_t pause) {
  if (!S) return fail(MCL_EINVAL, "server_pause: NULL server");
  std::lock_guard<std::mutex> lk(S->mu);
  S->paused = pause != 0;
  S->cv.notify_all();
  return MCL_OK;
}

mcl_status mcl_server_destroy(mcl_server_t S) {
  if (!S) return MCL_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    S->paused = false;
    S->cv.notify_all();
  }
  if (S->th.joinable()) S->th.join();
  std::vector<mcl_session_s*> open;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    open = S->sessions;
  }
  for (mcl_session_s* ss : open) mcl_session_close(ss);
  for (Slot* sl : S->slots) {
    if (sl->st) cudaStreamSynchronize(sl->st);
    if (sl->st) cudaStreamDestroy(sl->st);
    cudaFree(sl->d_tab);
    cudaFreeHost(sl->h_tab);
    cudaFree(sl->d_est);
    cudaFreeHost(sl->h_est);
    delete sl;
  }
  delete S;
  return MCL_OK;
}

}  // extern "C"
