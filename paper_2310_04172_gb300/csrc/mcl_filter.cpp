// Whole filter steps on the device (Sec. III: motion update, sensor update,
// pose estimate, resampling), optionally replayed from CUDA graphs.
//
// The filter owns one device allocation holding its particles, weights,
// scan buffer, estimate, per-step inputs and the sensor / resampling
// scratch, sized at creation for the largest scan; every pointer a step uses
// is fixed, so a captured step stays valid. The values that change per step
// (odometry increment, noise counter, resampling offset) travel in a 48-byte
// StepIn record copied to the device before each step from a ring of pinned
// host slots, and the kernels read them when they run.
#include <cmath>
#include <cstring>
#include <list>
#include <vector>

#include "runtime.h"

using namespace mcl;

namespace {

constexpr int kSlots = 8;  // pinned StepIn slots, reused round robin

struct GraphEntry {
  int64_t N;
  cudaGraphExec_t exec;
  int kernels;  // kernel nodes in the graph
};

}  // namespace

struct mcl_filter_s {
  int device = 0;
  mcl_map_t map = nullptr;
  int64_t P = 0, maxN = 0;
  mcl_sensor_params prm{};
  float msig[6] = {};
  uint64_t seed = 0;
  bool use_graph = false;
  int max_graphs = 8;
  int64_t steps = 0, graph_launches = 0;
  double last_r = 0.0;
  char* d = nullptr;
  size_t bytes = 0;
  float *part = nullptr, *part2 = nullptr, *logw = nullptr, *w = nullptr, *scan = nullptr;
  int32_t* idx = nullptr;
  mcl_estimate* est = nullptr;
  StepIn* d_in = nullptr;
  char* ws = nullptr;
  double *cum = nullptr, *tot = nullptr;
  long long* last = nullptr;
  StepIn* h_in = nullptr;
  cudaEvent_t ev[kSlots] = {};
  unsigned* status = nullptr;
  cudaStream_t cap = nullptr;
  std::list<GraphEntry> graphs;  // most recently used first
};

namespace {

void release(mcl_filter_s* f) {
  for (auto& g : f->graphs) cudaGraphExecDestroy(g.exec);
  f->graphs.clear();
  for (auto& e : f->ev)
    if (e) cudaEventDestroy(e);
  if (f->cap) cudaStreamDestroy(f->cap);
  if (f->h_in) cudaFreeHost(f->h_in);
  if (f->d) cudaFree(f->d);
  delete f;
}

// The work of one step for scans of N points, enqueued on s.
mcl_status enqueue_step(mcl_filter_s* f, int64_t N, cudaStream_t s) {
  Plan pl;
  if (mcl_status rc = make_plan(f->map, f->P, N, &f->prm, &pl)) return rc;
  const int P = (int)f->P;
  {
    PhaseScope ps(MCL_PHASE_MOTION, s);
    MCL_CUDA(launch_motion(f->part, P, nullptr, f->msig, f->seed, 0, s, f->d_in));
  }
  if (mcl_status rc = enqueue_sensor(f->map, f->part, f->P, f->scan, N, &f->prm, f->logw, f->w,
                                     f->est, pl, f->ws, f->status, s))
    return rc;
  {
    PhaseScope ps(MCL_PHASE_RESAMPLE, s, resample_kernels(P));
    MCL_CUDA(launch_resample(f->w, P, 0.0, f->idx, f->part, f->part2, f->cum, f->tot, f->last, s,
                             &f->d_in->r));
    MCL_CUDA(cudaMemcpyAsync(f->part, f->part2, (size_t)P * 6 * sizeof(float),
                             cudaMemcpyDeviceToDevice, s));
  }
  return MCL_OK;
}

// The graph of the step for N points: found (and moved to the front) or
// captured on the filter's own stream and instantiated.
mcl_status graph_for(mcl_filter_s* f, int64_t N, GraphEntry* out) {
  for (auto it = f->graphs.begin(); it != f->graphs.end(); ++it)
    if (it->N == N) {
      f->graphs.splice(f->graphs.begin(), f->graphs, it);
      *out = f->graphs.front();
      return MCL_OK;
    }
  cudaGraph_t g = nullptr;
  mcl_status rc;
  cudaError_t e;
  {
    NoProfileScope np;
    MCL_CUDA(cudaStreamBeginCapture(f->cap, cudaStreamCaptureModeThreadLocal));
    rc = enqueue_step(f, N, f->cap);
    e = cudaStreamEndCapture(f->cap, &g);
  }
  if (rc != MCL_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  MCL_CUDA(e);
  size_t n_nodes = 0;
  int kernels = 0;
  e = cudaGraphGetNodes(g, nullptr, &n_nodes);
  std::vector<cudaGraphNode_t> nodes(n_nodes);
  if (e == cudaSuccess && n_nodes) e = cudaGraphGetNodes(g, nodes.data(), &n_nodes);
  for (size_t i = 0; e == cudaSuccess && i < n_nodes; ++i) {
    cudaGraphNodeType t;
    e = cudaGraphNodeGetType(nodes[i], &t);
    kernels += t == cudaGraphNodeTypeKernel;
  }
  cudaGraphExec_t ex = nullptr;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  MCL_CUDA(e);
  f->graphs.push_front({N, ex, kernels});
  while ((int)f->graphs.size() > f->max_graphs) {
    cudaGraphExecDestroy(f->graphs.back().exec);  // an in-flight replay completes first
    f->graphs.pop_back();
  }
  *out = f->graphs.front();
  return MCL_OK;
}

}  // namespace

extern "C" {

mcl_status mcl_filter_create(const mcl_filter_desc* d, const float* particles, mcl_filter_t* out) {
  if (!d || !particles || !out) return fail(MCL_EINVAL, "filter_create: NULL argument");
  *out = nullptr;
  if (d->struct_size < sizeof(mcl_filter_desc)) return fail(MCL_EINVAL, "filter_create: struct_size");
  if (!d->map) return fail(MCL_EINVAL, "filter_create: NULL map");
  if (d->P < 1 || d->P > kMaxCount) return fail(MCL_EINVAL, "filter_create: P = %lld", (long long)d->P);
  if (d->max_points < 1 || d->max_points > kMaxCount)
    return fail(MCL_EINVAL, "filter_create: max_points = %lld", (long long)d->max_points);
  if (d->max_graphs < 0) return fail(MCL_EINVAL, "filter_create: max_graphs < 0");
  if (d->first_step < 0) return fail(MCL_EINVAL, "filter_create: first_step < 0");
  for (int k = 0; k < 6; ++k)
    if (!(d->motion_sigma[k] >= 0.f && d->motion_sigma[k] < 3.4e38f))
      return fail(MCL_EINVAL, "filter_create: motion_sigma[%d]", k);
  if (!aligned(particles, 4)) return fail(MCL_EINVAL, "filter_create: particles need 4-byte alignment");
  if (mcl_status rc = check_params(&d->sensor)) return rc;
  if (mcl_status rc = check_device(d->map)) return rc;
  DeviceState st;
  int dev = 0;
  if (mcl_status rc = device_state(&dev, &st)) return rc;
  Plan pl;
  if (mcl_status rc = make_plan(d->map, d->P, d->max_points, &d->sensor, &pl)) return rc;

  mcl_filter_s* f = new mcl_filter_s;
  f->device = dev;
  f->map = d->map;
  f->P = d->P;
  f->maxN = d->max_points;
  f->prm = d->sensor;
  std::memcpy(f->msig, d->motion_sigma, sizeof(f->msig));
  f->seed = d->seed;
  f->use_graph = d->use_graph != 0;
  f->max_graphs = d->max_graphs > 0 ? d->max_graphs : 8;
  f->steps = d->first_step;
  f->status = st.status;
  const size_t P = (size_t)d->P, N = (size_t)d->max_points;
  const size_t nt = (size_t)resample_tiles((int)d->P);
  size_t o = 0;
  const size_t o_part = o;  o = align256(o + P * 6 * sizeof(float));
  const size_t o_part2 = o; o = align256(o + P * 6 * sizeof(float));
  const size_t o_logw = o;  o = align256(o + P * sizeof(float));
  const size_t o_w = o;     o = align256(o + P * sizeof(float));
  const size_t o_idx = o;   o = align256(o + P * sizeof(int32_t));
  const size_t o_scan = o;  o = align256(o + N * 3 * sizeof(float));
  const size_t o_est = o;   o = align256(o + sizeof(mcl_estimate));
  const size_t o_in = o;    o = align256(o + sizeof(StepIn));
  const size_t o_ws = o;    o = align256(o + pl.total);
  const size_t o_cum = o;   o = align256(o + P * sizeof(double));
  const size_t o_tot = o;   o = align256(o + (nt + 1) * sizeof(double));
  const size_t o_last = o;  o = align256(o + (nt + 1) * sizeof(long long));
  f->bytes = o;
  cudaError_t e = cudaMalloc((void**)&f->d, o);
  if (e != cudaSuccess) {
    release(f);
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? fail(MCL_ENOMEM, "filter_create: %zu device bytes", o)
                                          : cuda_fail(e, "cudaMalloc");
  }
  f->part = (float*)(f->d + o_part);
  f->part2 = (float*)(f->d + o_part2);
  f->logw = (float*)(f->d + o_logw);
  f->w = (float*)(f->d + o_w);
  f->idx = (int32_t*)(f->d + o_idx);
  f->scan = (float*)(f->d + o_scan);
  f->est = (mcl_estimate*)(f->d + o_est);
  f->d_in = (StepIn*)(f->d + o_in);
  f->ws = f->d + o_ws;
  f->cum = (double*)(f->d + o_cum);
  f->tot = (double*)(f->d + o_tot);
  f->last = (long long*)(f->d + o_last);
  e = cudaMallocHost((void**)&f->h_in, kSlots * sizeof(StepIn));
  for (int k = 0; e == cudaSuccess && k < kSlots; ++k)
    e = cudaEventCreateWithFlags(&f->ev[k], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&f->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMemset(f->d, 0, o);
  if (e == cudaSuccess)
    e = cudaMemcpy(f->part, particles, P * 6 * sizeof(float), cudaMemcpyDeviceToDevice);
  if (e != cudaSuccess) {
    release(f);
    return cuda_fail(e, "filter_create");
  }
  std::memset(f->h_in, 0, kSlots * sizeof(StepIn));
  *out = f;
  return MCL_OK;
}

mcl_status mcl_filter_step(mcl_filter_t f, const float* delta, const float* scan, int64_t N,
                           mcl_estimate* out, mcl_stream_t stream) {
  if (!f || !scan) return fail(MCL_EINVAL, "filter_step: NULL filter or scan");
  if (N < 1 || N > f->maxN)
    return fail(MCL_EINVAL, "filter_step: N = %lld outside [1, %lld]", (long long)N, (long long)f->maxN);
  if (!aligned(scan, 4) || !aligned(out, 8)) return fail(MCL_EINVAL, "filter_step: misaligned pointer");
  if (delta)
    for (int k = 0; k < 6; ++k)
      if (!std::isfinite(delta[k])) return fail(MCL_EINVAL, "filter_step: delta[%d] not finite", k);
  if (mcl_status rc = check_device(f->map)) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const int k = (int)(f->steps % kSlots);
  MCL_CUDA(cudaEventSynchronize(f->ev[k]));  // the slot's previous copy has been read
  StepIn& in = f->h_in[k];
  std::memset(&in, 0, sizeof(in));
  if (delta) std::memcpy(in.delta, delta, sizeof(in.delta));
  in.motion = delta ? 1 : 0;
  in.step = (unsigned long long)f->steps;
  in.r = resample_offset(f->seed, (uint64_t)f->steps);
  MCL_CUDA(cudaMemcpyAsync(f->d_in, &in, sizeof(StepIn), cudaMemcpyHostToDevice, s));
  MCL_CUDA(cudaEventRecord(f->ev[k], s));
  MCL_CUDA(cudaMemcpyAsync(f->scan, scan, (size_t)N * 3 * sizeof(float), cudaMemcpyDeviceToDevice, s));
  if (f->use_graph) {
    GraphEntry g{};
    if (mcl_status rc = graph_for(f, N, &g)) return rc;
    PhaseScope ps(MCL_PHASE_OTHER, s, g.kernels);
    MCL_CUDA(cudaGraphLaunch(g.exec, s));
    ++f->graph_launches;
  } else if (mcl_status rc = enqueue_step(f, N, s)) {
    return rc;
  }
  if (out) MCL_CUDA(cudaMemcpyAsync(out, f->est, sizeof(mcl_estimate), cudaMemcpyDeviceToDevice, s));
  f->last_r = in.r;
  ++f->steps;
  return MCL_OK;
}

mcl_status mcl_filter_reset(mcl_filter_t f, const float* particles, mcl_stream_t stream) {
  if (!f || !particles) return fail(MCL_EINVAL, "filter_reset: NULL argument");
  if (!aligned(particles, 4)) return fail(MCL_EINVAL, "filter_reset: particles need 4-byte alignment");
  if (mcl_status rc = check_device(f->map)) return rc;
  MCL_CUDA(cudaMemcpyAsync(f->part, particles, (size_t)f->P * 6 * sizeof(float),
                           cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return MCL_OK;
}

mcl_status mcl_filter_get_state(mcl_filter_t f, mcl_filter_state* out) {
  if (!f || !out) return fail(MCL_EINVAL, "filter_get_state: NULL argument");
  if (out->struct_size < sizeof(mcl_filter_state)) return fail(MCL_EINVAL, "filter_get_state: struct_size");
  out->particles = f->part;
  out->logw = f->logw;
  out->w = f->w;
  out->idx = f->idx;
  out->estimate = f->est;
  out->P = f->P;
  out->steps = f->steps;
  out->graph_launches = f->graph_launches;
  out->last_r = f->last_r;
  out->device_bytes = (int64_t)f->bytes;
  out->graphs = (int32_t)f->graphs.size();
  out->reserved = 0;
  return MCL_OK;
}

mcl_status mcl_filter_destroy(mcl_filter_t f) {
  if (!f) return MCL_OK;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(f->device);
  const cudaError_t e = cudaDeviceSynchronize();
  release(f);
  cudaSetDevice(prev);
  return e == cudaSuccess ? MCL_OK : cuda_fail(e, "filter_destroy");
}

}  // extern "C"
