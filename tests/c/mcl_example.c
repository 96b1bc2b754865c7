/*
 * A plain C user of the library's C ABI (no Python, no PyTorch): reads a
 * dense TSDF, particles and a scan from binary files, runs the sensor update
 * with the fused pose estimate and the systematic resampling on the GPU, and
 * writes log-weights, weights, resampled indices and the estimate back.
 *
 *   mcl_example DIR      reads DIR/map.bin, DIR/particles.bin, DIR/scan.bin,
 *                        writes DIR/out.bin
 *
 * map.bin:       int64 nx, ny, nz; float origin[3], voxel, truncation;
 *                float values[nz][ny][nx]
 * particles.bin: int64 P; float [P][6]
 * scan.bin:      int64 N; float [N][3]
 * out.bin:       float logw[P], float w[P], int32 idx[P], mcl_estimate
 */
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "mcl.h"

static void* read_file(const char* dir, const char* name, size_t* size) {
  char path[4096];
  snprintf(path, sizeof path, "%s/%s", dir, name);
  FILE* f = fopen(path, "rb");
  if (!f) return NULL;
  fseek(f, 0, SEEK_END);
  long n = ftell(f);
  fseek(f, 0, SEEK_SET);
  void* buf = malloc((size_t)n);
  if (buf && fread(buf, 1, (size_t)n, f) != (size_t)n) {
    free(buf);
    buf = NULL;
  }
  fclose(f);
  *size = (size_t)n;
  return buf;
}

#define CHECK(call)                                                            \
  do {                                                                         \
    mcl_status s_ = (call);                                                    \
    if (s_ != MCL_OK) {                                                        \
      fprintf(stderr, "%s failed: %d %s\n", #call, s_, mcl_last_error());      \
      return 1;                                                                \
    }                                                                          \
  } while (0)

#define CUDA(call)                                                             \
  do {                                                                         \
    cudaError_t e_ = (call);                                                   \
    if (e_ != cudaSuccess) {                                                   \
      fprintf(stderr, "%s failed: %s\n", #call, cudaGetErrorString(e_));       \
      return 1;                                                                \
    }                                                                          \
  } while (0)

int main(int argc, char** argv) {
  if (argc != 2) {
    fprintf(stderr, "usage: %s DIR\n", argv[0]);
    return 2;
  }
  size_t map_size = 0, part_size = 0, scan_size = 0;
  char* map = (char*)read_file(argv[1], "map.bin", &map_size);
  char* parts = (char*)read_file(argv[1], "particles.bin", &part_size);
  char* scan = (char*)read_file(argv[1], "scan.bin", &scan_size);
  if (!map || !parts || !scan) {
    fprintf(stderr, "cannot read the inputs\n");
    return 1;
  }
  int64_t dims[3];
  float hdr[5];
  memcpy(dims, map, sizeof dims);
  memcpy(hdr, map + sizeof dims, sizeof hdr);
  const float* values = (const float*)(map + sizeof dims + sizeof hdr);
  int64_t P = 0, N = 0;
  memcpy(&P, parts, sizeof P);
  memcpy(&N, scan, sizeof N);

  mcl_map_desc d;
  memset(&d, 0, sizeof d);
  d.struct_size = sizeof d;
  d.kind = MCL_MAP_DENSE;
  d.dtype = MCL_F32;
  d.origin[0] = hdr[0];
  d.origin[1] = hdr[1];
  d.origin[2] = hdr[2];
  d.voxel = hdr[3];
  d.truncation = hdr[4];
  for (int k = 0; k < 3; ++k) d.dims[k] = dims[k];
  mcl_map_t m = NULL;
  CHECK(mcl_map_create(&d, values, &m));

  float *d_parts = NULL, *d_scan = NULL, *d_logw = NULL, *d_w = NULL;
  int32_t* d_idx = NULL;
  mcl_estimate* d_est = NULL;
  CUDA(cudaMalloc((void**)&d_parts, (size_t)P * 6 * sizeof(float)));
  CUDA(cudaMalloc((void**)&d_scan, (size_t)N * 3 * sizeof(float)));
  CUDA(cudaMalloc((void**)&d_logw, (size_t)P * sizeof(float)));
  CUDA(cudaMalloc((void**)&d_w, (size_t)P * sizeof(float)));
  CUDA(cudaMalloc((void**)&d_idx, (size_t)P * sizeof(int32_t)));
  CUDA(cudaMalloc((void**)&d_est, sizeof(mcl_estimate)));
  CUDA(cudaMemcpy(d_parts, parts + sizeof P, (size_t)P * 6 * sizeof(float), cudaMemcpyHostToDevice));
  CUDA(cudaMemcpy(d_scan, scan + sizeof N, (size_t)N * 3 * sizeof(float), cudaMemcpyHostToDevice));

  mcl_sensor_params prm;
  memset(&prm, 0, sizeof prm);
  prm.struct_size = sizeof prm;
  prm.sigma_hit = 0.1f;
  prm.mode = MCL_LOGPROD;
  CHECK(mcl_sensor_update_estimate(m, d_parts, P, d_scan, N, &prm, d_logw, d_w, d_est, NULL));
  CHECK(mcl_resample(d_w, P, 0.5, d_idx, NULL, NULL, NULL));
  CHECK(mcl_sync(NULL));

  const size_t out_size = (size_t)P * (2 * sizeof(float) + sizeof(int32_t)) + sizeof(mcl_estimate);
  char* out = (char*)malloc(out_size);
  CUDA(cudaMemcpy(out, d_logw, (size_t)P * sizeof(float), cudaMemcpyDeviceToHost));
  CUDA(cudaMemcpy(out + (size_t)P * sizeof(float), d_w, (size_t)P * sizeof(float), cudaMemcpyDeviceToHost));
  CUDA(cudaMemcpy(out + (size_t)P * 2 * sizeof(float), d_idx, (size_t)P * sizeof(int32_t),
                  cudaMemcpyDeviceToHost));
  CUDA(cudaMemcpy(out + (size_t)P * (2 * sizeof(float) + sizeof(int32_t)), d_est, sizeof(mcl_estimate),
                  cudaMemcpyDeviceToHost));
  char path[4096];
  snprintf(path, sizeof path, "%s/out.bin", argv[1]);
  FILE* f = fopen(path, "wb");
  if (!f || fwrite(out, 1, out_size, f) != out_size) {
    fprintf(stderr, "cannot write %s\n", path);
    return 1;
  }
  fclose(f);
  cudaFree(d_parts);
  cudaFree(d_scan);
  cudaFree(d_logw);
  cudaFree(d_w);
  cudaFree(d_idx);
  cudaFree(d_est);
  CHECK(mcl_map_destroy(m));
  free(out);
  free(map);
  free(parts);
  free(scan);
  printf("ok P=%lld N=%lld\n", (long long)P, (long long)N);
  return 0;
}
