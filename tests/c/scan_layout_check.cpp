// Host-side check of the scan staging order (ScanLayout::source, patch_rings):
// with a ring count the staged order is the 4-ring x 8-point patches of a
// ring-major scan, written here as four nested loops, and a bijection of the
// N points; without one it is the order given; the ring count applies
// exactly when it divides N, is a multiple of 4 and N / rings one of 8. Also
// the pair layout's sizes: a chunk of cnt points takes ceil(cnt / 2G) G
// pairs, and every point's (step, lane, half) slot lies inside them.
#include <cstdio>
#include <vector>

#include "runtime.h"

using namespace mcl;

static int check_order(int rings, int az) {
  const int N = rings * az;
  if (patch_rings(N, rings) != rings) return printf("rule rejects %d x %d\n", rings, az), 1;
  const ScanLayout L{2048, 32, rings, az};
  std::vector<int> want;
  for (int band = 0; band < rings / 4; ++band)
    for (int col = 0; col < az / 8; ++col)
      for (int ring = 0; ring < 4; ++ring)
        for (int a = 0; a < 8; ++a) want.push_back((band * 4 + ring) * az + col * 8 + a);
  std::vector<int> hit(N, 0);
  for (int j = 0; j < N; ++j) {
    const int s = L.source(j);
    if (s != want[j]) return printf("%d x %d: place %d holds %d, want %d\n", rings, az, j, s, want[j]), 1;
    if (s < 0 || s >= N || hit[s]++) return printf("%d x %d: not a permutation at %d\n", rings, az, j), 1;
  }
  const ScanLayout G{2048, 32, 0, 0};
  for (int j = 0; j < N; ++j)
    if (G.source(j) != j) return printf("order as given changed at %d\n", j), 1;
  return 0;
}

static int check_pairs(int chunk, int g) {
  const ScanLayout L{chunk, g, 0, 0};
  for (int cnt = 1; cnt <= chunk; ++cnt) {
    const int np = L.pairs(cnt);
    if (np % g || 2 * np < cnt || 2 * np >= cnt + 2 * g)  // whole steps of G pairs, none spare
      return printf("pairs(%d) = %d for G = %d\n", cnt, np, g), 1;
    std::vector<int> used(2 * np, 0);
    for (int i = 0; i < cnt; ++i) {
      const int slot = (i / (2 * g)) * g + i % g, half = (i / g) & 1;
      if (slot >= np || used[2 * slot + half]++) return printf("chunk %d G %d: point %d slot\n", cnt, g, i), 1;
    }
    if (L.chunk_bytes(cnt) != (uint32_t)np * 24u) return printf("chunk_bytes(%d)\n", cnt), 1;
  }
  if (L.chunk_offset(3) != (size_t)3 * L.full_pairs() * 24) return printf("chunk_offset\n"), 1;
  const int N = 5 * chunk + 7;
  if (L.total_bytes(N) != (size_t)6 * L.full_pairs() * 24) return printf("total_bytes\n"), 1;
  return 0;
}

int main() {
  const int fits[][2] = {{4, 8}, {4, 16}, {8, 8}, {16, 64}, {16, 1800}, {64, 1024}, {12, 24}, {128, 2048}};
  for (const auto& f : fits)
    if (check_order(f[0], f[1])) return 1;
  // ring counts that do not fit: not dividing N, not a multiple of 4, N / R
  // not a multiple of 8, zero or negative
  const long long bad[][2] = {{1024, 3}, {1024, 6}, {900, 16}, {1024, 2}, {96, 16}, {1024, 0}, {1024, -16},
                              {1000, 1000}, {65536, 65536}};
  for (const auto& b : bad)
    if (patch_rings(b[0], (int)b[1]) != 0) return printf("rule accepts N %lld R %lld\n", b[0], b[1]), 1;
  if (patch_rings(65536, 64) != 64 || patch_rings(512, 16) != 16) return printf("rule rejects a fit\n"), 1;
  for (int g : {8, 16, 32})
    for (int chunk : {32, 256, 2048})
      if (check_pairs(chunk, g)) return 1;
  printf("ok\n");
  return 0;
}
