// Host side of the batched side launches (SideSeg / SegBlocks, mcl_internal.h):
// per launch kind the blocks each session needs, their prefix arrays, and the
// launch itself. Used by the batched sensor update and the serving loop, so
// that a step over many sessions costs the same number of launches as a step
// over one.
#include <algorithm>
#include <cstring>

#include "runtime.h"

namespace mcl {

int side_blocks(int kind, const SideSeg& g) {
  switch (kind) {
    case kSideMotion: return side_blocks_motion(g);
    case kSideOrderZero:
    case kSideOrderKeys:
    case kSideOrderTiles:
    case kSideOrderTotals:
    case kSideOrderScatter: return side_blocks_order(kind, g);
    case kSidePosePack: return side_blocks_pose(g);
    case kSideStats:
    case kSideNormalise:
    case kSideEstimate: return side_blocks_normalise(kind, g);
    case kSideTileScan:
    case kSideTileOffsets:
    case kSideSystematic: return side_blocks_resample(kind, g);
    default: return 0;
  }
}

cudaError_t launch_side(int kind, const SideSeg* segs, const SegBlocks& b, cudaStream_t s) {
  switch (kind) {
    case kSideMotion: return launch_side_motion(segs, b, s);
    case kSideOrderZero:
    case kSideOrderKeys:
    case kSideOrderTiles:
    case kSideOrderTotals:
    case kSideOrderScatter: return launch_side_order(kind, segs, b, s);
    case kSidePosePack: return launch_side_pose(segs, b, s);
    case kSideStats:
    case kSideNormalise:
    case kSideEstimate: return launch_side_normalise(kind, segs, b, s);
    case kSideTileScan:
    case kSideTileOffsets:
    case kSideSystematic: return launch_side_resample(kind, segs, b, s);
    default: return cudaErrorInvalidValue;
  }
}

long long item_segments(const std::vector<SegSession>& s, long long slots, bool interleave, int max_rounds,
                        std::vector<int>* sweeps, std::vector<ItemSeg>* segs) {
  const int n = (int)s.size();
  segs->clear();
  sweeps->assign(n, 0);
  long long pos = 0;
  if (!interleave) {
    for (int i = 0; i < n; ++i) {
      (*sweeps)[i] = s[i].sweep;
      segs->push_back(ItemSeg{pos, 0, i, 0});
      pos += (long long)s[i].nblk * s[i].K;
    }
  } else {
    std::vector<char> done(n, 0);
    for (int i = 0; i < n; ++i) {
      if (done[i]) continue;
      std::vector<int> on;  // the sessions on this map, in order
      long long items = 0;
      for (int j = i; j < n; ++j)
        if (!done[j] && s[j].values == s[i].values) {
          on.push_back(j);
          done[j] = 1;
          items += (long long)s[j].nblk * s[j].K;
        }
      if (on.size() == 1) {  // alone on its map: its own sweeps, one segment
        (*sweeps)[i] = s[i].sweep;
        segs->push_back(ItemSeg{pos, 0, i, 0});
        pos += (long long)s[i].nblk * s[i].K;
        continue;
      }
      const long long R = std::max<long long>(1, std::min<long long>(max_rounds, (items + slots - 1) / std::max<long long>(1, slots)));
      long long rounds = 0;
      for (int j : on) {
        const int sw = (int)std::max<long long>(1, (s[j].nblk + R - 1) / R);
        (*sweeps)[j] = sw;
        rounds = std::max<long long>(rounds, (s[j].nblk + sw - 1) / sw);
      }
      for (long long r = 0; r < rounds; ++r)
        for (int j : on) {
          const long long b0 = r * (*sweeps)[j];
          if (b0 >= s[j].nblk) continue;
          segs->push_back(ItemSeg{pos, b0 * s[j].K, j, 0});
          pos += std::min<long long>((*sweeps)[j], s[j].nblk - b0) * s[j].K;
        }
    }
  }
  segs->push_back(ItemSeg{pos, 0, -1, 0});
  return pos;
}

size_t side_table_bytes(int n) {
  return align256((size_t)n * sizeof(SideSeg)) + align256((size_t)kSideLaunches * (n + 1) * sizeof(int));
}

void side_tables(const std::vector<SideSeg>& segs, char* h, char* d, SideTables* out) {
  const int n = (int)segs.size();
  std::memcpy(h, segs.data(), (size_t)n * sizeof(SideSeg));
  out->segs = reinterpret_cast<const SideSeg*>(d);
  const size_t off_first = align256((size_t)n * sizeof(SideSeg));
  int* hf = reinterpret_cast<int*>(h + off_first);
  const int* df = reinterpret_cast<const int*>(d + off_first);
  for (int k = 0; k < kSideLaunches; ++k) {
    int* f = hf + (size_t)k * (n + 1);
    f[0] = 0;
    for (int i = 0; i < n; ++i) f[i + 1] = f[i] + side_blocks(k, segs[i]);
    out->b[k] = SegBlocks{df + (size_t)k * (n + 1), n, f[n]};
  }
}

mcl_status enqueue_side(const SideTables& t, int kind, cudaStream_t s) {
  MCL_CUDA(launch_side(kind, t.segs, t.b[kind], s));
  return MCL_OK;
}

int side_launch_count(const SideTables& t) {
  int k = 0;
  for (int i = 0; i < kSideLaunches; ++i) k += t.b[i].blocks > 0 ? 1 : 0;
  return k;
}

}  // namespace mcl
