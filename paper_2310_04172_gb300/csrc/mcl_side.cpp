// Host side of the batched side launches (SideSeg / SegBlocks, mcl_internal.h):
// per launch kind the blocks each session needs, their prefix arrays, and the
// launch itself. Used by the batched sensor update and the serving loop, so
// that a step over many sessions costs the same number of launches as a step
// over one.
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
