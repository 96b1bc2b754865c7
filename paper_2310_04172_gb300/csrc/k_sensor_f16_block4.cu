// Sensor kernel instances for f16 brick maps with the hash index (4x4x4-block bricks) (one unit per storage type
// and map kind, so they compile in parallel).
#include "k_sensor_impl.cuh"

namespace mcl {

void* sensor_kernel_f16_block4(int mode, const SensorShape& sh, bool batch) {
  return sensor::pick_kind<kKindBrickBlock4, MCL_F16>(mode, sh, batch);
}

}  // namespace mcl
