// Sensor kernel instances for f32 brick maps with the hash index (linear bricks) (one unit per storage type
// and map kind, so they compile in parallel).
#include "k_sensor_impl.cuh"

namespace mcl {

void* sensor_kernel_f32_hash(int mode, const SensorShape& sh, bool batch) {
  return sensor::pick_kind<MCL_MAP_BRICK, MCL_F32>(mode, sh, batch);
}

}  // namespace mcl
