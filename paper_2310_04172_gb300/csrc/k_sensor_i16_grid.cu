// Sensor kernel instances for i16 brick maps with the grid index (one unit per storage type
// and map kind, so they compile in parallel).
#include "k_sensor_impl.cuh"

namespace mcl {

void* sensor_kernel_i16_grid(int mode, const SensorShape& sh, bool batch) {
  return sensor::pick_kind<kKindBrickGrid, MCL_I16>(mode, sh, batch);
}

}  // namespace mcl
