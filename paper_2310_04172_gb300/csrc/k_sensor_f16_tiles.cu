// Sensor kernel instances for f16 dense maps stored in 8 x 4 tiles (one
// unit per storage type and map kind, so they compile in parallel).
#include "k_sensor_impl.cuh"

namespace mcl {

void* sensor_kernel_f16_tiles(int mode, const SensorShape& sh, bool batch) {
  return sensor::pick_kind<kKindDenseTiles, MCL_F16>(mode, sh, batch);
}

}  // namespace mcl
