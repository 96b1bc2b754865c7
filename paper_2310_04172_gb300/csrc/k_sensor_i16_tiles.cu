// Sensor kernel instances for i16 dense maps stored in 8 x 4 tiles (one
// unit per storage type and map kind, so they compile in parallel).
#include "k_sensor_impl.cuh"

namespace mcl {

void* sensor_kernel_i16_tiles(int mode, const SensorShape& sh, bool batch) {
  return sensor::pick_kind<kKindDenseTiles, MCL_I16>(mode, sh, batch);
}

}  // namespace mcl
