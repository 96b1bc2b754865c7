// Sensor kernel instances for i16 dense maps (one unit per storage type
// and map kind, so they compile in parallel).
#include "k_sensor_impl.cuh"

namespace mcl {

void* sensor_kernel_i16_dense(int mode, const SensorShape& sh, bool batch) {
  return sensor::pick_kind<MCL_MAP_DENSE, MCL_I16>(mode, sh, batch);
}

}  // namespace mcl
