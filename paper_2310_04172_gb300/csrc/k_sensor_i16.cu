// Sensor kernel instances for i16 maps (compiled as their own unit so the
// storage types build in parallel).
#include "k_sensor_impl.cuh"

namespace mcl {

void* sensor_kernel_i16(int kind, int layout, int mode, const SensorShape& sh, bool batch) {
  return sensor::pick_dtype<MCL_I16>(kind, layout, mode, sh, batch);
}

}  // namespace mcl
