// Sensor kernel instances for f16 maps (compiled as their own unit so the
// storage types build in parallel).
#include "k_sensor_impl.cuh"

namespace mcl {

void* sensor_kernel_f16(int kind, int layout, int mode, const SensorShape& sh, bool batch) {
  return sensor::pick_dtype<MCL_F16>(kind, layout, mode, sh, batch);
}

}  // namespace mcl
