// Learned plan selector -- placeholder until the MLP cost model lands.
#include "internal.h"
namespace cosma {
int learned_plan(int64_t, int64_t, int64_t, int, const DeviceInfo&, const cosma_config&,
                 cosma_plan*) {
  return COSMA_ERR_UNSUPPORTED;
}
}  // namespace cosma
