// K-GROUPED -- placeholder until the persistent grouped kernel lands.
#include "internal.h"
namespace cosma {
int grouped_gemm(int, const cosma_problem*, int, const DeviceInfo&, void*, long long, int*,
                 long long, cudaStream_t, long long* needed) {
  if (needed) *needed = 0;
  return COSMA_ERR_UNSUPPORTED;
}
}  // namespace cosma
