// K-BF16 (tcgen05) -- placeholder until the tensor-core kernel lands.
#include "internal.h"
namespace cosma {
int launch_tc_bf16(const GemmArgs&, const Sched&, const cosma_plan&, void*, long long, int*,
                   long long, cudaStream_t) {
  return COSMA_ERR_UNSUPPORTED;
}
}  // namespace cosma
