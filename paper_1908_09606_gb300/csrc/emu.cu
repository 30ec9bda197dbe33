// K-SPLIT / K-EMU -- placeholder until the emulated FP64 path lands.
#include "internal.h"
namespace cosma {
long long emu_workspace_bytes(int64_t, int64_t, int64_t, const cosma_config&) { return 0; }
int launch_emu_bf16(const GemmArgs&, const Sched&, const cosma_plan&, const cosma_config&, void*,
                    long long, int*, long long, cudaStream_t) {
  return COSMA_ERR_UNSUPPORTED;
}
}  // namespace cosma
