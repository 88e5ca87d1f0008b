// Instantiation of the fine-operator hop passes for bf16 storage.
#include "dwf_kernels.cuh"

namespace hdcg {
void launch_hop_bf16(int v, int pass, bool mob, const HopArgs& a, dim3 grid, cudaStream_t st) {
  launch_hop_variant<bf16_t>(v, pass, mob, a, grid, st);
}
}  // namespace hdcg
