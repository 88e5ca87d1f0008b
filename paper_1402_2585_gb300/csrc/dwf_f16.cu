// Instantiation of the fine-operator hop passes for f16 storage.
#include "dwf_kernels.cuh"

namespace hdcg {
void launch_hop_f16(int v, int pass, bool mob, const HopArgs& a, dim3 grid, cudaStream_t st) {
  launch_hop_variant<f16_t>(v, pass, mob, a, grid, st);
}
}  // namespace hdcg
