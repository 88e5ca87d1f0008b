// Instantiation of the fine-operator hop passes for bf16t storage.
#include "dwf_kernels.cuh"

namespace hdcg {
void launch_hop_bf16t(int v, int pass, bool mob, const HopArgs& a, dim3 grid, cudaStream_t st) {
  launch_hop_variant<bf16t_t>(v, pass, mob, a, grid, st);
}
}  // namespace hdcg
