// Instantiation of the fine-operator hop passes for double-float storage.
#include "dwf_kernels.cuh"

namespace hdcg {
void launch_hop_df(int v, int pass, bool mob, const HopArgs& a, dim3 grid, cudaStream_t st) {
  launch_hop_variant<df_t>(v, pass, mob, a, grid, st);
}
}  // namespace hdcg
