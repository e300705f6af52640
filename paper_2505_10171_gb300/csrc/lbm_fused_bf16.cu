// Fused fluid kernel instantiated for __nv_bfloat16 storage.
#include "lbm_fused.cuh"

namespace lbmg {
template void launch_fused_form<__nv_bfloat16>(const Lattice &, int, const FluidLaunch &, cudaStream_t);
}  // namespace lbmg
