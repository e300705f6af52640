// Fused fluid kernel instantiated for __half storage.
#include "lbm_fused.cuh"

namespace lbmg {
template void launch_fused_form<__half>(const Lattice &, int, const FluidLaunch &, cudaStream_t);
}  // namespace lbmg
