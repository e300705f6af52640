// Fused fluid kernel instantiated for double storage.
#include "lbm_fused.cuh"

namespace lbmg {
template void launch_fused_form<double>(const Lattice &, int, const FluidLaunch &, cudaStream_t);
}  // namespace lbmg
