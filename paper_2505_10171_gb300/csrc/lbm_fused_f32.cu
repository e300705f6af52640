// Fused fluid kernel instantiated for float storage.
#include "lbm_fused.cuh"

namespace lbmg {
template void launch_fused_form<float>(const Lattice &, int, const FluidLaunch &, cudaStream_t);
}  // namespace lbmg
