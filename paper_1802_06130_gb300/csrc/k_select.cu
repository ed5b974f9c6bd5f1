// Selector-only instantiations of the fused level kernel (bucket map output).
#include "k_level.cuh"
namespace mdn {
int launch_select_f32(const LevelArgs& a, cudaStream_t s) { return lvl::run<3, -1, false, float, float, false, false>(a, s); }
int launch_select_f16(const LevelArgs& a, cudaStream_t s) { return lvl::run<3, -1, false, __half, float, false, false>(a, s); }
}  // namespace mdn
