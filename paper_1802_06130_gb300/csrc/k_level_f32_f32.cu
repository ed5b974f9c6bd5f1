// Instantiations of the fused level kernel for storage type float, bank type float.
#include "k_level.cuh"
namespace mdn {
int launch_level_f32_f32(const LevelArgs& a, cudaStream_t s) { return lvl::dispatch<float, float>(a, s); }
}  // namespace mdn
