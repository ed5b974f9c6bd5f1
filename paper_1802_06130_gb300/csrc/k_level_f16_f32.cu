// Instantiations of the fused level kernel for storage type __half, bank type float.
#include "k_level.cuh"
namespace mdn {
int launch_level_f16_f32(const LevelArgs& a, cudaStream_t s) { return lvl::dispatch<__half, float>(a, s); }
}  // namespace mdn
