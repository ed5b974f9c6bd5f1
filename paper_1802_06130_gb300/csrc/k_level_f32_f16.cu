// Instantiations of the fused level kernel for storage type float, bank type __half.
#include "k_level.cuh"
namespace mdn {
int launch_level_f32_f16(const LevelArgs& a, cudaStream_t s) { return lvl::dispatch<float, __half>(a, s); }
}  // namespace mdn
