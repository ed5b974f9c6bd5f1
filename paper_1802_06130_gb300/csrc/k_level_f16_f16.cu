// Instantiations of the fused level kernel for storage type __half, bank type __half.
#include "k_level.cuh"
namespace mdn {
int launch_level_f16_f16(const LevelArgs& a, cudaStream_t s) { return lvl::dispatch<__half, __half>(a, s); }
}  // namespace mdn
