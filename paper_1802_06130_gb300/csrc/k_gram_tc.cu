// k_gram_tc.cu -- tensor-core (tcgen05) Gram accumulation.  Placeholder
// until the tcgen05 kernel lands: reports the precision as unsupported.
#include "train_common.cuh"

namespace mdn {
int launch_gram_tc(const GatherArgs&, int, const int4*, int, const int*, float*, cudaStream_t) {
    return fail(MDN_EINVAL, "train: tensor-core Gram precisions are not available in this build");
}
}  // namespace mdn
