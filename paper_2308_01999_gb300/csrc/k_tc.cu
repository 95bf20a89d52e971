// k_tc.cu -- fused 6-qubit gate application on the tensor cores (placeholder
// until the tcgen05 kernel lands: reports the path as unsupported).
#include "sv_internal.h"

namespace svk {

bool tc6_supported(int, const int *) { return false; }

cudaError_t launch_tc6(const LaunchCtx &, void *, int, const int *, const double *, sv_precision_t, void *, int *) {
    return cudaErrorNotSupported;
}

}  // namespace svk
