// Split-precision complex products on the tcgen05 tensor cores.
#include "kernels.h"

namespace tz {
namespace dev {

bool cgemm_tc_supported(int, int64_t, int64_t, int64_t) { return false; }
size_t cgemm_tc_scratch_bytes(int, int64_t, int64_t, int64_t) { return 0; }
cudaError_t launch_cgemm_tc(int, const float2 *, const float2 *, float2 *, int64_t, int64_t, int64_t, int64_t,
                            int64_t, int64_t, int64_t, void *, size_t, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace dev
}  // namespace tz
