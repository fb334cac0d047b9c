// Split-precision HSUMMA, step 3 with int8 slices: placeholder until the
// warp-level int8 MMA kernel lands (tcgen05 has no int8 kind on sm_103a).
#include "internal.h"
#include "../../include/hsumma.h"

namespace hs {

int int8_cluster_limit(int *limit) {
  *limit = 16;
  return HSUMMA_OK;
}

int launch_split_int8(const GridPlan &, int, const void *, const void *, int32_t *,
                      cudaStream_t) {
  set_error("INT8 slices are not built yet");
  return HSUMMA_ERR_UNSUPPORTED;
}

}  // namespace hs
