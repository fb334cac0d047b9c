// Learned cost model kernels: placeholder entry points until the MLP kernels
// land; every call reports HSUMMA_ERR_UNSUPPORTED.
#include "internal.h"
#include "../../include/hsumma.h"

using namespace hs;

extern "C" {
int hsumma_mlp_forward(int, const float *, const float *, float *, float *, void *) {
  set_error("MLP kernels are not built yet");
  return HSUMMA_ERR_UNSUPPORTED;
}
int hsumma_mlp_backward(int, const float *, const float *, const float *, float *, float *,
                        void *) {
  set_error("MLP kernels are not built yet");
  return HSUMMA_ERR_UNSUPPORTED;
}
int hsumma_mlp_adam(int, float *, const float *, float *, float *, int, float, float, float,
                    float, void *) {
  set_error("MLP kernels are not built yet");
  return HSUMMA_ERR_UNSUPPORTED;
}
int hsumma_mlp_pick(int, const float *, const float *, float *, int32_t *, void *) {
  set_error("MLP kernels are not built yet");
  return HSUMMA_ERR_UNSUPPORTED;
}
int hsumma_mlp_load(const float *, const float *, const float *) {
  set_error("MLP kernels are not built yet");
  return HSUMMA_ERR_UNSUPPORTED;
}
}
