// Host side of the learned cost model (device kernels in mlp.cu).
#include "runtime.h"

namespace compar {

int mlp_predict(compar_ctx* ctx, const float* feats, int rows, float* out_host) {
  (void)ctx;
  (void)feats;
  (void)rows;
  (void)out_host;
  return COMPAR_ERR_UNSUPPORTED;
}

void mlp_release(compar_ctx* ctx) { (void)ctx; }

}  // namespace compar
