// Kernels for the StoreF32 population storage.
#include "lb_inst.cuh"

namespace lbgb {
const StorageOps &ops_f32() {
  static const StorageOps o = Instance<StoreF32>::make();
  return o;
}
}  // namespace lbgb
