// Kernels for the StoreF16 population storage.
#include "lb_inst.cuh"

namespace lbgb {
const StorageOps &ops_f16() {
  static const StorageOps o = Instance<StoreF16>::make();
  return o;
}
}  // namespace lbgb
