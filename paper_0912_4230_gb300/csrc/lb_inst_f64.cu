// Kernels for the StoreF64 population storage.
#include "lb_inst.cuh"

namespace lbgb {
const StorageOps &ops_f64() {
  static const StorageOps o = Instance<StoreF64>::make();
  return o;
}
}  // namespace lbgb
