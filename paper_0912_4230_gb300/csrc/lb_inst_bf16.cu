// Kernels for the StoreBF16 population storage.
#include "lb_inst.cuh"

namespace lbgb {
const StorageOps &ops_bf16() {
  static const StorageOps o = Instance<StoreBF16>::make();
  return o;
}
}  // namespace lbgb
