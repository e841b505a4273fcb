// Instantiations of the path kernel for the single path on an FP32 design.
#include "path_kernel.cuh"

namespace lassogs {

const void* path_kernel_single_f32(int ngc, int cw) {
  if (cw == 1) return kernel_ptr<1, 1, false, false>();
  return ngc == 1 ? kernel_ptr<1, 4, false, false>()
         : ngc == 2 ? kernel_ptr<2, 4, false, false>() : kernel_ptr<4, 4, false, false>();
}

}  // namespace lassogs
