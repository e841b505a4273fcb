// Instantiations of the path kernel for the single path on an FP64 design
// (held as two FP32 planes).
#include "path_kernel.cuh"

namespace lassogs {

const void* path_kernel_single_f64(int ngc, int cw) {
  if (cw == 1) return kernel_ptr<1, 1, true, false>();
  return ngc == 1 ? kernel_ptr<1, 4, true, false>()
         : ngc == 2 ? kernel_ptr<2, 4, true, false>() : kernel_ptr<4, 4, true, false>();
}

}  // namespace lassogs
