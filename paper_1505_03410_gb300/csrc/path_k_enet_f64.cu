// Instantiations of the path kernel for the Elastic-Net on an FP64 design
// (held as two FP32 planes; single path, the augmented rows implicit).
#include "path_kernel.cuh"

namespace lassogs {

const void* path_kernel_enet_f64(int ngc, int cw) {
  if (cw == 1) return kernel_ptr<1, 1, true, false, 1, true>();
  return ngc == 1 ? kernel_ptr<1, 4, true, false, 1, true>()
         : ngc == 2 ? kernel_ptr<2, 4, true, false, 1, true>() : kernel_ptr<4, 4, true, false, 1, true>();
}

}  // namespace lassogs
