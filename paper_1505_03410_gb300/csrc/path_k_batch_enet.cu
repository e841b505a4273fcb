// Instantiations of the path kernel for the batched Elastic-Net (one CTA or a
// group of CTAs per problem; 1 or 2 resident CTAs per SM).
#include "path_kernel.cuh"

namespace lassogs {

const void* path_kernel_batch_enet(int ngc, int per_sm) {
  if (per_sm == 2)
    return ngc == 1 ? kernel_ptr<1, 4, false, true, 2, true>()
           : ngc == 2 ? kernel_ptr<2, 4, false, true, 2, true>() : kernel_ptr<4, 4, false, true, 2, true>();
  return ngc == 1 ? kernel_ptr<1, 4, false, true, 1, true>()
         : ngc == 2 ? kernel_ptr<2, 4, false, true, 1, true>() : kernel_ptr<4, 4, false, true, 1, true>();
}

}  // namespace lassogs
