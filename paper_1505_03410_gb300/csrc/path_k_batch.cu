// Instantiations of the path kernel for the batched solver (one CTA or a
// group of CTAs per problem; 1 or 2 resident CTAs per SM).
#include "path_kernel.cuh"

namespace lassogs {

const void* path_kernel_batch(int ngc, int per_sm) {
  if (per_sm == 2)
    return ngc == 1 ? kernel_ptr<1, 4, false, true, 2>()
           : ngc == 2 ? kernel_ptr<2, 4, false, true, 2>() : kernel_ptr<4, 4, false, true, 2>();
  return ngc == 1 ? kernel_ptr<1, 4, false, true, 1>()
         : ngc == 2 ? kernel_ptr<2, 4, false, true, 1>() : kernel_ptr<4, 4, false, true, 1>();
}

}  // namespace lassogs
