// batched_quad.cu -- one build of the batched kernel (batched.cuh).
#include "batched.cuh"

namespace edp {

void *batched_kernel_quad() { return reinterpret_cast<void *>(edp_batched_kernel<33, false, true>); }

}  // namespace edp
