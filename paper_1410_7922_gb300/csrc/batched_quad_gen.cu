// batched_quad_gen.cu -- one build of the batched kernel (batched.cuh).
#include "batched.cuh"

namespace edp {

void *batched_kernel_quad_gen() { return reinterpret_cast<void *>(edp_batched_kernel<33, true, true>); }

}  // namespace edp
