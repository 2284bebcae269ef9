// batched_lean.cu -- one build of the batched kernel (batched.cuh).
#include "batched.cuh"

namespace edp {

void *batched_kernel_lean() { return reinterpret_cast<void *>(edp_batched_kernel<33, false, false>); }

}  // namespace edp
