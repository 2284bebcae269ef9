// batched.cu -- many independent EDP problems (uneven sizes and label
// spaces) solved by one persistent launch.
//
// Work items are (scan pass, problem, row band), ordered pass-major.  Blocks
// take items in that order from one global counter.  Every dependency of an
// item is an earlier item:
//   - the previous band of the same pass and problem (the band bodies wait
//     for it row by row);
//   - the previous pass of the same problem (a per-problem counter of
//     finished bands, waited for with a bounded spin).
// A block therefore only ever waits for an item that an already running
// block owns.  Problems of different sizes fill the GPU together; the
// heterogeneity lives in the per-problem descriptors, passed by value as the
// kernel's parameter block (no host tables, so the launch can be captured in
// a CUDA graph).
#include "kernels.h"

namespace edp {

// the builds of the batched kernel (batched_*.cu)
void *batched_kernel_lean();      // lean multi-axis and one-axis bodies
void *batched_kernel_gen();       // + the lane-group multi-axis body
void *batched_kernel_quad();      // quadratic-prior bodies
void *batched_kernel_quad_gen();  // quadratic-prior and lane-group bodies

static void *batched_kernel_for(int lm, int gen) {
    // lm: 2 = the wave holds quadratic-prior problems (the lean body
    // dispatches on the line lengths itself otherwise)
    if (lm == 2) return gen ? batched_kernel_quad_gen() : batched_kernel_quad();
    return gen ? batched_kernel_gen() : batched_kernel_lean();
}
int edp_batched_occupancy(int lm, int gen, int threads, size_t smem) {
    void *k = batched_kernel_for(lm, gen);
    if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, threads, smem);
    return occ;
}

int launch_edp_batched(const BatchArgs &a, int lm, int gen, int threads, size_t smem, int grid, cudaStream_t st) {
    void *k = batched_kernel_for(lm, gen);
    if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    void *args[] = {const_cast<BatchArgs *>(&a)};
    return cudaLaunchKernel(k, dim3(grid), dim3(threads), args, smem, st) == cudaSuccess ? 0 : -2;
}

}  // namespace edp
