// edp_pass.cu -- the single-problem scan-pass kernel (any number of label
// axes); the band body is in pass_gen.cuh.
#include "pass_gen.cuh"

namespace edp {

template <int EM>
__global__ void __launch_bounds__(kMaxThreads) edp_pass_kernel(PassArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_band;
    __shared__ volatile int s_abort;
    if (threadIdx.x == 0) s_abort = (*(volatile int *)A.status != 0);
    __syncthreads();
    if (s_abort) return;
    while (true) {
        if (threadIdx.x == 0) s_band = atomicAdd(A.band_counter, 1);
        __syncthreads();
        const int band = s_band;
        if (band >= A.nbands) break;
        if (!gen_band<EM>(A, band, smem_raw, &s_abort)) return;
    }
}

int edp_pass_occupancy(int em, int threads, size_t smem) {
    int occ = 0;
    switch (em) {
#define EDP_OCC(N)                                                                            \
    case N:                                                                                   \
        if (smem > 48 * 1024)                                                                 \
            cudaFuncSetAttribute(edp_pass_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 (int)smem);                                                  \
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, edp_pass_kernel<N>, threads, smem); \
        break;
        EDP_OCC(2)
        EDP_OCC(4)
        EDP_OCC(8)
        EDP_OCC(16)
#undef EDP_OCC
    default:
        break;
    }
    return occ;
}

int launch_edp_pass(const PassArgs &a, int em, int threads, size_t smem, cudaStream_t st) {
    switch (em) {
#define EDP_CASE(N)                                                                          \
    case N: {                                                                                \
        auto k = edp_pass_kernel<N>;                                                         \
        if (smem > 48 * 1024)                                                                \
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        k<<<a.grid, threads, smem, st>>>(a);                                                 \
        break;                                                                               \
    }
        EDP_CASE(2)
        EDP_CASE(4)
        EDP_CASE(8)
        EDP_CASE(16)
#undef EDP_CASE
    default:
        return -1;
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace edp
