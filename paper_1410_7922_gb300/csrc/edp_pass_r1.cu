// edp_pass_r1.cu -- the single-problem warp-per-row scan-pass kernel; the
// band body is in pass_r1.cuh.
#include "pass_r1.cuh"

namespace edp {

template <bool QUAD>
__global__ void __launch_bounds__(QUAD ? 256 : kMaxThreads, 1) edp_pass_r1_kernel(PassR1Args A) {
    extern __shared__ __align__(16) int smem_i[];
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
        const bool ok =
            r1_dispatch(A.E, [&](auto e) { return r1_band<decltype(e)::value, QUAD>(A, band, smem_i, &s_abort); });
        if (!ok) return;
    }
}

size_t pass_r1_smem(int NWR, int E) {
    const size_t Qp = 32 * (size_t)E;
    return ((size_t)NWR * (kPf + 1) * 3 * Qp + (size_t)NWR * kMb * Qp + 2 * (size_t)NWR) * 4;
}

int launch_edp_pass_r1(const PassR1Args &a, int threads, size_t smem, cudaStream_t st) {
    auto k = a.l1 == 2 ? edp_pass_r1_kernel<true> : edp_pass_r1_kernel<false>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<a.grid, threads, smem, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace edp
