// edp_pass_r1.cu -- the single-problem warp-per-row scan-pass kernel; the
// band body is in pass_r1.cuh.
#include "pass_r1.cuh"

namespace edp {

// rows (warps) per block the build allows: 16 where the registers fit 512
// threads (E <= 4, linear prior), else 8
template <int E, bool QUAD>
constexpr int r1_max_rows() { return (E <= 4 && !QUAD) ? 16 : 8; }

template <int E, bool QUAD, bool WT>
__global__ void __launch_bounds__(32 * r1_max_rows<E, QUAD>(), 1) edp_pass_r1_kernel(PassR1Args A) {
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
        if (!r1_band<E, QUAD, WT>(A, band, smem_i, &s_abort)) return;
    }
}

// one build per labels-per-lane count (each allocates its own registers)
using R1Kernel = void (*)(PassR1Args);
template <bool QUAD, bool WT>
R1Kernel r1_kernel_for(int E) {
    switch (E) {
    case 1: return edp_pass_r1_kernel<1, QUAD, WT>;
    case 2: return edp_pass_r1_kernel<2, QUAD, WT>;
    case 3: return edp_pass_r1_kernel<3, QUAD, WT>;
    case 4: return edp_pass_r1_kernel<4, QUAD, WT>;
    case 5: return edp_pass_r1_kernel<5, QUAD, WT>;
    case 6: return edp_pass_r1_kernel<6, QUAD, WT>;
    case 7: return edp_pass_r1_kernel<7, QUAD, WT>;
    default: return edp_pass_r1_kernel<8, QUAD, WT>;
    }
}
R1Kernel r1_kernel_of(int E, int l1, bool wt) {
    if (wt) return l1 == 2 ? r1_kernel_for<true, true>(E) : r1_kernel_for<false, true>(E);
    return l1 == 2 ? r1_kernel_for<true, false>(E) : r1_kernel_for<false, false>(E);
}

int pass_r1_max_rows(int E, int l1) { return (E <= 4 && l1 != 2) ? 16 : 8; }

size_t pass_r1_smem(int NWR, int E) {
    const size_t Qp = 32 * (size_t)E;
    // staging rings, mailbox records, consumed counters
    return ((size_t)NWR * (kPf + 1) * 3 * Qp + 2 * (size_t)NWR * kMb * Qp + (size_t)NWR) * 4;
}

int edp_pass_r1_occupancy(int E, int l1, int threads, size_t smem) {
    const R1Kernel k = r1_kernel_of(E, l1, false);
    if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, threads, smem) != cudaSuccess) return 0;
    return occ;
}

int launch_edp_pass_r1(const PassR1Args &a, int threads, size_t smem, cudaStream_t st) {
    const R1Kernel k = r1_kernel_of(a.E, a.l1, a.wh != nullptr);
    if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<a.grid, threads, smem, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace edp
