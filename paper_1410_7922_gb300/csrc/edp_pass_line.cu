// edp_pass_line.cu -- the two-axis scan-pass kernels: one label line per
// lane (band body in pass_line.cuh) and each line split over two lanes
// (pass_line2.cuh).  One build per label-space shape (Q0 x Q1): the lines
// are held in registers with exact lengths.
#include <algorithm>

#include "pass_line2.cuh"

namespace edp {

template <int LA, int LB, bool QUAD = false>
__global__ void __launch_bounds__(line::kMaxThreads, 1) edp_pass_line_kernel(TeamArgs A) {
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
        if (!line_band<LA, LB, QUAD>(A, band, smem_i, &s_abort)) return;
    }
}

// lines split over lane pairs; CH: global loads per batch and lane; FUSED:
// the pair cost computed from the images instead of read from C
template <int LA, int LB, int CH, bool FUSED>
__global__ void __launch_bounds__(line2::kMaxThreads, 1) edp_pass_line2_kernel(TeamArgs A) {
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
        if (!line2_band<LA, LB, CH, FUSED>(A, band, smem_i, &s_abort)) return;
    }
}

static void *line2_kernel_for(int Q0, int Q1, int l1, bool fused = false) {
    if (l1 == 1 && Q0 == 65 && Q1 == 65)
        return fused ? reinterpret_cast<void *>(edp_pass_line2_kernel<65, 65, 5, true>)
                     : reinterpret_cast<void *>(edp_pass_line2_kernel<65, 65, 5, false>);
    return nullptr;
}

// the shapes with a build: (Q0, Q1) = (LB, LA); the truncated quadratic
// prior for the two shapes no other kernel serves with it
static void *line1_kernel_for(int Q0, int Q1, int l1) {
    if (l1 == 2) {
        if (Q0 == 27 && Q1 == 15) return reinterpret_cast<void *>(edp_pass_line_kernel<15, 27, true>);
        if (Q0 == 25 && Q1 == 25) return reinterpret_cast<void *>(edp_pass_line_kernel<25, 25, true>);
        return nullptr;
    }
    if (l1 != 1) return nullptr;
    if (Q0 == 65 && Q1 == 65) return reinterpret_cast<void *>(edp_pass_line_kernel<65, 65>);
    if (Q0 == 33 && Q1 == 33) return reinterpret_cast<void *>(edp_pass_line_kernel<33, 33>);
    if (Q0 == 25 && Q1 == 25) return reinterpret_cast<void *>(edp_pass_line_kernel<25, 25>);
    if (Q0 == 17 && Q1 == 17) return reinterpret_cast<void *>(edp_pass_line_kernel<17, 17>);
    if (Q0 == 27 && Q1 == 15) return reinterpret_cast<void *>(edp_pass_line_kernel<15, 27>);
    return nullptr;
}

static void *line_kernel_for(int Q0, int Q1, int l1, bool split) {
    return split ? line2_kernel_for(Q0, Q1, l1) : line1_kernel_for(Q0, Q1, l1);
}

bool pass_line_built(int Q0, int Q1, int l1) { return line1_kernel_for(Q0, Q1, l1) != nullptr; }

bool pass_line_split_built(int Q0, int Q1, int l1) { return line2_kernel_for(Q0, Q1, l1) != nullptr; }

int pass_line_split_max_lambda() { return line2::kMaxLambda; }

int pass_line_warps(int Q0, int Q1, bool split) {
    return split ? (std::max(Q0, Q1) + 15) / 16 : (std::max(Q0, Q1) + 31) / 32;
}

size_t pass_line_smem(int NT, int Q0, int Q1, bool split) {
    return (size_t)NT * (split ? line2::team_ints(Q1) : line::team_ints(Q1, Q0)) * 4;
}

int edp_pass_line_occupancy(int Q0, int Q1, int l1, bool split, int threads, size_t smem) {
    void *k = line_kernel_for(Q0, Q1, l1, split);
    if (!k) return 0;
    if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, threads, smem);
    return occ;
}

int launch_edp_pass_line(const TeamArgs &a, int Q0, int Q1, bool split, int threads, size_t smem, cudaStream_t st) {
    void *k = (split && a.fI1) ? line2_kernel_for(Q0, Q1, a.l1, true) : line_kernel_for(Q0, Q1, a.l1, split);
    if (!k) return -1;
    if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    void *args[] = {const_cast<TeamArgs *>(&a)};
    if (cudaLaunchKernel(k, dim3(a.grid), dim3(threads), args, smem, st) != cudaSuccess) return -2;
    return 0;
}

}  // namespace edp
