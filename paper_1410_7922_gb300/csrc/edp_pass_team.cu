// edp_pass_team.cu -- the single-problem multi-axis scan-pass kernel; the
// band body is in pass_team.cuh.
#include "pass_team.cuh"

namespace edp {

template <int EM, bool LEAN, bool WIN, bool WT>
__global__ void __launch_bounds__(WIN || LEAN || EM > 17 ? 256 : 384, 1) edp_pass_team_kernel(TeamArgs A) {
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
        if (!team_band<EM, LEAN, WIN, WT>(A, band, smem_i, &s_abort)) return;
    }
}

size_t pass_team_smem(int NT, int Qm, int R, int nbuf, int kmb) {
    return (size_t)NT * team::team_ints(Qm, R, nbuf, kmb) * 4;
}

template <int EM, bool LEAN, bool WIN = false, bool WT = false>
static void *team_kernel() {
    return reinterpret_cast<void *>(edp_pass_team_kernel<EM, LEAN, WIN, WT>);
}
static void *team_kernel_for(int em, int lean, int win = 0, bool wt = false) {
    // the windowed body dispatches on the box side; em is its prior power
    if (win) return em == 2 ? team_kernel<2, false, true>() : team_kernel<1, false, true>();
    // the lean body dispatches on the line lengths itself: 9/17/33, or 65 only;
    // per-edge prior multipliers have builds of their own
    if (lean && wt)
        return em == 2 ? team_kernel<2, true, false, true>()
                       : (em == 65 ? team_kernel<65, true, false, true>() : team_kernel<33, true, false, true>());
    if (lean) return em == 2 ? team_kernel<2, true>() : (em == 65 ? team_kernel<65, true>() : team_kernel<33, true>());
    return em == 9 ? team_kernel<9, false>() : (em == 17 ? team_kernel<17, false>() : team_kernel<33, false>());
}

int edp_pass_team_occupancy(int em, int lean, int win, int threads, size_t smem) {
    void *k = team_kernel_for(em, lean, win);
    if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, threads, smem);
    return occ;
}

int launch_edp_pass_team(const TeamArgs &a, int threads, size_t smem, cudaStream_t st) {
    void *k = team_kernel_for(a.em, a.lean, a.win, a.wh != nullptr);
    if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    void *args[] = {const_cast<TeamArgs *>(&a)};
    if (cudaLaunchKernel(k, dim3(a.grid), dim3(threads), args, smem, st) != cudaSuccess) return -2;
    return 0;
}

}  // namespace edp
