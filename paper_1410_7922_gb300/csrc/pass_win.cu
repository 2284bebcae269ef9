// pass_win.cu -- the cost of per-pixel label boxes for the windowed form of
// EDP (used after a proposal): Eq. Cost_value restricted to each pixel's
// n^R box.  The windowed scan pass is the WIN form of the band body in
// pass_team.cuh.
#include "common.cuh"
#include "kernels.h"

namespace edp {

// Cost of every label in each pixel's box (Eq. Cost_value restricted to the
// box), one thread per (pixel, box label).
__global__ void cost_window_kernel(CostArgs A, const int *centre, int n) {
    const int Qw = (A.R == 2) ? n * n : n;
    const long long total = (long long)A.W * A.H * Qw;
    const int h = (n - 1) / 2;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long pix = e / Qw;
        const int i = (int)(e - pix * Qw);
        const int x = (int)(pix % A.W), y = (int)(pix / A.W);
        int c0 = min(max(centre[pix * A.R], h), A.Q0 - 1 - h);
        const int q0 = c0 - h + i % n;
        int q1 = 0;
        if (A.R == 2) {
            const int c1 = min(max(centre[pix * 2 + 1], h), A.Q1 - 1 - h);
            q1 = c1 - h + i / n;
        }
        const int o0 = A.vmin[0] + A.step[0] * q0;
        const int o1 = A.R == 2 ? A.vmin[1] + A.step[1] * q1 : 0;
        const int xs0 = x + o0, ys0 = y + o1;
        int c;
        auto term = [&](const uint8_t *I, int xs, int ys, bool &oob) {
            oob = xs < 0 || xs >= A.W || ys < 0 || ys >= A.H;
            if (oob) return 0;
            const int d = (int)I[(size_t)ys * A.pitch + xs] - (int)A.I0[(size_t)y * A.pitch + x];
            const int a = d < 0 ? -d : d;
            return A.l2 == 1 ? a : a * a;
        };
        bool oob1, oob2;
        if (A.mode == 2) {
            int c1 = term(A.I1, xs0, ys0, oob1);
            int c2 = term(A.I2, x - o0, y - o1, oob2);
            c1 = oob1 ? A.cmax : min(c1, A.cmax);
            c2 = oob2 ? A.cmax : min(c2, A.cmax);
            c = min(c1, c2);
        } else {
            c = term(A.I1, xs0, ys0, oob1);
            c = oob1 ? A.cmax : min(c, A.cmax);
        }
        A.C[e] = c;
    }
}

int launch_cost_window(const CostArgs &a, const int *centre, int n, cudaStream_t st) {
    const int Qw = (a.R == 2) ? n * n : n;
    const long long total = (long long)a.W * a.H * Qw;
    long long blocks = (total + 255) / 256;
    if (blocks > 152LL * 32) blocks = 152LL * 32;
    if (blocks < 1) blocks = 1;
    cost_window_kernel<<<(unsigned)blocks, 256, 0, st>>>(a, centre, n);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace edp
