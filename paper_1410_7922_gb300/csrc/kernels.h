// kernels.h -- argument blocks and launchers of the libedp kernels.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace edp {

constexpr int EDP_ERR_TIMEOUT_CODE = 5;  // == EDP_ERR_TIMEOUT of edp.h

// one EDP scan pass
struct PassArgs {
    const int *C;         // [H][W][Q]
    int *M[4];            // messages into each pixel from +x, -x, +y, -y
    int *labels;          // [H][W], written by the final pass
    unsigned *progress;   // [H] columns published per pass-order row
    unsigned *band_counter;
    int *status;
    int W, H, Q, R;
    AxisCfg ax[3];
    int lam;              // lambda
    int capv;             // lambda * g^l1 (clip addend)
    int mode;             // 0 joint, 1 per axis
    int pass;             // 0..3 = P1..P4
    int read_c, read_d;   // 0: the old message array is known to be zero
    int write_a, write_b; // 0: the outputs are never read again
    int final_;           // marginal + argmin in this pass
    int RB;               // rows per band
    int nbands;
    int grid;
    long long spin_limit;
    unsigned long long *trace;  // optional: per band {start ns, end ns, wait ns, sm id}
};
int launch_edp_pass(const PassArgs &a, int em, int threads, size_t smem, cudaStream_t st);
int edp_pass_occupancy(int em, int threads, size_t smem);

// one EDP scan pass, one label axis, one warp per row (edp_pass_r1.cu)
struct PassR1Args {
    const int *C;
    int *M[4];
    int *labels;
    int2 *ll;               // [nbands][W][Q] {value, tag} hand-off records between blocks
    unsigned *band_counter;
    int *status;
    int W, H, Q, E, EMt;    // E labels per lane (EMt: template bound)
    int lam, capv, kc;      // kc: lanes of carry in the truncated sweeps
    int pass, read_c, read_d, write_a, write_b, final_;
    int NWR;                // rows (warps) per block
    int nbands, grid, tag;
    long long spin_limit;
    unsigned long long *trace;
};
int launch_edp_pass_r1(const PassR1Args &a, int threads, size_t smem, cudaStream_t st);
size_t pass_r1_smem(int NWR, int E);

// scanline DP
struct ScanArgs {
    const int *C;
    int *labels;
    long long *row_energy;  // may be null
    void *ptr;              // back-pointers [H][W][Q] in global memory (if not in smem)
    int ptr_bytes;          // 1, 2 or 4
    int ptr_in_smem;
    int W, H, Q, R;
    AxisCfg ax[3];
    int lam, capv, mode;
    int RB;
};
int launch_scanline(const ScanArgs &a, int em, int threads, size_t smem, int grid, cudaStream_t st);

// cost volume
struct CostArgs {
    const uint8_t *I0, *I1, *I2;
    int W, H, pitch;
    int R, Q, Q0, Q1, Q2;
    int vmin[3], step[3];
    int l2, cmax, mode;
    int *C;
};
int launch_cost(const CostArgs &a, cudaStream_t st);

// energy
struct EnergyArgs {
    const int *C;  // may be null
    const int *labels;
    int W, H, Q, R, Q0, Q1;
    int lam, g, l1, mode;
    long long *out4;
};
int launch_energy(const EnergyArgs &a, cudaStream_t st);

}  // namespace edp
