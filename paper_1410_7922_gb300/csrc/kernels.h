// kernels.h -- argument blocks and launchers of the libedp kernels.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace edp {

constexpr int EDP_ERR_TIMEOUT_CODE = 5;  // == EDP_ERR_TIMEOUT of edp.h

// Which message vectors a scan pass reads and writes (pass 0..3 = P1..P4 of
// iteration it of iters).  An old vector is read only once some earlier pass
// wrote it; a new vector is written only if a later pass reads it before it
// is overwritten (P1's m_{+y} and P3's m_{-y} are overwritten by P2 / P4;
// the last pass of the last iteration writes none).
struct PassFlags {
    int read_c, read_d, write_a, write_b, final_;
};
__host__ __device__ inline PassFlags pass_flags(int it, int pass, int iters) {
    const bool last_it = (it == iters - 1);
    PassFlags f;
    f.read_c = (pass == 0) ? (it > 0) : 1;
    f.read_d = (pass <= 1) ? (it > 0) : 1;
    f.write_a = (pass == 3) ? !last_it : 1;
    f.write_b = (pass == 1) ? 1 : (pass == 3 ? !last_it : 0);
    f.final_ = (pass == 3 && last_it);
    return f;
}

// one EDP scan pass, any label axes, one team of T warps per row (pass_team.cuh)
struct TeamAxis {
    int L;        // labels on the axis (line length)
    int G;        // lanes per line segment group (power of two <= 32)
    int E;        // labels per lane, ceil(L / G)
    int nlines;   // Q / L
    int stride;   // distance of axis neighbours in the linear label index
    int kc;       // lanes of carry in the truncated sweeps
    int rounds;   // line groups per lane, ceil(nlines * G / (32 T))
};
struct TeamArgs {
    const int *C;           // [H][W][Q]
    int *M[4];              // [H][W][Qm] messages into each pixel from +x, -x, +y, -y
    int *labels;            // [H][W], written by the final pass
    int2 *ll;               // [nbands][ring][Qm] {value, tag} records between bands
    unsigned *cons;         // [nbands] columns of each band's records consumed ([nbands][8] per warp: line kernels)
    unsigned *rflag;        // line kernels: [nbands][8] columns of records each producing warp has written
    unsigned *band_counter;
    int *status;
    int W, H, Q, Qm, R;     // Qm: message stride, Q rounded up to a multiple of 4
    TeamAxis ax[3];
    int lam, capv, mode;    // mode 0 joint, 1 per axis truncation
    const uint8_t *wh, *wv; // optional [H][W] prior multipliers of the edges (x,y)-(x+1,y), (x,y)-(x,y+1) (lean form)
    int l1, g;              // prior power (1: linear sweeps, 2: quadratic taps, lean / windowed forms) and truncation
    int pass, read_c, read_d, write_a, write_b, final_;
    int pair;               // 1: passes pass and pass + 1 (pass 0 or 2) as one sweep of 2W columns per row
    int read_c2, write_a2, write_b2, final2;  // flags of the second pass of a pair (read_d is shared)
    int T, NT;              // warps per team (one row), teams per block
    int nbuf, kmb, ring;    // staging buffers, mailbox slots, record ring columns
    int tag0;               // tag of the first ring lap of this pass
    int lean;               // 1: lanes own whole lines of one vector (two or more axes)
    int win;                // > 0: windowed form, box side (odd, <= 15)
    const int *centre;      // windowed form: [H][W][R] box centres (label coordinates)
    int Q0w, Q1w;           // windowed form: full label space sizes
    int em;                 // instantiation bound: labels per lane, or line length (lean)
    int nbands, grid;
    long long spin_limit;
    int hold_band;          // test hook: > 0, the first row of this band waits for records never written
    unsigned long long *trace;  // optional: per band {start ns, end ns, 0, sm id}
    // split line kernel: the pair cost of Eq. Cost_value computed from the
    // images (fI1 non-null) instead of read from C: offsets (fv0 + ft0 q0,
    // fv1 + ft1 q1), truncation fcmax, power fl2
    const uint8_t *fI0, *fI1;
    int fpitch, fv0, fv1, ft0, ft1, fcmax, fl2;
};
int launch_edp_pass_team(const TeamArgs &a, int threads, size_t smem, cudaStream_t st);
int edp_pass_team_occupancy(int em, int lean, int win, int threads, size_t smem);
size_t pass_team_smem(int NT, int Qm, int R, int nbuf, int kmb);

// one EDP scan pass, two label axes, one label line per lane (edp_pass_line.cu);
// uses TeamArgs with T = warps per row, NT = rows per block
// split: the form with each label line shared by two lanes (pass_line2.cuh)
bool pass_line_built(int Q0, int Q1, int l1);
bool pass_line_split_built(int Q0, int Q1, int l1);
int pass_line_split_max_lambda();
int pass_line_warps(int Q0, int Q1, bool split);
size_t pass_line_smem(int NT, int Q0, int Q1, bool split);
int edp_pass_line_occupancy(int Q0, int Q1, int l1, bool split, int threads, size_t smem);
int launch_edp_pass_line(const TeamArgs &a, int Q0, int Q1, bool split, int threads, size_t smem, cudaStream_t st);
// per-band stride of the line kernels' record flags and consumed counters
// (one per warp of the producing / consuming team)
constexpr int kLineFlagStride = 8;

// one EDP scan pass, one label axis, one warp per row (edp_pass_r1.cu)
struct PassR1Args {
    const int *C;
    int *M[4];
    int *labels;
    int2 *ll;               // [nbands][W or 2W][Q] {value, tag} hand-off records between blocks
    unsigned *band_counter;
    int *status;
    int W, H, Q, Qm, E, EMt; // Qm: message stride; E labels per lane
    int vw;                 // ints per prefetch copy (1, 2, 4): divides E and Q, aligned
    int lam, capv, kc;      // kc: lanes of carry in the truncated sweeps
    int l1, g;              // prior power (1: linear sweeps, 2: quadratic taps) and truncation
    int pass, read_c, read_d, write_a, write_b, final_;
    int pair;               // 1: passes pass and pass + 1 (pass 0 or 2) as one sweep of 2W columns per row
    int read_c2, write_a2, write_b2, final2;  // flags of the second pass of a pair (read_d is shared)
    const uint8_t *wh, *wv; // optional [H][W] prior multipliers of the edges (x,y)-(x+1,y) and (x,y)-(x,y+1)
    int NWR;                // rows (warps) per block
    int nbands, grid, tag;
    long long spin_limit;
    int hold_band;          // test hook: > 0, the first row of this band waits for records never written
    unsigned long long *trace;
};
int launch_edp_pass_r1(const PassR1Args &a, int threads, size_t smem, cudaStream_t st);
int edp_pass_r1_occupancy(int E, int l1, int threads, size_t smem);
size_t pass_r1_smem(int NWR, int E);
int pass_r1_max_rows(int E, int l1);  // rows per block the one-axis build for E labels per lane allows

// batched solve: up to kMaxBatch problems of one wave, passed by value
constexpr int kMaxBatch = 64;
struct BatchProblem {
    int r1;            // 1: warp-per-row band body, 0: team band body
    int nbands;
    int iters;
    int laps;          // record ring laps per pass (team body)
    unsigned *cons;    // team body: [4*iters][nbands] consumed columns
    union {
        TeamArgs t;    // team body fields (pass / flags / tags set per item)
        PassR1Args o;  // one-axis body fields
    };
};
struct BatchArgs {
    int n;
    int pairs;            // 1: a slot is a paired sweep (P1 + P2 or P3 + P4)
    int slots;            // 4 * iters, or 2 * iters with pairs (shared by the wave)
    int per_slot;         // sum of nbands over the wave
    int prefix[kMaxBatch + 1];
    unsigned *queue;      // work-item counter
    unsigned *done;       // [n][slots] bands finished
    int *status;
    long long spin_limit;
    BatchProblem p[kMaxBatch];
};
// lm: line-length bound of the lean team body (9, 17, 33, 65); gen: the wave
// also holds problems for the generic team body
int launch_edp_batched(const BatchArgs &a, int lm, int gen, int threads, size_t smem, int grid, cudaStream_t st);
int edp_batched_occupancy(int lm, int gen, int threads, size_t smem);



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
    int l1, g;              // prior power (2: quadratic taps, one label axis) and truncation
    int RB;
    int *sums;              // optional [H][W][Q]: S of every column (min-marginal mode)
    int reverse;            // 1: the chain runs from column W-1 to 0
    int no_ptr;             // 1: no back-pointers and no backtrack (min-marginal mode)
};
int launch_scanline(const ScanArgs &a, int em, int threads, size_t smem, int grid, cudaStream_t st);
// S_Omega = F + B - C per pixel, lowest-index argmin (min-marginal mode)
int launch_marginal_argmin(const int *C, const int *F, const int *B, long long npix, int Q, int *labels, int *marg,
                           cudaStream_t st);

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
    const uint8_t *wh, *wv;  // optional per-edge prior multipliers (null: all 1)
    long long *out4;
    // C null and I1 non-null: the data term is the pair cost from the images
    const uint8_t *I0, *I1;
    int pitch, v0, v1, t0, t1, cmax, l2;
};
int launch_energy(const EnergyArgs &a, cudaStream_t st);
int launch_edge_weights(const uint8_t *I, int W, int H, int pitch, int thresh, int factor, uint8_t *wh, uint8_t *wv,
                        cudaStream_t st);

struct CostBatch {
    int n;
    CostArgs c[kMaxBatch];
};
struct EnergyBatch {
    int n;
    EnergyArgs e[kMaxBatch];
};
struct ZeroBatch {
    int n;
    void *ptr[2 * kMaxBatch + 1];
    size_t bytes[2 * kMaxBatch + 1];
};
int launch_cost_batched(const CostBatch &a, long long max_entries, cudaStream_t st);
int launch_energy_batched(const EnergyBatch &a, long long max_pixels, cudaStream_t st);
int launch_zero_batched(const ZeroBatch &a, cudaStream_t st);
int launch_cost_window(const CostArgs &a, const int *centre, int n, cudaStream_t st);

// proposal network (net.cu)
long long net_param_count();
void net_set_tensor_cores(int on);
size_t net_status_offset();
// tensor-core 3x3 convolution of 32 -> 32 channels (net_tc.cu): B image of a
// layer's weights (flip: the input-gradient form), and the convolution
// (mode 0: bias + ReLU; mode 2: input gradient masked by act > 0)
int net_prep_tc_launch(const float *w, int flip, void *out, cudaStream_t st);
int net_conv_tc_launch(const void *in, int N, int H, int W, const void *wB, const float *bias, int mode, void *out,
                       const void *act, int *status, cudaStream_t st);
// weight and bias gradients of a 32 -> 32 layer on the tensor cores: each
// block writes its partial sums to part (net_wgrad_tc_max_blocks() x
// net_wgrad_tc_part_floats() floats), then a reduction adds them to
// grad = dW [32][32][9] followed by db [32]
int net_wgrad_tc_max_blocks();
int net_wgrad_tc_part_floats();
int net_wgrad_tc_launch(const void *g, const void *x, int N, int H, int W, float *part, float *grad, int *status,
                        cudaStream_t st);
size_t net_workspace_bytes(long long npix);
size_t net_activation_offset(long long npix, int layer);
int net_forward(const float *params, const void *x, int N, int H, int W, float *out, unsigned char *ws,
                cudaStream_t st);
int net_backward(const float *params, const float *out, const float *target, int N, int H, int W, float *grad,
                 double *loss, unsigned char *ws, cudaStream_t st);
int net_adam_step(float *p, const float *g, float *m, float *v, long long n, float lr, float b1, float b2, float eps,
                  int step, cudaStream_t st);
int net_features_launch(const uint8_t *I0, const uint8_t *I1, const int *wta_q, const int *wta_cost, int W, int H,
                        int Q0, int Q1, float scale, float cmax, void *out, cudaStream_t st);
int net_centres_launch(const float *out, int n, int Q0, int Q1, int *centre, cudaStream_t st);
int wta_launch(const CostArgs &a, int radius, int *labels, int *cost, cudaStream_t st);
int pyr_down2_launch(const uint8_t *I, int W, int H, int pitch, uint8_t *out, cudaStream_t st);
int labels_up2_launch(const int *lc, int Wc, int Hc, int Qc0, int vminc0, int vminc1, int W, int H, int Q0, int Q1,
                      int vmin0, int vmin1, int *out, cudaStream_t st);
int net_features_lab_launch(const uint8_t *I0, const uint8_t *I1, const int *lab, int W, int H, int pitch, int Q0,
                            int Q1, int vmin0, int vmin1, int l2, int cmax, float scale, void *out, cudaStream_t st);
int net_centres_base_launch(const float *out, const int *base, int n, int Q0, int Q1, int min_shift, int *centre,
                            cudaStream_t st);
int net_targets_launch(const int *lab, const int *base, int n, int Q0, int Q1, float *t, cudaStream_t st);
int window_edge_count_launch(const int *labels, const int *centre, int n, int win, int Q0, int Q1,
                             unsigned long long *count, cudaStream_t st);

}  // namespace edp
