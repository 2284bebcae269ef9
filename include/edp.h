/*
 * edp.h -- C ABI of libedp.so, a GB300 (sm_103a) implementation of the
 * energy minimisation of M. G. Mozerov, "Extended Dynamic Programming and
 * Fast Multidimensional Search Algorithm for Energy Minimization in Stereo
 * and Motion" (arXiv 1410.7922).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Pointers named `*_host` are host memory; every other pointer is device
 *    memory on the current CUDA device.  All memory is owned by the caller;
 *    the library never allocates.  Scratch space is the caller's workspace
 *    `ws` of `ws_bytes` bytes (query the size with edp_workspace_size; the
 *    pointer must be 256-byte aligned).
 *  - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *    stream) and the call returns without synchronising, except where noted.
 *  - Images are uint8 luminance, row-major [H][pitch] (pitch >= W bytes).
 *  - Cost volumes and sums are int32, layout [H][W][Q]: the Q label costs of
 *    one pixel are contiguous.  Labels are int32 [H][W] linear label indexes.
 *  - Return value: EDP_OK or an EDP_ERR_* code.  Argument errors are detected
 *    on the host before anything is enqueued.  Errors detected on the device
 *    (a bounded inter-block wait that expired) are written to the status word
 *    inside the workspace; read it with edp_get_device_status.
 *
 * Label space (Sec. 2, Eq. v_r_x_d)
 * ----------------------------------
 *  R label axes (1..3), Q[r] labels on axis r, axis 0 fastest:
 *      q = q0 + Q[0] * (q1 + Q[1] * q2),   Q = Q[0] * Q[1] * Q[2].
 *  Label coordinate q_r means the displacement  vmin[r] + step[r] * q_r
 *  (step[r] = +1 or -1: the affine relabelling the paper allows below
 *  Eq. v_r_x_d).  Axis 0 displaces x into I1, axis 1 displaces y into I1;
 *  axis 2 (R = 3) displaces x into a third image I2.  Unused entries of
 *  Q must be 1.  A stereo pair is R = 1, vmin = 0, step = -1 (label d reads
 *  I1 at x - d).
 *
 * Parameters (Sec. 5: lambda, g, l1, l2, C_max, j)
 * -------------------------------------------------
 *  Prior, Eq. Smooth_value_t with f(u) = |u|^l1:
 *    EDP_PRIOR_JOINT     V(q, q') = lambda * min(sum_r |q_r - q'_r|^l1, g^l1)
 *    EDP_PRIOR_PER_AXIS  V(q, q') = sum_r lambda * min(|q_r - q'_r|^l1, g^l1)
 *  (identical for R = 1).  l1 = 1 (truncated linear) is evaluated with the
 *  LRMS sweeps of Sec. 3.2 everywhere.  l1 = 2 (truncated quadratic, the
 *  generalized RMS of Eq. M_decmp: per axis the 2g - 1 taps |u| < g, then
 *  the clip) is built for edp_solve / edp_solve_images / edp_solve_batched
 *  when every label axis is served by the one-axis kernel (R = 1, Q <= 256)
 *  or by the whole-line form of the multi-axis kernel (all axes of 9, 17 or
 *  33 labels, or all of 65), for edp_solve / edp_solve_images on the
 *  two-axis spaces 27 x 15 (the paper's +-13 x +-7 motion space) and
 *  25 x 25 (the two-axis line kernel), for edp_solve_windowed, and for
 *  edp_scanline_dp / edp_scanline_marginals on one label axis; other shapes
 *  return EDP_ERR_UNSUPPORTED for l1 = 2.
 *  Cost, Eq. Cost_value: C(x, q) = min(|I1(x + o(q)) - I0(x)|^l2, cmax),
 *  cmax where x + o(q) leaves the image.
 */
#ifndef EDP_H
#define EDP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *edp_stream_t; /* == cudaStream_t */

enum edp_status {
    EDP_OK = 0,
    EDP_ERR_INVALID_ARG = 1, /* null pointer, bad size, bad enum value        */
    EDP_ERR_UNSUPPORTED = 2, /* valid by the paper but not built for this shape */
    EDP_ERR_WORKSPACE = 3,   /* ws_bytes smaller than edp_workspace_size      */
    EDP_ERR_RANGE = 4,       /* sizes or values could overflow int32          */
    EDP_ERR_TIMEOUT = 5,     /* a bounded device-side wait expired            */
    EDP_ERR_CUDA = 6         /* a CUDA runtime call failed                    */
};

enum { EDP_PRIOR_JOINT = 0, EDP_PRIOR_PER_AXIS = 1 };

/* Cost models (edp_params.cost_mode):
 *  EDP_COST_PAIR          Eq. Cost_value between I0 and I1 (R = 1 or 2).
 *  EDP_COST_PAIR_STEREO3  R = 3: min(|I1(x+o0, y+o1) - I0|^l2
 *                                    + |I2(x+o2, y) - I0|^l2, cmax),
 *                         cmax if either displaced pixel leaves the image.
 *  EDP_COST_COMPOSITE     Eq. Cost_cmp (occlusion handling with a third
 *                         image): min(C_{I0->I1}(x, o), C_{I0->I2}(x, -o)),
 *                         each term truncated by Eq. Cost_value (R = 1, 2). */
enum { EDP_COST_PAIR = 0, EDP_COST_PAIR_STEREO3 = 1, EDP_COST_COMPOSITE = 2 };

typedef struct {
    int32_t R;       /* number of label axes, 1..3                      */
    int32_t Q[3];    /* labels per axis (unused axes: 1)                */
    int32_t vmin[3]; /* displacement of label coordinate 0 on each axis */
    int32_t step[3]; /* +1 or -1                                        */
} edp_label_space;

typedef struct {
    int32_t lambda;     /* prior weight, >= 0                            */
    int32_t g;          /* truncation threshold, >= 1                    */
    int32_t l1;         /* prior power, 1 or 2 (see above)               */
    int32_t prior_mode; /* EDP_PRIOR_*                                   */
    int32_t l2;         /* cost power, 1 or 2                            */
    int32_t cmax;       /* cost truncation C_max, >= 0                   */
    int32_t cost_mode;  /* EDP_COST_*                                    */
    int32_t iters;      /* EDP iterations j (Algorithm 1, step 3), >= 1  */
} edp_params;

/* Operations for edp_workspace_size. */
enum {
    EDP_OP_SCANLINE_DP = 1,
    EDP_OP_SOLVE = 2,
    EDP_OP_SOLVE_IMAGES = 3, /* edp_solve_images and edp_solve_images_host */
    EDP_OP_COARSE = 4,       /* edp_coarse_labels */
    EDP_OP_SCANLINE_MARGINALS = 5 /* edp_scanline_marginals */
};

/* Library version (major * 10000 + minor * 100 + patch). */
int edp_version(void);

/* Human-readable name of a status code (static storage). */
const char *edp_status_string(int status);

/* Bytes of workspace `op` needs for a W x H image (params->iters matters
 * for the EDP operations).  Returns 0 for invalid arguments. */
size_t edp_workspace_size(int op, int W, int H, const edp_label_space *space,
                          const edp_params *params);

/* Process-wide launch shape of the DP kernels (0 = automatic, the default):
 *   rows_per_block   rows of the image per block (scanline DP, both
 *                    scan-pass kernels);
 *   labels_per_lane  target labels per lane on one label line (scanline DP);
 *   warps_per_row    warps that share one image row in the multi-axis
 *                    scan-pass kernel (1..12);
 *   general_kernel   1: one-axis label spaces also take the multi-axis
 *                    scan-pass kernel instead of the warp-per-row one;
 *                    2: in addition, multi-axis spaces take its lane-group
 *                    form instead of the whole-line form;
 *                    3: two-axis spaces take the multi-axis kernel instead
 *                    of the two-axis line kernel; 4: two-axis spaces take
 *                    the line kernel wherever it is built (Q0 x Q1 = 17 x
 *                    17, 25 x 25, 33 x 33, 65 x 65 and 27 x 15, l1 = 1;
 *                    by default it serves 65 x 65); 5: as 4, with one lane
 *                    per label line also at 65 x 65 (by default the lines
 *                    of 65 x 65 are split over two lanes when lambda <=
 *                    2^30 / (34 * 255)).
 * Used by the autotuner and the tests; results never depend on it.  A shape
 * the kernels cannot run makes the next solve return EDP_ERR_UNSUPPORTED.
 * Not thread-safe with concurrent solves. */
int edp_set_tuning(int rows_per_block, int labels_per_lane, int warps_per_row, int general_kernel);

/* Pass schedule of edp_solve, edp_solve_images, edp_solve_windowed and
 * edp_solve_batched (Sec. 4.2: P1..P4 per iteration).  P1 and P2, and P3 and
 * P4, share their vertical direction and can run as one paired sweep each:
 * every row sweeps left to right, then right to left, so the second pass
 * starts on a row as soon as the first has finished it (two launches per
 * iteration instead of four).
 *   mode 0: one launch per pass;
 *   mode 1: paired sweeps always;
 *   mode 2 (the default): paired sweeps when every row band of the problem
 *           has a block at once (a paired band holds its block twice as long,
 *           which costs more than it saves when bands wait for blocks);
 *           edp_solve_batched pairs only in mode 1 (its bands share the
 *           blocks).
 * Results never depend on it.  Returns EDP_ERR_INVALID_ARG unless mode is 0,
 * 1 or 2.  Not thread-safe with concurrent solves. */
int edp_set_pass_pairs(int mode);

/* Cost volume of edp_solve_images / edp_solve_images_host.  1: where the
 * pair cost (Eq. Cost_value, cost_mode pair) of a two-axis label space runs
 * on the split form of the two-axis line kernel, the scan passes and the
 * energy compute C(x, q) from the images as they need it and no cost volume
 * is built (the values are those edp_cost_volume stores).  0 (the default):
 * the cost volume is always built first (measured faster at 640x480 with
 * 65 x 65 labels: the scan passes' byte loads of 65 image rows per column
 * cost more than the cost volume saves).  Results never depend on it.
 * Returns EDP_ERR_INVALID_ARG unless on is 0 or 1.  Not thread-safe with
 * concurrent solves. */
int edp_set_fused_cost(int on);

/* Scan-pass launches of the most recent edp_solve, edp_solve_images or
 * edp_solve_windowed call in this process (2 per iteration for paired
 * sweeps, else 4; 0 before the first solve).  The launches are counted as by
 * edp_set_profile_events.  Not thread-safe with concurrent solves. */
int edp_last_pass_launches(void);

/* Name of the scan-pass kernel the most recent edp_solve, edp_solve_images
 * or edp_solve_windowed call in this process launched (static storage; ""
 * before the first solve).  Not thread-safe with concurrent solves. */
const char *edp_last_pass_kernel(void);

/* Per-launch timing hook: while set, edp_solve (and edp_solve_images) record
 * events[2*i] / events[2*i + 1] (cudaEvent_t handles created by the caller)
 * on the solve's stream immediately before / after scan-pass launch i
 * (i counts the launches of one solve in order: 4 * iteration + pass, or
 * 2 * iteration + pair for paired sweeps), for i < n_events / 2.  NULL / 0
 * disables.
 * The library keeps the pointer, not a copy: the array must outlive the
 * solves that use it. */
int edp_set_profile_events(void *const *events, int n_events);

/* Bound of every wait between row bands of the scan-pass kernels (polls of
 * the awaited flag or record before the wait gives up and the launch sets
 * EDP_ERR_TIMEOUT in the device status word); 0 restores the default of
 * 4,000,000.  Applies to the solves enqueued after the call.  Returns
 * EDP_ERR_INVALID_ARG for a negative value.  Not thread-safe with
 * concurrent solves. */
int edp_set_spin_limit(long long polls);

/* Test hook for the timeout path (0, the default, turns it off): in the
 * solves enqueued after the call (edp_solve, edp_solve_images,
 * edp_solve_weighted), the first row of row band `band` (> 0) waits for
 * hand-off data that is never published (records of a tag no producer
 * writes, or a column past the last one).  Its wait runs out after the
 * spin limit, the launch sets EDP_ERR_TIMEOUT in the device status word and
 * every kernel of the solve returns; the labels are then undefined.  Makes
 * the wait expire without a fault.  Not thread-safe with concurrent solves. */
int edp_test_hold_band(int band);

/* Per-band trace of the scan passes (tracing hook): while set, scan-pass
 * launch i of a solve (counted as for edp_set_profile_events) writes, for
 * every row band b, four uint64 at device_buffer[(i * nbands + b) * 4 ...]:
 * start and end %globaltimer (ns), ns spent waiting for the previous band,
 * and the SM id.  Launches whose record would not fit in `bytes` are not
 * traced.  NULL / 0 disables. */
int edp_set_trace(void *device_buffer, size_t bytes);

/* Cost volume (DSI), Eq. Cost_value (Algorithm 1, step 1).
 *  I0, I1: uint8 [H][pitch]; I2: third image for EDP_COST_PAIR_STEREO3 and
 *  EDP_COST_COMPOSITE, else NULL.  Writes C int32 [H][W][Q].
 *  Uses params->l2, cmax, cost_mode. */
int edp_cost_volume(const uint8_t *I0, const uint8_t *I1, const uint8_t *I2, int W, int H,
                    int pitch, const edp_label_space *space, const edp_params *params,
                    int32_t *C, edp_stream_t stream);

/* Scanline DP, Sec. 4.1: every row is an independent chain (Eq. One_d, the
 * vertical prior set to zero).  Forward recurrence Eq. base with the
 * boundary of Eq. DP_1D_2 (S(0) = C(0)), the min search done by the RMS
 * (Sec. 3), optimal-choice indexes stored during the forward pass, then the
 * backward recovery from argmin_q S(W-1, q).  Ties take the lowest label
 * index: at the last column, and at each back-pointer.
 *  C: int32 [H][W][Q].  labels: int32 [H][W].  row_energy: int64 [H]
 *  (min_q S(W-1, q), the optimal chain energy), or NULL. */
int edp_scanline_dp(const int32_t *C, int W, int H, const edp_label_space *space,
                    const edp_params *params, int32_t *labels, int64_t *row_energy, void *ws,
                    size_t ws_bytes, edp_stream_t stream);

/* Min-marginal mode of the scanline DP (the modified DP of Sec. 4.1,
 * Eq. DP_1D_3): per image row the forward sums F (Eq. base, from the left
 * end) and the backward sums B (the same recurrence from the right end);
 * the marginal is S_Omega(x, q) = M(F(x-1))(q) + C(x, q) + M(B(x+1))(q)
 * = F(x, q) + B(x, q) - C(x, q), and labels[y][x] is its lowest-index
 * argmin.  marginals: optional int32 [H][W][Q] output of S_Omega (NULL:
 * not written).  ws: edp_workspace_size(EDP_OP_SCANLINE_MARGINALS, ...)
 * bytes, 256-byte aligned.  l1 = 1, or l1 = 2 on one label axis
 * (EDP_ERR_UNSUPPORTED otherwise);
 * EDP_ERR_RANGE when W * (cmax + R * lambda * g^l1) >= 2^29. */
int edp_scanline_marginals(const int32_t *C, int W, int H, const edp_label_space *space, const edp_params *params,
                           int32_t *labels, int32_t *marginals, void *ws, size_t ws_bytes, edp_stream_t stream);

/* EDP, Sec. 4.2 / Algorithm 1 steps 2-5: params->iters iterations of the
 * four scan passes P1..P4 (Eq. DP_2D_base with the data term added, D = 2,
 * messages M(floor(S_k(x_k) / 2)), zero outside the image), then the
 * marginal estimate S_Omega = C + sum_k M(floor(S_k(x_k) / 2)) (Eq. DP_2D_1)
 * and its argmin (Eq. DP_2D_2), lowest label index on ties.
 *  C: int32 [H][W][Q].  labels: int32 [H][W].  ws: >= edp_workspace_size(
 *  EDP_OP_SOLVE, ...) bytes.  Device status word: EDP_ERR_TIMEOUT if a wait
 *  between row bands expired (the labels are then undefined).
 *  Returns EDP_ERR_RANGE when N * (cmax + 2 * R * lambda * g) * 2 >= 2^31
 *  (the sums could leave int32). */
int edp_solve(const int32_t *C, int W, int H, const edp_label_space *space,
              const edp_params *params, int32_t *labels, void *ws, size_t ws_bytes,
              edp_stream_t stream);

/* Energy, Eq. GE_objective_function on the 4-connected grid:
 *  out4[0] = sum_x C(x, v(x))                 (data term)
 *  out4[1] = sum over horizontal edges V       (x, x+1)
 *  out4[2] = sum over vertical edges V         (y, y+1)
 *  out4[3] = out4[0] + out4[1] + out4[2].
 *  C may be NULL (data term 0).  out4: int64 [4], device memory. */
int edp_energy(const int32_t *C, const int32_t *labels, int W, int H,
               const edp_label_space *space, const edp_params *params, int64_t *out4,
               edp_stream_t stream);

/* Locally adaptive prior (the text below Eq. Smooth_value_t: lambda(x) =
 * 2 lambda where the local gradient of the image is below 10, lambda
 * elsewhere), read as one multiplier per grid edge: the prior of the edge
 * (x, y)-(x+1, y) is wh[y][x] * lambda * f, that of (x, y)-(x, y+1) is
 * wv[y][x] * lambda * f.  (The paper's printed rule gives 2 lambda on both
 * branches; the second is read as lambda.)
 *
 * edp_edge_weights: the multipliers of that rule from an image I (uint8
 * [H][pitch]): an edge whose intensity step |I(x') - I(x)| is below
 * `threshold` gets `factor` (0..255), every other edge 1; entries without an
 * edge (last column of wh, last row of wv) are 1.  wh, wv: uint8 [H][W],
 * device memory. */
int edp_edge_weights(const uint8_t *I, int W, int H, int pitch, int threshold, int factor, uint8_t *wh,
                     uint8_t *wv, edp_stream_t stream);

/* edp_solve with the per-edge multipliers wh, wv (uint8 [H][W], device
 * memory, every entry in 0..max_weight): the message from a pixel into its
 * neighbour is the min search M with the prior of the edge between them.
 * One-axis label spaces with Q <= 256, and multi-axis spaces whose lines all
 * hold 9, 17 or 33 labels, or all 65 (the whole-line form of the multi-axis
 * kernel); EDP_ERR_UNSUPPORTED otherwise.
 * ws: >= edp_workspace_size(EDP_OP_SOLVE, ...).  The range check of
 * edp_solve applies with lambda * max_weight. */
int edp_solve_weighted(const int32_t *C, int W, int H, const edp_label_space *space, const edp_params *params,
                       const uint8_t *wh, const uint8_t *wv, int max_weight, int32_t *labels, void *ws,
                       size_t ws_bytes, edp_stream_t stream);

/* edp_energy with the per-edge multipliers: out4[1] = sum over horizontal
 * edges of wh * V, out4[2] = sum over vertical edges of wv * V. */
int edp_energy_weighted(const int32_t *C, const int32_t *labels, int W, int H, const edp_label_space *space,
                        const edp_params *params, const uint8_t *wh, const uint8_t *wv, int64_t *out4,
                        edp_stream_t stream);

/* Images to labels on the device: edp_cost_volume into the workspace,
 * edp_solve, edp_energy.  labels: int32 [H][W]; energy4: int64 [4] or NULL. */
int edp_solve_images(const uint8_t *I0, const uint8_t *I1, const uint8_t *I2, int W, int H,
                     int pitch, const edp_label_space *space, const edp_params *params,
                     int32_t *labels, int64_t *energy4, void *ws, size_t ws_bytes,
                     edp_stream_t stream);

/* Same as edp_solve_images with HOST images and HOST outputs: copies the
 * images (dense [H][W]) into the workspace, runs the pipeline and copies the
 * labels and the energy back.  Synchronises `stream` before returning.
 * Pinned host buffers give the fastest copies. */
int edp_solve_images_host(const uint8_t *I0_host, const uint8_t *I1_host,
                          const uint8_t *I2_host, int W, int H, const edp_label_space *space,
                          const edp_params *params, int32_t *labels_host,
                          int64_t *energy4_host, void *ws, size_t ws_bytes, edp_stream_t stream);

/* Windowed EDP (the learned-proposal form; not in the paper).  Every pixel
 * keeps only the win^R labels of a box centred on a proposed label
 * (centre: int32 [H][W][R] label coordinates, clamped so that the box lies
 * inside the label space).  Costs, messages and sums live in box
 * coordinates; a message between neighbouring boxes is the exact
 * min-convolution of Eq. M_strf restricted to the two boxes, evaluated with
 * the RMS sweeps of Sec. 3.2 per axis.  With every box equal to the whole
 * space this is edp_solve.  Supported: R = 1 or 2, odd win <= 15,
 * win <= Q[r], l1 = 1 or 2 (quadratic taps between the boxes).
 *  Cw: int32 [H][W][win^R] box costs from edp_cost_window.  labels: int32
 *  [H][W] full-space linear label indexes. */
size_t edp_workspace_size_windowed(int W, int H, const edp_label_space *space, const edp_params *params,
                                   int win);
int edp_cost_window(const uint8_t *I0, const uint8_t *I1, const uint8_t *I2, int W, int H, int pitch,
                    const edp_label_space *space, const edp_params *params, const int32_t *centre, int win,
                    int32_t *Cw, edp_stream_t stream);
int edp_solve_windowed(const int32_t *Cw, const int32_t *centre, int win, int W, int H,
                       const edp_label_space *space, const edp_params *params, int32_t *labels, void *ws,
                       size_t ws_bytes, edp_stream_t stream);

/* Winner-take-all over the full label space, straight from the images (no
 * cost volume): labels[x] = lowest-index argmin_q of Eq. Cost_value summed
 * over the (2 radius + 1)^2 pixels around x (edge pixels repeated; radius 0
 * is the plain cost, radius <= 15), cost[x] = that minimum (may be NULL).
 * R = 1 or 2, EDP_COST_PAIR. */
int edp_wta(const uint8_t *I0, const uint8_t *I1, int W, int H, int pitch, const edp_label_space *space,
            const edp_params *params, int radius, int32_t *labels, int32_t *cost, edp_stream_t stream);

/* Learned proposal network (not in the paper): six 3x3 convolutions, channels
 * 5 -> 32 -> 32 -> 32 -> 32 -> 32 -> 2, ReLU between layers, predicting the
 * label-space centre of each pixel (R = 2) for edp_solve_windowed.
 * bfloat16 weights and activations (round to nearest even), float32
 * accumulation; parameters are a flat float32 array (layer by layer:
 * W[Co][Ci][3][3], then b[Co]), edp_net_param_count() values.
 * Features x: bf16 [N][H][W][5] (from edp_net_features).  Output and target:
 * float32 [N][H][W][2], label coordinates relative to the space's middle. */
long long edp_net_param_count(void);
size_t edp_net_workspace_size(int N, int H, int W);
/* Byte offset in the network workspace of the input of layer `layer` (0..5;
 * layer 0's input is the feature tensor), which edp_net_forward leaves
 * there for edp_net_backward: bf16 [N][H][W][C], C = 5, 32, 32, 32, 32, 32.
 * (size_t)-1 for invalid arguments.  For inspection and tests. */
size_t edp_net_activation_offset(int N, int H, int W, int layer);
/* Forward pass; keeps the activations in ws for edp_net_backward. */
int edp_net_forward(const float *params, const void *x, int N, int H, int W, float *out, void *ws, size_t ws_bytes,
                    edp_stream_t stream);
/* Smooth-L1 loss (mean) of the last forward's output against target and
 * the gradient of every parameter (grad: float32, same layout as params).
 * loss: device float64 [1]. */
int edp_net_backward(const float *params, const float *out, const float *target, int N, int H, int W, float *grad,
                     double *loss, void *ws, size_t ws_bytes, edp_stream_t stream);
/* Where the 3x3 convolutions of 32 -> 32 channels run (layers 1-4 forward,
 * their input gradients and their weight gradients): 1 (the default) on the
 * tensor cores
 * (tcgen05.mma, bf16 operands, float32 accumulation in tensor memory, one
 * implicit GEMM per 8 x 16 pixel tile: M = 128 pixels, N = 32 channels,
 * K = 9 x 32), 0 on the CUDA cores (float32 FMA).  The two forms round the
 * same bf16 products and differ only in the order of the float32 sums.
 * Returns EDP_ERR_INVALID_ARG unless on is 0 or 1.  Not thread-safe with
 * concurrent calls. */
int edp_set_net_tensor_cores(int on);
/* The network workspace's status word (0, or EDP_ERR_TIMEOUT when a bounded
 * wait of a tensor-core convolution ran out; cleared by edp_net_forward),
 * read after the work queued on `stream`.  Synchronises the stream. */
int edp_net_get_device_status(const void *ws, size_t ws_bytes, int *status, edp_stream_t stream);
/* One Adam step (step >= 1) on the float32 parameters. */
int edp_net_adam(float *params, const float *grad, float *m, float *v, float lr, float beta1, float beta2, float eps,
                 int step, edp_stream_t stream);
/* Features of one image pair: I0/255, I1/255, the WTA label coordinates
 * (centred, / scale) and the WTA cost / cmax, as bf16 [H][W][5]. */
int edp_net_features(const uint8_t *I0, const uint8_t *I1, const int32_t *wta_labels, const int32_t *wta_cost,
                     int W, int H, const edp_label_space *space, float scale, float cmax, void *x,
                     edp_stream_t stream);
/* Box centres (int32 [n][2], label coordinates) from network outputs:
 * round to the nearest label, clamp into the space. */
int edp_net_centres(const float *out, int n, const edp_label_space *space, int32_t *centre, edp_stream_t stream);

/* Coarse-level labeling for the proposal (no counterpart in the paper; an
 * input of the proposal network).  Two-axis spaces with step +1 only
 * (EDP_ERR_UNSUPPORTED otherwise).  I0, I1: device uint8 [H][pitch].  Both
 * images are halved (2x2 averages rounded half up, (W+1)/2 x (H+1)/2), full
 * EDP (Algorithm 1, params->iters iterations, the given prior and cost) runs
 * there on the label space with halved offsets (ceil(vmin/2) ..
 * floor(vmax/2) per axis), and each full-resolution pixel (x, y) gets the
 * label of coarse pixel (x/2, y/2) with its offsets doubled and clamped into
 * `space`.  labels: device int32 [H][W] (linear label index of `space`).
 * ws: edp_workspace_size(EDP_OP_COARSE, ...) bytes, 256-byte aligned; the
 * coarse solve's status word is the workspace's first int at offset 256.
 * Errors as edp_solve_images. */
int edp_coarse_labels(const uint8_t *I0, const uint8_t *I1, int W, int H, int pitch, const edp_label_space *space,
                      const edp_params *params, int32_t *labels, void *ws, size_t ws_bytes, edp_stream_t stream);

/* Network input (bf16 [H][W][5]) from a labeling of a two-axis space with
 * step +1: I0/255, I1/255, the label's coordinates minus (Q_r - 1)/2,
 * divided by `scale`, and its data cost (Eq. Cost_value with params->l2,
 * params->cmax) / cmax.  Images uint8 [H][pitch], labels int32 [H][W]. */
int edp_net_features_labels(const uint8_t *I0, const uint8_t *I1, const int32_t *labels, int W, int H, int pitch,
                            const edp_label_space *space, const edp_params *params, float scale, void *x,
                            edp_stream_t stream);

/* Box centres (int32 [n][2]) as a correction of a base labeling: the base
 * label's coordinates plus the network output (label units) rounded half away
 * from zero; a correction whose larger component is below min_shift labels
 * is dropped (0: every correction applies); clamped into the space.
 * out: float [n][2]; base: int32 [n]. */
int edp_net_centres_residual(const float *out, const int32_t *base, int n, const edp_label_space *space,
                             int min_shift, int32_t *centre, edp_stream_t stream);

/* Training targets (float [n][2], label units) of a labeling: its label
 * coordinates minus those of `base` (int32 [n]), or minus (Q_r - 1)/2 when
 * base is NULL. */
int edp_net_targets(const int32_t *labels, const int32_t *base, int n, const edp_label_space *space, float *target,
                    edp_stream_t stream);

/* Fallback trigger of the proposal path (not in the paper): the number of
 * pixels whose label (int32 [n], full-space linear index) lies on an inner
 * edge of its win x win box (centre: int32 [n][2], clamped into the space as
 * edp_solve_windowed does) -- an edge that is not also an edge of the label
 * space, so a better label may lie outside the box.  Two-axis spaces.
 * count: device int64 [1], overwritten. */
int edp_window_edge_count(const int32_t *labels, const int32_t *centre, int n, int win,
                          const edp_label_space *space, int64_t *count, edp_stream_t stream);

/* One problem of a batch: a device image pair (or triple) in, labels and
 * energy out.  Images are uint8 [H][pitch]. */
typedef struct {
    const uint8_t *I0, *I1, *I2;
    int32_t W, H, pitch;
    edp_label_space space;
    edp_params params;
    int32_t *labels;  /* device int32 [H][W]          */
    int64_t *energy4; /* device int64 [4], or NULL    */
} edp_problem;

/* Workspace bytes for edp_solve_batched to keep all n problems resident at
 * once.  A smaller workspace also works as long as it holds the largest
 * single problem: the problems are then solved in waves that fit. */
size_t edp_batch_workspace_size(const edp_problem *probs, int n);

/* Batched form of edp_solve_images for many independent problems of uneven
 * sizes and label spaces (one, two and three label axes mixed).  Per wave of
 * resident problems: one launch zeroes the control words, one builds every
 * cost volume, ONE persistent launch runs every scan pass of every problem
 * (work items (pass, problem, row band) taken in order from a global queue,
 * with bounded waits on the previous band and the previous pass of the same
 * problem), and one launch evaluates every energy.  Results are identical to
 * solving each problem alone.  `probs` is host memory and is read during the
 * call only.  The call enqueues work and returns; it can be captured in a
 * CUDA graph (after one uncaptured call has set the kernels' attributes).
 * Problems at or above the size set by edp_set_batch_split run with launches
 * of their own inside the call. */
int edp_solve_batched(const edp_problem *probs, int n, void *ws, size_t ws_bytes, edp_stream_t stream);

/* Split of edp_solve_batched (process-wide): a problem of at least
 * `min_pixels` pixels fills the GPU by itself and is solved with its own
 * launches in the problem's best shape (cost volume, scan passes, energy),
 * the smaller problems of a wave share one persistent launch.  0 puts every
 * problem into the persistent launch.  The default is 172,800 pixels
 * (480 x 360).  Results never depend on it.  Not thread-safe with
 * concurrent solves. */
int edp_set_batch_split(long long min_pixels);

/* Reads the device status word of a workspace used by edp_solve /
 * edp_solve_images / edp_scanline_dp.  Synchronises `stream`. */
int edp_get_device_status(const void *ws, size_t ws_bytes, int *status, edp_stream_t stream);


/* edp_solve without a workspace argument (the paper has no counterpart).
 * For callers that cannot allocate device memory at all -- their device
 * memory is entirely reserved up front by another allocator (a framework's
 * fixed pool, an embedded or real-time loop with a fixed budget), or they
 * must not call cudaMalloc because it may synchronise the device.  The
 * caller still passes C and labels (as for edp_solve); the scratch is a
 * static array of EDP_NOALLOC_SCRATCH_BYTES in the library's device memory,
 * which every GPU that loads the library holds until the process exits.
 * The call is edp_solve with that array as its workspace: the same argument
 * checks in the same order and the same return codes, EDP_ERR_WORKSPACE for
 * a problem whose edp_workspace_size(EDP_OP_SOLVE, ...) exceeds the array
 * (nothing is enqueued then).  The first call on a device looks up the
 * array's device address (once per device, with that device current); make
 * that first call before any stream capture.  The address belongs to the
 * device's primary context: after cudaDeviceReset of a device, do not call
 * this entry point (or edp_noalloc_get_device_status) on it again in the
 * same process.  Every call shares the one array and it keeps the previous
 * call's contents: calls whose work overlaps on the GPU (other streams,
 * other threads) race and must be ordered by the caller. */
#define EDP_NOALLOC_SCRATCH_BYTES (64u << 20)
int edp_solve_noalloc(const int32_t *C, int W, int H, const edp_label_space *space,
                      const edp_params *params, int32_t *labels, edp_stream_t stream);

/* Device status word of the most recent edp_solve_noalloc on the current
 * device (EDP_ERR_TIMEOUT if a wait between row bands expired; the labels
 * are then undefined), as edp_get_device_status reads it for a workspace.
 * Synchronises `stream`. */
int edp_noalloc_get_device_status(int *status, edp_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* EDP_H */
