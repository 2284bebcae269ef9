// net.cu -- the learned proposal network (not in the paper): six 3x3
// convolutions (channels 5 -> 32 -> 32 -> 32 -> 32 -> 32 -> 2, ReLU after all
// but the last) predicting a per-pixel label centre for windowed EDP, with its
// training kernels.
//
// Precision: weights and activations are stored as bfloat16 (round to
// nearest even), every product is accumulated in float32, the biases, the
// master weights, the optimiser state and the network output are float32.
// The gradient entering each layer is stored as bfloat16.
//
// Layout: activations NHWC ([N][H][W][C], channels contiguous), parameters a
// flat float32 array, layer by layer: W[Co][Ci][3][3] then b[Co].
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"

namespace edp {

namespace {
constexpr int kT = 16;  // output tile side (pixels)

__device__ __forceinline__ float bf2f(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ __nv_bfloat16 f2bf(float v) { return __float2bfloat16_rn(v); }
}  // namespace

// Weights of one layer, bf16-rounded, re-laid as float32 [9][Cin][Cout] for
// the forward conv (Cin = Ci, Cout = Co), or flipped and transposed as
// [9][Co][Ci] for the input gradient (a forward conv of the output gradient
// with w'[ci][co][2-dy][2-dx]).
__global__ void net_prep_weights(const float *w, int Co, int Ci, int flip, float *out) {
    const int n = Co * Ci * 9;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const int tap = e % 9, ci = (e / 9) % Ci, co = e / (9 * Ci);
        const float v = bf2f(f2bf(w[e]));
        if (!flip)
            out[((size_t)tap * Ci + ci) * Co + co] = v;
        else
            out[((size_t)(8 - tap) * Co + co) * Ci + ci] = v;
    }
}

// 3x3 convolution, zero padding, one output pixel per thread, all output
// channels in registers.  in: bf16 [N][H][W][Cin].  wf: float [9][Cin][Cout].
// mode 0: out_bf = bf16(relu(z + b)); mode 1: out_f = z + b (float32);
// mode 2 (input gradient): out_bf = bf16(z * (act > 0)) with act bf16
// [N][H][W][Cout] the activation at this gradient's position.
template <int COUT>
__global__ void __launch_bounds__(256) net_conv3x3(const __nv_bfloat16 *in, int N, int H, int W, int Cin,
                                                  const float *wf, const float *bias, int mode,
                                                  __nv_bfloat16 *out_bf, float *out_f,
                                                  const __nv_bfloat16 *act) {
    extern __shared__ float sm[];
    // the tile's pixels are CP = Cin | 1 floats apart (odd), so that the
    // lanes of a warp, which read neighbouring pixels, hit distinct banks
    const int CP = Cin | 1;
    float *ws = sm;                                  // [9][Cin][COUT]
    float *tile = sm + 9 * Cin * COUT;               // [(kT+2)^2][CP]
    const int n = blockIdx.z;
    const int x0 = blockIdx.x * kT, y0 = blockIdx.y * kT;
    for (int e = threadIdx.x; e < 9 * Cin * COUT; e += blockDim.x) ws[e] = wf[e];
    const int TW = kT + 2;
    for (int e = threadIdx.x; e < TW * TW * Cin; e += blockDim.x) {
        const int c = e % Cin, p = e / Cin;
        const int ty = p / TW, tx = p % TW;
        const int y = y0 + ty - 1, x = x0 + tx - 1;
        float v = 0.f;
        if (y >= 0 && y < H && x >= 0 && x < W) v = bf2f(in[(((size_t)n * H + y) * W + x) * Cin + c]);
        tile[p * CP + c] = v;
    }
    __syncthreads();
    const int lx = threadIdx.x % kT, ly = threadIdx.x / kT;
    const int x = x0 + lx, y = y0 + ly;
    float acc[COUT];
#pragma unroll
    for (int c = 0; c < COUT; ++c) acc[c] = 0.f;
    for (int dy = 0; dy < 3; ++dy)
        for (int dx = 0; dx < 3; ++dx) {
            const float *t = tile + ((ly + dy) * TW + (lx + dx)) * CP;
            const float *wt = ws + (dy * 3 + dx) * Cin * COUT;
            for (int ci = 0; ci < Cin; ++ci) {
                const float v = t[ci];
                const float *wr = wt + ci * COUT;
#pragma unroll
                for (int c = 0; c < COUT; ++c) acc[c] = fmaf(v, wr[c], acc[c]);
            }
        }
    if (x >= W || y >= H) return;
    const size_t o = (((size_t)n * H + y) * W + x) * COUT;
    if (mode == 0) {
#pragma unroll
        for (int c = 0; c < COUT; ++c) out_bf[o + c] = f2bf(fmaxf(acc[c] + bias[c], 0.f));
    } else if (mode == 1) {
#pragma unroll
        for (int c = 0; c < COUT; ++c) out_f[o + c] = acc[c] + bias[c];
    } else {
#pragma unroll
        for (int c = 0; c < COUT; ++c) out_bf[o + c] = f2bf(bf2f(act[o + c]) > 0.f ? acc[c] : 0.f);
    }
}

// Weight and bias gradients of one layer: dW[co][ci][dy][dx] += sum over the
// tile's pixels of g[p][co] * x[p + (dy-1, dx-1)][ci]; db[co] += sum g[p][co].
// Thread = (tap, group of 4 input channels, group of 8 output channels).
__global__ void __launch_bounds__(288) net_wgrad(const __nv_bfloat16 *g, const __nv_bfloat16 *x, int N, int H, int W,
                                                 int Ci, int Co, float *dW, float *db) {
    extern __shared__ float sm[];
    const int TW = kT + 2;
    // odd strides between pixels: the threads of a warp read different taps
    // and channel groups of one pixel without sharing a bank
    const int CiP = Ci | 1, CoP = Co | 1;
    float *xt = sm;                        // [(kT+2)^2][CiP]
    float *gt = sm + TW * TW * CiP;        // [kT*kT][CoP]
    const int n = blockIdx.z;
    const int x0 = blockIdx.x * kT, y0 = blockIdx.y * kT;
    for (int e = threadIdx.x; e < TW * TW * Ci; e += blockDim.x) {
        const int c = e % Ci, p = e / Ci;
        const int yy = y0 + p / TW - 1, xx = x0 + p % TW - 1;
        xt[p * CiP + c] = (yy >= 0 && yy < H && xx >= 0 && xx < W) ? bf2f(x[(((size_t)n * H + yy) * W + xx) * Ci + c]) : 0.f;
    }
    for (int e = threadIdx.x; e < kT * kT * Co; e += blockDim.x) {
        const int c = e % Co, p = e / Co;
        const int yy = y0 + p / kT, xx = x0 + p % kT;
        gt[p * CoP + c] = (yy < H && xx < W) ? bf2f(g[(((size_t)n * H + yy) * W + xx) * Co + c]) : 0.f;
    }
    __syncthreads();
    const int cig = (Ci + 3) / 4, cog = (Co + 7) / 8;
    const int t = threadIdx.x;
    if (t < 9 * cig * cog) {
        const int tap = t % 9, ci0 = ((t / 9) % cig) * 4, co0 = (t / (9 * cig)) * 8;
        const int dy = tap / 3, dx = tap % 3;
        float acc[4][8];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
        for (int p = 0; p < kT * kT; ++p) {
            const int py = p / kT, px = p % kT;
            const float *xr = xt + ((py + dy) * TW + (px + dx)) * CiP;
            const float *gr = gt + p * CoP;
            float xv[4], gv[8];
#pragma unroll
            for (int a = 0; a < 4; ++a) xv[a] = (ci0 + a < Ci) ? xr[ci0 + a] : 0.f;
#pragma unroll
            for (int b = 0; b < 8; ++b) gv[b] = (co0 + b < Co) ? gr[co0 + b] : 0.f;
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(gv[b], xv[a], acc[a][b]);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 8; ++b)
                if (ci0 + a < Ci && co0 + b < Co)
                    atomicAdd(dW + (((size_t)(co0 + b) * Ci + ci0 + a) * 9 + tap), acc[a][b]);
    }
    if (t < Co) {
        float s = 0.f;
        for (int p = 0; p < kT * kT; ++p) s += gt[p * CoP + t];
        atomicAdd(db + t, s);
    }
}

// Smooth-L1 (beta = 1) over out - target, mean over all elements; writes the
// bf16 output gradient and adds the loss (already divided by the count).
__global__ void net_loss(const float *out, const float *target, long long n, __nv_bfloat16 *g, double *loss) {
    double part = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float d = out[i] - target[i];
        const float a = fabsf(d);
        part += a < 1.f ? 0.5 * (double)d * d : (double)a - 0.5;
        const float gr = (a < 1.f ? d : copysignf(1.f, d)) / (float)n;
        g[i] = f2bf(gr);
    }
    __shared__ double red[32];
    for (int d = 16; d >= 1; d >>= 1) part += __shfl_xor_sync(0xffffffffu, part, d);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        atomicAdd(loss, s / (double)n);
    }
}

// Adam on the float32 master parameters.
__global__ void net_adam(float *p, const float *g, float *m, float *v, long long n, float lr, float b1, float b2,
                         float eps, float c1, float c2) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// Network input [H][W][5] bf16: I0 / 255, I1 / 255, the winner-take-all label
// coordinates (centred, / scale) and the winner-take-all cost / cmax.
__global__ void net_features(const uint8_t *I0, const uint8_t *I1, const int *wta_q, const int *wta_cost, int W, int H,
                             int Q0, int Q1, float scale, float cmax, __nv_bfloat16 *out) {
    const int n = W * H;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int q = wta_q[i];
        const float q0 = (float)(q % Q0) - 0.5f * (Q0 - 1), q1 = (float)(q / Q0) - 0.5f * (Q1 - 1);
        __nv_bfloat16 *o = out + (size_t)i * 5;
        o[0] = f2bf(I0[i] / 255.f);
        o[1] = f2bf(I1[i] / 255.f);
        o[2] = f2bf(q0 / scale);
        o[3] = f2bf(q1 / scale);
        o[4] = f2bf(wta_cost[i] / cmax);
    }
}

// Centres from the network output: label coordinates rounded to the nearest
// integer (ties away from zero) and clamped into the label space.
__global__ void net_centres(const float *out, int n, int Q0, int Q1, int *centre) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int c0 = (int)roundf(out[2 * i] + 0.5f * (Q0 - 1));
        const int c1 = (int)roundf(out[2 * i + 1] + 0.5f * (Q1 - 1));
        centre[2 * i] = min(max(c0, 0), Q0 - 1);
        centre[2 * i + 1] = min(max(c1, 0), Q1 - 1);
    }
}

// Coarse level of the proposal: 2x2 box average of an image, rounded half
// up (edge pixels repeat on odd sizes).
__global__ void pyr_down2(const uint8_t *I, int W, int H, int pitch, uint8_t *out, int Wc, int Hc) {
    const int n = Wc * Hc;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int xc = i % Wc, yc = i / Wc;
        const int x0 = min(2 * xc, W - 1), x1 = min(2 * xc + 1, W - 1);
        const int y0 = min(2 * yc, H - 1), y1 = min(2 * yc + 1, H - 1);
        const int sum = I[(size_t)y0 * pitch + x0] + I[(size_t)y0 * pitch + x1] + I[(size_t)y1 * pitch + x0] +
                        I[(size_t)y1 * pitch + x1];
        out[i] = (uint8_t)((sum + 2) >> 2);
    }
}

// Coarse labels to full resolution: pixel (x, y) takes the label of coarse
// pixel (x/2, y/2); its offsets double and are clamped into the full space.
__global__ void labels_up2(const int *lc, int Wc, int Hc, int Qc0, int vminc0, int vminc1, int W, int H, int Q0,
                           int Q1, int vmin0, int vmin1, int *out) {
    const int n = W * H;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int x = i % W, y = i / W;
        const int q = lc[min(y / 2, Hc - 1) * Wc + min(x / 2, Wc - 1)];
        const int o0 = 2 * (vminc0 + q % Qc0), o1 = 2 * (vminc1 + q / Qc0);
        const int q0 = min(max(o0 - vmin0, 0), Q0 - 1), q1 = min(max(o1 - vmin1, 0), Q1 - 1);
        out[i] = q0 + Q0 * q1;
    }
}

// Network input from a labeling: I0/255, I1/255, the label's coordinates
// centred on the space's middle / scale, and its data cost (Eq. Cost_value)
// / cmax.
__global__ void net_features_lab(const uint8_t *I0, const uint8_t *I1, const int *lab, int W, int H, int pitch,
                                 int Q0, int Q1, int vmin0, int vmin1, int l2, int cmax, float scale,
                                 __nv_bfloat16 *out) {
    const int n = W * H;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int x = i % W, y = i / W;
        const int q = lab[i], q0 = q % Q0, q1 = q / Q0;
        const int xs = x + vmin0 + q0, ys = y + vmin1 + q1;
        int c = cmax;
        if (xs >= 0 && xs < W && ys >= 0 && ys < H) {
            const int d = abs((int)I1[(size_t)ys * pitch + xs] - (int)I0[(size_t)y * pitch + x]);
            c = min(l2 == 1 ? d : d * d, cmax);
        }
        __nv_bfloat16 *o = out + (size_t)i * 5;
        o[0] = f2bf(I0[(size_t)y * pitch + x] / 255.f);
        o[1] = f2bf(I1[(size_t)y * pitch + x] / 255.f);
        o[2] = f2bf(((float)q0 - 0.5f * (Q0 - 1)) / scale);
        o[3] = f2bf(((float)q1 - 0.5f * (Q1 - 1)) / scale);
        o[4] = f2bf((float)c / (float)cmax);
    }
}

// Centres as a correction of a base labeling: base coordinates plus the
// network output (label units), rounded; a correction whose larger component
// is below min_shift labels is dropped; clamped into the label space.
__global__ void net_centres_base(const float *out, const int *base, int n, int Q0, int Q1, int min_shift,
                                 int *centre) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int b0 = base[i] % Q0, b1 = base[i] / Q0;
        int r0 = (int)roundf(out[2 * i]), r1 = (int)roundf(out[2 * i + 1]);
        if (max(abs(r0), abs(r1)) < min_shift) r0 = r1 = 0;
        const int c0 = b0 + r0;
        const int c1 = b1 + r1;
        centre[2 * i] = min(max(c0, 0), Q0 - 1);
        centre[2 * i + 1] = min(max(c1, 0), Q1 - 1);
    }
}

// Training targets: label coordinates minus those of the base labeling, or
// centred on the space's middle without one (label units).
__global__ void net_targets(const int *lab, const int *base, int n, int Q0, int Q1, float *t) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float b0 = base ? (float)(base[i] % Q0) : 0.5f * (Q0 - 1);
        const float b1 = base ? (float)(base[i] / Q0) : 0.5f * (Q1 - 1);
        t[2 * i] = (float)(lab[i] % Q0) - b0;
        t[2 * i + 1] = (float)(lab[i] / Q0) - b1;
    }
}

// Pixels whose label (full-space linear index) lies on an inner edge of its
// win x win box (centre clamped into the space as the windowed solve does):
// on an edge that is not also an edge of the label space, so a better label
// may lie outside the box.  One count per launch, reduced per block.
__global__ void window_edge_count(const int *labels, const int *centre, int n, int win, int Q0, int Q1,
                                  unsigned long long *count) {
    __shared__ unsigned s_cnt;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    const int h = (win - 1) / 2;
    unsigned local = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int q = labels[i];
        const int l0 = q % Q0, l1 = q / Q0;
        const int lo0 = min(max(centre[2 * i], h), Q0 - 1 - h) - h;
        const int lo1 = min(max(centre[2 * i + 1], h), Q1 - 1 - h) - h;
        const bool e0 = (l0 == lo0 && lo0 > 0) || (l0 == lo0 + win - 1 && lo0 + win - 1 < Q0 - 1);
        const bool e1 = (l1 == lo1 && lo1 > 0) || (l1 == lo1 + win - 1 && lo1 + win - 1 < Q1 - 1);
        local += (e0 || e1) ? 1u : 0u;
    }
    local = __reduce_add_sync(0xffffffffu, local);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(&s_cnt, local);
    __syncthreads();
    if (threadIdx.x == 0 && s_cnt) atomicAdd(count, (unsigned long long)s_cnt);
}

// Winner-take-all over the full label space straight from the images (no
// cost volume): lowest-index minimum of Eq. Cost_value per pixel, summed over
// a (2 radius + 1)^2 window of pixels around it (radius 0: the plain cost),
// one warp per pixel.
__global__ void wta_kernel(CostArgs A, int radius, int *labels, int *cost) {
    const int lane = threadIdx.x & 31;
    const long long npix = (long long)A.W * A.H;
    for (long long pix = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32; pix < npix;
         pix += (long long)gridDim.x * blockDim.x / 32) {
        const int x = (int)(pix % A.W), y = (int)(pix / A.W);
        int best = 0x7fffffff, bq = 0x7fffffff;
        for (int q = lane; q < A.Q; q += 32) {
            const int q0 = q % A.Q0, q1 = (q / A.Q0) % A.Q1;
            const int o0 = A.vmin[0] + A.step[0] * q0;
            const int o1 = A.R >= 2 ? A.vmin[1] + A.step[1] * q1 : 0;
            int c = 0;
            for (int dy = -radius; dy <= radius; ++dy) {
                const int yy = min(max(y + dy, 0), A.H - 1);
                for (int dx = -radius; dx <= radius; ++dx) {
                    const int xx = min(max(x + dx, 0), A.W - 1);
                    const int xs = xx + o0, ys = yy + o1;
                    int cc = A.cmax;
                    if (xs >= 0 && xs < A.W && ys >= 0 && ys < A.H) {
                        const int d = abs((int)A.I1[(size_t)ys * A.pitch + xs] - (int)A.I0[(size_t)yy * A.pitch + xx]);
                        cc = min(A.l2 == 1 ? d : d * d, A.cmax);
                    }
                    c += cc;
                }
            }
            if (c < best) {
                best = c;
                bq = q;
            }
        }
        const int vb = __reduce_min_sync(0xffffffffu, best);
        const int qb = __reduce_min_sync(0xffffffffu, best == vb ? bq : 0x7fffffff);
        if (lane == 0) {
            labels[pix] = qb;
            if (cost) cost[pix] = vb;
        }
    }
}

// ----------------------------------------------------------------------------
// host side
// ----------------------------------------------------------------------------

namespace {
constexpr int kLayers = 6;
const int kChan[kLayers + 1] = {5, 32, 32, 32, 32, 32, 2};

long long param_offset(int l) {
    long long o = 0;
    for (int i = 0; i < l; ++i) o += (long long)kChan[i + 1] * kChan[i] * 9 + kChan[i + 1];
    return o;
}

size_t al(size_t v) { return (v + 255) / 256 * 256; }

struct NetLayout {
    size_t status;        // int: EDP_ERR_TIMEOUT when a tensor-core wait ran out
    size_t act[kLayers];  // bf16 inputs of every layer (act[0] = features)
    size_t g0, g1;        // bf16 gradient ping-pong [N][H][W][32]
    size_t wprep;         // float [9][32][32]
    size_t wtc;           // bf16 B image of a 32 -> 32 layer for the tensor-core convolution
    size_t wpart;         // float [blocks][32*32*9 + 32]: per-block weight / bias gradients
    size_t end;
};
NetLayout net_layout(long long npix) {
    NetLayout L;
    L.status = 0;
    size_t off = 256;
    for (int l = 0; l < kLayers; ++l) {
        L.act[l] = off;
        off = al(off + (size_t)npix * kChan[l] * 2);
    }
    L.g0 = off;
    off = al(off + (size_t)npix * 32 * 2);
    L.g1 = off;
    off = al(off + (size_t)npix * 32 * 2);
    L.wprep = off;
    off = al(off + 9 * 32 * 32 * 4);
    L.wtc = off;
    off = al(off + 9 * 32 * 32 * 2);
    L.wpart = off;
    off = al(off + (size_t)net_wgrad_tc_max_blocks() * net_wgrad_tc_part_floats() * 4);
    L.end = off;
    return L;
}

int conv(const __nv_bfloat16 *in, int N, int H, int W, int Cin, int Cout, const float *wf, const float *bias, int mode,
         __nv_bfloat16 *out_bf, float *out_f, const __nv_bfloat16 *act, cudaStream_t st) {
    dim3 grid((W + kT - 1) / kT, (H + kT - 1) / kT, N);
    const size_t smem = (size_t)(9 * Cin * Cout + (kT + 2) * (kT + 2) * (Cin | 1)) * 4;
    if (Cout == 32) {
        cudaFuncSetAttribute(net_conv3x3<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        net_conv3x3<32><<<grid, kT * kT, smem, st>>>(in, N, H, W, Cin, wf, bias, mode, out_bf, out_f, act);
    } else if (Cout == 2) {
        cudaFuncSetAttribute(net_conv3x3<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        net_conv3x3<2><<<grid, kT * kT, smem, st>>>(in, N, H, W, Cin, wf, bias, mode, out_bf, out_f, act);
    } else if (Cout == 5) {
        cudaFuncSetAttribute(net_conv3x3<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        net_conv3x3<5><<<grid, kT * kT, smem, st>>>(in, N, H, W, Cin, wf, bias, mode, out_bf, out_f, act);
    } else {
        return -1;
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}
}  // namespace

// 32 -> 32 convolutions on the tensor cores (1, the default) or on the CUDA
// cores (0)
int g_net_tc = 1;

long long net_param_count() { return param_offset(kLayers); }
void net_set_tensor_cores(int on) { g_net_tc = on ? 1 : 0; }
size_t net_status_offset() { return 0; }
size_t net_workspace_bytes(long long npix) { return net_layout(npix).end; }
size_t net_activation_offset(long long npix, int layer) { return net_layout(npix).act[layer]; }

int net_forward(const float *params, const void *x, int N, int H, int W, float *out, unsigned char *ws, cudaStream_t st) {
    const long long npix = (long long)N * H * W;
    const NetLayout L = net_layout(npix);
    auto *act0 = reinterpret_cast<__nv_bfloat16 *>(ws + L.act[0]);
    int *status = reinterpret_cast<int *>(ws + L.status);
    if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return -2;
    if (cudaMemcpyAsync(act0, x, (size_t)npix * 5 * 2, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return -2;
    float *wprep = reinterpret_cast<float *>(ws + L.wprep);
    for (int l = 0; l < kLayers; ++l) {
        const int Ci = kChan[l], Co = kChan[l + 1];
        const float *w = params + param_offset(l);
        const float *b = w + (long long)Co * Ci * 9;
        const auto *in = reinterpret_cast<const __nv_bfloat16 *>(ws + L.act[l]);
        if (g_net_tc && Ci == 32 && Co == 32 && l < kLayers - 1) {
            if (net_prep_tc_launch(w, 0, ws + L.wtc, st)) return -2;
            if (net_conv_tc_launch(in, N, H, W, ws + L.wtc, b, 0, ws + L.act[l + 1], nullptr, status, st)) return -2;
            continue;
        }
        net_prep_weights<<<36, 256, 0, st>>>(w, Co, Ci, 0, wprep);
        if (l < kLayers - 1) {
            auto *o = reinterpret_cast<__nv_bfloat16 *>(ws + L.act[l + 1]);
            if (conv(in, N, H, W, Ci, Co, wprep, b, 0, o, nullptr, nullptr, st)) return -2;
        } else {
            if (conv(in, N, H, W, Ci, Co, wprep, b, 1, nullptr, out, nullptr, st)) return -2;
        }
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int net_backward(const float *params, const float *out, const float *target, int N, int H, int W, float *grad,
                 double *loss, unsigned char *ws, cudaStream_t st) {
    const long long npix = (long long)N * H * W;
    const NetLayout L = net_layout(npix);
    if (cudaMemsetAsync(grad, 0, net_param_count() * 4, st) != cudaSuccess) return -2;
    if (cudaMemsetAsync(loss, 0, sizeof(double), st) != cudaSuccess) return -2;
    auto *g = reinterpret_cast<__nv_bfloat16 *>(ws + L.g0);
    auto *g2 = reinterpret_cast<__nv_bfloat16 *>(ws + L.g1);
    net_loss<<<152 * 4, 256, 0, st>>>(out, target, npix * 2, g, loss);
    float *wprep = reinterpret_cast<float *>(ws + L.wprep);
    dim3 grid((W + kT - 1) / kT, (H + kT - 1) / kT, N);
    for (int l = kLayers - 1; l >= 0; --l) {
        const int Ci = kChan[l], Co = kChan[l + 1];
        const long long po = param_offset(l);
        const auto *xin = reinterpret_cast<const __nv_bfloat16 *>(ws + L.act[l]);
        if (g_net_tc && Ci == 32 && Co == 32) {
            if (net_wgrad_tc_launch(g, xin, N, H, W, reinterpret_cast<float *>(ws + L.wpart), grad + po,
                                    reinterpret_cast<int *>(ws + L.status), st))
                return -2;
        } else {
            const size_t smw = (size_t)((kT + 2) * (kT + 2) * (Ci | 1) + kT * kT * (Co | 1)) * 4;
            cudaFuncSetAttribute(net_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smw);
            net_wgrad<<<grid, 288, smw, st>>>(g, xin, N, H, W, Ci, Co, grad + po, grad + po + (long long)Co * Ci * 9);
        }
        if (l > 0) {
            // input gradient of layer l = output gradient of layer l-1, masked by its ReLU
            if (g_net_tc && Ci == 32 && Co == 32) {
                if (net_prep_tc_launch(params + po, 1, ws + L.wtc, st)) return -2;
                if (net_conv_tc_launch(g, N, H, W, ws + L.wtc, nullptr, 2, g2, xin,
                                       reinterpret_cast<int *>(ws + L.status), st))
                    return -2;
            } else {
                net_prep_weights<<<36, 256, 0, st>>>(params + po, Co, Ci, 1, wprep);
                if (conv(g, N, H, W, Co, Ci, wprep, nullptr, 2, g2, nullptr, xin, st)) return -2;
            }
            auto *t = g;
            g = g2;
            g2 = t;
        }
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int net_adam_step(float *p, const float *g, float *m, float *v, long long n, float lr, float b1, float b2, float eps,
                  int step, cudaStream_t st) {
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    net_adam<<<152, 256, 0, st>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int net_features_launch(const uint8_t *I0, const uint8_t *I1, const int *wta_q, const int *wta_cost, int W, int H,
                        int Q0, int Q1, float scale, float cmax, void *out, cudaStream_t st) {
    net_features<<<152 * 4, 256, 0, st>>>(I0, I1, wta_q, wta_cost, W, H, Q0, Q1, scale, cmax,
                                          static_cast<__nv_bfloat16 *>(out));
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int pyr_down2_launch(const uint8_t *I, int W, int H, int pitch, uint8_t *out, cudaStream_t st) {
    pyr_down2<<<152 * 4, 256, 0, st>>>(I, W, H, pitch, out, (W + 1) / 2, (H + 1) / 2);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}
int labels_up2_launch(const int *lc, int Wc, int Hc, int Qc0, int vminc0, int vminc1, int W, int H, int Q0, int Q1,
                      int vmin0, int vmin1, int *out, cudaStream_t st) {
    labels_up2<<<152 * 4, 256, 0, st>>>(lc, Wc, Hc, Qc0, vminc0, vminc1, W, H, Q0, Q1, vmin0, vmin1, out);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}
int net_features_lab_launch(const uint8_t *I0, const uint8_t *I1, const int *lab, int W, int H, int pitch, int Q0,
                            int Q1, int vmin0, int vmin1, int l2, int cmax, float scale, void *out, cudaStream_t st) {
    net_features_lab<<<152 * 4, 256, 0, st>>>(I0, I1, lab, W, H, pitch, Q0, Q1, vmin0, vmin1, l2, cmax, scale,
                                               reinterpret_cast<__nv_bfloat16 *>(out));
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}
int net_centres_base_launch(const float *out, const int *base, int n, int Q0, int Q1, int min_shift, int *centre,
                            cudaStream_t st) {
    net_centres_base<<<152 * 4, 256, 0, st>>>(out, base, n, Q0, Q1, min_shift, centre);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}
int net_targets_launch(const int *lab, const int *base, int n, int Q0, int Q1, float *t, cudaStream_t st) {
    net_targets<<<152 * 4, 256, 0, st>>>(lab, base, n, Q0, Q1, t);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}
int net_centres_launch(const float *out, int n, int Q0, int Q1, int *centre, cudaStream_t st) {
    net_centres<<<152 * 4, 256, 0, st>>>(out, n, Q0, Q1, centre);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int window_edge_count_launch(const int *labels, const int *centre, int n, int win, int Q0, int Q1,
                             unsigned long long *count, cudaStream_t st) {
    if (cudaMemsetAsync(count, 0, sizeof(unsigned long long), st) != cudaSuccess) return -2;
    window_edge_count<<<152 * 4, 256, 0, st>>>(labels, centre, n, win, Q0, Q1, count);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int wta_launch(const CostArgs &a, int radius, int *labels, int *cost, cudaStream_t st) {
    wta_kernel<<<152 * 16, 256, 0, st>>>(a, radius, labels, cost);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace edp
