// cost_energy.cu -- cost volume (Eq. Cost_value, Eq. Cost_cmp) and energy
// (Eq. GE_objective_function) kernels, sm_103a.
#include <cstdint>

#include "common.cuh"
#include "kernels.h"

namespace edp {

__device__ __forceinline__ int cost_term(const uint8_t *I, const uint8_t *I0, int W, int H, int pitch,
                                         int x, int y, int dx, int dy, int l2, bool &oob) {
    const int xs = x + dx, ys = y + dy;
    oob = (xs < 0 || xs >= W || ys < 0 || ys >= H);
    if (oob) return 0;
    const int d = (int)I[(size_t)ys * pitch + xs] - (int)I0[(size_t)y * pitch + x];
    const int a = d < 0 ? -d : d;
    return l2 == 1 ? a : a * a;
}

// One block-row of threads per pixel tile: blockIdx.x walks pixels, the
// threads of a block cover that pixel's labels (consecutive threads write
// consecutive labels, so the stores coalesce).  All index arithmetic is
// 32-bit; the label coordinates come from a per-label table in shared memory.
__device__ __forceinline__ void cost_body(const CostArgs &A) {
    __shared__ int s_o0[1024], s_o1[1024], s_o2[1024];
    const int npix = A.W * A.H;
    const int Q = A.Q;
    // labels are processed in chunks of up to 1024 (one offset table each)
    for (int qb = 0; qb < Q; qb += 1024) {
        const int qn = min(1024, Q - qb);
        __syncthreads();
        for (int t = threadIdx.x; t < qn; t += blockDim.x) {
            const int q = qb + t;
            const int q0 = q % A.Q0, q1 = (q / A.Q0) % A.Q1, q2 = q / (A.Q0 * A.Q1);
            s_o0[t] = A.vmin[0] + A.step[0] * q0;
            s_o1[t] = A.R >= 2 ? A.vmin[1] + A.step[1] * q1 : 0;
            s_o2[t] = A.R >= 3 ? A.vmin[2] + A.step[2] * q2 : 0;
        }
        __syncthreads();
        // element e = pix * qn + t, walked with a fixed stride: (pix, t) are
        // advanced incrementally, no division in the loop
        const long long e0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
        const long long stride = (long long)gridDim.x * blockDim.x;
        const int sp = (int)(stride / qn), st = (int)(stride % qn);
        int pix = (int)(e0 / qn), t = (int)(e0 % qn);
        int y = pix / A.W, x = pix - y * A.W;
        const int sy = sp / A.W, sx = sp - sy * A.W;
        for (; pix < npix; pix += sp, t += st, x += sx, y += sy) {
            if (t >= qn) {
                t -= qn;
                ++pix;
                ++x;
            }
            if (x >= A.W) {
                x -= A.W;
                ++y;
            }
            if (pix >= npix) break;
            const int o0 = s_o0[t], o1 = s_o1[t], o2 = s_o2[t];
            int c;
            bool oob1, oob2;
            if (A.mode == 0) {  // pair
                c = cost_term(A.I1, A.I0, A.W, A.H, A.pitch, x, y, o0, o1, A.l2, oob1);
                c = oob1 ? A.cmax : min(c, A.cmax);
            } else if (A.mode == 1) {  // pair + stereo partner on axis 2
                const int c1 = cost_term(A.I1, A.I0, A.W, A.H, A.pitch, x, y, o0, o1, A.l2, oob1);
                const int c2 = cost_term(A.I2, A.I0, A.W, A.H, A.pitch, x, y, o2, 0, A.l2, oob2);
                c = (oob1 || oob2) ? A.cmax : min(c1 + c2, A.cmax);
            } else {  // composite: C_{I0->I1}(x, o) ^ C_{I0->I2}(x, -o)
                int c1 = cost_term(A.I1, A.I0, A.W, A.H, A.pitch, x, y, o0, o1, A.l2, oob1);
                int c2 = cost_term(A.I2, A.I0, A.W, A.H, A.pitch, x, y, -o0, -o1, A.l2, oob2);
                c1 = oob1 ? A.cmax : min(c1, A.cmax);
                c2 = oob2 ? A.cmax : min(c2, A.cmax);
                c = min(c1, c2);
            }
            A.C[(size_t)pix * Q + qb + t] = c;
        }
    }
}

// C(x, o) of one entry (Eq. Cost_value / Eq. Cost_cmp), as cost_body computes it
__device__ __forceinline__ int cost_entry(const CostArgs &A, int x, int y, int o0, int o1, int o2) {
    bool oob1, oob2;
    if (A.mode == 0) {
        const int c = cost_term(A.I1, A.I0, A.W, A.H, A.pitch, x, y, o0, o1, A.l2, oob1);
        return oob1 ? A.cmax : min(c, A.cmax);
    }
    if (A.mode == 1) {
        const int c1 = cost_term(A.I1, A.I0, A.W, A.H, A.pitch, x, y, o0, o1, A.l2, oob1);
        const int c2 = cost_term(A.I2, A.I0, A.W, A.H, A.pitch, x, y, o2, 0, A.l2, oob2);
        return (oob1 || oob2) ? A.cmax : min(c1 + c2, A.cmax);
    }
    int c1 = cost_term(A.I1, A.I0, A.W, A.H, A.pitch, x, y, o0, o1, A.l2, oob1);
    int c2 = cost_term(A.I2, A.I0, A.W, A.H, A.pitch, x, y, -o0, -o1, A.l2, oob2);
    c1 = oob1 ? A.cmax : min(c1, A.cmax);
    c2 = oob2 ? A.cmax : min(c2, A.cmax);
    return min(c1, c2);
}

// Position of one entry of the flat [H][W][Q] array: pixel (x, y) and label
// coordinates (q0, q1, q2), advanced by mixed-radix increments.
struct CostPos {
    int x, y, q0, q1, q2;
};
__device__ __forceinline__ void cost_step(CostPos &p, const CostArgs &A, int d0, int d1, int d2, int dx, int dy) {
    p.q0 += d0;
    int c = p.q0 >= A.Q0;
    p.q0 -= c * A.Q0;
    p.q1 += d1 + c;
    c = p.q1 >= A.Q1;
    p.q1 -= c * A.Q1;
    p.q2 += d2 + c;
    c = p.q2 >= A.Q2;
    p.q2 -= c * A.Q2;
    p.x += dx + c;
    p.y += dy;
    if (p.x >= A.W) {
        p.x -= A.W;
        ++p.y;
    }
}

// The same cost volume with four consecutive entries of the flat array per
// thread and step, stored as one 16-byte word (the pixel boundaries need not
// be aligned: Q may be odd).  C must be 16-byte aligned.  The positions of
// the four entries follow from the first by mixed-radix increments; the pair
// cost (mode 0) is computed inline, without the per-mode dispatch.
__device__ __forceinline__ void cost_vec_body(const CostArgs &A) {
    const long long N = (long long)A.W * A.H * A.Q;
    const long long nv = N >> 2;
    const long long k0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    // per step the flat index advances by 4 stride = sp pixels + st labels
    const long long es = 4 * stride;
    const int sp = (int)(es / A.Q), st = (int)(es % A.Q);
    const int s0 = st % A.Q0, s1 = (st / A.Q0) % A.Q1, s2 = st / (A.Q0 * A.Q1);
    const int spy = sp / A.W, spx = sp - spy * A.W;
    CostPos p;
    {
        const long long e0 = 4 * k0;
        const long long pix = e0 / A.Q;
        const int q = (int)(e0 - pix * A.Q);
        p.q0 = q % A.Q0;
        p.q1 = (q / A.Q0) % A.Q1;
        p.q2 = q / (A.Q0 * A.Q1);
        p.y = (int)(pix / A.W);
        p.x = (int)(pix - (long long)p.y * A.W);
    }
    const int v1 = A.R >= 2 ? A.vmin[1] : 0, t1 = A.R >= 2 ? A.step[1] : 0;
    const int v2 = A.R >= 3 ? A.vmin[2] : 0, t2 = A.R >= 3 ? A.step[2] : 0;
    int4 *const C4 = reinterpret_cast<int4 *>(A.C);
    for (long long k = k0; k < nv; k += stride) {
        int v[4];
        CostPos e = p;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int o0 = A.vmin[0] + A.step[0] * e.q0, o1 = v1 + t1 * e.q1;
            if (A.mode == 0) {
                const int xs = e.x + o0, ys = e.y + o1;
                if (xs < 0 || xs >= A.W || ys < 0 || ys >= A.H) {
                    v[j] = A.cmax;
                } else {
                    const int d = abs((int)A.I1[(size_t)ys * A.pitch + xs] - (int)A.I0[(size_t)e.y * A.pitch + e.x]);
                    v[j] = min(A.l2 == 1 ? d : d * d, A.cmax);
                }
            } else {
                v[j] = cost_entry(A, e.x, e.y, o0, o1, v2 + t2 * e.q2);
            }
            if (j < 3) cost_step(e, A, 1, 0, 0, 0, 0);
        }
        C4[k] = make_int4(v[0], v[1], v[2], v[3]);
        cost_step(p, A, s0, s1, s2, spx, spy);
    }
    // the last N mod 4 entries
    if (k0 == 0) {
        for (long long e = nv * 4; e < N; ++e) {
            const long long pix = e / A.Q;
            const int q = (int)(e - pix * A.Q);
            const int y = (int)(pix / A.W), x = (int)(pix - (long long)y * A.W);
            const int q0 = q % A.Q0, q1 = (q / A.Q0) % A.Q1, q2 = q / (A.Q0 * A.Q1);
            A.C[e] = cost_entry(A, x, y, A.vmin[0] + A.step[0] * q0, v1 + t1 * q1, v2 + t2 * q2);
        }
    }
}

// The pair cost (mode 0) of one- and two-axis spaces whose axis 0 holds 32
// labels or more, one warp per pixel: lane l walks the pixel's labels l,
// l + 32, ... (consecutive lanes: consecutive labels, so the stores of C and
// the byte loads of one row of I1 coalesce); the label coordinates advance
// by 32 with at most one wrap of axis 0 per step.
__global__ void cost_pix_kernel(CostArgs A) {
    const int lane = threadIdx.x & 31;
    const long long npix = (long long)A.W * A.H;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const int Q = A.Q, Q0 = A.Q0;
    const int v0 = A.vmin[0], t0 = A.step[0];
    const int v1 = A.R >= 2 ? A.vmin[1] : 0, t1 = A.R >= 2 ? A.step[1] : 0;
    for (long long pix = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; pix < npix; pix += nw) {
        const int y = (int)(pix / A.W), x = (int)(pix - (long long)y * A.W);
        const int i0 = A.I0[(size_t)y * A.pitch + x];
        int q0 = lane, q1 = 0;
        int *out = A.C + pix * Q + lane;
        for (int q = lane; q < Q; q += 32, out += 32) {
            const int xs = x + v0 + t0 * q0, ys = y + v1 + t1 * q1;
            int c = A.cmax;
            if ((unsigned)xs < (unsigned)A.W && (unsigned)ys < (unsigned)A.H) {
                const int d = abs((int)A.I1[(size_t)ys * A.pitch + xs] - i0);
                c = min(A.l2 == 1 ? d : d * d, A.cmax);
            }
            *out = c;
            q0 += 32;
            if (q0 >= Q0) {
                q0 -= Q0;
                ++q1;
            }
        }
    }
}

__global__ void cost_kernel(CostArgs A) { cost_body(A); }
__global__ void cost_vec_kernel(CostArgs A) { cost_vec_body(A); }

// one launch for a wave of problems: blockIdx.y selects the problem
__global__ void cost_batched_kernel(const __grid_constant__ CostBatch B) { cost_body(B.c[blockIdx.y]); }

int launch_cost_batched(const CostBatch &a, long long max_entries, cudaStream_t st) {
    const int threads = 256;
    long long blocks = (max_entries + threads - 1) / threads;
    if (blocks > 152LL * 8) blocks = 152LL * 8;
    if (blocks < 1) blocks = 1;
    cost_batched_kernel<<<dim3((unsigned)blocks, a.n), threads, 0, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_cost(const CostArgs &a, cudaStream_t st) {
    const long long n = (long long)a.W * a.H * a.Q;
    const int threads = 256;
    if (a.mode == 0 && a.R <= 2 && a.Q0 >= 32) {  // one warp per pixel
        long long blocks = ((long long)a.W * a.H + 7) / 8;
        if (blocks > 152LL * 16) blocks = 152LL * 16;
        if (blocks < 1) blocks = 1;
        cost_pix_kernel<<<(unsigned)blocks, threads, 0, st>>>(a);
        return cudaGetLastError() == cudaSuccess ? 0 : -2;
    }
    if ((reinterpret_cast<uintptr_t>(a.C) & 15) == 0) {  // four entries per thread and step
        long long blocks = (n / 4 + threads - 1) / threads;
        if (blocks > 152LL * 8) blocks = 152LL * 8;
        if (blocks < 1) blocks = 1;
        cost_vec_kernel<<<(unsigned)blocks, threads, 0, st>>>(a);
        return cudaGetLastError() == cudaSuccess ? 0 : -2;
    }
    long long blocks = (n + threads - 1) / threads;
    if (blocks > 152LL * 16) blocks = 152LL * 16;
    if (blocks < 1) blocks = 1;
    cost_kernel<<<(unsigned)blocks, threads, 0, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

// V(q, q') of Eq. Smooth_value_t (l1 = 1 or 2).
__device__ __forceinline__ long long prior_v(int a, int b, const EnergyArgs &A) {
    const int a0 = a % A.Q0, b0 = b % A.Q0;
    const int a1 = (a / A.Q0) % A.Q1, b1 = (b / A.Q0) % A.Q1;
    const int a2 = a / (A.Q0 * A.Q1), b2 = b / (A.Q0 * A.Q1);
    int d[3] = {abs(a0 - b0), abs(a1 - b1), abs(a2 - b2)};
    const long long cap = A.l1 == 1 ? A.g : (long long)A.g * A.g;
    if (A.mode == 0) {
        long long f = 0;
        for (int r = 0; r < 3; ++r) f += A.l1 == 1 ? d[r] : (long long)d[r] * d[r];
        return (long long)A.lam * min(f, cap);
    }
    long long v = 0;
    for (int r = 0; r < 3; ++r) {
        const long long f = A.l1 == 1 ? d[r] : (long long)d[r] * d[r];
        v += (long long)A.lam * min(f, cap);
    }
    return v;
}

__device__ __forceinline__ void energy_body(const EnergyArgs &A) {
    long long e[3] = {0, 0, 0};
    const long long n = (long long)A.W * A.H;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % A.W), y = (int)(i / A.W);
        // labels outside [0, Q) are clamped so that every read stays in bounds
        const int l = min(max(A.labels[i], 0), A.Q - 1);
        if (A.C) {
            e[0] += A.C[i * A.Q + l];
        } else if (A.I1) {  // the pair cost of Eq. Cost_value from the images
            const int xs = x + A.v0 + A.t0 * (l % A.Q0), ys = y + A.v1 + A.t1 * (l / A.Q0);
            int c = A.cmax;
            if ((unsigned)xs < (unsigned)A.W && (unsigned)ys < (unsigned)A.H) {
                const int d = abs((int)A.I1[(size_t)ys * A.pitch + xs] - (int)A.I0[(size_t)y * A.pitch + x]);
                c = min(A.l2 == 1 ? d : d * d, A.cmax);
            }
            e[0] += c;
        }
        // per-edge multipliers of the locally adaptive prior (null: all 1)
        if (x + 1 < A.W) e[1] += (A.wh ? A.wh[i] : 1) * prior_v(l, min(max(A.labels[i + 1], 0), A.Q - 1), A);
        if (y + 1 < A.H) e[2] += (A.wv ? A.wv[i] : 1) * prior_v(l, min(max(A.labels[i + A.W], 0), A.Q - 1), A);
    }
    __shared__ long long red[3][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < 3; ++k) {
        long long v = e[k];
        for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
        if (lane == 0) red[k][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        long long s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[threadIdx.x][w];
        atomicAdd(reinterpret_cast<unsigned long long *>(A.out4 + threadIdx.x), (unsigned long long)s);
        atomicAdd(reinterpret_cast<unsigned long long *>(A.out4 + 3), (unsigned long long)s);
    }
}

__global__ void energy_kernel(EnergyArgs A) { energy_body(A); }

__global__ void energy_batched_kernel(const __grid_constant__ EnergyBatch B) {
    if (B.e[blockIdx.y].out4) energy_body(B.e[blockIdx.y]);
}

int launch_energy_batched(const EnergyBatch &a, long long max_pixels, cudaStream_t st) {
    const int threads = 256;
    long long blocks = (max_pixels + threads - 1) / threads;
    if (blocks > 152LL * 2) blocks = 152LL * 2;
    if (blocks < 1) blocks = 1;
    energy_batched_kernel<<<dim3((unsigned)blocks, a.n), threads, 0, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

// zero a list of device regions (control words, hand-off records, energy
// accumulators of a wave) in one launch: blockIdx.y selects the region
__global__ void zero_batched_kernel(const __grid_constant__ ZeroBatch Z) {
    unsigned char *p = static_cast<unsigned char *>(Z.ptr[blockIdx.y]);
    const size_t n = Z.bytes[blockIdx.y];
    const size_t n16 = ((reinterpret_cast<uintptr_t>(p) & 15) == 0) ? n / 16 : 0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += (size_t)gridDim.x * blockDim.x)
        reinterpret_cast<int4 *>(p)[i] = make_int4(0, 0, 0, 0);
    for (size_t i = n16 * 16 + (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        p[i] = 0;
}

int launch_zero_batched(const ZeroBatch &a, cudaStream_t st) {
    if (a.n == 0) return 0;
    zero_batched_kernel<<<dim3(64, a.n), 256, 0, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

// Per-edge multipliers of the locally adaptive prior (the text below Eq.
// Smooth_value_t: 2 lambda where the local image gradient is below 10), read
// per grid edge: an edge whose intensity step is below `thresh` gets
// `factor`, every other edge 1; entries without an edge are 1.
__global__ void edge_weights_kernel(const uint8_t *I, int W, int H, int pitch, int thresh, int factor, uint8_t *wh,
                                    uint8_t *wv) {
    const long long n = (long long)W * H;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % W), y = (int)(i / W);
        const uint8_t *p = I + (size_t)y * pitch + x;
        const int v = *p;
        wh[i] = (uint8_t)((x + 1 < W && abs((int)p[1] - v) < thresh) ? factor : 1);
        wv[i] = (uint8_t)((y + 1 < H && abs((int)p[pitch] - v) < thresh) ? factor : 1);
    }
}

int launch_edge_weights(const uint8_t *I, int W, int H, int pitch, int thresh, int factor, uint8_t *wh, uint8_t *wv,
                        cudaStream_t st) {
    const long long n = (long long)W * H;
    long long blocks = (n + 255) / 256;
    if (blocks > 152LL * 8) blocks = 152LL * 8;
    edge_weights_kernel<<<(unsigned)blocks, 256, 0, st>>>(I, W, H, pitch, thresh, factor, wh, wv);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_energy(const EnergyArgs &a, cudaStream_t st) {
    const long long n = (long long)a.W * a.H;
    const int threads = 256;
    long long blocks = (n + threads - 1) / threads;
    if (blocks > 152LL * 8) blocks = 152LL * 8;
    if (blocks < 1) blocks = 1;
    if (cudaMemsetAsync(a.out4, 0, 4 * sizeof(long long), st) != cudaSuccess) return -2;
    energy_kernel<<<(unsigned)blocks, threads, 0, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace edp
