// pass_win.cu -- EDP scan pass on per-pixel label boxes (the windowed form
// used after a learned proposal), one or two label axes, box side n <= 15.
//
// Every pixel x keeps only the n^R labels of its box B(x) (origin lo(x),
// from a proposed centre clamped into the label space).  Costs, messages and
// sums are stored in the coordinates of the pixel's own box.  A message from
// x to a neighbour x' is the exact min-convolution between the two boxes,
//     m(v) = min_{u in B(x)} floor(S(x, u) / 2) + V(u, v),   v in B(x'),
// computed per label axis as in Sec. 3.2: the forward / backward sweeps
// (Eq. L_dec3, Eq. L_dec5) along the source box's line give the L1 distance
// transform D at every source position; a target coordinate t outside the
// source range takes D at the nearest source end plus lambda times the
// distance (all candidates then lie on one side).  The per-axis clip (line
// minimum + lambda g) follows each axis; the joint clip (box minimum +
// lambda g, Eq. derivation1) follows the last axis.
//
// Schedule as in pass_r1.cuh: one warp per image row, m_a in registers, m_b
// through a shared-memory mailbox inside a block and tagged records between
// blocks, C / m_c / m_d prefetched with cp.async.
#include "common.cuh"
#include "kernels.h"

namespace edp {

namespace {
constexpr int kPfW = 5;  // prefetch distance in columns
constexpr int kMbW = 4;  // mailbox ring depth
constexpr int kNMax = 16;

__device__ __forceinline__ int ldv(const int *p) { return *reinterpret_cast<const volatile int *>(p); }
__device__ __forceinline__ void stv(int *p, int v) { *reinterpret_cast<volatile int *>(p) = v; }
__device__ __forceinline__ int2 ld_rec(const int2 *p) {
    int2 r;
    asm volatile("ld.relaxed.gpu.global.v2.s32 {%0, %1}, [%2];" : "=r"(r.x), "=r"(r.y) : "l"(p) : "memory");
    return r;
}
__device__ __forceinline__ void st_rec(int2 *p, int v, int tag) {
    asm volatile("st.relaxed.gpu.global.v2.s32 [%0], {%1, %2};" ::"l"(p), "r"(v), "r"(tag) : "memory");
}

// box origin of pixel p on both axes
__device__ __forceinline__ void box_lo(const WinArgs &A, size_t pix, int &lo0, int &lo1) {
    const int h = (A.n - 1) / 2;
    int c0 = A.centre[pix * A.R];
    c0 = min(max(c0, h), A.Q0 - 1 - h);
    lo0 = c0 - h;
    lo1 = 0;
    if (A.R == 2) {
        int c1 = A.centre[pix * 2 + 1];
        c1 = min(max(c1, h), A.Q1 - 1 - h);
        lo1 = c1 - h;
    }
}

// One line of n values (stride in shared memory): L1 distance transform,
// line minimum, and the values at target coordinates t = 0..n-1 shifted by
// delta (source coordinate of target t is t + delta), clipped by the line
// minimum + cap when per_axis.  `scratch` is this lane's private n ints.
__device__ __forceinline__ void line_to_target(const int *src, int sstride, int *dst, int dstride, int n,
                                               int delta, int lam, int cap, bool per_axis, int *scratch) {
    int d[kNMax];
    int lmin = kBig;
#pragma unroll
    for (int i = 0; i < kNMax; ++i)
        if (i < n) {
            d[i] = src[i * sstride];
            lmin = min(lmin, d[i]);
        }
#pragma unroll
    for (int i = 1; i < kNMax; ++i)
        if (i < n) d[i] = min(d[i], d[i - 1] + lam);
#pragma unroll
    for (int i = kNMax - 2; i >= 0; --i)
        if (i < n - 1) d[i] = min(d[i], d[i + 1] + lam);
#pragma unroll
    for (int i = 0; i < kNMax; ++i)
        if (i < n) scratch[i] = d[i];
#pragma unroll
    for (int t = 0; t < kNMax; ++t)
        if (t < n) {
            const int u = t + delta;
            const int p = min(max(u, 0), n - 1);
            int v = scratch[p] + lam * abs(u - p);
            if (per_axis) v = min(v, lmin + cap);
            dst[t * dstride] = v;
        }
}
}  // namespace

template <int EM>
__global__ void __launch_bounds__(kMaxThreads) edp_pass_win_kernel(WinArgs A) {
    extern __shared__ __align__(16) int smem_i[];
    __shared__ int s_band;
    __shared__ volatile int s_abort;
    const int Q = A.Qw, E = A.E, W = A.W, H = A.H, NWR = A.NWR, n = A.n;
    const int Qp = 32 * E;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const size_t per_warp = (size_t)(kPfW + 1) * 3 * Qp + 6 * (size_t)Qp + 32 * kNMax;
    int *ring = smem_i + (size_t)w * per_warp;  // [kPfW+1][3][Qp]
    int *Hs = ring + (size_t)(kPfW + 1) * 3 * Qp;  // [2][Qp] halved sums
    int *T1 = Hs + 2 * Qp;                          // [2][Qp] after the first axis
    int *OUT = T1 + 2 * Qp;                         // [2][Qp] messages
    int *scr = OUT + 2 * Qp + lane * kNMax;         // per-lane scratch
    int *mbox = smem_i + (size_t)NWR * per_warp;    // [NWR][kMbW][Qp]
    int *produced = mbox + (size_t)NWR * kMbW * Qp;
    int *consumed = produced + NWR;

    const bool incx = (A.pass == 0 || A.pass == 2);
    const bool incy = (A.pass < 2);
    int *const Ma = incx ? A.M[0] : A.M[1];
    int *const Mb = incy ? A.M[2] : A.M[3];
    const int *const Mc = incx ? A.M[1] : A.M[0];
    const int *const Md = incy ? A.M[3] : A.M[2];
    const bool per_axis = (A.mode == 1);

    if (tid == 0) s_abort = (*(volatile int *)A.status != 0);
    __syncthreads();
    if (s_abort) return;

    while (true) {
        if (tid == 0) s_band = atomicAdd(A.band_counter, 1);
        if (tid < NWR) {
            produced[tid] = 0;
            consumed[tid] = 0;
        }
        __syncthreads();
        const int band = s_band;
        if (band >= A.nbands) break;
        const int r = band * NWR + w;
        if (w < NWR && r < H) {
            const int y = incy ? r : H - 1 - r;
            const bool has_next = r + 1 < H;
            const int y_next = incy ? y + 1 : y - 1;
            const bool last_in_band = (w == NWR - 1);
            const bool d_ok = A.read_d && (incy ? y + 1 < H : y - 1 >= 0);
            const size_t rowp = (size_t)y * W;
            const size_t rowpn = (size_t)(has_next ? y_next : y) * W;
            const int2 *ll_in = A.ll + (size_t)(band - 1) * W * Q;
            int2 *ll_out = A.ll + (size_t)band * W * Q;
            const int q0 = lane * E;
            auto prefetch = [&](int s) {
                if (s < W) {
                    const int x = incx ? s : W - 1 - s;
                    const bool c_ok = A.read_c && (incx ? x + 1 < W : x - 1 >= 0);
                    const size_t pix = (rowp + x) * Q;
                    int *dst = ring + (s % (kPfW + 1)) * 3 * Qp;
#pragma unroll
                    for (int i = 0; i < EM; ++i) {
                        const int q = q0 + i;
                        if (i < E && q < Q) {
                            cp_async4(dst + q, A.Cw + pix + q, true);
                            cp_async4(dst + Qp + q, Mc + pix + q, c_ok);
                            cp_async4(dst + 2 * Qp + q, Md + pix + q, d_ok);
                        }
                    }
                }
                cp_async_commit();
            };
            for (int s = 0; s < kPfW; ++s) prefetch(s);
            int ma[EM];
#pragma unroll
            for (int i = 0; i < EM; ++i) ma[i] = 0;
            long long spins = 0;
            for (int s = 0; s < W; ++s) {
                const int x = incx ? s : W - 1 - s;
                prefetch(s + kPfW);
                cp_async_wait_n<kPfW>();
                const int *src = ring + (s % (kPfW + 1)) * 3 * Qp;
                int mb[EM];
#pragma unroll
                for (int i = 0; i < EM; ++i) mb[i] = 0;
                if (r > 0) {
                    if (w > 0) {
                        if (lane == 0) {
                            spins = 0;
                            while (ldv(produced + w - 1) < s + 1) {
                                if (++spins > A.spin_limit || s_abort) {
                                    atomicCAS(A.status, 0, EDP_ERR_TIMEOUT_CODE);
                                    s_abort = 1;
                                    break;
                                }
                            }
                        }
                        __syncwarp();
                        __threadfence_block();
                        const int *mbx = mbox + ((w - 1) * kMbW + s % kMbW) * Qp;
#pragma unroll
                        for (int i = 0; i < EM; ++i)
                            if (i < E) mb[i] = ldv(mbx + q0 + i);
                        __syncwarp();
                        if (lane == 0) stv(consumed + w, s + 1);
                    } else {
                        const int2 *p = ll_in + (size_t)s * Q;
                        spins = 0;
                        while (true) {
                            bool ok = true;
#pragma unroll
                            for (int i = 0; i < EM; ++i) {
                                const int q = q0 + i;
                                if (i < E && q < Q) {
                                    const int2 t = ld_rec(p + q);
                                    mb[i] = t.x;
                                    ok = ok && (t.y == A.tag);
                                }
                            }
                            if (__all_sync(0xffffffffu, ok)) break;
                            const bool bail =
                                ++spins > A.spin_limit || s_abort || *(volatile int *)A.status != 0;
                            if (__any_sync(0xffffffffu, bail)) {
                                if (lane == 0) {
                                    atomicCAS(A.status, 0, EDP_ERR_TIMEOUT_CODE);
                                    s_abort = 1;
                                }
                                break;
                            }
                            __nanosleep(20);
                        }
                    }
                }
                __syncwarp();
                if (__any_sync(0xffffffffu, s_abort != 0)) break;
                // boxes of this pixel and of the two targets
                int lo0, lo1, la0 = 0, la1 = 0, lb0 = 0, lb1 = 0;
                box_lo(A, rowp + x, lo0, lo1);
                const int xn = incx ? x + 1 : x - 1;
                const bool has_a = (s + 1 < W);
                if (has_a) box_lo(A, rowp + xn, la0, la1);
                if (has_next) box_lo(A, rowpn + x, lb0, lb1);
                // Old messages no pass has written yet come from sums that are
                // still zero: M(0) between the two boxes, lambda times the
                // (truncated) distance from each label to the source box.
                const int xc = incx ? x + 1 : x - 1;
                const int yd = incy ? y + 1 : y - 1;
                const bool c_m0 = !A.read_c && xc >= 0 && xc < W;
                const bool d_m0 = !A.read_d && yd >= 0 && yd < H;
                int lc0 = 0, lc1 = 0, ld0 = 0, ld1 = 0;
                if (c_m0) box_lo(A, rowp + xc, lc0, lc1);
                if (d_m0) box_lo(A, (size_t)yd * W + x, ld0, ld1);
                auto m0 = [&](int q, int s0, int s1) {
                    const int a0 = lo0 + q % n, a1 = lo1 + q / n;
                    const int d0 = max(0, max(s0 - a0, a0 - (s0 + n - 1)));
                    const int d1 = A.R == 2 ? max(0, max(s1 - a1, a1 - (s1 + n - 1))) : 0;
                    if (per_axis) return min(A.lam * d0, A.capv) + min(A.lam * d1, A.capv);
                    return min(A.lam * (d0 + d1), A.capv);
                };
                // ---- sums (Eq. DP_2D_base) in this pixel's box ----
                int mina = kBig, minb = kBig;
                int so_v = kBig, so_q = 0x7fffffff;
#pragma unroll
                for (int i = 0; i < EM; ++i) {
                    const int q = q0 + i;
                    if (i < E && q < Q) {
                        const int Cv = src[q];
                        const int mc = c_m0 ? m0(q, lc0, lc1) : src[Qp + q];
                        const int md = d_m0 ? m0(q, ld0, ld1) : src[2 * Qp + q];
                        const int ha = floor_half(Cv + ma[i] + mb[i] + md - mc);
                        const int hb = floor_half(Cv + ma[i] + mb[i] + mc - md);
                        Hs[q] = ha;
                        Hs[Qp + q] = hb;
                        mina = min(mina, ha);
                        minb = min(minb, hb);
                        if (A.final_) {
                            const int so = Cv + ma[i] + mb[i] + mc + md;
                            if (so < so_v) {
                                so_v = so;
                                so_q = q;
                            }
                        }
                    }
                }
                const int ga = __reduce_min_sync(0xffffffffu, mina);
                const int gb = __reduce_min_sync(0xffffffffu, minb);
                if (A.final_) {
                    const int vbest = __reduce_min_sync(0xffffffffu, so_v);
                    const int qbest = __reduce_min_sync(0xffffffffu, so_v == vbest ? so_q : 0x7fffffff);
                    if (lane == 0) {
                        const int i0 = qbest % n, i1 = qbest / n;
                        A.labels[rowp + x] = (A.R == 1) ? lo0 + i0 : (lo0 + i0) + A.Q0 * (lo1 + i1);
                    }
                }
                __syncwarp();
                // ---- first axis: lines along axis 0, one lane per (vector, line) ----
                const int nl = (A.R == 2) ? n : 1;
                if (lane < 2 * nl) {
                    const int v = lane / nl, l = lane % nl;
                    const int delta = v == 0 ? (la0 - lo0) : (lb0 - lo0);
                    int *dst = (A.R == 2 ? T1 : OUT) + v * Qp + l * n;
                    line_to_target(Hs + v * Qp + l * n, 1, dst, 1, n, delta, A.lam, A.capv,
                                   per_axis || A.R == 1, scr);
                }
                __syncwarp();
                // ---- second axis: lines along axis 1 ----
                if (A.R == 2) {
                    if (lane < 2 * n) {
                        const int v = lane / n, t0 = lane % n;
                        const int delta = v == 0 ? (la1 - lo1) : (lb1 - lo1);
                        line_to_target(T1 + v * Qp + t0, n, OUT + v * Qp + t0, n, n, delta, A.lam, A.capv, per_axis,
                                       scr);
                    }
                    __syncwarp();
                }
                // ---- joint clip, outputs ----
                const int clipa = per_axis ? kBig : ga + A.capv;
                const int clipb = per_axis ? kBig : gb + A.capv;
                int ob[EM];
#pragma unroll
                for (int i = 0; i < EM; ++i) {
                    const int q = q0 + i;
                    ma[i] = (i < E && q < Q) ? min(OUT[q], clipa) : 0;
                    ob[i] = (i < E && q < Q) ? min(OUT[Qp + q], clipb) : 0;
                }
                __syncwarp();
                if (A.write_a && has_a) {
                    int *dst = Ma + (rowp + xn) * Q;
#pragma unroll
                    for (int i = 0; i < EM; ++i)
                        if (i < E && q0 + i < Q) dst[q0 + i] = ma[i];
                }
                if (has_next) {
                    if (A.write_b) {
                        int *dst = Mb + (rowpn + x) * Q;
#pragma unroll
                        for (int i = 0; i < EM; ++i)
                            if (i < E && q0 + i < Q) dst[q0 + i] = ob[i];
                    }
                    if (!last_in_band) {
                        if (lane == 0 && s >= kMbW) {
                            spins = 0;
                            while (ldv(consumed + w + 1) < s - kMbW + 1) {
                                if (++spins > A.spin_limit || s_abort) {
                                    atomicCAS(A.status, 0, EDP_ERR_TIMEOUT_CODE);
                                    s_abort = 1;
                                    break;
                                }
                            }
                        }
                        __syncwarp();
                        int *mbx = mbox + (w * kMbW + s % kMbW) * Qp;
#pragma unroll
                        for (int i = 0; i < EM; ++i)
                            if (i < E) stv(mbx + q0 + i, ob[i]);
                        __threadfence_block();
                        __syncwarp();
                        if (lane == 0) stv(produced + w, s + 1);
                    } else {
                        int2 *p = ll_out + (size_t)s * Q;
#pragma unroll
                        for (int i = 0; i < EM; ++i)
                            if (i < E && q0 + i < Q) st_rec(p + q0 + i, ob[i], A.tag);
                    }
                }
            }
            cp_async_wait_0();
        }
        __syncthreads();
        if (s_abort) break;
    }
}

size_t pass_win_smem(int NWR, int E) {
    const size_t Qp = 32 * (size_t)E;
    const size_t per_warp = (size_t)(kPfW + 1) * 3 * Qp + 6 * Qp + 32 * kNMax;
    return ((size_t)NWR * per_warp + (size_t)NWR * kMbW * Qp + 2 * (size_t)NWR) * 4;
}

int launch_edp_pass_win(const WinArgs &a, int threads, size_t smem, cudaStream_t st) {
    switch (a.EMt) {
#define EDP_CASE(N)                                                                          \
    case N: {                                                                                \
        auto k = edp_pass_win_kernel<N>;                                                     \
        if (smem > 48 * 1024)                                                                \
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        k<<<a.grid, threads, smem, st>>>(a);                                                 \
        break;                                                                               \
    }
        EDP_CASE(1)
        EDP_CASE(2)
        EDP_CASE(4)
        EDP_CASE(8)
#undef EDP_CASE
    default:
        return -1;
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

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
