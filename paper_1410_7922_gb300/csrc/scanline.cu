// scanline.cu -- scanline DP (Sec. 4.1) on sm_103a.
//
// Every image row is an independent chain (Eq. One_d: the vertical prior is
// zero).  Forward recurrence Eq. base,
//     S(x, q) = C(x, q) + min_q' [ S(x-1, q') + V(q', q) ],
// with S(0) = C(0) (the boundary of Eq. DP_1D_2).  The min search runs on
// 64-bit keys (S << 32 | q') through the RMS sweeps of Sec. 3.2, so every
// minimum carries the lowest label index reaching it; that index is the
// optimal-choice index stored during the forward pass (back-pointer).  The
// backward recovery starts from the lowest-index argmin of S(W-1) and follows
// the back-pointers (Sec. 4.1, Fig. 6a).
//
// A block owns RB rows and advances them together, one column per step.
//
// Min-marginal mode (the modified DP of Eq. DP_1D_3): the forward sums F and
// the backward sums B (the same recurrence run from the right end) of every
// column are stored; S_Omega(x) = M(F(x-1)) + C(x) + M(B(x+1)) = F(x) + B(x)
// - C(x), and the label is its lowest-index argmin.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace edp {

template <int EM>
__global__ void __launch_bounds__(kMaxThreads) scanline_kernel(ScanArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Q = A.Q, RB = A.RB, W = A.W, H = A.H;
    long long *gkey = reinterpret_cast<long long *>(smem_raw);  // [RB][2]
    long long *tmpk = gkey + 2 * RB;                            // [RB][Q] (R >= 2)
    int *Sv = reinterpret_cast<int *>(tmpk + (A.R >= 2 ? RB * Q : 0));  // [RB][Q]
    int *stgC = Sv + RB * Q;                                              // [2][RB][Q]
    unsigned char *sptr = reinterpret_cast<unsigned char *>(stgC + 2 * RB * Q);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const unsigned full = 0xffffffffu;
    const long long lam_k = (long long)A.lam << 32;
    const long long cap_k = (long long)A.capv << 32;
    const bool per_axis = (A.mode == 1);

    const int r0 = blockIdx.x * RB;
    const int nrows = min(RB, H - r0);
    const AxisCfg a0 = A.ax[0];
    const int gpw0 = 32 / a0.G;
    const int j0 = lane % a0.G;
    const int ngroups0 = nrows * a0.nlines;

    for (int i = tid; i < 2 * RB; i += blockDim.x) gkey[i] = kBigKey;

    auto xe = [&](int x) { return A.reverse ? W - 1 - x : x; };  // column of chain step x
    auto put_sum = [&](int w, int x, int q, int v) {
        if (A.sums) A.sums[((size_t)(r0 + w) * W + xe(x)) * Q + q] = v;
    };
    auto ptr_index = [&](int w, int x, int q) -> size_t {
        return A.ptr_in_smem ? ((size_t)w * W + x) * Q + q : ((size_t)(r0 + w) * W + x) * Q + q;
    };
    unsigned char *pbase = A.ptr_in_smem ? sptr : reinterpret_cast<unsigned char *>(A.ptr);
    auto put_ptr = [&](int w, int x, int q, unsigned v) {
        if (A.no_ptr) return;
        const size_t idx = ptr_index(w, x, q);
        if (A.ptr_bytes == 1)
            pbase[idx] = (unsigned char)v;
        else if (A.ptr_bytes == 2)
            reinterpret_cast<unsigned short *>(pbase)[idx] = (unsigned short)v;
        else
            reinterpret_cast<unsigned *>(pbase)[idx] = v;
    };
    auto get_ptr = [&](int w, int x, int q) -> unsigned {
        const size_t idx = ptr_index(w, x, q);
        if (A.ptr_bytes == 1) return pbase[idx];
        if (A.ptr_bytes == 2) return reinterpret_cast<const unsigned short *>(pbase)[idx];
        return reinterpret_cast<const unsigned *>(pbase)[idx];
    };
    // stage C(x) of every row this lane serves (the lanes of phase A)
    auto stage = [&](int x, int buf) {
        if (x < W) {
            for (int gb = warp * gpw0; gb < ngroups0; gb += nwarps * gpw0) {
                const int gi = gb + lane / a0.G;
                if (gi >= ngroups0) continue;
                const int w = gi / a0.nlines, l = gi % a0.nlines;
                const int base = line_base(a0, l);
                const size_t gpix = ((size_t)(r0 + w) * W + xe(x)) * Q;
#pragma unroll
                for (int i = 0; i < EM; ++i) {
                    const int p = j0 * a0.E + i;
                    if (i < a0.E && p < a0.L) cp_async4(stgC + (buf * RB + w) * Q + base + p, A.C + gpix + base + p, true);
                }
            }
        }
        cp_async_commit();
    };
    stage(0, 0);
    __syncthreads();

    for (int x = 0; x < W; ++x) {
        const int par = x & 1;
        for (int i = tid; i < RB; i += blockDim.x) gkey[i * 2 + (par ^ 1)] = kBigKey;
        stage(x + 1, par ^ 1);
        cp_async_wait_1();
        // ---- phase A: axis-0 lines of S(x-1) ----
        for (int gb = warp * gpw0; gb < ngroups0; gb += nwarps * gpw0) {
            const int gi = gb + lane / a0.G;
            const bool gvalid = gi < ngroups0;
            const int w0 = gvalid ? gi / a0.nlines : 0;
            const int l0 = gvalid ? gi % a0.nlines : 0;
            const int base0 = line_base(a0, l0);
            const int *cx = stgC + (par * RB + w0) * Q;
            if (x == 0) {
                if (gvalid) {
#pragma unroll
                    for (int i = 0; i < EM; ++i) {
                        const int p = j0 * a0.E + i;
                        if (i < a0.E && p < a0.L) {
                            Sv[w0 * Q + base0 + p] = cx[base0 + p];
                            put_sum(w0, 0, base0 + p, cx[base0 + p]);
                        }
                    }
                }
                continue;
            }
            long long k[EM];
#pragma unroll
            for (int i = 0; i < EM; ++i) {
                const int p = j0 * a0.E + i;
                const int q = base0 + p;
                k[i] = (gvalid && i < a0.E && p < a0.L) ? (((long long)Sv[w0 * Q + q] << 32) | (unsigned)q)
                                                        : kBigKey;
            }
            long long lmin;
            if (A.l1 == 2 && A.R == 1) {
                // truncated quadratic prior (Eq. M_decmp, l1 = 2) on one label
                // axis: the taps |d| < g on keys, read from this row's S(x - 1)
                // in shared memory (farther sources cost at least the clip)
                lmin = kBigKey;
#pragma unroll
                for (int i = 0; i < EM; ++i) lmin = min(lmin, k[i]);
                for (int d = a0.G >> 1; d >= 1; d >>= 1) lmin = min(lmin, __shfl_xor_sync(full, lmin, d, a0.G));
                const int dmax = min(A.g, a0.L);
#pragma unroll
                for (int i = 0; i < EM; ++i) {
                    const int p = j0 * a0.E + i;
                    if (!(gvalid && i < a0.E && p < a0.L)) continue;
                    long long o = k[i];
                    for (int d = 1; d < dmax; ++d) {
                        const long long w = (long long)(A.lam * d * d) << 32;
                        if (p + d < a0.L)
                            o = min(o, (((long long)Sv[w0 * Q + base0 + p + d] << 32) | (unsigned)(base0 + p + d)) + w);
                        if (p - d >= 0)
                            o = min(o, (((long long)Sv[w0 * Q + base0 + p - d] << 32) | (unsigned)(base0 + p - d)) + w);
                    }
                    k[i] = o;
                }
                __syncwarp();  // every lane of the line has read S(x - 1) before it is overwritten
            } else {
                lmin = line_dt_key<EM>(k, a0.E, a0.G, j0, lam_k);
            }
            if (!gvalid) continue;
            if (A.R == 1) {
#pragma unroll
                for (int i = 0; i < EM; ++i) {
                    const int p = j0 * a0.E + i;
                    if (i < a0.E && p < a0.L) {
                        const int q = base0 + p;
                        const long long o = min(k[i], lmin + cap_k);
                        Sv[w0 * Q + q] = cx[q] + (int)(o >> 32);
                        put_sum(w0, x, q, cx[q] + (int)(o >> 32));
                        put_ptr(w0, x, q, (unsigned)(o & 0xffffffffLL));
                    }
                }
            } else {
#pragma unroll
                for (int i = 0; i < EM; ++i) {
                    const int p = j0 * a0.E + i;
                    if (i < a0.E && p < a0.L) {
                        const int q = base0 + p;
                        tmpk[w0 * Q + q] = per_axis ? min(k[i], lmin + cap_k) : k[i];
                    }
                }
                if (!per_axis && j0 == 0) atomicMin(&gkey[w0 * 2 + par], lmin);
            }
        }
        __syncthreads();
        // ---- remaining axes ----
        if (x > 0) {
            for (int r = 1; r < A.R; ++r) {
                const AxisCfg ax = A.ax[r];
                const int gpw = 32 / ax.G;
                const int ngroups = nrows * ax.nlines;
                const int jj = lane % ax.G;
                const bool last_axis = (r == A.R - 1);
                for (int gb = warp * gpw; gb < ngroups; gb += nwarps * gpw) {
                    const int gi = gb + lane / ax.G;
                    const bool gvalid = gi < ngroups;
                    const int w = gvalid ? gi / ax.nlines : 0;
                    const int l = gvalid ? gi % ax.nlines : 0;
                    const int base = line_base(ax, l);
                    long long k[EM];
#pragma unroll
                    for (int i = 0; i < EM; ++i) {
                        const int p = jj * ax.E + i;
                        k[i] = (gvalid && i < ax.E && p < ax.L) ? tmpk[w * Q + base + p * ax.stride] : kBigKey;
                    }
                    const long long lmin = line_dt_key<EM>(k, ax.E, ax.G, jj, lam_k);
                    if (!gvalid) continue;
                    long long clip = per_axis ? lmin + cap_k : kBigKey;
                    if (last_axis && !per_axis) clip = gkey[w * 2 + par] + cap_k;
                    const int *cx = stgC + (par * RB + w) * Q;
#pragma unroll
                    for (int i = 0; i < EM; ++i) {
                        const int p = jj * ax.E + i;
                        if (i < ax.E && p < ax.L) {
                            const int q = base + p * ax.stride;
                            const long long o = min(k[i], clip);
                            if (last_axis) {
                                Sv[w * Q + q] = cx[q] + (int)(o >> 32);
                                put_sum(w, x, q, cx[q] + (int)(o >> 32));
                                put_ptr(w, x, q, (unsigned)(o & 0xffffffffLL));
                            } else {
                                tmpk[w * Q + q] = o;
                            }
                        }
                    }
                }
                __syncthreads();
            }
        }
    }
    cp_async_wait_0();
    if (A.no_ptr) return;  // min-marginal mode: the sums are the output
    // ---- argmin of S(W-1), lowest index on ties ----
    for (int i = tid; i < RB; i += blockDim.x) gkey[i * 2 + 0] = kBigKey;
    __syncthreads();
    for (int gb = warp * gpw0; gb < ngroups0; gb += nwarps * gpw0) {
        const int gi = gb + lane / a0.G;
        const bool gvalid = gi < ngroups0;
        const int w0 = gvalid ? gi / a0.nlines : 0;
        const int base0 = line_base(a0, gvalid ? gi % a0.nlines : 0);
        long long kmin = kBigKey;
        if (gvalid) {
#pragma unroll
            for (int i = 0; i < EM; ++i) {
                const int p = j0 * a0.E + i;
                if (i < a0.E && p < a0.L) {
                    const int q = base0 + p;
                    kmin = min(kmin, ((long long)Sv[w0 * Q + q] << 32) | (unsigned)q);
                }
            }
        }
        for (int d = a0.G >> 1; d >= 1; d >>= 1) kmin = min(kmin, __shfl_xor_sync(full, kmin, d, a0.G));
        if (gvalid && j0 == 0) atomicMin(&gkey[w0 * 2 + 0], kmin);
    }
    __syncthreads();
    // ---- backward recovery, one thread per row ----
    for (int w = tid; w < nrows; w += blockDim.x) {
        const long long kk = gkey[w * 2 + 0];
        unsigned lab = (unsigned)(kk & 0xffffffffLL);
        const int y = r0 + w;
        if (A.row_energy) A.row_energy[y] = (long long)(int)(kk >> 32);
        A.labels[(size_t)y * W + W - 1] = (int)lab;
        for (int x = W - 1; x >= 1; --x) {
            if (lab >= (unsigned)Q) lab = 0;  // unreachable for in-range sums; keeps reads in bounds
            lab = get_ptr(w, x, (int)lab);
            A.labels[(size_t)y * W + x - 1] = (int)lab;
        }
    }
}

// S_Omega = F + B - C and its lowest-index argmin, one warp per pixel.
__global__ void marginal_argmin_kernel(const int *C, const int *F, const int *B, long long npix, int Q, int *labels,
                                       int *marg) {
    const int lane = threadIdx.x & 31;
    for (long long pix = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32; pix < npix;
         pix += (long long)gridDim.x * blockDim.x / 32) {
        const size_t o = (size_t)pix * Q;
        int best = 0x7fffffff, bq = 0x7fffffff;
        for (int q = lane; q < Q; q += 32) {
            const int v = F[o + q] + B[o + q] - C[o + q];
            if (marg) marg[o + q] = v;
            if (v < best) {
                best = v;
                bq = q;
            }
        }
        const int vb = __reduce_min_sync(0xffffffffu, best);
        const int qb = __reduce_min_sync(0xffffffffu, best == vb ? bq : 0x7fffffff);
        if (lane == 0) labels[pix] = qb;
    }
}

int launch_marginal_argmin(const int *C, const int *F, const int *B, long long npix, int Q, int *labels, int *marg,
                           cudaStream_t st) {
    long long blocks = (npix * 32 + 255) / 256;
    if (blocks > 152LL * 16) blocks = 152LL * 16;
    marginal_argmin_kernel<<<(unsigned)std::max(1LL, blocks), 256, 0, st>>>(C, F, B, npix, Q, labels, marg);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_scanline(const ScanArgs &a, int em, int threads, size_t smem, int grid, cudaStream_t st) {
    switch (em) {
#define EDP_CASE(N)                                                                          \
    case N: {                                                                                \
        auto k = scanline_kernel<N>;                                                         \
        if (smem > 48 * 1024)                                                                \
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        k<<<grid, threads, smem, st>>>(a);                                                   \
        break;                                                                               \
    }
        EDP_CASE(2)
        EDP_CASE(4)
        EDP_CASE(8)
        EDP_CASE(16)
#undef EDP_CASE
    default:
        return -1;
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace edp
