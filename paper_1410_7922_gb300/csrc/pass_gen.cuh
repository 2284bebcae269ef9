// pass_gen.cuh -- one row band of an EDP scan pass, any number of label axes.
//
// What is stored.  The paper keeps the four directional sums S_k.  Every
// use of S_k is through the message  m_k(x) = M(floor(S_k(x_k) / 2))  into
// the neighbour x of x_k (Eq. DP_2D_1, Eq. DP_2D_base), so this kernel stores
// the messages instead: M[k] at pixel x holds m_k(x), computed once by the
// pixel x_k that produces S_k(x_k).  The values are identical; what changes
// is that a pass computes the min search twice per pixel (for the two sums it
// updates) instead of four times, and reads two "old" message vectors
// instead of two sums plus their min search.
//
// A pass p updates the sums a (x direction) and b (y direction):
//   P1: a = +x, b = +y   P2: a = -x, b = +y   P3: a = +x, b = -y   P4: a = -x, b = -y
// with c = opposite(a), d = opposite(b) read from the previous passes, and
//   S_a = C + m_a + m_b + m_d - m_c,    S_b = C + m_a + m_b + m_c - m_d
// (Eq. DP_2D_base with the data term: all k except -k', minus m_{-k'}).
// The new messages M(floor(S_a / 2)) and M(floor(S_b / 2)) go to the next
// pixel of the row and to the same column of the next row.  In the last pass
// the marginal S_Omega = C + m_a + m_b + m_c + m_d and its lowest-index argmin
// (Eq. DP_2D_1, Eq. DP_2D_2) are taken at the same time: all four messages
// into a pixel are final when the last pass reaches it.
//
// Schedule.  The recursion is in place (Sec. 4.2: recursion, not iteration),
// so pixel (x, y) of a pass needs (x -/+ 1, y) and (x, y -/+ 1) of the same
// pass.  A block owns a band of RB consecutive rows (in pass order) and
// advances them in lock step, row w of the band lagging row w-1 by one column
// (a skewed wavefront inside the block; the m_b hand-off between its rows
// goes through shared memory).  Bands are taken in order from a global
// counter, so a band only ever waits for a band that an already running
// block owns; the first row of a band waits, with a bounded spin, for the
// progress counter of the previous band's last row, whose m_b vectors it
// reads from global memory.
#pragma once
#include "common.cuh"
#include "kernels.h"

namespace edp {

// One row band of one scan pass.  Every thread of the block calls it with the
// same band; returns false when the pass was aborted (a wait timed out).
template <int EM>
__device__ __forceinline__ bool gen_band(const PassArgs &A, const int band, unsigned char *smem_raw,
                                         volatile int *s_abort) {
    const int Q = A.Q, RB = A.RB, W = A.W, H = A.H;
    unsigned long long *argk = reinterpret_cast<unsigned long long *>(smem_raw);  // [RB][2]
    int *gmin = reinterpret_cast<int *>(argk + 2 * RB);                          // [RB][2 vec][2 par]
    int *msgA = gmin + 4 * RB;                                                     // [RB][Q]
    int *ringB = msgA + RB * Q;                                                    // [RB][2][Q]
    int *stg = ringB + 2 * RB * Q;                                                 // [2][RB][3][Q]
    int *tmpA = stg + 6 * RB * Q;                                                  // [RB][Q] (R >= 2)
    int *tmpB = tmpA + RB * Q;                                                     // [RB][Q]

    const bool incx = (A.pass == 0 || A.pass == 2);
    const bool incy = (A.pass < 2);
    int *const Ma = incx ? A.M[0] : A.M[1];
    int *const Mb = incy ? A.M[2] : A.M[3];
    const int *const Mc = incx ? A.M[1] : A.M[0];
    const int *const Md = incy ? A.M[3] : A.M[2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const unsigned full = 0xffffffffu;


    const AxisCfg a0 = A.ax[0];
    const int gpw0 = 32 / a0.G;
    const int j0 = lane % a0.G;

    const int r0 = band * RB;
    const int nrows = min(RB, H - r0);
    const int ngroups0 = nrows * a0.nlines;
    for (int i = tid; i < 4 * RB; i += blockDim.x) gmin[i] = kBig;
    for (int i = tid; i < 2 * RB; i += blockDim.x) argk[i] = ~0ull;
    unsigned seen = 0;  // progress of the previous band's last row seen by this warp
    unsigned long long t_band0 = 0, t_wait = 0;
    if (A.trace && tid == 0) t_band0 = global_ns();

    // Stage C, m_c, m_d of column s of every row this lane serves into
    // stg[buf]; vectors known to be zero (not written yet, or from
    // outside the image) are zero-filled.
    auto stage = [&](int t_for, int buf) {
        for (int gb = warp * gpw0; gb < ngroups0; gb += nwarps * gpw0) {
            const int gi = gb + lane / a0.G;
            if (gi >= ngroups0) continue;
            const int w = gi / a0.nlines, l = gi % a0.nlines;
            const int s = t_for - w;
            if (s < 0 || s >= W) continue;
            const int r = r0 + w;
            const int y = incy ? r : H - 1 - r;
            const int x = incx ? s : W - 1 - s;
            const bool cval = A.read_c && (incx ? x + 1 < W : x - 1 >= 0);
            const bool dval = A.read_d && (incy ? y + 1 < H : y - 1 >= 0);
            const size_t gpix = ((size_t)y * W + x) * Q;
            const int base = line_base(a0, l);
            int *dst = stg + ((size_t)(buf * RB + w) * 3) * Q;
#pragma unroll
            for (int i = 0; i < EM; ++i) {
                const int p = j0 * a0.E + i;
                if (i < a0.E && p < a0.L) {
                    const int q = base + p;
                    cp_async4(dst + q, A.C + gpix + q, true);
                    cp_async4(dst + Q + q, Mc + gpix + q, cval);
                    cp_async4(dst + 2 * Q + q, Md + gpix + q, dval);
                }
            }
        }
        cp_async_commit();
    };
    stage(0, 0);
    __syncthreads();

    const int nsteps = W + nrows;  // last row's last column at W + nrows - 2, then a drain step
    for (int t = 0; t < nsteps; ++t) {
        const int par = t & 1;
        // ---------------- phase A: sums and the axis-0 sweeps ----------------
        for (int i = tid; i < 2 * RB; i += blockDim.x) {
            gmin[(i >> 1) * 4 + (i & 1) * 2 + (par ^ 1)] = kBig;
            argk[(i >> 1) * 2 + (par ^ 1)] = ~0ull;
        }
        stage(t + 1, par ^ 1);
        cp_async_wait_1();  // this step's staged inputs (own copies) have landed
        for (int gb = warp * gpw0; gb < ngroups0; gb += nwarps * gpw0) {
            const int gi = gb + lane / a0.G;
            const bool gvalid = gi < ngroups0;
            const int w0 = gvalid ? gi / a0.nlines : 0;
            const int l0 = gvalid ? gi % a0.nlines : 0;
            const int base0 = line_base(a0, l0);
            const int r_me = r0 + w0;
            const int y_me = incy ? r_me : H - 1 - r_me;
            const bool has_next_row = (r_me + 1 < H);
            const int y_next = incy ? y_me + 1 : y_me - 1;
            const int s = t - w0;
            const bool compute = gvalid && s >= 0 && s < W;
            const bool drain = gvalid && s >= 1 && s <= W;
            const int x = incx ? s : W - 1 - s;
            // the previous band's last row must have published column t
            const bool need_glob = compute && w0 == 0 && r_me > 0;
            if (__any_sync(full, need_glob)) {
                if (lane == 0 && seen < (unsigned)(t + 1)) {
                    const unsigned long long tw = A.trace ? global_ns() : 0;
                    const long long got =
                        wait_progress(A.progress + (r0 - 1), (unsigned)(t + 1), A.spin_limit, A.status);
                    if (A.trace) t_wait += global_ns() - tw;
                    if (got < 0) {
                        atomicCAS(A.status, 0, EDP_ERR_TIMEOUT_CODE);
                        *s_abort = 1;
                    } else {
                        seen = (unsigned)got;
                    }
                }
                __syncwarp();
            }
            int ha[EM], hb[EM];
            unsigned long long okey = ~0ull;
            const size_t gpix = ((size_t)y_me * W + (compute ? x : 0)) * Q;
            const int xprev = incx ? x - 1 : x + 1;  // column of step t-1
            const int *src = stg + ((size_t)(par * RB + w0) * 3) * Q;
#pragma unroll
            for (int i = 0; i < EM; ++i) {
                const int p = j0 * a0.E + i;
                const bool in = gvalid && i < a0.E && p < a0.L;
                const int q = base0 + p;
                int ma = 0, mb = 0;
                if (in && compute) {
                    if (s > 0) ma = msgA[w0 * Q + q];
                    if (r_me > 0)
                        mb = (w0 > 0) ? ringB[((w0 - 1) * 2 + (par ^ 1)) * Q + q] : ld_cg(Mb + gpix + q);
                    // deferred global write of the m_a vector into this pixel
                    if (s > 0 && A.write_a) Ma[gpix + q] = ma;
                }
                if (in && drain && has_next_row && (A.write_b || w0 == nrows - 1)) {
                    // deferred global write of the m_b vector produced at step t-1
                    Mb[((size_t)y_next * W + xprev) * Q + q] = ringB[(w0 * 2 + (par ^ 1)) * Q + q];
                }
                if (in && compute) {
                    const int Cv = src[q], mc = src[Q + q], md = src[2 * Q + q];
                    const int sa = Cv + ma + mb + md - mc;
                    const int sb = Cv + ma + mb + mc - md;
                    ha[i] = floor_half(sa);
                    hb[i] = floor_half(sb);
                    if (A.final_) {
                        const int so = Cv + ma + mb + mc + md;
                        const unsigned long long k =
                            ((unsigned long long)((unsigned)so ^ 0x80000000u) << 32) | (unsigned)q;
                        okey = min(okey, k);
                    }
                } else {
                    ha[i] = kBig;
                    hb[i] = kBig;
                }
            }
            const int la = line_dt<EM>(ha, a0.E, a0.G, j0, A.lam);
            const int lb = line_dt<EM>(hb, a0.E, a0.G, j0, A.lam);
            if (A.final_) {
                for (int d = a0.G >> 1; d >= 1; d >>= 1)
                    okey = min(okey, (unsigned long long)__shfl_xor_sync(full, okey, d, a0.G));
            }
            if (!compute) continue;
            if (A.R == 1) {
                // one line is the whole vector: clip and emit
#pragma unroll
                for (int i = 0; i < EM; ++i) {
                    const int p = j0 * a0.E + i;
                    if (i < a0.E && p < a0.L) {
                        const int q = base0 + p;
                        msgA[w0 * Q + q] = min(ha[i], la + A.capv);
                        ringB[(w0 * 2 + par) * Q + q] = min(hb[i], lb + A.capv);
                    }
                }
                if (A.final_ && j0 == 0) A.labels[(size_t)y_me * W + x] = (int)(okey & 0xffffffffu);
            } else {
                const bool per_axis = (A.mode == 1);
#pragma unroll
                for (int i = 0; i < EM; ++i) {
                    const int p = j0 * a0.E + i;
                    if (i < a0.E && p < a0.L) {
                        const int q = base0 + p;
                        tmpA[w0 * Q + q] = per_axis ? min(ha[i], la + A.capv) : ha[i];
                        tmpB[w0 * Q + q] = per_axis ? min(hb[i], lb + A.capv) : hb[i];
                    }
                }
                if (j0 == 0) {
                    if (!per_axis) {
                        atomicMin(&gmin[w0 * 4 + 0 * 2 + par], la);
                        atomicMin(&gmin[w0 * 4 + 1 * 2 + par], lb);
                    }
                    if (A.final_) atomicMin(&argk[w0 * 2 + par], okey);
                }
            }
        }
        __syncthreads();
        if (*s_abort) goto done;
        // the last row of the band has written column t - (nrows-1) - 1 to global
        if (tid == 0) {
            const int sl = t - (nrows - 1);
            if (sl >= 1 && sl <= W && r0 + nrows < H)
                publish_progress(A.progress + (r0 + nrows - 1), (unsigned)sl);
        }
        // ---------------- phases B, C: remaining axes ----------------
        for (int r = 1; r < A.R; ++r) {
            const AxisCfg ax = A.ax[r];
            const int gpw = 32 / ax.G;
            const int ngroups = nrows * ax.nlines;
            const int jj = lane % ax.G;
            const bool last_axis = (r == A.R - 1);
            const bool per_axis = (A.mode == 1);
            for (int gb = warp * gpw; gb < ngroups; gb += nwarps * gpw) {
                const int gi = gb + lane / ax.G;
                const bool gvalid = gi < ngroups;
                const int w = gvalid ? gi / ax.nlines : 0;
                const int l = gvalid ? gi % ax.nlines : 0;
                const int s = t - w;
                const bool compute = gvalid && s >= 0 && s < W;
                const int base = line_base(ax, l);
                int va[EM], vb[EM];
#pragma unroll
                for (int i = 0; i < EM; ++i) {
                    const int p = jj * ax.E + i;
                    const bool in = compute && i < ax.E && p < ax.L;
                    const int q = base + p * ax.stride;
                    va[i] = in ? tmpA[w * Q + q] : kBig;
                    vb[i] = in ? tmpB[w * Q + q] : kBig;
                }
                const int la = line_dt<EM>(va, ax.E, ax.G, jj, A.lam);
                const int lb = line_dt<EM>(vb, ax.E, ax.G, jj, A.lam);
                if (compute) {
                    int clipa = per_axis ? la + A.capv : kBig;
                    int clipb = per_axis ? lb + A.capv : kBig;
                    if (last_axis && !per_axis) {
                        clipa = gmin[w * 4 + 0 * 2 + par] + A.capv;
                        clipb = gmin[w * 4 + 1 * 2 + par] + A.capv;
                    }
#pragma unroll
                    for (int i = 0; i < EM; ++i) {
                        const int p = jj * ax.E + i;
                        if (i < ax.E && p < ax.L) {
                            const int q = base + p * ax.stride;
                            const int oa = min(va[i], clipa), ob = min(vb[i], clipb);
                            if (last_axis) {
                                msgA[w * Q + q] = oa;
                                ringB[(w * 2 + par) * Q + q] = ob;
                            } else {
                                tmpA[w * Q + q] = oa;
                                tmpB[w * Q + q] = ob;
                            }
                        }
                    }
                }
            }
            if (last_axis && A.final_) {
                for (int w = tid; w < nrows; w += blockDim.x) {
                    const int s = t - w;
                    if (s >= 0 && s < W) {
                        const int rr = r0 + w;
                        const int yy = incy ? rr : H - 1 - rr;
                        const int xx = incx ? s : W - 1 - s;
                        A.labels[(size_t)yy * W + xx] = (int)(argk[w * 2 + par] & 0xffffffffu);
                    }
                }
            }
            __syncthreads();
        }
    }
    cp_async_wait_0();
    if (A.trace && tid == 0) {
        A.trace[band * 4 + 0] = t_band0;
        A.trace[band * 4 + 1] = global_ns();
        A.trace[band * 4 + 2] = t_wait;
        A.trace[band * 4 + 3] = sm_id();
    }
    __syncthreads();
    return true;
done:
    cp_async_wait_0();
    return false;
}

}  // namespace edp
