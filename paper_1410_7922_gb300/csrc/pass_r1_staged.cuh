// pass_r1_staged.cuh -- the one-axis band body of the batched kernel: one
// scan pass per call (no paired sweeps), C, m_c, m_d staged through a
// shared-memory ring (cp.async, kPf columns ahead) instead of a register
// ring, so that it fits beside the multi-axis bodies in the one batched
// kernel without spilling.  Same arithmetic and hand-off protocol as the
// single-problem body in pass_r1.cuh (Sec. 4.2, Eq. DP_2D_base with the data
// term, messages M(floor(S_k / 2)) stored at the receiving pixel); m_b moves
// through a shared-memory mailbox (release / acquire counters) inside the
// block and through tagged records in global memory between blocks.
#pragma once
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace edp {
namespace staged {

constexpr int kPf = 7;   // prefetch distance in columns (ring of kPf + 1)
constexpr int kMb = 8;   // mailbox ring depth between rows of a block
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ int redux_min(int v) { return __reduce_min_sync(kFull, v); }

__device__ __forceinline__ int ld_acq_shared(const int *p) {
    int v;
    asm volatile("ld.acquire.cta.shared.u32 %0, [%1];" : "=r"(v) : "r"((unsigned)__cvta_generic_to_shared(p)) : "memory");
    return v;
}
__device__ __forceinline__ void st_rel_shared(int *p, int v) {
    asm volatile("st.release.cta.shared.u32 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(p)), "r"(v) : "memory");
}
__device__ __forceinline__ int2 ld_rec(const int2 *p) {
    int2 r;
    asm volatile("ld.relaxed.gpu.global.v2.s32 {%0, %1}, [%2];" : "=r"(r.x), "=r"(r.y) : "l"(p) : "memory");
    return r;
}
__device__ __forceinline__ void st_rec(int2 *p, int v, int tag) {
    asm volatile("st.relaxed.gpu.global.v2.s32 [%0], {%1, %2};" ::"l"(p), "r"(v), "r"(tag) : "memory");
}
__device__ __forceinline__ void cp_async_bytes(int *dst, const int *src, int bytes, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const int n = valid ? bytes : 0;
    if (bytes == 16)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
    else if (bytes == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
}

// Truncated L1 distance transform of two row vectors a, b (E labels per
// lane), carries from kc <= 4 lanes on each side (full lane scan otherwise).
template <int E>
__device__ __forceinline__ void dt_pair(int (&a)[E], int (&b)[E], int lane, int lam, int kc) {
    int fa[E], ba[E], fb[E], bb[E];
    fa[0] = a[0];
    fb[0] = b[0];
#pragma unroll
    for (int i = 1; i < E; ++i) {
        fa[i] = min(a[i], fa[i - 1] + lam);
        fb[i] = min(b[i], fb[i - 1] + lam);
    }
    ba[E - 1] = a[E - 1];
    bb[E - 1] = b[E - 1];
#pragma unroll
    for (int i = E - 2; i >= 0; --i) {
        ba[i] = min(a[i], ba[i + 1] + lam);
        bb[i] = min(b[i], bb[i + 1] + lam);
    }
    int cfa = kBig, cba = kBig, cfb = kBig, cbb = kBig;
    if (kc <= 4) {
#pragma unroll
        for (int d = 1; d <= 4; ++d) {
            if (d > kc) break;
            const int t0 = __shfl_up_sync(kFull, fa[E - 1], d);
            const int t1 = __shfl_up_sync(kFull, fb[E - 1], d);
            const int t2 = __shfl_down_sync(kFull, ba[0], d);
            const int t3 = __shfl_down_sync(kFull, bb[0], d);
            const int gap = lam * ((d - 1) * E + 1);
            if (lane >= d) {
                cfa = min(cfa, t0 + gap);
                cfb = min(cfb, t1 + gap);
            }
            if (lane + d < 32) {
                cba = min(cba, t2 + gap);
                cbb = min(cbb, t3 + gap);
            }
        }
    } else {
        // min-plus prefix / suffix scans over all lanes
        int pa = fa[E - 1] - lam * E * lane, pb = fb[E - 1] - lam * E * lane;
        int sa = ba[0] + lam * E * lane, sb = bb[0] + lam * E * lane;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int t0 = __shfl_up_sync(kFull, pa, d), t1 = __shfl_up_sync(kFull, pb, d);
            const int t2 = __shfl_down_sync(kFull, sa, d), t3 = __shfl_down_sync(kFull, sb, d);
            if (lane >= d) {
                pa = min(pa, t0);
                pb = min(pb, t1);
            }
            if (lane + d < 32) {
                sa = min(sa, t2);
                sb = min(sb, t3);
            }
        }
        const int xa = __shfl_up_sync(kFull, pa, 1), xb = __shfl_up_sync(kFull, pb, 1);
        const int ya = __shfl_down_sync(kFull, sa, 1), yb = __shfl_down_sync(kFull, sb, 1);
        if (lane > 0) {
            cfa = xa + lam * (E * (lane - 1) + 1);
            cfb = xb + lam * (E * (lane - 1) + 1);
        }
        if (lane < 31) {
            cba = ya - lam * (lane * E + E - 1);
            cbb = yb - lam * (lane * E + E - 1);
        }
    }
#pragma unroll
    for (int i = 0; i < E; ++i) {
        a[i] = min(min(fa[i], cfa + lam * i), min(ba[i], cba + lam * (E - 1 - i)));
        b[i] = min(min(fb[i], cfb + lam * i), min(bb[i], cbb + lam * (E - 1 - i)));
    }
}

// Truncated quadratic prior (l1 = 2, Eq. M_decmp: the generalized RMS): the
// min-convolution of two row vectors a, b with lambda d^2 over the taps
// |d| < g (farther sources cost at least the clip value lambda g^2 applied
// afterwards).  The window slides one label per tap: every lane shifts its E
// values and takes the boundary value from its neighbour lane.  Positions
// past the vector hold kBig.
template <int E>
__device__ __forceinline__ void quad_pair(int (&a)[E], int (&b)[E], int lane, int lam, int g) {
    int oa[E], ob[E], ua[E], ub[E], da[E], db[E];
#pragma unroll
    for (int i = 0; i < E; ++i) {
        oa[i] = ua[i] = da[i] = a[i];
        ob[i] = ub[i] = db[i] = b[i];
    }
    const int dmax = min(g, 32 * E);
    for (int d = 1; d < dmax; ++d) {
        // u: value at position p + d; v: value at position p - d
        const int na = __shfl_down_sync(kFull, ua[0], 1), nb = __shfl_down_sync(kFull, ub[0], 1);
        const int pa = __shfl_up_sync(kFull, da[E - 1], 1), pb = __shfl_up_sync(kFull, db[E - 1], 1);
#pragma unroll
        for (int i = 0; i < E - 1; ++i) {
            ua[i] = ua[i + 1];
            ub[i] = ub[i + 1];
        }
        ua[E - 1] = lane < 31 ? na : kBig;
        ub[E - 1] = lane < 31 ? nb : kBig;
#pragma unroll
        for (int i = E - 1; i > 0; --i) {
            da[i] = da[i - 1];
            db[i] = db[i - 1];
        }
        da[0] = lane > 0 ? pa : kBig;
        db[0] = lane > 0 ? pb : kBig;
        const int w = lam * d * d;
#pragma unroll
        for (int i = 0; i < E; ++i) {
            oa[i] = min(oa[i], min(ua[i], da[i]) + w);
            ob[i] = min(ob[i], min(ub[i], db[i]) + w);
        }
    }
#pragma unroll
    for (int i = 0; i < E; ++i) {
        a[i] = oa[i];
        b[i] = ob[i];
    }
}

// vector shared-memory load / store of a lane's E consecutive ints
template <int E>
__device__ __forceinline__ void lds_vec(const int *p, int (&v)[E]) {
    if constexpr (E % 4 == 0) {
#pragma unroll
        for (int i = 0; i < E; i += 4) {
            const int4 t = *reinterpret_cast<const int4 *>(p + i);
            v[i] = t.x;
            v[i + 1] = t.y;
            v[i + 2] = t.z;
            v[i + 3] = t.w;
        }
    } else if constexpr (E % 2 == 0) {
#pragma unroll
        for (int i = 0; i < E; i += 2) {
            const int2 t = *reinterpret_cast<const int2 *>(p + i);
            v[i] = t.x;
            v[i + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < E; ++i) v[i] = p[i];
    }
}
template <int E>
__device__ __forceinline__ void sts_vec(int *p, const int (&v)[E]) {
    if constexpr (E % 4 == 0) {
#pragma unroll
        for (int i = 0; i < E; i += 4) *reinterpret_cast<int4 *>(p + i) = make_int4(v[i], v[i + 1], v[i + 2], v[i + 3]);
    } else if constexpr (E % 2 == 0) {
#pragma unroll
        for (int i = 0; i < E; i += 2) *reinterpret_cast<int2 *>(p + i) = make_int2(v[i], v[i + 1]);
    } else {
#pragma unroll
        for (int i = 0; i < E; ++i) p[i] = v[i];
    }
}

// One row band (NWR rows, one warp each) of one scan pass.  Every thread of
// the block calls it with the same band; returns false when the pass was
// aborted (a wait timed out).
// QUAD: the build for the truncated quadratic prior (l1 = 2).
template <int E, bool QUAD = false>
__device__ __forceinline__ bool r1_band_staged(const PassR1Args &A, const int band, int *smem_i, volatile int *s_abort) {
    const int Q = A.Q, W = A.W, H = A.H, NWR = A.NWR;
    constexpr int Qp = 32 * E;  // padded vector length in shared memory
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    int *ring = smem_i + (size_t)w * (kPf + 1) * 3 * Qp;  // [kPf+1][3][Qp] per warp
    int *mbox = smem_i + (size_t)NWR * (kPf + 1) * 3 * Qp;  // [NWR][kMb][Qp]
    int *produced = mbox + (size_t)NWR * kMb * Qp;          // [NWR]
    int *consumed = produced + NWR;                         // [NWR]
    const bool incx = (A.pass == 0 || A.pass == 2);
    const bool incy = (A.pass < 2);
    int *const Ma = incx ? A.M[0] : A.M[1];
    int *const Mb = incy ? A.M[2] : A.M[3];
    const int *const Mc = incx ? A.M[1] : A.M[0];
    const int *const Md = incy ? A.M[3] : A.M[2];
    if (tid < NWR) {
        produced[tid] = 0;
        consumed[tid] = 0;
    }
    __syncthreads();
    unsigned long long t_band0 = (A.trace && tid == 0) ? global_ns() : 0, t_wait = 0;
    const int r = band * NWR + w;
    if (w < NWR && r < H) {
        const int y = incy ? r : H - 1 - r;
        const bool has_next = r + 1 < H;
        const int y_next = incy ? y + 1 : y - 1;
        const bool last_in_band = (w == NWR - 1);
        const bool d_ok = A.read_d && (incy ? y + 1 < H : y - 1 >= 0);
        const int q0 = lane * E;
        const bool lane_on = q0 < Q;
        const int vw = A.vw;          // ints per cp.async (1, 2 or 4)
        // pixel pointers advance by +/-Q (cost) and +/-Qm (messages) per column
        const int Qm = A.Qm;
        const long long dq = incx ? Q : -Q, dqm = incx ? Qm : -Qm;
        const int *pC = A.C + ((size_t)y * W + (incx ? 0 : W - 1)) * Q + q0;
        const size_t m0 = ((size_t)y * W + (incx ? 0 : W - 1)) * Qm + q0;
        const size_t mn = ((size_t)(has_next ? y_next : y) * W + (incx ? 0 : W - 1)) * Qm + q0;
        const int *pc = Mc + m0;
        const int *pd = Md + m0;
        int *pa_out = Ma + m0;   // message into the column, written one column ahead
        int *pb_out = Mb + mn;
        const int2 *ll_in = A.ll + (size_t)(band - 1) * W * Q + q0;  // previous band's last row
        int2 *ll_out = A.ll + (size_t)band * W * Q + q0;
        const int mb_src = (w - 1) * kMb;

        auto prefetch = [&](int s) {
            if (s < W && lane_on) {
                const long long off = (long long)s * dq, offm = (long long)s * dqm;
                const int x = incx ? s : W - 1 - s;
                const bool c_ok = A.read_c && (incx ? x + 1 < W : x - 1 >= 0);
                int *dst = ring + (s % (kPf + 1)) * 3 * Qp + q0;
#pragma unroll
                for (int i = 0; i < E; i += 1) {
                    // vw divides both E and Q: a vw-chunk is wholly inside or outside the vector
                    if (i % vw || q0 + i >= Q) continue;
                    cp_async_bytes(dst + i, pC + off + i, 4 * vw, true);
                    cp_async_bytes(dst + Qp + i, pc + offm + i, 4 * vw, c_ok);
                    cp_async_bytes(dst + 2 * Qp + i, pd + offm + i, 4 * vw, d_ok);
                }
            }
            cp_async_commit();
        };
        for (int s = 0; s < kPf; ++s) prefetch(s);

        int ma[E];
#pragma unroll
        for (int i = 0; i < E; ++i) ma[i] = 0;
        for (int s = 0; s < W; ++s) {
            prefetch(s + kPf);
            cp_async_wait_n<kPf>();
            // ---- work that does not wait for the row above ----
            const int *src = ring + (s % (kPf + 1)) * 3 * Qp + q0;
            int cv[E], mc[E], md[E], pa[E], pb[E], po[E];
            lds_vec<E>(src, cv);
            lds_vec<E>(src + Qp, mc);
            lds_vec<E>(src + 2 * Qp, md);
#pragma unroll
            for (int i = 0; i < E; ++i) {
                pa[i] = cv[i] + ma[i] + md[i] - mc[i];
                pb[i] = cv[i] + ma[i] + mc[i] - md[i];
                po[i] = cv[i] + ma[i] + mc[i] + md[i];
            }
            // ---- m_b from the row above ----
            int mb[E];
#pragma unroll
            for (int i = 0; i < E; ++i) mb[i] = 0;
            if (r > 0) {
                long long spins = 0;
                if (w > 0) {
                    while (true) {
                        const bool ok = ld_acq_shared(produced + w - 1) >= s + 1;
                        if (__all_sync(kFull, ok)) break;
                        if (__any_sync(kFull, ++spins > A.spin_limit || *s_abort != 0)) {
                            if (lane == 0) {
                                atomicCAS(A.status, 0, EDP_ERR_TIMEOUT_CODE);
                                *s_abort = 1;
                            }
                            break;
                        }
                    }
                    lds_vec<E>(mbox + (mb_src + s % kMb) * Qp + q0, mb);
                    __syncwarp();
                    if (lane == 0) st_rel_shared(consumed + w, s + 1);
                } else {
                    const unsigned long long tw = A.trace ? global_ns() : 0;
                    const int2 *p = ll_in + (size_t)s * Q;
                    while (true) {
                        bool ok = true;
#pragma unroll
                        for (int i = 0; i < E; ++i) {
                            if (q0 + i < Q) {
                                const int2 t = ld_rec(p + i);
                                mb[i] = t.x;
                                ok = ok && (t.y == A.tag);
                            }
                        }
                        if (__all_sync(kFull, ok)) break;
                        if (__any_sync(kFull, ++spins > A.spin_limit || *s_abort != 0 ||
                                                  *(volatile int *)A.status != 0)) {
                            if (lane == 0) {
                                atomicCAS(A.status, 0, EDP_ERR_TIMEOUT_CODE);
                                *s_abort = 1;
                            }
                            break;
                        }
                        __nanosleep(20);
                    }
                    if (A.trace) t_wait += global_ns() - tw;
                }
                if (__any_sync(kFull, *s_abort != 0)) break;
            }
            // ---- sums (Eq. DP_2D_base), halving, min search M ----
            int ha[E], hb[E];
            int la = kBig, lb = kBig;
#pragma unroll
            for (int i = 0; i < E; ++i) {
                const bool on = q0 + i < Q;
                ha[i] = on ? floor_half(pa[i] + mb[i]) : kBig;
                hb[i] = on ? floor_half(pb[i] + mb[i]) : kBig;
                la = min(la, ha[i]);
                lb = min(lb, hb[i]);
            }
            const int ga = redux_min(la), gb = redux_min(lb);
            if constexpr (QUAD)
                quad_pair<E>(ha, hb, lane, A.lam, A.g);
            else
                dt_pair<E>(ha, hb, lane, A.lam, A.kc);
            const int clipa = ga + A.capv, clipb = gb + A.capv;
#pragma unroll
            for (int i = 0; i < E; ++i) {
                ha[i] = min(ha[i], clipa);
                hb[i] = min(hb[i], clipb);
            }
            // ---- hand-off of m_b to the row below, then the global stores ----
            if (has_next) {
                if (!last_in_band) {
                    if (s >= kMb) {
                        long long spins = 0;
                        while (true) {
                            const bool ok = ld_acq_shared(consumed + w + 1) >= s - kMb + 1;
                            if (__all_sync(kFull, ok)) break;
                            if (__any_sync(kFull, ++spins > A.spin_limit || *s_abort != 0)) {
                                if (lane == 0) {
                                    atomicCAS(A.status, 0, EDP_ERR_TIMEOUT_CODE);
                                    *s_abort = 1;
                                }
                                break;
                            }
                        }
                    }
                    sts_vec<E>(mbox + (w * kMb + s % kMb) * Qp + q0, hb);
                    __syncwarp();
                    if (lane == 0) st_rel_shared(produced + w, s + 1);
                } else {
                    int2 *p = ll_out + (size_t)s * Q;
#pragma unroll
                    for (int i = 0; i < E; ++i)
                        if (q0 + i < Q) st_rec(p + i, hb[i], A.tag);
                }
                if (A.write_b) {
                    int *p = pb_out + (long long)s * dqm;
#pragma unroll
                    for (int i = 0; i < E; ++i)
                        if (q0 + i < Q) p[i] = hb[i];
                }
            }
            if (A.write_a && s + 1 < W) {
                int *p = pa_out + (long long)(s + 1) * dqm;
#pragma unroll
                for (int i = 0; i < E; ++i)
                    if (q0 + i < Q) p[i] = ha[i];
            }
            if (A.final_) {
                // marginal S_Omega = C + all four messages, lowest-index argmin
                int sv = kBig, sq = 0x7fffffff;
#pragma unroll
                for (int i = 0; i < E; ++i) {
                    const int v = po[i] + mb[i];
                    if (q0 + i < Q && v < sv) {
                        sv = v;
                        sq = q0 + i;
                    }
                }
                const int vbest = redux_min(sv);
                const int qbest = redux_min(sv == vbest ? sq : 0x7fffffff);
                if (lane == 0) {
                    const int x = incx ? s : W - 1 - s;
                    A.labels[(size_t)y * W + x] = qbest;
                }
            }
#pragma unroll
            for (int i = 0; i < E; ++i) ma[i] = ha[i];
        }
        cp_async_wait_0();
    }
    if (A.trace && tid == 0) {
        A.trace[band * 4 + 0] = t_band0;
        A.trace[band * 4 + 1] = global_ns();
        A.trace[band * 4 + 2] = t_wait;
        A.trace[band * 4 + 3] = sm_id();
    }
    __syncthreads();
    return *s_abort == 0;
}


}  // namespace staged

}  // namespace edp
