// pass_r1.cuh -- one row band of an EDP scan pass for one label axis (Q <= 256).
//
// Sec. 4.2, Eq. DP_2D_base with the data term, messages M(floor(S_k / 2))
// stored at the receiving pixel (the arithmetic of pass_team.cuh), with a
// schedule built for the latency of the pass's wavefront: one warp owns one
// image row and keeps the message into its next pixel (m_a) in registers;
// lane j holds the E labels j*E .. j*E+E-1 of the row's current pixel.
//
// The column step is a chain of dependent instructions (the warp's own m_a
// feeds the next column), so the loop body is kept short and compact (one
// copy of it, hot in the instruction cache): C, m_c, m_d are staged kPf
// columns ahead into a shared-memory ring by cp.async from running pointers,
// the output addresses advance by one add per column, and the back-pressure
// check loads the consumer's counter only when the cached value is too old.
// What waits for the row above is: two adds, the halving, the min search M
// and the hand-off of m_b.
//
//  - m_b from the row above: inside the block a shared-memory mailbox ring
//    of "value + tag" 8-byte records (tag = column + 1; one 64-bit access
//    per record, so a tag that matches carries its value), polled until
//    every tag of the column matches, with a consumed-column counter for
//    back-pressure; between blocks the same records in global memory, one
//    per column and label, tagged with the launch.  No fence is on the path:
//    a release would also wait for this warp's earlier global stores.
//    Global message stores are issued after the hand-off.
//  - M of the truncated linear prior: per-lane forward / backward sweeps
//    (Eq. L_dec3, Eq. L_dec5), carries from the lanes within distance < g
//    (farther labels cost at least the clip value), the vector minimum by
//    redux.sync, then the clip of Eq. derivation1.
#pragma once
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace edp {

namespace {
constexpr int kPf = 7;   // prefetch distance in columns (ring of kPf + 1 slots, a power of two)
constexpr int kMb = 8;   // mailbox ring depth between rows of a block (a power of two)
static_assert(((kPf + 1) & kPf) == 0 && (kMb & (kMb - 1)) == 0, "ring sizes must be powers of two");
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ int redux_min(int v) { return __reduce_min_sync(kFull, v); }

// tagged mailbox records in shared memory: {value, tag} as one 64-bit access
__device__ __forceinline__ int2 lds_rec(const int2 *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.cta.shared.b64 %0, [%1];" : "=l"(v) : "r"((unsigned)__cvta_generic_to_shared(p)) : "memory");
    return make_int2((int)(unsigned)v, (int)(unsigned)(v >> 32));
}
__device__ __forceinline__ void sts_rec(int2 *p, int value, int tag) {
    const unsigned long long v = (unsigned long long)(unsigned)value | ((unsigned long long)(unsigned)tag << 32);
    asm volatile("st.relaxed.cta.shared.b64 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(p)), "l"(v) : "memory");
}
__device__ __forceinline__ int ld_relaxed_shared(const int *p) {
    int v;
    asm volatile("ld.relaxed.cta.shared.u32 %0, [%1];" : "=r"(v) : "r"((unsigned)__cvta_generic_to_shared(p)) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_shared(int *p, int v) {
    asm volatile("st.relaxed.cta.shared.u32 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(p)), "r"(v) : "memory");
}
__device__ __forceinline__ int2 ld_rec(const int2 *p) {
    int2 r;
    asm volatile("ld.relaxed.gpu.global.v2.s32 {%0, %1}, [%2];" : "=r"(r.x), "=r"(r.y) : "l"(p) : "memory");
    return r;
}
__device__ __forceinline__ void st_rec(int2 *p, int v, int tag) {
    asm volatile("st.relaxed.gpu.global.v2.s32 [%0], {%1, %2};" ::"l"(p), "r"(v), "r"(tag) : "memory");
}
// cp.async of a lane's E consecutive ints in chunks of V ints (V divides E);
// chunks at or past Q labels are not copied, all are zero-filled when !ok.
template <int E, int V>
__device__ __forceinline__ void cp_chunks(unsigned dst, const int *src, int q0, int Q, bool ok) {
    const int n = ok ? 4 * V : 0;
#pragma unroll
    for (int i = 0; i < E; i += V) {
        if (q0 + i < Q) {
            if constexpr (V == 4)
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst + 4 * i), "l"(src + i), "r"(n) : "memory");
            else if constexpr (V == 2)
                asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst + 4 * i), "l"(src + i), "r"(n) : "memory");
            else
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst + 4 * i), "l"(src + i), "r"(n) : "memory");
        }
    }
}
// widest chunk that divides E (message vectors: 16-byte aligned pixel
// vectors, so a lane's E-aligned run of labels is E * 4-byte aligned)
template <int E>
constexpr int msg_chunk() { return E % 4 == 0 ? 4 : (E % 2 == 0 ? 2 : 1); }
// vector shared-memory load of a lane's E consecutive ints
template <int E>
__device__ __forceinline__ void lds_vec(unsigned a, int (&v)[E]) {
    constexpr int V = msg_chunk<E>();
#pragma unroll
    for (int i = 0; i < E; i += V) {
        if constexpr (V == 4) {
            asm volatile("ld.shared.v4.s32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(v[i]), "=r"(v[i + 1]), "=r"(v[i + 2]), "=r"(v[i + 3]) : "r"(a + 4 * i));
        } else if constexpr (V == 2) {
            asm volatile("ld.shared.v2.s32 {%0, %1}, [%2];" : "=r"(v[i]), "=r"(v[i + 1]) : "r"(a + 4 * i));
        } else {
            asm volatile("ld.shared.s32 %0, [%1];" : "=r"(v[i]) : "r"(a + 4 * i));
        }
    }
}

// store of a lane's E message values (message vectors have stride Qm, a
// multiple of 4, so E-aligned chunks of a lane that starts below Q stay
// inside its pixel's vector)
template <int E>
__device__ __forceinline__ void stg_vec(int *p, const int (&v)[E], int q0, int Q) {
    constexpr int V = E % 4 == 0 ? 4 : (E % 2 == 0 ? 2 : 1);
#pragma unroll
    for (int i = 0; i < E; i += V) {
        if (q0 + i < Q) {
            if constexpr (V == 4)
                *reinterpret_cast<int4 *>(p + i) = make_int4(v[i], v[i + 1], v[i + 2], v[i + 3]);
            else if constexpr (V == 2)
                *reinterpret_cast<int2 *>(p + i) = make_int2(v[i], v[i + 1]);
            else
                p[i] = v[i];
        }
    }
}

// Truncated L1 distance transform of two row vectors a, b (E labels per
// lane) with slopes la, lb (the prior of each vector's edge), carries from
// kc <= 4 lanes on each side (full lane scan otherwise).
template <int E>
__device__ __forceinline__ void dt_pair(int (&a)[E], int (&b)[E], int lane, int la, int lb, int kc) {
    int fa[E], ba[E], fb[E], bb[E];
    fa[0] = a[0];
    fb[0] = b[0];
#pragma unroll
    for (int i = 1; i < E; ++i) {
        fa[i] = min(a[i], fa[i - 1] + la);
        fb[i] = min(b[i], fb[i - 1] + lb);
    }
    ba[E - 1] = a[E - 1];
    bb[E - 1] = b[E - 1];
#pragma unroll
    for (int i = E - 2; i >= 0; --i) {
        ba[i] = min(a[i], ba[i + 1] + la);
        bb[i] = min(b[i], bb[i + 1] + lb);
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
            const int gapa = la * ((d - 1) * E + 1), gapb = lb * ((d - 1) * E + 1);
            if (lane >= d) {
                cfa = min(cfa, t0 + gapa);
                cfb = min(cfb, t1 + gapb);
            }
            if (lane + d < 32) {
                cba = min(cba, t2 + gapa);
                cbb = min(cbb, t3 + gapb);
            }
        }
    } else {
        // min-plus prefix / suffix scans over all lanes
        int pa = fa[E - 1] - la * E * lane, pb = fb[E - 1] - lb * E * lane;
        int sa = ba[0] + la * E * lane, sb = bb[0] + lb * E * lane;
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
            cfa = xa + la * (E * (lane - 1) + 1);
            cfb = xb + lb * (E * (lane - 1) + 1);
        }
        if (lane < 31) {
            cba = ya - la * (lane * E + E - 1);
            cbb = yb - lb * (lane * E + E - 1);
        }
    }
#pragma unroll
    for (int i = 0; i < E; ++i) {
        a[i] = min(min(fa[i], cfa + la * i), min(ba[i], cba + la * (E - 1 - i)));
        b[i] = min(min(fb[i], cfb + lb * i), min(bb[i], cbb + lb * (E - 1 - i)));
    }
}

// Truncated quadratic prior (l1 = 2, Eq. M_decmp: the generalized RMS): the
// min-convolution of two row vectors a, b with la d^2, lb d^2 over the taps
// |d| < g (farther sources cost at least the clip value lambda g^2 applied
// afterwards).  The window slides one label per tap: every lane shifts its E
// values and takes the boundary value from its neighbour lane.  Positions
// past the vector hold kBig.
template <int E>
__device__ __forceinline__ void quad_pair(int (&a)[E], int (&b)[E], int lane, int la, int lb, int g) {
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
        const int wa = la * d * d, wb = lb * d * d;
#pragma unroll
        for (int i = 0; i < E; ++i) {
            oa[i] = min(oa[i], min(ua[i], da[i]) + wa);
            ob[i] = min(ob[i], min(ub[i], db[i]) + wb);
        }
    }
#pragma unroll
    for (int i = 0; i < E; ++i) {
        a[i] = oa[i];
        b[i] = ob[i];
    }
}

}  // namespace

// One row band (NWR rows, one warp each) of one scan pass, or of two passes
// that share the vertical direction (A.pair: P1 then P2, or P3 then P4).  A
// paired sweep runs 2W columns per row: the first half is pass A.pass from
// left to right, the second half pass A.pass + 1 from right to left.  This is
// the same Gauss-Seidel order as two separate passes: pixel (x, y) of the
// second pass reads m_{+x} of the first pass at (x - 1, y) (written by this
// lane in its first half), its own pass at (x + 1, y) and (x, y -+ 1), and
// m_{-+y} from the opposite vertical direction, which neither pass writes.
// The wavefront of the pair is H + 2W columns long instead of 2 (H + W).
// Every thread of the block calls it with the same band; returns false when
// the pass was aborted (a wait timed out).
// QUAD: the build for the truncated quadratic prior (l1 = 2).  WT: the build
// for per-edge prior multipliers A.wh / A.wv (the locally adaptive prior):
// the message into the next pixel of the row uses its horizontal edge, the
// message into the next row its vertical edge.
template <int E, bool QUAD = false, bool WT = false>
__device__ __forceinline__ bool r1_band(const PassR1Args &A, const int band, int *smem_i, volatile int *s_abort) {
    constexpr int Qp = 32 * E;  // padded vector length in shared memory
    constexpr int VM = msg_chunk<E>();
    const int Q = A.Q, W = A.W, H = A.H, NWR = A.NWR, Qm = A.Qm;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    // [NWR][kPf+1][3][Qp] staging ring, then [NWR][kMb][Qp] {value, tag} mailbox records
    int *const ring = smem_i + (size_t)w * (kPf + 1) * 3 * Qp;
    int2 *const mbox = reinterpret_cast<int2 *>(smem_i + (size_t)NWR * (kPf + 1) * 3 * Qp);
    int *const consumed = reinterpret_cast<int *>(mbox + (size_t)NWR * kMb * Qp);  // [NWR]
    const bool incy = (A.pass < 2);
    const int ncol = A.pair ? 2 * W : W;
    int *const Mb = incy ? A.M[2] : A.M[3];
    const int *const Md = incy ? A.M[3] : A.M[2];
    // no stale tag may match: records from an earlier band (or launch) are cleared
    for (int i = tid; i < NWR * kMb * Qp; i += blockDim.x) mbox[i] = make_int2(0, 0);
    if (tid < NWR) consumed[tid] = 0;
    __syncthreads();
    unsigned long long t_band0 = (A.trace && tid == 0) ? global_ns() : 0, t_wait = 0;
    const int r = band * NWR + w;
    // tag of the records from the previous band (the test hook hold_band makes
    // one band expect a tag no producer writes, so its wait runs out)
    const int tag_in = A.tag + (band == A.hold_band ? 0x20000000 : 0);
    bool aborted = false;
    if (w < NWR && r < H) {
        const int y = incy ? r : H - 1 - r;
        const bool has_next = r + 1 < H;
        const int y_next = has_next ? (incy ? y + 1 : y - 1) : y;
        const bool last_in_band = (w == NWR - 1);
        const bool d_ok = A.read_d && (incy ? y + 1 < H : y - 1 >= 0);
        const int q0 = lane * E;
        const int vw = A.vw;  // ints per C load (1, 2 or 4): divides E and Q, aligned
        const int2 *const ll_in = A.ll + (size_t)(band - 1) * ncol * Q + q0;  // previous band's last row
        int2 *const ll_out = A.ll + (size_t)band * ncol * Q + q0;
        const int2 *const mb_in = mbox + (size_t)(w - 1) * kMb * Qp + q0;  // used when w > 0
        int2 *const mb_out = mbox + (size_t)w * kMb * Qp + q0;
        const int *const Crow = A.C + (size_t)y * W * Q + q0;
        const size_t mrow = (size_t)y * W * Qm + q0;
        const int *const Mdrow = Md + mrow;
        int *const Mbrow = Mb + (size_t)y_next * W * Qm + q0;
        // The row's role is fixed for the band: FAST is the common one (a row
        // inside a block with rows above and below it, both hand-offs through
        // the shared-memory mailbox), built without the role branches.
        const bool fast_role = r > 0 && w > 0 && has_next && !last_in_band;
        auto run_row = [&](auto fast_c) {
            constexpr bool FAST = decltype(fast_c)::value;
            int cons_seen = 0;  // the consumer's progress as last read (producer side)
            const unsigned ring_s = (unsigned)__cvta_generic_to_shared(ring + q0);
            constexpr unsigned kSlot = 3 * Qp * 4;  // bytes per ring slot
            for (int h = 0; h < (A.pair ? 2 : 1) && !aborted; ++h) {
                // half h: pass A.pass + h, pixel x = incx ? xs : W - 1 - xs at column xs
                const bool incx = ((A.pass + h) & 1) == 0;
                const bool read_c = h ? A.read_c2 : A.read_c;
                const bool write_a = h ? A.write_a2 : A.write_a;
                const bool write_b = (FAST || has_next) && (h ? A.write_b2 : A.write_b);
                const bool fin = h ? A.final2 : A.final_;
                const int x0 = incx ? 0 : W - 1;
                const int dC = incx ? Q : -Q, dM = incx ? Qm : -Qm;
                // running source pointers of the prefetch (column xp of the half)
                const int *pfC = Crow + (size_t)x0 * Q;
                const int *pfc = (incx ? A.M[1] : A.M[0]) + mrow + (size_t)x0 * Qm;
                const int *pfd = Mdrow + (size_t)x0 * Qm;
                int xp = 0;
                auto prefetch = [&]() {
                    if (xp < W && q0 < Q) {
                        const unsigned dst = ring_s + ((unsigned)(h * W + xp) & kPf) * kSlot;
                        if (vw == 4)
                            cp_chunks<E, (E % 4 == 0 ? 4 : 1)>(dst, pfC, q0, Q, true);
                        else if (vw == 2)
                            cp_chunks<E, (E % 2 == 0 ? 2 : 1)>(dst, pfC, q0, Q, true);
                        else
                            cp_chunks<E, 1>(dst, pfC, q0, Q, true);
                        cp_chunks<E, VM>(dst + Qp * 4, pfc, q0, Q, read_c && xp + 1 < W);
                        cp_chunks<E, VM>(dst + 2 * Qp * 4, pfd, q0, Q, d_ok);
                    }
                    cp_async_commit();
                    ++xp;
                    pfC += dC;
                    pfc += dM;
                    pfd += dM;
                };
                for (int t = 0; t < kPf; ++t) prefetch();
                // running output pointers: m_a into the next pixel, m_b into the next row
                int *pa_out = (incx ? A.M[0] : A.M[1]) + mrow + (long long)(x0 + (incx ? 1 : -1)) * Qm;
                int *pb_out = Mbrow + (size_t)x0 * Qm;
                int ma[E];
    #pragma unroll
                for (int i = 0; i < E; ++i) ma[i] = 0;
    #pragma unroll 1
                for (int xs = 0; xs < W; ++xs) {
                    const int s = h * W + xs;  // column of the launch (ring slots, mailbox tags, records)
                    prefetch();
                    cp_async_wait_n<kPf>();
                    // ---- work that does not wait for the row above ----
                    const unsigned src = ring_s + ((unsigned)s & kPf) * kSlot;
                    int cv[E], mc[E], md[E], pa[E], pb[E];
                    lds_vec<E>(src, cv);
                    lds_vec<E>(src + Qp * 4, mc);
                    lds_vec<E>(src + 2 * Qp * 4, md);
    #pragma unroll
                    for (int i = 0; i < E; ++i) {
                        pa[i] = cv[i] + ma[i] + md[i] - mc[i];
                        pb[i] = cv[i] + ma[i] + mc[i] - md[i];
                    }
                    // multipliers of this column's two outgoing edges: into the next
                    // pixel of the sweep (x, x +- 1) and into the next row (y, y -+ 1)
                    int wgt_a = 1, wgt_b = 1;
                    if constexpr (WT) {
                        const int x = incx ? xs : W - 1 - xs;
                        const int xe = (xs + 1 < W) ? (incx ? x : x - 1) : 0;  // left pixel of the edge
                        wgt_a = __ldg(A.wh + (size_t)y * W + xe);
                        wgt_b = has_next ? __ldg(A.wv + (size_t)(incy ? y : y - 1) * W + x) : 1;
                    }
                    // ---- m_b from the row above ----
                    int mb[E];
    #pragma unroll
                    for (int i = 0; i < E; ++i) mb[i] = 0;
                    if (FAST || r > 0) {
                        long long spins = 0;
                        bool bad = false;
                        const int2 *p = (FAST || w > 0) ? mb_in + (s & (kMb - 1)) * Qp : ll_in + (size_t)s * Q;
                        const int want = (FAST || w > 0) ? s + 1 : tag_in;
                        const unsigned long long tw = (!FAST && A.trace && w == 0) ? global_ns() : 0;
                        // first look straight-line (the record is usually there), then the
                        // bounded spin
                        bool ok0 = true;
                        if (FAST || w > 0) {
    #pragma unroll
                            for (int i = 0; i < E; ++i) {
                                if (q0 + i < Q) {
                                    const int2 t = lds_rec(p + i);
                                    mb[i] = t.x;
                                    ok0 = ok0 && (t.y == want);
                                }
                            }
                        } else {
    #pragma unroll
                            for (int i = 0; i < E; ++i) {
                                if (q0 + i < Q) {
                                    const int2 t = ld_rec(p + i);
                                    mb[i] = t.x;
                                    ok0 = ok0 && (t.y == want);
                                }
                            }
                        }
                        if (!__all_sync(kFull, ok0)) while (true) {
                            bool ok = true;
    #pragma unroll
                            for (int i = 0; i < E; ++i) {
                                if (q0 + i < Q) {
                                    const int2 t = (FAST || w > 0) ? lds_rec(p + i) : ld_rec(p + i);
                                    mb[i] = t.x;
                                    ok = ok && (t.y == want);
                                }
                            }
                            if (__all_sync(kFull, ok)) break;
                            if (__any_sync(kFull, ++spins > A.spin_limit || *s_abort != 0 ||
                                                      (w == 0 && *(volatile int *)A.status != 0))) {
                                bad = true;
                                break;
                            }
                            if (w == 0) __nanosleep(20);
                        }
                        if (tw) t_wait += global_ns() - tw;
                        if (bad) {
                            if (lane == 0) {
                                atomicCAS(A.status, 0, EDP_ERR_TIMEOUT_CODE);
                                *s_abort = 1;
                            }
                            aborted = true;
                            break;
                        }
                        // issued after the vote on every lane's loaded tags: the
                        // loads of the slot have returned before the producer can
                        // see this count and overwrite it
                        // (every lane stores the same count: no divergent branch)
                        if (FAST || w > 0) st_relaxed_shared(consumed + w, s + 1);
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
                    const int lam_a = WT ? A.lam * wgt_a : A.lam, lam_b = WT ? A.lam * wgt_b : A.lam;
                    if constexpr (QUAD)
                        quad_pair<E>(ha, hb, lane, lam_a, lam_b, A.g);
                    else
                        dt_pair<E>(ha, hb, lane, lam_a, lam_b, A.kc);
                    const int clipa = ga + (WT ? A.capv * wgt_a : A.capv), clipb = gb + (WT ? A.capv * wgt_b : A.capv);
    #pragma unroll
                    for (int i = 0; i < E; ++i) {
                        ha[i] = min(ha[i], clipa);
                        hb[i] = min(hb[i], clipb);
                    }
                    // ---- hand-off of m_b to the row below, then the global stores ----
                    if (FAST || has_next) {
                        if (FAST || !last_in_band) {
                            const int need = s - kMb + 1;  // the slot's previous column was read
                            if (cons_seen < need) {
                                long long spins = 0;
                                bool bad = false;
                                while (true) {
                                    cons_seen = ld_relaxed_shared(consumed + w + 1);
                                    if (__all_sync(kFull, cons_seen >= need)) break;
                                    if (__any_sync(kFull, ++spins > A.spin_limit || *s_abort != 0)) {
                                        bad = true;
                                        break;
                                    }
                                }
                                if (bad) {
                                    if (lane == 0) {
                                        atomicCAS(A.status, 0, EDP_ERR_TIMEOUT_CODE);
                                        *s_abort = 1;
                                    }
                                    aborted = true;
                                    break;
                                }
                            }
                            int2 *p = mb_out + (s & (kMb - 1)) * Qp;
    #pragma unroll
                            for (int i = 0; i < E; ++i)
                                if (q0 + i < Q) sts_rec(p + i, hb[i], s + 1);
                        } else {
                            int2 *p = ll_out + (size_t)s * Q;
    #pragma unroll
                            for (int i = 0; i < E; ++i)
                                if (q0 + i < Q) st_rec(p + i, hb[i], A.tag);
                        }
                        if (write_b) stg_vec<E>(pb_out, hb, q0, Q);
                    }
                    if (write_a && xs + 1 < W) stg_vec<E>(pa_out, ha, q0, Q);
                    pa_out += dM;
                    pb_out += dM;
                    if (fin) {
                        // marginal S_Omega = C + all four messages, lowest-index argmin
                        int sv = kBig, sq = 0x7fffffff;
    #pragma unroll
                        for (int i = 0; i < E; ++i) {
                            const int v = cv[i] + ma[i] + mc[i] + md[i] + mb[i];
                            if (q0 + i < Q && v < sv) {
                                sv = v;
                                sq = q0 + i;
                            }
                        }
                        const int vbest = redux_min(sv);
                        const int qbest = redux_min(sv == vbest ? sq : 0x7fffffff);
                        if (lane == 0) A.labels[(size_t)y * W + (incx ? xs : W - 1 - xs)] = qbest;
                    }
    #pragma unroll
                    for (int i = 0; i < E; ++i) ma[i] = ha[i];
                }
                cp_async_wait_0();
            }
        };
        if (fast_role)
            run_row(std::true_type());
        else
            run_row(std::false_type());
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

// dispatch on the labels per lane
template <typename F>
__device__ __forceinline__ bool r1_dispatch(int E, F &&f) {
    switch (E) {
    case 1: return f(std::integral_constant<int, 1>());
    case 2: return f(std::integral_constant<int, 2>());
    case 3: return f(std::integral_constant<int, 3>());
    case 4: return f(std::integral_constant<int, 4>());
    case 5: return f(std::integral_constant<int, 5>());
    case 6: return f(std::integral_constant<int, 6>());
    case 7: return f(std::integral_constant<int, 7>());
    default: return f(std::integral_constant<int, 8>());
    }
}

}  // namespace edp
