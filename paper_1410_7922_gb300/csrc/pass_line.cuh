// pass_line.cuh -- EDP scan pass for two-axis label spaces, one label line
// per lane.
//
// Same messages, flags and pass schedule as pass_team.cuh (the kernels store
// the messages m_k(x) = M(floor(S_k(x_k) / 2)) of Eq. DP_2D_1 / DP_2D_base;
// a pass p updates the sums a (x direction) and b (y direction), with c, d
// the opposite directions read from earlier passes).  What differs is the
// mapping of the min search M onto the lanes, for label spaces of Q0 x Q1
// labels (axis 0 contiguous in the linear label index, axis 1 with stride
// Q0):
//   phase A  lane j of the row's team owns label column q0 = j, the line of
//            axis 1.  It loads C, m_c, m_d of its Q1 labels straight from
//            global memory (consecutive lanes read consecutive labels, so
//            every load is coalesced), adds m_a and m_b from shared memory,
//            halves the two sums of Eq. DP_2D_base and runs the LRMS sweeps
//            of Sec. 3.2 (Eq. L_dec5 backward, then Eq. L_dec3 forward over
//            the result) along axis 1 in registers;
//   phase B  after a transpose through shared memory, lane j owns label row
//            q1 = j, the line of axis 0, and runs the sweeps along axis 0.
// The min search is separable (the prior is a sum over axes, Eq. M_decmp),
// so the order of the axes does not change any value.  Per-axis truncation
// clips every line with its minimum + lambda f(g) after its sweeps; joint
// truncation clips the result with the vector minimum + lambda f(g)
// (Eq. derivation1).
//
// Messages leave a pixel in row layout (phase B) and enter the next one in
// column layout (phase A), so every global message store is done by the
// receiving pixel in phase A: it writes the m_a and m_b it received into the
// message arrays M[a], M[b] (coalesced), where later passes read them.
//
// Between rows.  The team of the row below gets m_b through a mailbox slot
// in shared memory (two slots per team, column parity; the slot of column s
// also holds the halved S_b sums of column s during its own phases), with
// per-warp release / acquire counters.  The first row of a block gets it from
// a ring of {value, tag} records in global memory written by the last row of
// the block above (in column layout, after a shared-memory round trip), with
// per-warp progress flags that only time the poll: the tags carry validity,
// so no fence is on the path.  Every wait is a bounded spin that sets the
// launch's status word when it runs out.
#pragma once
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace edp {
namespace line {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxWarps = 4;  // warps per team (lines of up to 128 labels)
constexpr int kMaxThreads = 384;
// control ints of one team: [0, 4) produced columns per warp (written by this
// team for the team below), [4, 8) consumed columns per warp (this team's
// slots, for the team above), [8, 12) / [12, 16) warp minima of the halved
// S_a / S_b sums, [16, 24) warp argmin keys (four 64-bit)
constexpr int kCtl = 32;

// row pitch of the [Q1][P0] buffers: odd, so that lanes owning rows hit
// distinct banks
__host__ __device__ constexpr int pitch0(int LB) { return LB | 1; }
// ints of shared memory of one team: control (first, so that its 64-bit
// words are 8-byte aligned), X_a [LA][P0], two mailbox slots; rounded up to
// 16 bytes so that every team's region starts 16-byte aligned
__host__ __device__ constexpr size_t team_ints(int LA, int LB) {
    return (kCtl + 3 * (size_t)LA * pitch0(LB) + 3) / 4 * 4;
}

__device__ __forceinline__ int ld_acq_cta(const int *p) {
    int v;
    asm volatile("ld.acquire.cta.shared.u32 %0, [%1];" : "=r"(v) : "r"((unsigned)__cvta_generic_to_shared(p)) : "memory");
    return v;
}
__device__ __forceinline__ void st_rel_cta(int *p, int v) {
    asm volatile("st.release.cta.shared.u32 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(p)), "r"(v) : "memory");
}
// {value, tag} record of another block as one 64-bit word (value in the low
// half, tag in the high half; an aligned 64-bit access is single-copy
// atomic, so a matching tag carries its value).  No memory clobber: the
// surrounding loads and stores may be scheduled around it (the tag alone
// decides whether the value is the awaited one).
__device__ __forceinline__ unsigned long long ld_rec(const int2 *p) {
    unsigned long long r;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(r) : "l"(p));
    return r;
}
__device__ __forceinline__ unsigned long long ld_rec_weak(const int2 *p) {
    return __ldcg(reinterpret_cast<const unsigned long long *>(p));
}
__device__ __forceinline__ void st_rec(int2 *p, int v, int tag) {
    const unsigned long long w = (unsigned long long)(unsigned)v | ((unsigned long long)(unsigned)tag << 32);
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(w));
}
__device__ __forceinline__ unsigned ld_relaxed_gpu(const unsigned *p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_gpu(unsigned *p, unsigned v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// L2 prefetch of the cache line holding p (inside an allocation)
__device__ __forceinline__ void prefetch_line_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }
// barrier of the TW warps of team tm (named barriers 1..NT)
__device__ __forceinline__ void team_sync(int tm, int TW) {
    if (TW == 1) {
        __syncwarp();
        return;
    }
    asm volatile("barrier.sync %0, %1;" ::"r"(tm + 1), "r"(32 * TW) : "memory");
}
__device__ __forceinline__ bool team_sync_or(int tm, int TW, bool pred) {
    if (TW == 1) return __any_sync(kFull, pred);
    int r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.s32 p, %1, 0;\n\t"
        "barrier.red.or.pred q, %2, %3, p;\n\t"
        "selp.s32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((int)pred), "r"(tm + 1), "r"(32 * TW)
        : "memory");
    return r != 0;
}
// (value, label) key of the argmin: lexicographic, lowest label on ties
__device__ __forceinline__ unsigned long long argmin_key(int v, int q) {
    return ((unsigned long long)((unsigned)v ^ 0x80000000u) << 32) | (unsigned)q;
}
__device__ __forceinline__ unsigned long long warp_min_key(unsigned long long k) {
    const unsigned hi = __reduce_min_sync(kFull, (unsigned)(k >> 32));
    const unsigned lo = __reduce_min_sync(kFull, (unsigned)(k >> 32) == hi ? (unsigned)k : 0xffffffffu);
    return ((unsigned long long)hi << 32) | lo;
}

// Truncated-L1 distance transform of one line of L labels held by one lane,
// in place: the backward sweep (Eq. L_dec5), then the forward sweep
// (Eq. L_dec3) over its result, then the clip.  A step min(h[i], h[i -/+ 1]
// + lambda) is one add-min instruction.
template <int L>
__device__ __forceinline__ void line_sweeps1(int (&h)[L], int lam, int clip) {
#pragma unroll
    for (int i = L - 2; i >= 0; --i) h[i] = __viaddmin_s32(h[i + 1], lam, h[i]);
#pragma unroll
    for (int i = 1; i < L; ++i) h[i] = __viaddmin_s32(h[i - 1], lam, h[i]);
#pragma unroll
    for (int i = 0; i < L; ++i) h[i] = min(h[i], clip);
}

// Truncated quadratic prior (l1 = 2, the generalized RMS of Eq. M_decmp) on
// one line of L labels held by one lane: h[i] <- min over the taps |d| < g of
// input[i + d] + lambda d^2 (sources farther away cost at least the clip
// lambda g^2), then the clip.  The input is read from the lane's own copy of
// the line in shared memory, src[i * st]; no other lane writes it meanwhile.
template <int L>
__device__ __forceinline__ void line_quad(int (&h)[L], const int *src, int st, int lam, int g, int clip) {
    const int dmax = min(g, L);
    for (int d = 1; d < dmax; ++d) {
        const int w = lam * d * d;
#pragma unroll
        for (int i = 0; i < L; ++i) {
            int c = kBig;
            if (i + d < L) c = src[(i + d) * st];
            if (i - d >= 0) c = min(c, src[(i - d) * st]);
            h[i] = min(h[i], c + w);
        }
    }
#pragma unroll
    for (int i = 0; i < L; ++i) h[i] = min(h[i], clip);
}

}  // namespace line

// Phase A loads of one label column (axis-1 line) of one pixel: C, the old
// messages m_c and m_d (global, coalesced across the lanes), m_a from xa and
// m_b from xb (shared memory, the lane's own column; or m_b from the record
// ring: RING), the messages this pixel received written to the message
// arrays, and the two halved sums of Eq. DP_2D_base: S_a into hv, S_b over
// m_b in xb.  xa is only read, so the column can be loaded again when a
// record was not there yet.  The global loads are issued in batches of CH
// labels, one batch ahead of the arithmetic on the previous one.  VOL: record
// loads as relaxed loads at GPU scope (the retry after a tag that did not
// match); otherwise plain L2 loads, whose tags are checked the same way.
// Returns whether every record tag matched.
template <int LA, int LB, int P0, bool RING, bool VOL>
__device__ __forceinline__ bool line_load(const int *__restrict__ Cp, const int *__restrict__ Mcp,
                                          const int *__restrict__ Mdp, int *__restrict__ Map, int *__restrict__ Mbp,
                                          const int2 *__restrict__ recp, const int *__restrict__ xa,
                                          int *__restrict__ xb, const bool c_ok, const bool d_ok, const bool has_ma,
                                          const bool mbox, const bool st_a, const bool st_b, const bool fin,
                                          const int tag, const int q0, int (&hv)[LA], int &lmin_a, int &lmin_b,
                                          unsigned long long &key) {
    constexpr int CHmax = LA > 40 ? (RING ? 6 : 10) : (RING ? 8 : 13);
    constexpr int NB = (LA + CHmax - 1) / CHmax;
    constexpr int CH = (LA + NB - 1) / NB;  // equal batches
    int cv[2][CH], mcv[2][CH], mdv[2][CH];
    unsigned long long rv[2][RING ? CH : 1];
    auto issue = [&](const int b, const int k) {
#pragma unroll
        for (int j = 0; j < CH; ++j) {
            const int i = b * CH + j;
            if (i < LA) {
                const int o = i * LB;
                // read once per pass: evict first, so the hand-off records stay in L2
                cv[k][j] = __ldcs(Cp + o);
                mcv[k][j] = c_ok ? __ldcs(Mcp + o) : 0;
                mdv[k][j] = d_ok ? __ldcs(Mdp + o) : 0;
                if constexpr (RING) rv[k][j] = VOL ? line::ld_rec(recp + o) : line::ld_rec_weak(recp + o);
            }
        }
    };
    bool ok = true;
    issue(0, 0);
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        if (b + 1 < NB) issue(b + 1, (b + 1) & 1);
        const int k = b & 1;
#pragma unroll
        for (int j = 0; j < CH; ++j) {
            const int i = b * CH + j;
            if (i < LA) {
                const int o = i * LB;  // label q = o + q0
                const int c = cv[k][j], mc = mcv[k][j], md = mdv[k][j];
                const int ma = has_ma ? xa[i * P0] : 0;
                int mb = 0;
                if constexpr (RING) {
                    mb = (int)(unsigned)rv[k][j];
                    ok = ok && (int)(unsigned)(rv[k][j] >> 32) == tag;
                } else {
                    if (mbox) mb = xb[i * P0];
                }
                // the messages this pixel received, into the message arrays
                if (st_a) __stcs(Map + o, ma);
                if (st_b) __stcs(Mbp + o, mb);
                const int t = c + ma + mb, e = md - mc;
                const int ha = floor_half(t + e), hb = floor_half(t - e);
                if (fin) key = min(key, line::argmin_key(t + mc + md, o + q0));
                hv[i] = ha;
                xb[i * P0] = hb;
                lmin_a = min(lmin_a, ha);
                lmin_b = min(lmin_b, hb);
            }
        }
    }
    return ok;
}

// One row band of one scan pass (or paired sweep) for a label space of
// LB x LA labels (axis 0: LB labels, contiguous; axis 1: LA labels).  Every
// thread of the block calls it with the same band; returns false when the
// pass was aborted (a wait timed out).
// QUAD: the build for the truncated quadratic prior (l1 = 2).
template <int LA, int LB, bool QUAD = false>
__device__ __forceinline__ bool line_band(const TeamArgs &A, const int band, int *smem, volatile int *s_abort) {
    using namespace line;
    constexpr int P0 = pitch0(LB);
    constexpr int XS = LA * P0;  // ints of one [LA][P0] buffer
    constexpr size_t TI = team_ints(LA, LB);
    const int W = A.W, H = A.H, Q = A.Q, Qm = A.Qm, TW = A.T, NT = A.NT, ring = A.ring;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tm = warp / TW, wt = warp - tm * TW, tl = wt * 32 + lane;
    for (int i = tid; i < NT * kCtl; i += blockDim.x) smem[(size_t)(i / kCtl) * TI + i % kCtl] = 0;
    __syncthreads();
    const unsigned long long t_band0 = (A.trace && tid == 0) ? global_ns() : 0;

    const int r = band * NT + tm;
    if (tm < NT && r < H) {
        const bool incy = A.pass < 2;
        int *const Mb = incy ? A.M[2] : A.M[3];
        const int *const Md = incy ? A.M[3] : A.M[2];
        const int y = incy ? r : H - 1 - r;
        const bool has_next = r + 1 < H;
        const bool to_mbox = has_next && tm + 1 < NT;
        const bool to_ring = has_next && tm + 1 == NT;
        const bool from_mbox = r > 0 && tm > 0;
        const bool from_ring = r > 0 && tm == 0;
        const bool d_ok = A.read_d && (incy ? y + 1 < H : y - 1 >= 0);
        const bool per_axis = A.mode == 1;
        int *const ctl = smem + (size_t)tm * TI;
        int *const Xa = ctl + kCtl;
        int *const nx_slots = to_mbox ? smem + (size_t)(tm + 1) * TI + kCtl + XS : nullptr;
        const int *const nx_ctl = to_mbox ? smem + (size_t)(tm + 1) * TI : nullptr;
        const int *const pv_ctl = from_mbox ? smem + (size_t)(tm - 1) * TI : nullptr;
        // record ring and progress flags between blocks: [band][ring][Qm]
        // records, [band][warp] flags and consumed counters
        const int2 *const ll_in = from_ring ? A.ll + (size_t)(band - 1) * ring * Qm : nullptr;
        int2 *const ll_out = to_ring ? A.ll + (size_t)band * ring * Qm : nullptr;
        const unsigned *const flag_in = from_ring ? A.rflag + (size_t)(band - 1) * kLineFlagStride + wt : nullptr;
        unsigned *const flag_out = to_ring ? A.rflag + (size_t)band * kLineFlagStride + wt : nullptr;
        unsigned *const cons_in = from_ring ? A.cons + (size_t)(band - 1) * kLineFlagStride + wt : nullptr;
        const unsigned *const cons_out = to_ring ? A.cons + (size_t)band * kLineFlagStride + wt : nullptr;
        // the test hook hold_band makes one band expect tags no producer writes
        const int tag_in0 = A.tag0 + (band == A.hold_band ? 0x20000000 : 0);
        const int ncol = A.pair ? 2 * W : W;
        const bool colA = tl < LB, rowB = tl < LA;
        unsigned cons_seen = 0, flag_seen = 0;
        bool aborted = false;
        for (int s = 0; s < ncol; ++s) {
            const int hh = s >= W ? 1 : 0;  // half of a paired sweep
            const int xs = s - hh * W;
            const bool incx = ((A.pass + hh) & 1) == 0;
            const bool fin = hh ? A.final2 : A.final_;
            const bool read_c = hh ? A.read_c2 : A.read_c;
            const bool write_a = hh ? A.write_a2 : A.write_a;
            const bool write_b = hh ? A.write_b2 : A.write_b;
            int *const Ma = incx ? A.M[0] : A.M[1];
            const int *const Mc = incx ? A.M[1] : A.M[0];
            const int x = incx ? xs : W - 1 - xs;
            const size_t pix = (size_t)y * W + x;
            const bool has_ma = xs > 0, nxt = xs + 1 < W;
            const bool c_ok = read_c && (incx ? x + 1 < W : x - 1 >= 0);
            int *const Xb = Xa + (1 + (s & 1)) * XS;  // this column's slot
            // L2 prefetch of the next column's inputs (C, m_c, m_d): every lane of
            // the team one 128-byte line per vector and step
            if (s + 1 < ncol) {
                const int s2 = s + 1, h2 = s2 >= W ? 1 : 0, xs2 = s2 - h2 * W;
                const bool incx2 = ((A.pass + h2) & 1) == 0;
                const int x2 = incx2 ? xs2 : W - 1 - xs2;
                const size_t p2 = (size_t)y * W + x2;
                const bool rc2 = (h2 ? A.read_c2 : A.read_c) && (incx2 ? x2 + 1 < W : x2 - 1 >= 0);
                const int *const pc = A.C + p2 * Q;
                const int *const pm = (incx2 ? A.M[1] : A.M[0]) + p2 * Qm;
                const int *const pd = Md + p2 * Qm;
                for (int o = tl * 32; o < Q; o += 32 * 32 * TW) {
                    prefetch_line_l2(pc + o);
                    if (rc2) prefetch_line_l2(pm + o);
                    if (d_ok) prefetch_line_l2(pd + o);
                }
            }
            // prior of the two outgoing edges (per-edge multipliers, or 1)
            int lam_a = A.lam, lam_b = A.lam, cap_a = A.capv, cap_b = A.capv;
            if (A.wh) {
                const int wa = nxt ? __ldg(A.wh + (size_t)y * W + (incx ? x : x - 1)) : 1;
                const int wb = has_next ? __ldg(A.wv + (size_t)(incy ? y : y - 1) * W + x) : 1;
                lam_a *= wa;
                cap_a *= wa;
                lam_b *= wb;
                cap_b *= wb;
            }

            // ---- waits (each warp for itself; warp-uniform outcomes) ----
            bool bad = false;
            long long spins = 0;
            if (from_mbox) {  // m_b of column s from every warp of the team above
                while (true) {
                    const bool ok = lane >= TW || ld_acq_cta(pv_ctl + lane) >= s + 1;
                    if (__all_sync(kFull, ok)) break;
                    if (__any_sync(kFull, ++spins > A.spin_limit || *s_abort != 0)) {
                        bad = true;
                        break;
                    }
                }
                __syncwarp();
            } else if (from_ring) {  // the producing warp's progress (times the poll only)
                while ((int)flag_seen < s + 1) {
                    flag_seen = __shfl_sync(kFull, lane == 0 ? ld_relaxed_gpu(flag_in) : 0u, 0);
                    if ((int)flag_seen >= s + 1) break;
                    if (__any_sync(kFull, ++spins > A.spin_limit || *s_abort != 0 ||
                                              ((spins & 63) == 0 && *(volatile int *)A.status != 0))) {
                        bad = true;
                        break;
                    }
                    __nanosleep(32);
                }
            }
            if (!bad && to_mbox) {  // the slot of this column in the team below is free
                spins = 0;
                while (true) {
                    const bool ok = lane >= TW || ld_acq_cta(nx_ctl + 4 + lane) >= s - 1;
                    if (__all_sync(kFull, ok)) break;
                    if (__any_sync(kFull, ++spins > A.spin_limit || *s_abort != 0)) {
                        bad = true;
                        break;
                    }
                }
            }

            // ---- phase A: sums of Eq. DP_2D_base, halving, sweeps along axis 1 ----
            unsigned long long key = ~0ull;  // final pass: (S_Omega, q) minimum
            int lmin_a = kBig, lmin_b = kBig;
            int hv[LA];
            const int tag = tag_in0 + s / ring;
            const bool st_a = write_a && has_ma, st_b = write_b && r > 0;
            const int2 *const recp = from_ring ? ll_in + (size_t)(s % ring) * Qm + tl : nullptr;
            auto load_column = [&](auto vol) -> bool {
                lmin_a = kBig;
                lmin_b = kBig;
                key = ~0ull;
                if (!colA) return true;
                if (from_ring)
                    return line_load<LA, LB, P0, true, decltype(vol)::value>(
                        A.C + pix * Q + tl, Mc + pix * Qm + tl, Md + pix * Qm + tl, Ma + pix * Qm + tl,
                        Mb + pix * Qm + tl, recp, Xa + tl, Xb + tl, c_ok, d_ok, has_ma, false, st_a, st_b, fin, tag,
                        tl, hv, lmin_a, lmin_b, key);
                return line_load<LA, LB, P0, false, false>(
                    A.C + pix * Q + tl, Mc + pix * Qm + tl, Md + pix * Qm + tl, Ma + pix * Qm + tl,
                    Mb + pix * Qm + tl, nullptr, Xa + tl, Xb + tl, c_ok, d_ok, has_ma, from_mbox, st_a, st_b, fin,
                    tag, tl, hv, lmin_a, lmin_b, key);
            };
            if (!bad) {
                bool ok = load_column(std::false_type());
                if (from_ring) {
                    // a record whose tag does not match yet: wait and load the column again
                    spins = 0;
                    while (!__all_sync(kFull, ok)) {
                        if (__any_sync(kFull, ++spins > A.spin_limit || *s_abort != 0 ||
                                                  ((spins & 15) == 0 && *(volatile int *)A.status != 0))) {
                            bad = true;
                            break;
                        }
                        __nanosleep(64);
                        ok = load_column(std::true_type());
                    }
                    // the records of this column have been read: the producer may reuse the slot
                    if (!bad && lane == 0) st_relaxed_gpu(cons_in, (unsigned)(s + 1));
                }
            }
            if (!bad && colA) {
                if constexpr (QUAD) {
                    // the taps read the column from shared memory (m_a is no longer needed)
#pragma unroll
                    for (int i = 0; i < LA; ++i) Xa[i * P0 + tl] = hv[i];
                    line_quad<LA>(hv, Xa + tl, P0, lam_a, A.g, per_axis ? lmin_a + cap_a : kBig);
                } else {
                    line_sweeps1<LA>(hv, lam_a, per_axis ? lmin_a + cap_a : kBig);
                }
#pragma unroll
                for (int i = 0; i < LA; ++i) Xa[i * P0 + tl] = hv[i];
#pragma unroll
                for (int i = 0; i < LA; ++i) hv[i] = Xb[i * P0 + tl];
                if constexpr (QUAD)
                    line_quad<LA>(hv, Xb + tl, P0, lam_b, A.g, per_axis ? lmin_b + cap_b : kBig);
                else
                    line_sweeps1<LA>(hv, lam_b, per_axis ? lmin_b + cap_b : kBig);
#pragma unroll
                for (int i = 0; i < LA; ++i) Xb[i * P0 + tl] = hv[i];
            }
            if (!per_axis) {
                const int ja = __reduce_min_sync(kFull, lmin_a), jb = __reduce_min_sync(kFull, lmin_b);
                if (lane == 0) {
                    ctl[8 + wt] = ja;
                    ctl[12 + wt] = jb;
                }
            }
            if (fin) {
                key = warp_min_key(key);
                if (lane == 0) reinterpret_cast<unsigned long long *>(ctl + 16)[wt] = key;
            }
            if (bad) {
                atomicCAS(A.status, 0, EDP_ERR_TIMEOUT_CODE);
                *s_abort = 1;
            }
            if (team_sync_or(tm, TW, bad || *s_abort != 0)) {  // barrier: phase A done
                aborted = true;
                break;
            }
            if (fin && tl == 0) {
                unsigned long long best = reinterpret_cast<unsigned long long *>(ctl + 16)[0];
                for (int w = 1; w < TW; ++w) best = min(best, reinterpret_cast<unsigned long long *>(ctl + 16)[w]);
                A.labels[pix] = (int)(best & 0xffffffffu);
            }

            // ---- phase B: sweeps along axis 0, clip, outputs ----
            if (rowB) {
                int ga = kBig, gb = kBig;  // joint truncation: minima of the halved sums
                if (!per_axis)
                    for (int w = 0; w < TW; ++w) {
                        ga = min(ga, ctl[8 + w]);
                        gb = min(gb, ctl[12 + w]);
                    }
                int *const ra = Xa + tl * P0;
                int *const rb = Xb + tl * P0;
                int gv[LB];
                int lm = kBig;
#pragma unroll
                for (int j = 0; j < LB; ++j) {
                    gv[j] = ra[j];
                    lm = min(lm, gv[j]);
                }
                if constexpr (QUAD)
                    line_quad<LB>(gv, ra, 1, lam_a, A.g, (per_axis ? lm : ga) + cap_a);
                else
                    line_sweeps1<LB>(gv, lam_a, (per_axis ? lm : ga) + cap_a);
                if (nxt) {  // m_a of the next column of the row
#pragma unroll
                    for (int j = 0; j < LB; ++j) ra[j] = gv[j];
                }
                lm = kBig;
#pragma unroll
                for (int j = 0; j < LB; ++j) {
                    gv[j] = rb[j];
                    lm = min(lm, gv[j]);
                }
                if constexpr (QUAD)
                    line_quad<LB>(gv, rb, 1, lam_b, A.g, (per_axis ? lm : gb) + cap_b);
                else
                    line_sweeps1<LB>(gv, lam_b, (per_axis ? lm : gb) + cap_b);
                if (to_mbox) {  // m_b of this column of the row below
                    int *const nb = nx_slots + (s & 1) * XS + tl * P0;
#pragma unroll
                    for (int j = 0; j < LB; ++j) nb[j] = gv[j];
                } else if (to_ring) {
#pragma unroll
                    for (int j = 0; j < LB; ++j) rb[j] = gv[j];
                }
            }
            if (to_mbox) {
                __syncwarp();
                if (lane == 0) st_rel_cta(ctl + wt, s + 1);
            }
            team_sync(tm, TW);  // barrier: rows of X_a (and of the outgoing slot) written

            // ---- phase C (last row of the block): m_b as records, column layout ----
            if (to_ring) {
                spins = 0;
                const int need = s - ring + 1;
                while ((int)cons_seen < need) {
                    cons_seen = __shfl_sync(kFull, lane == 0 ? ld_relaxed_gpu(cons_out) : 0u, 0);
                    if ((int)cons_seen >= need) break;
                    if (__any_sync(kFull, ++spins > A.spin_limit || *s_abort != 0 ||
                                              ((spins & 63) == 0 && *(volatile int *)A.status != 0))) {
                        bad = true;
                        break;
                    }
                    __nanosleep(32);
                }
                if (!bad && colA) {
                    int2 *const dst = ll_out + (size_t)(s % ring) * Qm + tl;
                    const int tag_out = A.tag0 + s / ring;
#pragma unroll
                    for (int i = 0; i < LA; ++i) st_rec(dst + i * LB, Xb[i * P0 + tl], tag_out);
                }
                __syncwarp();
                if (!bad && lane == 0) st_relaxed_gpu(flag_out, (unsigned)(s + 1));
                if (bad) {
                    atomicCAS(A.status, 0, EDP_ERR_TIMEOUT_CODE);
                    *s_abort = 1;
                }
            }
            if (from_mbox) {  // this column's slot is free again for the team above
                __syncwarp();
                if (lane == 0) st_rel_cta(ctl + 4 + wt, s + 1);
            }
        }
        (void)aborted;
    }
    if (A.trace && tid == 0) {
        A.trace[band * 4 + 0] = t_band0;
        A.trace[band * 4 + 1] = global_ns();
        A.trace[band * 4 + 2] = 0;
        A.trace[band * 4 + 3] = sm_id();
    }
    __syncthreads();
    return *s_abort == 0;
}

}  // namespace edp
