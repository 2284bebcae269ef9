// pass_team.cuh -- one row band of an EDP scan pass, any number of label axes.
//
// What is stored.  The paper keeps the four directional sums S_k.  Every use
// of S_k is through the message  m_k(x) = M(floor(S_k(x_k) / 2))  into the
// neighbour x of x_k (Eq. DP_2D_1, Eq. DP_2D_base), so the kernels store the
// messages instead: M[k] at pixel x holds m_k(x), computed once by the pixel
// x_k that produces S_k(x_k).  A pass p updates the sums a (x direction) and
// b (y direction):
//   P1: a = +x, b = +y   P2: a = -x, b = +y   P3: a = +x, b = -y   P4: a = -x, b = -y
// with c = opposite(a), d = opposite(b) read from the previous passes, and
//   S_a = C + m_a + m_b + m_d - m_c,    S_b = C + m_a + m_b + m_c - m_d
// (Eq. DP_2D_base with the data term: all k except -k', minus m_{-k'}).  The
// new messages M(floor(S_a / 2)) and M(floor(S_b / 2)) go to the next pixel
// of the row and to the same column of the next row.  In the last pass the
// marginal S_Omega = C + m_a + m_b + m_c + m_d and its lowest-index argmin
// (Eq. DP_2D_1, Eq. DP_2D_2) are taken on the way.
//
// Schedule.  The recursion is in place (Sec. 4.2), so pixel (x, y) of a pass
// needs (x -/+ 1, y) and (x, y -/+ 1) of the same pass: a wavefront.  One
// team of T warps owns one image row and walks it column by column; a block
// holds NT teams (NT consecutive rows, a "band").  Per column a team:
//   1. prefetches C, m_c, m_d of a later column into shared memory
//      (cp.async, 16-byte copies, nbuf - 1 columns ahead);
//   2. gets m_b: from the team above through a shared-memory mailbox
//      (release / acquire flags), or, for the first row of a band, from a
//      ring of "value + tag" records in global memory written by the last
//      row of the previous band (polled until every tag matches; no fence);
//   3. phase 0: sums, halving and the sweeps of label axis 0 -- lane groups
//      own line segments of axis 0 in registers (Eq. L_dec3, Eq. L_dec5);
//   4. phases 1..R-1: the same for axes 1, 2 after a transpose through
//      shared memory (named barrier of the team);
//   5. the clip of Eq. derivation1 (joint: vector minimum + lambda f(g);
//      per-axis: line minimum + lambda f(g) after every axis), then the two
//      messages go to the next column (shared memory + global M[a]) and to
//      the next row (mailbox or record ring + global M[b]).
// Between blocks the producer may run at most `ring` columns ahead of its
// consumer (a consumed-column counter per band).  Every wait is a bounded
// spin that sets the launch's status word on timeout.
#pragma once
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace edp {
namespace team {

constexpr unsigned kAllLanes = 0xffffffffu;
constexpr int kMaxT = 12;   // warps per team
// per-team control words (ints): [0, 16) produced columns per warp, [16]
// consumed columns, [24, 48) warp minima (a, b), [48, 72) warp argmin keys
constexpr int kMisc = 96;

__device__ __forceinline__ void sync(int tm, int T) {
    if (T == 1) {
        __syncwarp();
        return;
    }
    asm volatile("barrier.sync %0, %1;" ::"r"(tm + 1), "r"(32 * T) : "memory");
}
// team barrier that also returns the OR of `pred` over the team
__device__ __forceinline__ bool sync_or(int tm, int T, bool pred) {
    if (T == 1) return __any_sync(kAllLanes, pred);
    int r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.s32 p, %1, 0;\n\t"
        "barrier.red.or.pred q, %2, %3, p;\n\t"
        "selp.s32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((int)pred), "r"(tm + 1), "r"(32 * T)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ int ld_acq_cta(const int *p) {
    int v;
    asm volatile("ld.acquire.cta.shared.u32 %0, [%1];" : "=r"(v) : "r"((unsigned)__cvta_generic_to_shared(p)) : "memory");
    return v;
}
__device__ __forceinline__ void st_rel_cta(int *p, int v) {
    asm volatile("st.release.cta.shared.u32 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(p)), "r"(v) : "memory");
}
__device__ __forceinline__ int4 ld_rec2(const int2 *p) {
    int4 r;
    asm volatile("ld.relaxed.gpu.global.v4.s32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "l"(p)
                 : "memory");
    return r;
}
__device__ __forceinline__ void st_record(int2 *p, int v, int tag) {
    asm volatile("st.relaxed.gpu.global.v2.s32 [%0], {%1, %2};" ::"l"(p), "r"(v), "r"(tag) : "memory");
}
__device__ __forceinline__ unsigned ld_relaxed_gpu(const unsigned *p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_gpu(unsigned *p, unsigned v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void cp16(int *dst, const int *src, int bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src),
                 "r"(bytes)
                 : "memory");
}
// 32-bit shared-memory addressing (the buffers below live in dynamic shared memory)
__device__ __forceinline__ unsigned saddr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ int lds(unsigned a) {
    int v;
    asm volatile("ld.shared.s32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ void sts(unsigned a, int v) { asm volatile("st.shared.s32 [%0], %1;" ::"r"(a), "r"(v) : "memory"); }
__device__ __forceinline__ void wait_groups(int keep) {
    switch (keep) {
    case 0: cp_async_wait_0(); break;
    case 1: cp_async_wait_n<1>(); break;
    case 2: cp_async_wait_n<2>(); break;
    default: cp_async_wait_n<3>(); break;
    }
}

// Truncated-L1 distance transform (Eq. L_dec3, Eq. L_dec5) of two vectors a,
// b along one label line, in place.  Lane j of a group of G lanes holds the
// positions j*E .. j*E+E-1; positions past the line hold kBig.  Carries come
// from the kc nearest lanes of the group on each side: a source farther than
// g - 1 labels costs at least the clip value lambda f(g) applied afterwards,
// so the clipped result is exact.  Returns the minima of a and b over the
// line (of the input).
template <int EM>
__device__ __forceinline__ int2 seg_dt2(int (&a)[EM], int (&b)[EM], const int E, const int G, const int j,
                                        const int lam, const int kc) {
    int mina = kBig, minb = kBig;
#pragma unroll
    for (int i = 0; i < EM; ++i)
        if (i < E) {
            mina = min(mina, a[i]);
            minb = min(minb, b[i]);
        }
    int cfa = kBig, cfb = kBig, cba = kBig, cbb = kBig;
    if (G > 1) {
        // value of the lane's own labels at its last position (forward) and
        // at its first position (backward)
        int Fa = kBig, Fb = kBig, Ba = kBig, Bb = kBig;
#pragma unroll
        for (int i = 0; i < EM; ++i)
            if (i < E) {
                Fa = min(Fa + lam, a[i]);
                Fb = min(Fb + lam, b[i]);
                Ba = min(Ba, a[i] + lam * i);
                Bb = min(Bb, b[i] + lam * i);
            }
        const int kcl = min(kc, G - 1);
        for (int d = 1; d <= kcl; ++d) {
            const int t0 = __shfl_up_sync(kAllLanes, Fa, d, G), t1 = __shfl_up_sync(kAllLanes, Fb, d, G);
            const int t2 = __shfl_down_sync(kAllLanes, Ba, d, G), t3 = __shfl_down_sync(kAllLanes, Bb, d, G);
            const int gap = lam * ((d - 1) * E + 1);
            if (j >= d) {
                cfa = min(cfa, t0 + gap);
                cfb = min(cfb, t1 + gap);
            }
            if (j + d < G) {
                cba = min(cba, t2 + gap);
                cbb = min(cbb, t3 + gap);
            }
        }
        for (int d = G >> 1; d >= 1; d >>= 1) {
            mina = min(mina, __shfl_xor_sync(kAllLanes, mina, d, G));
            minb = min(minb, __shfl_xor_sync(kAllLanes, minb, d, G));
        }
    }
    int fa[EM], fb[EM];
    int ra = cfa, rb = cfb;
#pragma unroll
    for (int i = 0; i < EM; ++i)
        if (i < E) {
            ra = min(a[i], i == 0 ? ra : ra + lam);
            rb = min(b[i], i == 0 ? rb : rb + lam);
            fa[i] = ra;
            fb[i] = rb;
        }
    int sa = cba, sb = cbb;
    bool started = false;
#pragma unroll
    for (int i = EM - 1; i >= 0; --i)
        if (i < E) {
            sa = min(a[i], started ? sa + lam : sa);
            sb = min(b[i], started ? sb + lam : sb);
            started = true;
            a[i] = min(fa[i], sa);
            b[i] = min(fb[i], sb);
        }
    return make_int2(mina, minb);
}

// ints of shared memory of one team
// stage of one column: C, m_c, m_d (Qm + 4 ints each) and 8 ints of box centres
__host__ __device__ inline size_t stage_ints(int Qm) { return 3 * ((size_t)Qm + 4) + 8; }
__host__ __device__ inline size_t team_ints(int Qm, int R, int nbuf, int kmb) {
    return (size_t)nbuf * stage_ints(Qm) + (size_t)Qm * (1 + (R >= 2 ? 2 : 0) + kmb) + kMisc;
}

}  // namespace team

// One row band of one scan pass.  Every thread of the block calls it with the
// same band; returns false when the pass was aborted (a wait timed out).
// ---- lean form: one lane owns one whole line (L labels) of one vector ----

// Backward sweep into b, forward sweep combined with it and the clip cl
// (Eq. L_dec3, Eq. L_dec5 over a whole line held by one lane): h <- min(fwd,
// bwd, cl).  Returns the line minimum of the input.
template <int L>
__device__ __forceinline__ int lean_dt(int (&h)[L], int lam, int cl_add, bool per_axis, int cl_fixed) {
    int b[L];
    int lmin = h[L - 1], sw = h[L - 1];
    b[L - 1] = sw;
#pragma unroll
    for (int i = L - 2; i >= 0; --i) {
        lmin = min(lmin, h[i]);
        sw = min(h[i], sw + lam);
        b[i] = sw;
    }
    const int cl = per_axis ? lmin + cl_add : cl_fixed;
    int f = h[0];
    h[0] = min(b[0], cl);
#pragma unroll
    for (int i = 1; i < L; ++i) {
        f = min(h[i], f + lam);
        h[i] = min(min(f, b[i]), cl);
    }
    return lmin;
}

// Same, with the backward sweep kept in shared memory at ab + i * st4 (the
// line's own slots; lines longer than 33 labels).
template <int L>
__device__ __forceinline__ int lean_dt_smem(int (&h)[L], int lam, int cl_add, bool per_axis, int cl_fixed,
                                            unsigned ab, unsigned st4) {
    int lmin = h[L - 1], sw = h[L - 1];
    team::sts(ab + (L - 1) * st4, sw);
#pragma unroll
    for (int i = L - 2; i >= 0; --i) {
        lmin = min(lmin, h[i]);
        sw = min(h[i], sw + lam);
        team::sts(ab + i * st4, sw);
    }
    const int cl = per_axis ? lmin + cl_add : cl_fixed;
    int f = h[0];
    h[0] = min(team::lds(ab), cl);
#pragma unroll
    for (int i = 1; i < L; ++i) {
        f = min(h[i], f + lam);
        h[i] = min(min(f, team::lds(ab + i * st4)), cl);
    }
    return lmin;
}

// Truncated quadratic prior (l1 = 2, Eq. M_decmp, the generalized RMS) on a
// whole line held by one lane: the input is first stored at ab + i * st4;
// h[i] <- min over taps |d| < g of input[i + d] + lambda d^2 (farther sources
// cost at least the clip lambda g^2), then the clip.  Returns the line minimum.
template <int L>
__device__ __forceinline__ int lean_quad(int (&h)[L], int lam, int g, int cl_add, bool per_axis, int cl_fixed,
                                         unsigned ab, unsigned st4) {
    int lmin = kBig;
#pragma unroll
    for (int i = 0; i < L; ++i) {
        team::sts(ab + i * st4, h[i]);
        lmin = min(lmin, h[i]);
    }
    const int dmax = min(g, L);
    for (int d = 1; d < dmax; ++d) {
        const int w = lam * d * d;
#pragma unroll
        for (int i = 0; i < L; ++i) {
            int c = kBig;
            if (i + d < L) c = team::lds(ab + (i + d) * st4);
            if (i - d >= 0) c = min(c, team::lds(ab + (i - d) * st4));
            h[i] = min(h[i], c + w);
        }
    }
    const int cl = per_axis ? lmin + cl_add : cl_fixed;
#pragma unroll
    for (int i = 0; i < L; ++i) h[i] = min(h[i], cl);
    return lmin;
}

// Phase 0 of one line of axis 0 (contiguous labels q0 .. q0 + L - 1): the
// halved sums of Eq. DP_2D_base for vector `vsel` from the staged inputs,
// the final-pass argmin key (vector a lanes), the sweeps; result into X.
template <int L, bool QUAD = false>
__device__ __forceinline__ int lean_phase0(unsigned aC, unsigned aCc, unsigned aCd, unsigned aMa, unsigned aMb,
                                           unsigned aX, int q0, int vsel, bool final_a, bool per_axis, int lam,
                                           int capv, unsigned long long &key, int g) {
    const unsigned o = 4u * (unsigned)q0;
    int h[L];
    if (final_a) {
#pragma unroll
        for (int i = 0; i < L; ++i) {
            const int c = team::lds(aCc + o + 4 * i), d = team::lds(aCd + o + 4 * i);
            const int t = team::lds(aC + o + 4 * i) + team::lds(aMa + o + 4 * i) + team::lds(aMb + o + 4 * i);
            const int so = t + c + d;
            key = min(key, ((unsigned long long)((unsigned)so ^ 0x80000000u) << 32) | (unsigned)(q0 + i));
            h[i] = floor_half(t + d - c);
        }
    } else {
        const int sgn = vsel ? -1 : 1;
#pragma unroll
        for (int i = 0; i < L; ++i) {
            const int e = team::lds(aCd + o + 4 * i) - team::lds(aCc + o + 4 * i);
            h[i] = floor_half(team::lds(aC + o + 4 * i) + team::lds(aMa + o + 4 * i) + team::lds(aMb + o + 4 * i) +
                              sgn * e);
        }
    }
    int lmin;
    if constexpr (QUAD)
        lmin = lean_quad<L>(h, lam, g, capv, per_axis, kBig, aX + o, 4u);
    else if constexpr (L > 33)
        lmin = lean_dt_smem<L>(h, lam, capv, per_axis, kBig, aX + o, 4u);
    else
        lmin = lean_dt<L>(h, lam, capv, per_axis, kBig);
#pragma unroll
    for (int i = 0; i < L; ++i) team::sts(aX + o + 4 * i, h[i]);
    return lmin;
}

// Phase r >= 1 of one line (first label qb, neighbour stride st): sweeps of
// the values in X, clip; result back into X or, on the last axis, out as
// the messages.
struct LeanOut {
    unsigned aMa, aBox;    // shared: m_a of the next column, mailbox slot of the next row (0: none)
    bool zero_a;           // no next column in this sweep direction: m_a of the next column is zero
    int *pMa, *pMb;        // global M[a], M[b] (null: not written)
    int2 *pRec;            // record ring slot (null: none)
    int tag;
};
template <int L, bool QUAD = false>
__device__ __forceinline__ void lean_phase_r(unsigned aX, int qb, int st, bool last, int vsel, bool per_axis, int lam,
                                             int capv, int gv, const LeanOut &O, int g) {
    const unsigned o = aX + 4u * (unsigned)qb, st4 = 4u * (unsigned)st;
    int h[L];
#pragma unroll
    for (int i = 0; i < L; ++i) h[i] = team::lds(o + i * st4);
    if constexpr (QUAD)
        lean_quad<L>(h, lam, g, capv, per_axis, last ? gv + capv : kBig, o, st4);
    else if constexpr (L > 33)
        lean_dt_smem<L>(h, lam, capv, per_axis, last ? gv + capv : kBig, o, st4);
    else
        lean_dt<L>(h, lam, capv, per_axis, last ? gv + capv : kBig);
    if (!last) {
#pragma unroll
        for (int i = 0; i < L; ++i) team::sts(o + i * st4, h[i]);
    } else if (vsel == 0) {
        const unsigned om = O.aMa + 4u * (unsigned)qb;
#pragma unroll
        for (int i = 0; i < L; ++i) team::sts(om + i * st4, O.zero_a ? 0 : h[i]);
        if (O.pMa) {
#pragma unroll
            for (int i = 0; i < L; ++i) O.pMa[qb + i * st] = h[i];
        }
    } else {
        if (O.aBox) {
            const unsigned ob = O.aBox + 4u * (unsigned)qb;
#pragma unroll
            for (int i = 0; i < L; ++i) team::sts(ob + i * st4, h[i]);
        } else if (O.pRec) {
#pragma unroll
            for (int i = 0; i < L; ++i) team::st_record(O.pRec + qb + i * st, h[i], O.tag);
        }
        if (O.pMb) {
#pragma unroll
            for (int i = 0; i < L; ++i) O.pMb[qb + i * st] = h[i];
        }
    }
}

// lean line lengths
__host__ __device__ inline bool lean_length(int L) { return L == 9 || L == 17 || L == 33 || L == 65; }

// EM: labels-per-lane bound (generic form) or line-length bound (LEAN: 33
// serves 9/17/33, 65 serves 65, 2 is the quadratic-prior build for all).
// WIN: EDP on per-pixel label boxes (windowed form, one warp per row); EM is
// then the prior power l1 of the build (1 linear sweeps, 2 quadratic taps).
// WT (whole-line form): per-edge multipliers of the prior, A.wh / A.wv.
template <int EM, bool LEAN, bool WIN = false, bool WT = false>
__device__ __forceinline__ bool team_band(const TeamArgs &A, const int band, int *smem, volatile int *s_abort) {
    using namespace team;
    const int Q = A.Q, Qm = A.Qm, W = A.W, H = A.H, T = A.T, NT = A.NT, R = A.R;
    const int nbuf = A.nbuf, kmb = A.kmb, ring = A.ring;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tm = warp / T;
    const int wt = warp - tm * T;
    const int tl = wt * 32 + lane;
    const int NL = 32 * T;
    const int Ralloc = WIN ? 2 : R;  // the windowed form uses the transpose buffers as scratch
    const size_t tints = team_ints(Qm, Ralloc, nbuf, kmb);
    const int Qs = Qm + 4;
    const int SS = (int)stage_ints(Qm);
    // regions of team i
    auto stg_of = [&](int i) { return smem + (size_t)i * tints; };
    auto ma_of = [&](int i) { return stg_of(i) + (size_t)nbuf * SS; };
    auto ta_of = [&](int i) { return ma_of(i) + Qm; };
    auto mbox_of = [&](int i) { return ma_of(i) + Qm * (1 + (Ralloc >= 2 ? 2 : 0)); };
    auto misc_of = [&](int i) { return mbox_of(i) + (size_t)kmb * Qm; };
    for (int i = tid; i < NT * 32; i += blockDim.x) misc_of(i >> 5)[i & 31] = 0;
    if (LEAN || WIN) {
        // m_a into the first column and m_b into the image's first row are zero
        for (int i = tid; i < NT * Qm; i += blockDim.x) ma_of(i / Qm)[i % Qm] = 0;
        if (band == 0)
            for (int i = tid; i < kmb * Qm; i += blockDim.x) mbox_of(0)[i] = 0;
    }
    __syncthreads();
    unsigned long long t_band0 = (A.trace && tid == 0) ? global_ns() : 0;

    const int r = band * NT + tm;
    if (tm < NT && r < H) {
        // A.pair: passes A.pass (left to right) and A.pass + 1 (right to left)
        // as one sweep of 2W columns per row (half h = column / W)
        const int ncol = A.pair ? 2 * W : W;
        auto incx_of = [&](int h) { return ((A.pass + h) & 1) == 0; };
        const bool incy = (A.pass < 2);
        int *const Mb = incy ? A.M[2] : A.M[3];
        const int *const Md = incy ? A.M[3] : A.M[2];
        const int y = incy ? r : H - 1 - r;
        const bool has_next = r + 1 < H;
        const int y_next = has_next ? (incy ? y + 1 : y - 1) : y;
        const bool to_mbox = has_next && tm + 1 < NT;
        const bool to_ring = has_next && tm + 1 == NT;
        const bool from_mbox = r > 0 && tm > 0;
        const bool from_ring = r > 0 && tm == 0;
        const bool d_ok = A.read_d && (incy ? y + 1 < H : y - 1 >= 0);
        const bool per_axis = (A.mode == 1);
        int *const stg = stg_of(tm);
        int *const maS = ma_of(tm);
        int *const tA = ta_of(tm);
        int *const tB = tA + Qm;
        int *const mbox = mbox_of(tm);
        int *const misc = misc_of(tm);
        int *const produced = misc;
        int *const wmin = misc + 24;
        unsigned long long *const wkey = reinterpret_cast<unsigned long long *>(misc + 48);
        int *const nx_mbox = to_mbox ? mbox_of(tm + 1) : nullptr;
        const int *const nx_consumed = to_mbox ? misc_of(tm + 1) + 16 : nullptr;
        const int *const pv_produced = from_mbox ? misc_of(tm - 1) : nullptr;
        const int2 *const ll_in = from_ring ? A.ll + (size_t)(band - 1) * ring * Qm : nullptr;
        int2 *const ll_out = to_ring ? A.ll + (size_t)band * ring * Qm : nullptr;
        const size_t NQ = (size_t)W * H * Q;
        // C is read in 16-byte chunks from the aligned-down base
        const int cshift = (int)((reinterpret_cast<uintptr_t>(A.C) & 15) >> 2);
        const int *const Cbase = A.C - cshift;

        // lane -> line segments: on an axis with groups of G lanes, lane tl
        // serves position jr = tl % G of line gi + k * gpt, gi = tl / G,
        // gpt = 32 T / G (round k)
        auto line_first = [&](const TeamAxis &X, int li) {
            return X.stride == 1 ? li * X.L : (li % X.stride) + (li / X.stride) * X.stride * X.L;
        };

        // column xt of the half sweeping in direction incx (column s of the
        // launch); its m_c source Mc, read only where read_c.  In the second
        // half of a pair, Mc holds the first half's m_a outputs (ordered
        // before this by the team barriers).
        auto prefetch = [&](int xt, int s, bool incx, const int *Mc, bool read_c) {
            if (xt < W) {
                const int x = incx ? xt : W - 1 - xt;
                const size_t pix = (size_t)y * W + x;
                const bool c_ok = read_c && (incx ? x + 1 < W : x - 1 >= 0);
                int *dst = stg + (size_t)(s % nbuf) * SS;
                const size_t e0 = pix * Q + cshift, e1 = e0 + Q, eend = NQ + cshift;
                const size_t c0 = e0 >> 2, c1 = (e1 + 3) >> 2;
                for (size_t c = c0 + tl; c < c1; c += NL) {
                    const size_t rem = eend - 4 * c;
                    cp16(dst + 4 * (c - c0), Cbase + 4 * c, rem >= 4 ? 16 : (int)rem * 4);
                }
                const int *sc = Mc + pix * Qm, *sd = Md + pix * Qm;
                for (int c = tl; c < Qm / 4; c += NL) {
                    cp16(dst + Qs + 4 * c, sc + 4 * c, c_ok ? 16 : 0);
                    cp16(dst + 2 * Qs + 4 * c, sd + 4 * c, d_ok ? 16 : 0);
                }
                if (WIN && tl < 3 * R) {
                    // box centres of this pixel, of the next pixel of the row and of
                    // the same column in the next row (zero where there is none)
                    const int which = tl / R, r_ = tl - which * R;
                    const bool ok = which == 0 || (which == 1 ? xt + 1 < W : has_next);
                    const size_t p2 = which == 0 ? pix : (which == 1 ? pix + (incx ? 1 : -1) : (size_t)y_next * W + x);
                    cp_async4(dst + 3 * Qs + tl, A.centre + (ok ? p2 : pix) * R + r_, ok);
                }
            }
            cp_async_commit();
        };
        // tag of the first ring lap of the records from the previous band (the
        // test hook hold_band makes one band expect a tag no producer writes)
        const int tag_in0 = A.tag0 + (band == A.hold_band ? 0x20000000 : 0);
        unsigned cons_seen = 0;     // consumer progress seen by this producer (lane tl == 0)
        int mb_cons_seen = 0;       // same, for the mailbox consumer
        bool aborted = false;
        for (int h = 0; h < (A.pair ? 2 : 1) && !aborted; ++h) {
        // half h of the sweep: pass A.pass + h, direction and flags
        const bool incx = incx_of(h);
        const bool fin = h ? A.final2 : A.final_;     // marginal and labels (last pass)
        const bool read_c = h ? A.read_c2 : A.read_c;
        const bool write_a = h ? A.write_a2 : A.write_a;
        const bool write_b = h ? A.write_b2 : A.write_b;
        int *const Ma = incx ? A.M[0] : A.M[1];
        const int *const Mc = incx ? A.M[1] : A.M[0];
        for (int t = 0; t < nbuf - 1; ++t) prefetch(t, h * W + t, incx, Mc, read_c);
        for (int xs = 0; xs < W; ++xs) {
            const int s = h * W + xs;  // column of the launch (ring slots, tags, counters)
            prefetch(xs + nbuf - 1, s + nbuf - 1, incx, Mc, read_c);
            wait_groups(nbuf - 1);
            bool bad = false;
            // ---- m_b of this column from the row above ----
            if (from_mbox) {
                if (wt == 0) {
                    long long spins = 0;
                    while (true) {
                        const bool ok = lane >= T || ld_acq_cta(pv_produced + lane) >= s + 1;
                        if (__all_sync(kAllLanes, ok)) break;
                        if (++spins > A.spin_limit || *s_abort) {
                            bad = true;
                            break;
                        }
                    }
                }
            } else if (from_ring) {
                const int2 *p = ll_in + (size_t)(s % ring) * Qm;
                const int tag = tag_in0 + s / ring;
                int *dst = mbox + (s % kmb) * Qm;
                // kRecBatch record pairs per lane in flight: the first loads of a
                // batch are independent, so a column costs about one L2 round
                // trip per batch rather than one per record pair
                constexpr int kRecBatch = 8;
                for (int q0 = 2 * tl; q0 < Q && !bad; q0 += 2 * NL * kRecBatch) {
                    int4 v[kRecBatch];
#pragma unroll
                    for (int u = 0; u < kRecBatch; ++u) {
                        const int q = q0 + 2 * NL * u;
                        if (q < Q) v[u] = ld_rec2(p + q);
                    }
#pragma unroll
                    for (int u = 0; u < kRecBatch; ++u) {
                        const int q = q0 + 2 * NL * u;
                        if (q >= Q || bad) continue;
                        long long spins = 0;
                        while (!(v[u].y == tag && (q + 1 >= Q || v[u].w == tag))) {
                            if (++spins > A.spin_limit ||
                                ((spins & 63) == 0 && (*s_abort || *(volatile int *)A.status != 0))) {
                                bad = true;
                                break;
                            }
                            v[u] = ld_rec2(p + q);
                        }
                        if (bad) break;
                        dst[q] = v[u].x;
                        if (q + 1 < Q) dst[q + 1] = v[u].z;
                    }
                }
            }
            // producer side: room in the consumer's mailbox / record ring
            if (tl == 0 && has_next) {
                long long spins = 0;
                if (to_mbox) {
                    const int need = s - kmb + 1;
                    while (mb_cons_seen < need) {
                        mb_cons_seen = ld_acq_cta(nx_consumed);
                        if (mb_cons_seen >= need) break;
                        if (++spins > A.spin_limit || *s_abort) {
                            bad = true;
                            break;
                        }
                    }
                } else {
                    const int need = s - ring + 1;
                    while ((int)cons_seen < need) {
                        cons_seen = ld_relaxed_gpu(A.cons + band);
                        if ((int)cons_seen >= need) break;
                        if (++spins > A.spin_limit || *s_abort ||
                            ((spins & 63) == 0 && *(volatile int *)A.status != 0)) {
                            bad = true;
                            break;
                        }
                        __nanosleep(32);
                    }
                }
            }
            if (bad) {
                atomicCAS(A.status, 0, EDP_ERR_TIMEOUT_CODE);
                *s_abort = 1;
            }
            if (sync_or(tm, T, bad || *s_abort)) {  // barrier 1
                aborted = true;
                break;
            }

            // ---- column s: inputs in shared memory, outputs ----
            const int x = incx ? xs : W - 1 - xs;
            const int *sb = stg + (size_t)(s % nbuf) * SS;
            const int *sC = sb + (int)((((size_t)y * W + x) * Q + cshift) & 3);
            const int *sc = sb + Qs, *sd = sb + 2 * Qs;
            const int *mbv = (r > 0) ? mbox + (s % kmb) * Qm : nullptr;
            const bool has_ma = xs > 0;       // a previous pixel in this direction
            const bool nxt = xs + 1 < W;      // a next pixel in this direction
            unsigned long long key = ~0ull;           // final pass: (S_Omega, q) minimum
            const int xn = incx ? x + 1 : x - 1;
            const bool a_out = write_a && nxt;
            const int tag_out = A.tag0 + s / ring;
            int *const pMa = a_out ? Ma + ((size_t)y * W + xn) * Qm : nullptr;
            int *const pMb = (has_next && write_b) ? Mb + ((size_t)y_next * W + x) * Qm : nullptr;
            int *const pBox = to_mbox ? nx_mbox + (s % kmb) * Qm : nullptr;
            int2 *const pRec = to_ring ? ll_out + (size_t)(s % ring) * Qm : nullptr;
            // message into the next column of the row (m_a) and into the next row (m_b)
            auto emit_a = [&](int q, int oa) {
                maS[q] = nxt ? oa : 0;  // the first pixel of a sweep direction gets a zero m_a
                if (pMa) pMa[q] = oa;
            };
            auto emit_b = [&](int q, int ob) {
                if (pBox) pBox[q] = ob;
                if (pRec) st_record(pRec + q, ob, tag_out);
                if (pMb) pMb[q] = ob;
            };
            auto emit = [&](int q, int oa, int ob) {
                emit_a(q, oa);
                emit_b(q, ob);
            };
            // windowed form: the box origin maps box labels to the full space
            int map_lo0 = 0, map_lo1 = 0;
            // warp minimum / argmin into the team's control words, barrier 2,
            // then the per-column bookkeeping of lane 0
            auto barrier2 = [&](int ja, int jb) -> bool {
                ja = __reduce_min_sync(kAllLanes, ja);
                jb = __reduce_min_sync(kAllLanes, jb);
                if (fin) {
                    const unsigned hi = __reduce_min_sync(kAllLanes, (unsigned)(key >> 32));
                    const unsigned lo =
                        __reduce_min_sync(kAllLanes, (unsigned)(key >> 32) == hi ? (unsigned)key : 0xffffffffu);
                    key = ((unsigned long long)hi << 32) | lo;
                }
                if (lane == 0) {
                    wmin[2 * wt] = ja;
                    wmin[2 * wt + 1] = jb;
                    if (fin) wkey[wt] = key;
                }
                if (sync_or(tm, T, *s_abort != 0)) return false;  // barrier 2
                // every lane of the team is done with this column's m_b
                if (tl == 0) {
                    if (from_mbox) st_rel_cta(misc + 16, s + 1);
                    // the consumer's record loads above have returned (their values
                    // went through shared memory and a barrier) before this store
                    if (from_ring && ((s & 3) == 3 || s + 1 == ncol)) st_relaxed_gpu(A.cons + band - 1, (unsigned)(s + 1));
                    if (fin) {
                        unsigned long long best = wkey[0];
                        for (int w = 1; w < T; ++w) best = min(best, wkey[w]);
                        int q = (int)(best & 0xffffffffu);
                        if (WIN) q = (map_lo0 + q % A.win) + A.Q0w * (map_lo1 + q / A.win);
                        A.labels[(size_t)y * W + x] = q;
                    }
                }
                return true;
            };
            if constexpr (WIN) {
            // Windowed form.  Every pixel x keeps only the N^R labels of its box
            // B(x) (origin lo(x), from a proposed centre clamped into the label
            // space); costs, messages and sums are in the coordinates of the
            // pixel's own box.  A message from x to a neighbour x' is the exact
            // min-convolution between the two boxes,
            //     m(v) = min_{u in B(x)} floor(S(x, u) / 2) + V(u, v),  v in B(x'),
            // per label axis as in Sec. 3.2: the sweeps (Eq. L_dec3, Eq. L_dec5)
            // along the source box's line give the L1 distance transform D at
            // every source position; a target coordinate outside the source
            // range takes D at the nearest source end plus lambda times the
            // distance (all candidates then lie on one side).  The per-axis
            // clip follows each axis; the joint clip (box minimum + lambda f(g),
            // Eq. derivation1) follows the last axis.  Lanes [0, N) own the
            // axis-0 lines of S_a's box, lanes [N, 2N) those of S_b (one line
            // each for one label axis); one warp per image row.
            const int N = A.win, hN = (N - 1) / 2;
            const int *cs = sb + 3 * Qs;
            auto origin = [&](int c, int Qr) { return min(max(c, hN), Qr - 1 - hN) - hN; };
            const int lo0 = origin(cs[0], A.Q0w), lo1 = R == 2 ? origin(cs[1], A.Q1w) : 0;
            const int la0 = nxt ? origin(cs[R], A.Q0w) : lo0;
            const int la1 = R == 2 ? (nxt ? origin(cs[R + 1], A.Q1w) : lo1) : 0;
            const int lb0 = has_next ? origin(cs[2 * R], A.Q0w) : lo0;
            const int lb1 = R == 2 ? (has_next ? origin(cs[2 * R + 1], A.Q1w) : lo1) : 0;
            map_lo0 = lo0;
            map_lo1 = lo1;
            // old messages no pass has written yet come from sums that are still
            // zero: M(0) between the boxes (the c neighbour is the next pixel of
            // the row, the d neighbour the same column of the next row)
            const bool c_m0 = !read_c && nxt, d_m0 = !A.read_d && has_next;
            const int v = R == 2 ? (lane < N ? 0 : (lane < 2 * N ? 1 : -1)) : (lane < 2 ? lane : -1);
            const int l = R == 2 ? lane - (v > 0 ? N : 0) : 0;
            const int d0 = (v == 1 ? lb0 : la0) - lo0, d1 = (v == 1 ? lb1 : la1) - lo1;
            const unsigned aX = saddr(v == 1 ? tB : tA);
            const unsigned aC = saddr(sC), aCc = saddr(sc), aCd = saddr(sd);
            const unsigned aMa = saddr(maS), aMb = saddr(mbox + (s % kmb) * Qm);
            const int lam = A.lam, capv = A.capv;
            auto m0 = [&](int i0, int i1, int s0, int s1) {
                const int a0 = lo0 + i0, a1 = lo1 + i1;
                // distances beyond g are clipped anyway (and must not overflow)
                int e0 = min(A.g, max(0, max(s0 - a0, a0 - (s0 + N - 1))));
                int e1 = R == 2 ? min(A.g, max(0, max(s1 - a1, a1 - (s1 + N - 1)))) : 0;
                if (A.l1 == 2) {  // f(u) = u^2
                    e0 *= e0;
                    e1 *= e1;
                }
                return per_axis ? min(lam * e0, capv) + min(lam * e1, capv) : min(lam * (e0 + e1), capv);
            };
            auto body = [&](auto nc) -> bool {
                constexpr int NN = decltype(nc)::value;
                int lmin0 = kBig;
                int out1[NN];  // one label axis: the messages, emitted after barrier 2
                if (v >= 0) {
                    // phase 0: halved sums of the own box, sweeps along axis 0,
                    // values at the target box's axis-0 coordinates
                    const int qb = R == 2 ? l * NN : 0;
                    int hv[NN], bv[NN];
#pragma unroll
                    for (int i = 0; i < NN; ++i) {
                        const int q = qb + i;
                        const unsigned o4 = 4u * (unsigned)q;
                        const int t = lds(aC + o4) + lds(aMa + o4) + lds(aMb + o4);
                        const int c = c_m0 ? m0(i, l, la0, la1) : lds(aCc + o4);
                        const int d = d_m0 ? m0(i, l, lb0, lb1) : lds(aCd + o4);
                        if (fin && v == 0)
                            key = min(key, ((unsigned long long)((unsigned)(t + c + d) ^ 0x80000000u) << 32) | (unsigned)q);
                        hv[i] = floor_half(v ? t + c - d : t + d - c);
                        lmin0 = min(lmin0, hv[i]);
                    }
                    const int cl = (R == 1 || per_axis) ? lmin0 + capv : kBig;
                    const unsigned ax = aX + 4u * (unsigned)qb;
                    if constexpr (EM == 2) {  // windowed build for the quadratic prior
                        // quadratic taps |u - (t + d0)| < g between the boxes
#pragma unroll
                        for (int tt = 0; tt < NN; ++tt) {
                            int o = kBig;
#pragma unroll
                            for (int u = 0; u < NN; ++u) {
                                const int dd = u - tt - d0;
                                if (abs(dd) < A.g) o = min(o, hv[u] + lam * dd * dd);
                            }
                            bv[tt] = min(o, cl);
                        }
                    } else {
                        int sw = hv[NN - 1];
                        bv[NN - 1] = sw;
#pragma unroll
                        for (int i = NN - 2; i >= 0; --i) {
                            sw = min(hv[i], sw + lam);
                            bv[i] = sw;
                        }
                        int f = hv[0];
                        hv[0] = min(f, bv[0]);
#pragma unroll
                        for (int i = 1; i < NN; ++i) {
                            f = min(hv[i], f + lam);
                            hv[i] = min(f, bv[i]);
                        }
                        // values at the target box's coordinates t: source position
                        // u = t + d0 clamped to the line, plus lambda per label beyond it
#pragma unroll
                        for (int i = 0; i < NN; ++i) sts(ax + 4u * i, hv[i]);
#pragma unroll
                        for (int tt = 0; tt < NN; ++tt) {
                            const int u = min(max(tt + d0, 0), NN - 1);
                            bv[tt] = min(lds(ax + 4u * (unsigned)u) + lam * abs(tt + d0 - u), cl);
                        }
                    }
                    if (R == 1) {
                        // m_a of this column is still being read by the S_b lane
#pragma unroll
                        for (int i = 0; i < NN; ++i) out1[i] = bv[i];
                    } else {
#pragma unroll
                        for (int i = 0; i < NN; ++i) sts(aX + 4u * (unsigned)(qb + i), bv[i]);
                    }
                }
                const int vma = __reduce_min_sync(kAllLanes, v == 0 ? lmin0 : kBig);
                const int vmb = __reduce_min_sync(kAllLanes, v == 1 ? lmin0 : kBig);
                if (!barrier2(vma, vmb)) return false;
                if (R == 1 && v == 0) {
#pragma unroll
                    for (int i = 0; i < NN; ++i) emit_a(i, out1[i]);
                } else if (R == 1 && v == 1) {
#pragma unroll
                    for (int i = 0; i < NN; ++i) emit_b(i, out1[i]);
                }
                if (R == 2 && v >= 0) {
                    // phase 1: sweeps along axis 1 of the target's axis-0 column l
                    int hv[NN], bv[NN];
                    int lmin = kBig;
#pragma unroll
                    for (int i = 0; i < NN; ++i) {
                        hv[i] = lds(aX + 4u * (unsigned)(l + NN * i));
                        lmin = min(lmin, hv[i]);
                    }
                    const int cl = (per_axis ? lmin : (v == 0 ? vma : vmb)) + capv;
                    const unsigned ax = aX + 4u * (unsigned)l;
                    if constexpr (EM == 2) {  // windowed build for the quadratic prior
#pragma unroll
                        for (int tt = 0; tt < NN; ++tt) {
                            int o = kBig;
#pragma unroll
                            for (int u = 0; u < NN; ++u) {
                                const int dd = u - tt - d1;
                                if (abs(dd) < A.g) o = min(o, hv[u] + lam * dd * dd);
                            }
                            bv[tt] = min(o, cl);
                        }
                    } else {
                        int sw = hv[NN - 1];
                        bv[NN - 1] = sw;
#pragma unroll
                        for (int i = NN - 2; i >= 0; --i) {
                            sw = min(hv[i], sw + lam);
                            bv[i] = sw;
                        }
                        int f = hv[0];
                        hv[0] = min(f, bv[0]);
#pragma unroll
                        for (int i = 1; i < NN; ++i) {
                            f = min(hv[i], f + lam);
                            hv[i] = min(f, bv[i]);
                        }
#pragma unroll
                        for (int i = 0; i < NN; ++i) sts(ax + 4u * (unsigned)(NN * i), hv[i]);
#pragma unroll
                        for (int tt = 0; tt < NN; ++tt) {
                            const int u = min(max(tt + d1, 0), NN - 1);
                            bv[tt] = min(lds(ax + 4u * (unsigned)(NN * u)) + lam * abs(tt + d1 - u), cl);
                        }
                    }
                    if (v == 0) {
#pragma unroll
                        for (int i = 0; i < NN; ++i) emit_a(l + NN * i, bv[i]);
                    } else {
#pragma unroll
                        for (int i = 0; i < NN; ++i) emit_b(l + NN * i, bv[i]);
                    }
                }
                return true;
            };
            bool ok;
            switch (N) {
            case 1: ok = body(std::integral_constant<int, 1>()); break;
            case 3: ok = body(std::integral_constant<int, 3>()); break;
            case 5: ok = body(std::integral_constant<int, 5>()); break;
            case 7: ok = body(std::integral_constant<int, 7>()); break;
            case 9: ok = body(std::integral_constant<int, 9>()); break;
            case 11: ok = body(std::integral_constant<int, 11>()); break;
            case 13: ok = body(std::integral_constant<int, 13>()); break;
            default: ok = body(std::integral_constant<int, 15>()); break;
            }
            if (!ok) {
                aborted = true;
                break;
            }
            } else if constexpr (LEAN) {
            // Lean form (two or more axes): lane lv of vector v (warps
            // [v*Tv, v*Tv + Tv)) owns whole lines; the backward sweep goes to the
            // vector's shared buffer X, the forward sweep combines on the way.
            // m_a (maS) and the first row's m_b (mbox) start zero-filled.
            const int Tv = T >> 1;
            const int vsel = wt / Tv;                  // 0: S_a / m_a, 1: S_b / m_b
            const int lv = (wt - vsel * Tv) * 32 + lane;
            const int NLV = 32 * Tv;
            const unsigned aX = saddr(vsel ? tB : tA);
            const unsigned aC = saddr(sC), aCc = saddr(sc), aCd = saddr(sd);
            const unsigned aMa = saddr(maS), aMb = saddr(mbox + (s % kmb) * Qm);
            // the prior of this vector's outgoing edge: per-edge multipliers of
            // the locally adaptive prior (into the next pixel of the sweep, or
            // into the next row), 1 without them
            int wsel = 1;
            if constexpr (WT) {
                if (vsel == 0)
                    wsel = nxt ? __ldg(A.wh + (size_t)y * W + (incx ? x : x - 1)) : 1;
                else
                    wsel = has_next ? __ldg(A.wv + (size_t)(incy ? y : y - 1) * W + x) : 1;
            }
            // (the build without multipliers reads lambda f(g) from the
            // parameter block, as an operand, not from a register)
            const int lam = WT ? A.lam * wsel : A.lam;
            const int capw = WT ? A.capv * wsel : 0;
            const bool final_a = fin && vsel == 0;
            int vmin = kBig;                           // minimum of this vector's halved sums
            {
                const int L = A.ax[0].L, nl = A.ax[0].nlines;
#pragma unroll 1
                for (int li = lv; li < nl; li += NLV) {
                    int lm;
                    if (EM >= 65 || (EM == 2 && L == 65)) {
                        lm = lean_phase0<65, EM == 2>(aC, aCc, aCd, aMa, aMb, aX, li * 65, vsel, final_a, per_axis, lam, WT ? capw : A.capv, key, A.g);
                    } else if (L == 33)
                        lm = lean_phase0<33, EM == 2>(aC, aCc, aCd, aMa, aMb, aX, li * 33, vsel, final_a, per_axis, lam, WT ? capw : A.capv, key, A.g);
                    else if (L == 17)
                        lm = lean_phase0<17, EM == 2>(aC, aCc, aCd, aMa, aMb, aX, li * 17, vsel, final_a, per_axis, lam, WT ? capw : A.capv, key, A.g);
                    else
                        lm = lean_phase0<9, EM == 2>(aC, aCc, aCd, aMa, aMb, aX, li * 9, vsel, final_a, per_axis, lam, WT ? capw : A.capv, key, A.g);
                    vmin = min(vmin, lm);
                }
            }
            if (!barrier2(vsel ? kBig : vmin, vsel ? vmin : kBig)) {
                aborted = true;
                break;
            }
            {
                int gv = kBig;
                if (!per_axis)
                    for (int w = vsel * Tv; w < vsel * Tv + Tv; ++w) gv = min(gv, wmin[2 * w + vsel]);
                LeanOut O;
                O.aMa = aMa;
                O.zero_a = !nxt;
                O.aBox = pBox ? saddr(pBox) : 0u;
                O.pMa = pMa;
                O.pMb = pMb;
                O.pRec = pRec;
                O.tag = tag_out;
#pragma unroll 1
                for (int ax = 1; ax < R; ++ax) {
                    if (ax == 2) sync(tm, T);
                    const TeamAxis Xr = A.ax[ax];
                    const bool last = (ax == R - 1);
#pragma unroll 1
                    for (int li = lv; li < Xr.nlines; li += NLV) {
                        const int qb = line_first(Xr, li);
                        if (EM >= 65 || (EM == 2 && Xr.L == 65))
                            lean_phase_r<65, EM == 2>(aX, qb, Xr.stride, last, vsel, per_axis, lam, WT ? capw : A.capv, gv, O, A.g);
                        else if (Xr.L == 33)
                            lean_phase_r<33, EM == 2>(aX, qb, Xr.stride, last, vsel, per_axis, lam, WT ? capw : A.capv, gv, O, A.g);
                        else if (Xr.L == 17)
                            lean_phase_r<17, EM == 2>(aX, qb, Xr.stride, last, vsel, per_axis, lam, WT ? capw : A.capv, gv, O, A.g);
                        else
                            lean_phase_r<9, EM == 2>(aX, qb, Xr.stride, last, vsel, per_axis, lam, WT ? capw : A.capv, gv, O, A.g);
                    }
                }
            }
            } else {
            int ja = kBig, jb = kBig;  // joint minima of the halved sums
            {
                const TeamAxis X = A.ax[0];
                const int lg = __ffs(X.G) - 1;
                const int jr = tl & (X.G - 1), gi = tl >> lg, gpt = NL >> lg;
#pragma unroll 1
                for (int k = 0; k < X.rounds; ++k) {
                    int ha[EM], hb[EM];
                    const int li = gi + k * gpt;
                    const bool gv = li < X.nlines;
                    const int p0 = jr * X.E;
                    const int qb = (gv ? line_first(X, li) : 0) + p0;
#pragma unroll
                    for (int i = 0; i < EM; ++i) {
                        ha[i] = kBig;
                        hb[i] = kBig;
                        if (gv && i < X.E && p0 + i < X.L) {
                            const int q = qb + i;
                            const int c = sc[q], d = sd[q];
                            int t = sC[q];
                            if (has_ma) t += maS[q];
                            if (mbv) t += mbv[q];
                            ha[i] = floor_half(t + d - c);
                            hb[i] = floor_half(t + c - d);
                            if (fin) {
                                const int so = t + c + d;
                                key = min(key, ((unsigned long long)((unsigned)so ^ 0x80000000u) << 32) | (unsigned)q);
                            }
                        }
                    }
                    const int2 lm = seg_dt2<EM>(ha, hb, X.E, X.G, jr, A.lam, X.kc);
                    if (gv) {
                        ja = min(ja, lm.x);
                        jb = min(jb, lm.y);
                    }
                    if (R == 1 || per_axis) {
                        const int ca = lm.x + A.capv, cb = lm.y + A.capv;
#pragma unroll
                        for (int i = 0; i < EM; ++i) {
                            ha[i] = min(ha[i], ca);
                            hb[i] = min(hb[i], cb);
                        }
                    }
                    if (gv) {
#pragma unroll
                        for (int i = 0; i < EM; ++i) {
                            if (i < X.E && p0 + i < X.L) {
                                const int q = qb + i;
                                if (R == 1) {
                                    emit(q, ha[i], hb[i]);
                                } else {
                                    tA[q] = ha[i];
                                    tB[q] = hb[i];
                                }
                            }
                        }
                    }
                }
            }
            if (!barrier2(ja, jb)) {
                aborted = true;
                break;
            }
            // ---- phases 1 .. R-1: sweeps of the other axes, clip, emit ----
            if (R >= 2) {
                int ga = kBig, gb = kBig;
                if (!per_axis) {
                    for (int w = 0; w < T; ++w) {
                        ga = min(ga, wmin[2 * w]);
                        gb = min(gb, wmin[2 * w + 1]);
                    }
                }
#pragma unroll 1
                for (int ax = 1; ax < R; ++ax) {
                    if (ax == 2) sync(tm, T);
                    const TeamAxis X = A.ax[ax];
                    const bool last = (ax == R - 1);
                    const int lg = __ffs(X.G) - 1;
                    const int jr = tl & (X.G - 1), gi = tl >> lg, gpt = NL >> lg;
#pragma unroll 1
                    for (int k = 0; k < X.rounds; ++k) {
                        int va[EM], vb[EM];
                        const int li = gi + k * gpt;
                        const bool gv = li < X.nlines;
                        const int p0 = jr * X.E;
                        const int qb = (gv ? line_first(X, li) : 0) + p0 * X.stride;
#pragma unroll
                        for (int i = 0; i < EM; ++i) {
                            va[i] = kBig;
                            vb[i] = kBig;
                            if (gv && i < X.E && p0 + i < X.L) {
                                va[i] = tA[qb + i * X.stride];
                                vb[i] = tB[qb + i * X.stride];
                            }
                        }
                        const int2 lm = seg_dt2<EM>(va, vb, X.E, X.G, jr, A.lam, X.kc);
                        const int ca = (per_axis ? lm.x : ga) + A.capv;
                        const int cb = (per_axis ? lm.y : gb) + A.capv;
                        if (gv) {
#pragma unroll
                            for (int i = 0; i < EM; ++i) {
                                if (i < X.E && p0 + i < X.L) {
                                    const int q = qb + i * X.stride;
                                    if (last) {
                                        emit(q, min(va[i], ca), min(vb[i], cb));
                                    } else {
                                        tA[q] = per_axis ? min(va[i], ca) : va[i];
                                        tB[q] = per_axis ? min(vb[i], cb) : vb[i];
                                    }
                                }
                            }
                        }
                    }
                }
            }
            }
            if (to_mbox) {
                __syncwarp();
                if (lane == 0) st_rel_cta(produced + wt, s + 1);
            }
        }
        }
        cp_async_wait_0();
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

// dispatch on the form and its bound
template <typename F>
__device__ __forceinline__ bool team_dispatch(int em, bool lean, F &&f) {
    if (lean) {
        switch (em) {
        case 9: return f(std::integral_constant<int, 9>(), std::true_type());
        case 17: return f(std::integral_constant<int, 17>(), std::true_type());
        default: return f(std::integral_constant<int, 33>(), std::true_type());
        }
    }
    switch (em) {
    case 9: return f(std::integral_constant<int, 9>(), std::false_type());
    case 17: return f(std::integral_constant<int, 17>(), std::false_type());
    default: return f(std::integral_constant<int, 33>(), std::false_type());
    }
}

}  // namespace edp
