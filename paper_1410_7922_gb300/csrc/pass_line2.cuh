// pass_line2.cuh -- EDP scan pass for two-axis label spaces whose lines hold
// 33 to 65 labels, each label line shared by two lanes.
//
// Same messages, flags, pass schedule and hand-off protocol as
// pass_line.cuh; what differs is that a line of L labels is split into a
// first half of 32 labels and a second half of L - 32, held by lanes l and
// l + 16 of one warp (a warp serves 16 lines).  A lane loads, sums and
// halves only its half of the line, so the per-lane state, the loads in
// flight per lane and the dependent sweep chains are half as long.
//
// The LRMS sweeps of Sec. 3.2 over a split line.  The backward sweep
// (Eq. L_dec5) is the minimum over j >= i of h[j] + lambda (j - i), so after
// each half ran it on its own the first half only misses the sources of the
// second half, which all reach label i through label 32:
//     b[i] = min(b_1st[i], b[32] + lambda (32 - i))     (i < 32),
// and b[32] is the second half's own first value.  Likewise the forward
// sweep (Eq. L_dec3) over b, f[i] = min over j <= i of b[j] + lambda (i - j),
// completes the second half with the first half's last value:
//     f[i] = min(f_2nd[i], f[31] + lambda (i - 31))     (i >= 32).
// Each completion is one shuffle and a set of independent add-mins.  The
// products lambda k (k <= 33) stay below 2^30, which the planner checks
// before it picks this kernel.
//
// Shared memory: the [LA][LB] transposition buffers (X_a and the two mailbox
// slots of each team) are stored as four quadrants (i < 32 or not, k < 32 or
// not) with a row pitch of 33 and bases placed so that, in both phases, the
// 16 lanes of the first halves and the 16 of the second halves fall on
// different banks.
//
// Between blocks the hand-off ships the mailbox slot as it is: a ring of
// slot images in global memory (the quadrant layout, plain 32-bit values,
// no {value, tag} words).  Each thread of the last row of a block copies its
// 16-byte chunks of the outgoing slot there, then one lane per warp
// publishes them with a release store of the warp's flag at GPU scope; the
// same thread of the first row of the block below acquires that flag and
// copies the same chunks into its own, otherwise unused, mailbox slot with
// asynchronous copies (no registers in flight), and after a team barrier
// the row runs as every other row.
#pragma once
#include "pass_line.cuh"

namespace edp {
namespace line2 {

constexpr int kPQ = 33;        // row pitch of a quadrant (odd)
constexpr int kMaxWarps = 8;   // warps per team (16 lines each)
constexpr int kMaxThreads = 640;
// control ints of one team: [0, 8) produced columns per warp, [8, 16)
// consumed columns per warp, [16, 24) / [24, 32) warp minima of the halved
// S_a / S_b sums, [32, 48) warp argmin keys (eight 64-bit); 64 in all, so
// that the buffers after it start on bank 0
constexpr int kCtl = 64;

// smallest y >= x with y = r (mod 32)
__host__ __device__ constexpr int up32(int x, int r) { return x + ((r - x) % 32 + 32) % 32; }
// base of quadrant (hi, hk) of an [LA][LB] buffer (rows i in [32 hi, ...),
// columns k in [32 hk, ...)); bases 0, 16, 16, 0 (mod 32)
__host__ __device__ constexpr int qbase(int LA, int hi, int hk) {
    return hi == 0 ? (hk == 0 ? 0 : up32(32 * kPQ, 16))
                   : (hk == 0 ? up32(up32(32 * kPQ, 16) + 32 * kPQ, 16)
                              : up32(up32(up32(32 * kPQ, 16) + 32 * kPQ, 16) + (LA - 32) * kPQ, 0));
}
__host__ __device__ constexpr int buf_ints(int LA) { return up32(qbase(LA, 1, 1) + (LA - 32) * kPQ, 0); }
// ints of shared memory of one team: control, X_a, two mailbox slots
__host__ __device__ constexpr size_t team_ints(int LA) { return kCtl + 3 * (size_t)buf_ints(LA); }
// the planner's bound on the prior weight (the completions add lambda * 33)
constexpr int kMaxLambda = (1 << 30) / 34;

// Global loads as volatile asm: issued in program order, so that a batch is
// in flight as a whole (the compiler does not sink them to their uses)
__device__ __forceinline__ int ld_cs(const int *p) {
    int v;
    asm volatile("ld.global.cs.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ int ld_cg(const int *p) {
    int v;
    asm volatile("ld.global.cg.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ unsigned ld_acq_gpu(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_rel_gpu(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// LRMS sweeps of one split line, in place: the lane holds labels [32 hf,
// 32 hf + n) of the line in h[0, n), kBig above; its partner lane (lane ^ 16)
// the other half.  Then the clip.  mask: the lanes of the warp that call it
// (partners together).
template <int N>
__device__ __forceinline__ void split_sweeps(int (&h)[N], const bool lo, const int lam, const int clip,
                                             const unsigned mask) {
#pragma unroll
    for (int i = N - 2; i >= 0; --i) h[i] = __viaddmin_s32(h[i + 1], lam, h[i]);
    const int cb = __shfl_xor_sync(mask, h[0], 16);  // b[32], from the second half
    if (lo) {
#pragma unroll
        for (int i = 0; i < 32; ++i) h[i] = __viaddmin_s32(cb, lam * (32 - i), h[i]);
    }
#pragma unroll
    for (int i = 1; i < N; ++i) h[i] = __viaddmin_s32(h[i - 1], lam, h[i]);
    const int cf = __shfl_xor_sync(mask, h[31], 16);  // f[31], from the first half
    if (!lo) {
#pragma unroll
        for (int i = 0; i < N; ++i) h[i] = __viaddmin_s32(cf, lam * (i + 1), h[i]);
    }
#pragma unroll
    for (int i = 0; i < N; ++i) h[i] = min(h[i], clip);
}

// Phase A loads of one half label column of one pixel: C straight into hv
// (all of it in flight at once, in the registers the line needs anyway),
// the old messages m_c and m_d (global, coalesced across the 16 lanes of
// each half) in batches of CH labels one batch ahead of the arithmetic, m_a
// from xa and m_b from xb (shared memory, stride kPQ); the messages this
// pixel received written to the message arrays, and the two halved sums of
// Eq. DP_2D_base: S_a into hv (kBig above the lane's n labels), S_b over m_b
// in xb.  Two batches are in flight ahead of the arithmetic.
template <int N, int LB, int CH>
__device__ __forceinline__ void issue_batch(const int *__restrict__ Mcp, const int *__restrict__ Mdp,
                                            const bool c_ok, const bool d_ok, const int n, const int b,
                                            int (&mcv)[CH], int (&mdv)[CH]) {
#pragma unroll
    for (int jj = 0; jj < CH; ++jj) {
        const int i = b * CH + jj;
        if (i < N && i < n) {
            const int o = i * LB;
            mcv[jj] = c_ok ? ld_cs(Mcp + o) : 0;
            mdv[jj] = d_ok ? ld_cs(Mdp + o) : 0;
        }
    }
}
// The pair cost of Eq. Cost_value for the lane's half column, computed from
// the images: label i of the half has I1 row ys0 + t1 i at column col (the
// lane's axis-0 offset); C = cmax outside the image, else
// min(|I1 - I0(x)|^l2, cmax) -- the same values the cost kernels store.
struct FusedCost {
    const uint8_t *col;  // I1 + the lane's column (read only when col_ok)
    bool col_ok;
    int ys0, t1, H, pitch, i0, cmax, l2;
};
template <int N, int LB, int CH, bool FUSED>
__device__ __forceinline__ void front_load(const int *__restrict__ Cp, const FusedCost &fc,
                                           const int *__restrict__ Mcp, const int *__restrict__ Mdp,
                                           const bool c_ok, const bool d_ok, const int n, int (&hv)[N],
                                           int (&mcv)[2][CH], int (&mdv)[2][CH]) {
    constexpr int NB = (N + CH - 1) / CH;
    if constexpr (FUSED) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            if (i < n) {
                const int ys = fc.ys0 + fc.t1 * i;
                int c = fc.cmax;
                if (fc.col_ok && (unsigned)ys < (unsigned)fc.H) {
                    const int d = abs((int)fc.col[(size_t)ys * fc.pitch] - fc.i0);
                    c = min(fc.l2 == 1 ? d : d * d, fc.cmax);
                }
                hv[i] = c;
            } else {
                hv[i] = kBig;
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) hv[i] = i < n ? ld_cs(Cp + i * LB) : kBig;
    }
    issue_batch<N, LB, CH>(Mcp, Mdp, c_ok, d_ok, n, 0, mcv[0], mdv[0]);
    if (NB > 1) issue_batch<N, LB, CH>(Mcp, Mdp, c_ok, d_ok, n, 1, mcv[1], mdv[1]);
}
template <int N, int LB, int CH, bool FUSED>
__device__ __forceinline__ void half_load(const int *__restrict__ Cp, const FusedCost &fc, const int *__restrict__ Mcp,
                                          const int *__restrict__ Mdp, int *__restrict__ Map,
                                          int *__restrict__ Mbp, const int *__restrict__ xa, int *__restrict__ xb,
                                          const bool c_ok, const bool d_ok, const bool has_ma, const bool mbox,
                                          const bool st_a, const bool st_b, const bool fin, const int n,
                                          const int q0, int (&hv)[N], int &lmin_a, int &lmin_b,
                                          unsigned long long &key) {
    constexpr int NB = (N + CH - 1) / CH;
    int mcv[2][CH], mdv[2][CH];
    front_load<N, LB, CH, FUSED>(Cp, fc, Mcp, Mdp, c_ok, d_ok, n, hv, mcv, mdv);
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int k = b & 1;
#pragma unroll
        for (int jj = 0; jj < CH; ++jj) {
            const int i = b * CH + jj;
            if (i < N && i < n) {
                const int o = i * LB;
                const int mc = mcv[k][jj], md = mdv[k][jj];
                const int ma = has_ma ? xa[i * kPQ] : 0;
                const int mb = mbox ? xb[i * kPQ] : 0;
                if (st_a) __stcs(Map + o, ma);
                if (st_b) __stcs(Mbp + o, mb);
                const int t = hv[i] + ma + mb, e = md - mc;
                const int ha = floor_half(t + e), hb = floor_half(t - e);
                if (fin) key = min(key, line::argmin_key(t + mc + md, q0 + o));
                hv[i] = ha;
                xb[i * kPQ] = hb;
                lmin_a = min(lmin_a, ha);
                lmin_b = min(lmin_b, hb);
            }
        }
        // the batch after next, into the registers just consumed
        if (b + 2 < NB) issue_batch<N, LB, CH>(Mcp, Mdp, c_ok, d_ok, n, b + 2, mcv[k], mdv[k]);
    }
}

// 16-byte asynchronous copy global -> shared (L2 only), and the wait for
// this thread's copies
__device__ __forceinline__ void cp_async16(int *sdst, const int *gsrc) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(sdst)),
                 "l"(gsrc)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

}  // namespace line2

// One row band of one scan pass (or paired sweep) for a label space of
// LB x LA labels (axis 0: LB labels, contiguous; axis 1: LA labels), lines
// split over lane pairs.  Every thread of the block calls it with the same
// band; returns false when the pass was aborted (a wait timed out).
template <int LA, int LB, int CH, bool FUSED>
__device__ __forceinline__ bool line2_band(const TeamArgs &A, const int band, int *smem, volatile int *s_abort) {
    using namespace line;
    using line2::kPQ;
    static_assert(LA >= 33 && LA <= 65 && LB >= 33 && LB <= 65, "lines of 33 to 65 labels");
    constexpr int NA = LA - 32 > 32 ? LA - 32 : 32;  // register line of phase A
    constexpr int NBr = LB - 32 > 32 ? LB - 32 : 32;  // and of phase B
    constexpr int XS = line2::buf_ints(LA);
    constexpr size_t TI = line2::team_ints(LA);
    constexpr int KC = line2::kCtl;
    const int W = A.W, H = A.H, Q = A.Q, Qm = A.Qm, TW = A.T, NT = A.NT, ring = A.ring;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tm = warp / TW, wt = warp - tm * TW, tl = wt * 32 + lane;
    const int hf = lane >> 4, j = wt * 16 + (lane & 15);  // half, line
    const bool lo = hf == 0;
    for (int i = tid; i < NT * KC; i += blockDim.x) smem[(size_t)(i / KC) * TI + i % KC] = 0;
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
        int *const Xa = ctl + KC;
        int *const nx_slots = to_mbox ? smem + (size_t)(tm + 1) * TI + KC + XS : nullptr;
        const int *const nx_ctl = to_mbox ? smem + (size_t)(tm + 1) * TI : nullptr;
        const int *const pv_ctl = from_mbox ? smem + (size_t)(tm - 1) * TI : nullptr;
        // the ring of slot images between blocks: [band][ring][XS] ints; the
        // team's thread tl moves the 16-byte chunks tl, tl + 32 TW, ...
        int *const llv = reinterpret_cast<int *>(A.ll);
        const int *const ll_in = from_ring ? llv + (size_t)(band - 1) * ring * XS : nullptr;
        int *const ll_out = to_ring ? llv + (size_t)band * ring * XS : nullptr;
        const unsigned *const flag_in = from_ring ? A.rflag + (size_t)(band - 1) * kLineFlagStride + wt : nullptr;
        unsigned *const flag_out = to_ring ? A.rflag + (size_t)band * kLineFlagStride + wt : nullptr;
        unsigned *const cons_in = from_ring ? A.cons + (size_t)(band - 1) * kLineFlagStride + wt : nullptr;
        const unsigned *const cons_out = to_ring ? A.cons + (size_t)band * kLineFlagStride + wt : nullptr;
        // the test hook hold_band makes one band wait for a column never published
        const int hold = band == A.hold_band ? 0x20000000 : 0;
        const int ncol = A.pair ? 2 * W : W;
        const bool colA = j < LB, rowB = j < LA;
        const unsigned mA = __ballot_sync(kFull, colA), mB = __ballot_sync(kFull, rowB);
        const int nA = lo ? 32 : LA - 32, nB = lo ? 32 : LB - 32;
        const int jj = j >= 32 ? j - 32 : j;
        const int offA = line2::qbase(LA, hf, j >= 32) + jj;        // X(32 hf + n, j) at offA + n kPQ
        const int offB = line2::qbase(LA, j >= 32, hf) + jj * kPQ;  // X(j, 32 hf + n) at offB + n
        const int q0 = hf * 32 * LB + j;                             // label of the lane's first phase-A entry
        unsigned cons_seen = 0;
        for (int s = 0; s < ncol; ++s) {
            const int hh = s >= W ? 1 : 0;
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
            int *const Xb = Xa + (1 + (s & 1)) * XS;
            if (s + 1 < ncol) {  // L2 prefetch of the next column's C, m_c, m_d
                const int s2 = s + 1, h2 = s2 >= W ? 1 : 0, xs2 = s2 - h2 * W;
                const bool incx2 = ((A.pass + h2) & 1) == 0;
                const int x2 = incx2 ? xs2 : W - 1 - xs2;
                const size_t p2 = (size_t)y * W + x2;
                const bool rc2 = (h2 ? A.read_c2 : A.read_c) && (incx2 ? x2 + 1 < W : x2 - 1 >= 0);
                const int *const pc = FUSED ? nullptr : A.C + p2 * Q;
                const int *const pm = (incx2 ? A.M[1] : A.M[0]) + p2 * Qm;
                const int *const pd = Md + p2 * Qm;
                for (int o = tl * 32; o < Q; o += 32 * 32 * TW) {
                    if (!FUSED) prefetch_line_l2(pc + o);
                    if (rc2) prefetch_line_l2(pm + o);
                    if (d_ok) prefetch_line_l2(pd + o);
                }
            }
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
            } else if (from_ring) {
                // the producing warp's chunks of column s: published flag
                // (acquired by every lane, which orders its copies after it)
                while (true) {
                    const bool ok = (int)line2::ld_acq_gpu(flag_in) >= s + 1 + hold;
                    if (__all_sync(kFull, ok)) break;
                    if (__any_sync(kFull, ++spins > A.spin_limit || *s_abort != 0 ||
                                              ((spins & 63) == 0 && *(volatile int *)A.status != 0))) {
                        bad = true;
                        break;
                    }
                    __nanosleep(32);
                }
                if (!bad) {
                    const int *const src = ll_in + (size_t)(s % ring) * XS;
                    for (int c = tl; c < XS / 4; c += 32 * TW) line2::cp_async16(Xb + 4 * c, src + 4 * c);
                    line2::cp_async_wait_all();
                    // the chunks are in shared memory: the producer may reuse them
                    __syncwarp();
                    if (lane == 0) st_relaxed_gpu(cons_in, (unsigned)(s + 1));
                }
                team_sync(tm, TW);  // every warp's chunks of the slot have arrived
            }
            if (!bad && to_mbox) {  // the slot of this column in the team below is free
                spins = 0;
                while (true) {
                    const bool ok = lane >= TW || ld_acq_cta(nx_ctl + 8 + lane) >= s - 1;
                    if (__all_sync(kFull, ok)) break;
                    if (__any_sync(kFull, ++spins > A.spin_limit || *s_abort != 0)) {
                        bad = true;
                        break;
                    }
                }
            }

            // ---- phase A: sums of Eq. DP_2D_base, halving, sweeps along axis 1 ----
            unsigned long long key = ~0ull;
            int lmin_a = kBig, lmin_b = kBig;
            int hv[NA];
            if (!bad && colA) {
                const bool st_a = write_a && has_ma, st_b = write_b && r > 0;
                line2::FusedCost fc{};
                if constexpr (FUSED) {
                    const int xs = x + A.fv0 + A.ft0 * j;
                    fc.col_ok = (unsigned)xs < (unsigned)W;
                    fc.col = A.fI1 + (fc.col_ok ? xs : 0);
                    fc.ys0 = y + A.fv1 + A.ft1 * 32 * hf;
                    fc.t1 = A.ft1;
                    fc.H = H;
                    fc.pitch = A.fpitch;
                    fc.i0 = A.fI0[(size_t)y * A.fpitch + x];
                    fc.cmax = A.fcmax;
                    fc.l2 = A.fl2;
                }
                line2::half_load<NA, LB, CH, FUSED>(FUSED ? nullptr : A.C + pix * Q + q0, fc, Mc + pix * Qm + q0,
                                                    Md + pix * Qm + q0,
                                             Ma + pix * Qm + q0, Mb + pix * Qm + q0, Xa + offA, Xb + offA, c_ok,
                                             d_ok, has_ma, r > 0, st_a, st_b, fin, nA, q0, hv, lmin_a, lmin_b,
                                             key);
                const int la = min(lmin_a, __shfl_xor_sync(mA, lmin_a, 16));
                const int lb = min(lmin_b, __shfl_xor_sync(mA, lmin_b, 16));
                line2::split_sweeps<NA>(hv, lo, lam_a, per_axis ? la + cap_a : kBig, mA);
#pragma unroll
                for (int i = 0; i < NA; ++i)
                    if (i < nA) Xa[offA + i * kPQ] = hv[i];
#pragma unroll
                for (int i = 0; i < NA; ++i) hv[i] = i < nA ? Xb[offA + i * kPQ] : kBig;
                line2::split_sweeps<NA>(hv, lo, lam_b, per_axis ? lb + cap_b : kBig, mA);
#pragma unroll
                for (int i = 0; i < NA; ++i)
                    if (i < nA) Xb[offA + i * kPQ] = hv[i];
            }
            if (!per_axis) {
                const int ja = __reduce_min_sync(kFull, lmin_a), jb = __reduce_min_sync(kFull, lmin_b);
                if (lane == 0) {
                    ctl[16 + wt] = ja;
                    ctl[24 + wt] = jb;
                }
            }
            if (fin) {
                key = warp_min_key(key);
                if (lane == 0) reinterpret_cast<unsigned long long *>(ctl + 32)[wt] = key;
            }
            if (bad) {
                atomicCAS(A.status, 0, EDP_ERR_TIMEOUT_CODE);
                *s_abort = 1;
            }
            if (team_sync_or(tm, TW, bad || *s_abort != 0)) break;  // barrier: phase A done
            if (fin && tl == 0) {
                unsigned long long best = reinterpret_cast<unsigned long long *>(ctl + 32)[0];
                for (int w = 1; w < TW; ++w) best = min(best, reinterpret_cast<unsigned long long *>(ctl + 32)[w]);
                A.labels[pix] = (int)(best & 0xffffffffu);
            }

            // ---- phase B: sweeps along axis 0, clip, outputs ----
            if (rowB) {
                int ga = kBig, gb = kBig;
                if (!per_axis)
                    for (int w = 0; w < TW; ++w) {
                        ga = min(ga, ctl[16 + w]);
                        gb = min(gb, ctl[24 + w]);
                    }
                int *const ra = Xa + offB;
                int *const rb = Xb + offB;
                int gv[NBr];
                int lm = kBig;
#pragma unroll
                for (int i = 0; i < NBr; ++i) {
                    gv[i] = i < nB ? ra[i] : kBig;
                    lm = min(lm, gv[i]);
                }
                lm = min(lm, __shfl_xor_sync(mB, lm, 16));
                line2::split_sweeps<NBr>(gv, lo, lam_a, (per_axis ? lm : ga) + cap_a, mB);
                if (nxt) {  // m_a of the next column of the row
#pragma unroll
                    for (int i = 0; i < NBr; ++i)
                        if (i < nB) ra[i] = gv[i];
                }
                lm = kBig;
#pragma unroll
                for (int i = 0; i < NBr; ++i) {
                    gv[i] = i < nB ? rb[i] : kBig;
                    lm = min(lm, gv[i]);
                }
                lm = min(lm, __shfl_xor_sync(mB, lm, 16));
                line2::split_sweeps<NBr>(gv, lo, lam_b, (per_axis ? lm : gb) + cap_b, mB);
                if (to_mbox) {  // m_b of this column of the row below
                    int *const nb = nx_slots + (s & 1) * XS + offB;
#pragma unroll
                    for (int i = 0; i < NBr; ++i)
                        if (i < nB) nb[i] = gv[i];
                } else if (to_ring) {
#pragma unroll
                    for (int i = 0; i < NBr; ++i)
                        if (i < nB) rb[i] = gv[i];
                }
            }
            if (to_mbox) {
                __syncwarp();
                if (lane == 0) st_rel_cta(ctl + wt, s + 1);
            }
            team_sync(tm, TW);  // barrier: rows of X_a (and of the outgoing slot) written

            // ---- phase C (last row of the block): the outgoing slot into the ring ----
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
                if (!bad) {
                    int *const dst = ll_out + (size_t)(s % ring) * XS;
                    for (int c = tl; c < XS / 4; c += 32 * TW)
                        __stcg(reinterpret_cast<int4 *>(dst) + c, reinterpret_cast<const int4 *>(Xb)[c]);
                }
                // publish column s: the warp's stores, then the flag (release at
                // GPU scope, cumulative over the stores the barrier ordered)
                __syncwarp();
                if (!bad && lane == 0) line2::st_rel_gpu(flag_out, (unsigned)(s + 1));
                if (bad) {
                    atomicCAS(A.status, 0, EDP_ERR_TIMEOUT_CODE);
                    *s_abort = 1;
                }
            }
            if (from_mbox) {  // this column's slot is free again for the team above
                __syncwarp();
                if (lane == 0) st_rel_cta(ctl + 8 + wt, s + 1);
            }
        }
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
