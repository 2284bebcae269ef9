// pass_r1.cuh -- one row band of an EDP scan pass for one label axis (Q <= 256).
//
// Same arithmetic as edp_pass.cu (Sec. 4.2, Eq. DP_2D_base with the data
// term, messages M(floor(S_k / 2)) stored at the receiving pixel), with a
// schedule built for latency: one warp owns one image row and keeps the
// message into its next pixel (m_a) in registers; lane j holds the E labels
// j*E .. j*E+E-1 of the row's current pixel.
//
//  - m_b from the previous row: through a shared-memory mailbox ring inside
//    the block (per-row produced / consumed counters, bounded spins), and
//    through a "value + tag" 8-byte record per label in global memory
//    between blocks: the consumer polls the records themselves until every
//    tag equals this pass's tag, so no memory fence sits on the path.
//  - C, m_c, m_d (read-only in the pass) are prefetched kPf columns ahead
//    with cp.async into a per-warp shared-memory ring.
//  - M of the truncated linear prior: per-lane forward/backward sweeps
//    (Eq. L_dec3, Eq. L_dec5), carries from the lanes within distance < g
//    (farther labels cost at least the clip value), the minimum by
//    redux.sync, then the clip of Eq. derivation1.
#pragma once
#include "common.cuh"
#include "kernels.h"

namespace edp {

namespace {
constexpr int kPf = 7;   // prefetch distance in columns (ring of kPf + 1)
constexpr int kMb = 4;   // mailbox ring depth between rows of a block

__device__ __forceinline__ int redux_min(int v) { return __reduce_min_sync(0xffffffffu, v); }

// In-place truncated L1 distance transform of one row vector held as
// v[0..E) per lane over a full warp; carries from `kc` lanes on each side.
template <int EM>
__device__ __forceinline__ void dt_trunc(int (&v)[EM], int E, int lane, int lam, int kc) {
    int f[EM], b[EM];
    f[0] = v[0];
#pragma unroll
    for (int i = 1; i < EM; ++i)
        if (i < E) f[i] = min(v[i], f[i - 1] + lam);
#pragma unroll
    for (int i = EM - 1; i >= 0; --i)
        if (i < E) b[i] = (i == E - 1) ? v[i] : min(v[i], b[i + 1] + lam);
    int F = f[0], B = b[0];
#pragma unroll
    for (int i = 0; i < EM; ++i)
        if (i == E - 1) F = f[i];
    int cf = kBig, cb = kBig;
    for (int d = 1; d <= kc; ++d) {
        const int tf = __shfl_up_sync(0xffffffffu, F, d);
        const int tb = __shfl_down_sync(0xffffffffu, B, d);
        const int gap = lam * ((d - 1) * E + 1);
        if (lane >= d) cf = min(cf, tf + gap);
        if (lane + d < 32) cb = min(cb, tb + gap);
    }
#pragma unroll
    for (int i = 0; i < EM; ++i)
        if (i < E) v[i] = min(min(f[i], cf + lam * i), min(b[i], cb + lam * (E - 1 - i)));
}

__device__ __forceinline__ int ld_volatile_shared(const int *p) {
    return *reinterpret_cast<const volatile int *>(p);
}
__device__ __forceinline__ void st_volatile_shared(int *p, int v) { *reinterpret_cast<volatile int *>(p) = v; }

__device__ __forceinline__ int2 ld_ll(const int2 *p) {
    int2 r;
    asm volatile("ld.relaxed.gpu.global.v2.s32 {%0, %1}, [%2];" : "=r"(r.x), "=r"(r.y) : "l"(p) : "memory");
    return r;
}
__device__ __forceinline__ void st_ll(int2 *p, int v, int tag) {
    asm volatile("st.relaxed.gpu.global.v2.s32 [%0], {%1, %2};" ::"l"(p), "r"(v), "r"(tag) : "memory");
}
}  // namespace

// One row band (NWR rows, one warp each) of one scan pass.  Every thread of
// the block calls it with the same band; returns false when the pass was
// aborted (a wait timed out).
template <int EM>
__device__ __forceinline__ bool r1_band(const PassR1Args &A, const int band, int *smem_i, volatile int *s_abort) {
    const int Q = A.Q, E = A.E, W = A.W, H = A.H, NWR = A.NWR;
    const int Qp = 32 * E;  // padded vector length in shared memory
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
        const size_t row0 = (size_t)y * W * Q;
        const size_t rown = (size_t)(has_next ? y_next : y) * W * Q;
        const int2 *ll_in = A.ll + (size_t)(band - 1) * W * Q;   // previous band's last row
        int2 *ll_out = A.ll + (size_t)band * W * Q;
        const int q0 = lane * E;

        auto prefetch = [&](int s) {
            if (s < W) {
                const int x = incx ? s : W - 1 - s;
                const bool c_ok = A.read_c && (incx ? x + 1 < W : x - 1 >= 0);
                const size_t pix = row0 + (size_t)x * Q;
                int *dst = ring + (s % (kPf + 1)) * 3 * Qp;
#pragma unroll
                for (int i = 0; i < EM; ++i) {
                    const int q = q0 + i;
                    if (i < E && q < Q) {
                        cp_async4(dst + q, A.C + pix + q, true);
                        cp_async4(dst + Qp + q, Mc + pix + q, c_ok);
                        cp_async4(dst + 2 * Qp + q, Md + pix + q, d_ok);
                    }
                }
            }
            cp_async_commit();
        };
        for (int s = 0; s < kPf; ++s) prefetch(s);

        int ma[EM];
#pragma unroll
        for (int i = 0; i < EM; ++i) ma[i] = 0;
        long long spins = 0;
        for (int s = 0; s < W; ++s) {
            const int x = incx ? s : W - 1 - s;
            prefetch(s + kPf);
            cp_async_wait_n<kPf>();
            const int *src = ring + (s % (kPf + 1)) * 3 * Qp;
            // ---- m_b from the previous row ----
            int mb[EM];
#pragma unroll
            for (int i = 0; i < EM; ++i) mb[i] = 0;
            if (r > 0) {
                if (w > 0) {
                    if (lane == 0) {
                        spins = 0;
                        while (ld_volatile_shared(produced + w - 1) < s + 1) {
                            if (++spins > A.spin_limit || (*s_abort)) {
                                atomicCAS(A.status, 0, EDP_ERR_TIMEOUT_CODE);
                                *s_abort = 1;
                                break;
                            }
                        }
                    }
                    __syncwarp();
                    __threadfence_block();
                    const int *mbx = mbox + ((w - 1) * kMb + s % kMb) * Qp;
#pragma unroll
                    for (int i = 0; i < EM; ++i)
                        if (i < E) mb[i] = ld_volatile_shared(mbx + q0 + i);
                    __syncwarp();
                    if (lane == 0) st_volatile_shared(consumed + w, s + 1);
                } else {
                    const unsigned long long tw = A.trace ? global_ns() : 0;
                    const int2 *p = ll_in + (size_t)s * Q;
                    bool ok = false;
                    spins = 0;
                    while (true) {
                        ok = true;
#pragma unroll
                        for (int i = 0; i < EM; ++i) {
                            const int q = q0 + i;
                            if (i < E && q < Q) {
                                const int2 t = ld_ll(p + q);
                                mb[i] = t.x;
                                ok = ok && (t.y == A.tag);
                            }
                        }
                        if (__all_sync(0xffffffffu, ok)) break;
                        const bool bail = ++spins > A.spin_limit || (*s_abort) ||
                                          *(volatile int *)A.status != 0;
                        if (__any_sync(0xffffffffu, bail)) {
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
            }
            __syncwarp();
            if (__any_sync(0xffffffffu, (*s_abort) != 0)) break;
            // ---- sums (Eq. DP_2D_base) and halving ----
            int ha[EM], hb[EM];
            int lmin_a = kBig, lmin_b = kBig;
            int so_v = kBig, so_q = 0x7fffffff;
#pragma unroll
            for (int i = 0; i < EM; ++i) {
                const int q = q0 + i;
                if (i < E && q < Q) {
                    const int Cv = src[q], mc = src[Qp + q], md = src[2 * Qp + q];
                    const int sa = Cv + ma[i] + mb[i] + md - mc;
                    const int sb = Cv + ma[i] + mb[i] + mc - md;
                    ha[i] = floor_half(sa);
                    hb[i] = floor_half(sb);
                    lmin_a = min(lmin_a, ha[i]);
                    lmin_b = min(lmin_b, hb[i]);
                    if (A.final_) {
                        const int so = Cv + ma[i] + mb[i] + mc + md;
                        if (so < so_v) {
                            so_v = so;
                            so_q = q;
                        }
                    }
                } else {
                    ha[i] = kBig;
                    hb[i] = kBig;
                }
            }
            // ---- min search M (RMS sweeps + clip) ----
            const int ga = redux_min(lmin_a), gb = redux_min(lmin_b);
            dt_trunc<EM>(ha, E, lane, A.lam, A.kc);
            dt_trunc<EM>(hb, E, lane, A.lam, A.kc);
            const int clipa = ga + A.capv, clipb = gb + A.capv;
#pragma unroll
            for (int i = 0; i < EM; ++i) {
                ma[i] = min(ha[i], clipa);
                hb[i] = min(hb[i], clipb);
            }
            if (A.final_) {
                const int vbest = redux_min(so_v);
                const int qbest = redux_min(so_v == vbest ? so_q : 0x7fffffff);
                if (lane == 0) A.labels[(size_t)y * W + x] = qbest;
            }
            // ---- outputs ----
            if (A.write_a && s + 1 < W) {
                const int xn = incx ? x + 1 : x - 1;
                int *dst = Ma + row0 + (size_t)xn * Q;
#pragma unroll
                for (int i = 0; i < EM; ++i)
                    if (i < E && q0 + i < Q) dst[q0 + i] = ma[i];
            }
            if (has_next) {
                if (A.write_b) {
                    int *dst = Mb + rown + (size_t)x * Q;
#pragma unroll
                    for (int i = 0; i < EM; ++i)
                        if (i < E && q0 + i < Q) dst[q0 + i] = hb[i];
                }
                if (!last_in_band) {
                    if (lane == 0 && s >= kMb) {
                        spins = 0;
                        while (ld_volatile_shared(consumed + w + 1) < s - kMb + 1) {
                            if (++spins > A.spin_limit || (*s_abort)) {
                                atomicCAS(A.status, 0, EDP_ERR_TIMEOUT_CODE);
                                *s_abort = 1;
                                break;
                            }
                        }
                    }
                    __syncwarp();
                    int *mbx = mbox + (w * kMb + s % kMb) * Qp;
#pragma unroll
                    for (int i = 0; i < EM; ++i)
                        if (i < E) st_volatile_shared(mbx + q0 + i, hb[i]);
                    __threadfence_block();
                    __syncwarp();
                    if (lane == 0) st_volatile_shared(produced + w, s + 1);
                } else {
                    int2 *p = ll_out + (size_t)s * Q;
#pragma unroll
                    for (int i = 0; i < EM; ++i)
                        if (i < E && q0 + i < Q) st_ll(p + q0 + i, hb[i], A.tag);
                }
            }
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

}  // namespace edp
