// common.cuh -- device helpers shared by the libedp kernels (sm_103a).
//
// The min search operator M of Eq. M_strf for the truncated linear prior is
// evaluated with the recursive minimum search of Sec. 3.2 (LRMS): per label
// axis r the operator L_r of Eq. L_dec6 -- a forward sweep (Eq. L_dec3) and a
// backward sweep (Eq. L_dec5) along every line of the label grid -- followed
// by the clip by S_min + lambda * f(g) of Eq. derivation1 (joint truncation)
// or by the line minimum + lambda * f(g) after every axis (per-axis
// truncation).
//
// GPU mapping of one line of L labels: a group of G lanes (G a power of two,
// G <= 32), lane j holding the E = ceil(L / G) consecutive labels
// j*E .. j*E + E - 1 in registers.  Each lane runs the two sweeps over its own
// E labels; the carries between lanes are a min-plus prefix (suffix) scan with
// __shfl_up_sync / __shfl_down_sync over the group, using
//   min_{u <= v} h(u) + lam (v - u) = lam v + min_{u <= v} (h(u) - lam u).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace edp {

constexpr int kEM = 16;                 // max labels per lane on one line
constexpr int kMaxThreads = 512;        // block size limit of the DP kernels
constexpr int kBig = 0x3fffffff;        // "no candidate" in int32 sweeps
constexpr int kMaxLine = 32 * kEM;      // longest label axis supported (512)
constexpr long long kBigKey = ((long long)kBig << 32) | 0xffffffffLL;

// floor(s / 2) for any sign (the 1/D factor of Eq. DP_2D_1 with D = 2).
__device__ __forceinline__ int floor_half(int s) { return s >> 1; }  // arithmetic shift

// One label axis of the grid as seen by the kernels.
struct AxisCfg {
    int L;       // labels on this axis (line length)
    int G;       // lanes per line (power of two)
    int E;       // labels per lane, ceil(L / G)
    int nlines;  // Q / L
    int stride;  // distance between neighbours on this axis in the linear index
};

// Linear index of the first label of line `l` on an axis with `stride`.
__device__ __forceinline__ int line_base(const AxisCfg &a, int l) {
    int inner = l % a.stride;
    int outer = l / a.stride;
    return inner + outer * a.stride * a.L;
}

// L1 distance transform of one line held as v[0..E) per lane (Eq. L_dec6),
// weight lam per label step, in place.  Positions >= L must hold kBig.
// Returns the minimum of the input over the whole line (all lanes of the
// group get it).  All 32 lanes of the warp must call this together with the
// same G (width of the shuffles).
template <int EM>
__device__ __forceinline__ int line_dt(int (&v)[EM], int E, int G, int j, int lam) {
    const unsigned full = 0xffffffffu;
    int f[EM], b[EM];
    int lmin = kBig;
#pragma unroll
    for (int i = 0; i < EM; ++i)
        if (i < E) lmin = min(lmin, v[i]);
    // forward sweep inside the lane
    f[0] = v[0];
#pragma unroll
    for (int i = 1; i < EM; ++i)
        if (i < E) f[i] = min(v[i], f[i - 1] + lam);
    // backward sweep inside the lane
    int last = v[0];
#pragma unroll
    for (int i = 0; i < EM; ++i)
        if (i == E - 1) last = v[i];
    b[EM - 1] = kBig;
#pragma unroll
    for (int i = EM - 1; i >= 0; --i) {
        if (i < E) {
            if (i == E - 1)
                b[i] = last;
            else
                b[i] = min(v[i], b[i + 1] + lam);
        }
    }
    if (G > 1) {
        int F = f[0];
#pragma unroll
        for (int i = 0; i < EM; ++i)
            if (i == E - 1) F = f[i];
        // prefix min over lanes of F_j - lam*E*j
        int a = F - lam * E * j;
        for (int d = 1; d < G; d <<= 1) {
            int t = __shfl_up_sync(full, a, d, G);
            if (j >= d) a = min(a, t);
        }
        int aex = __shfl_up_sync(full, a, 1, G);
        // suffix min over lanes of B_j + lam*E*j
        int c = b[0] + lam * E * j;
        for (int d = 1; d < G; d <<= 1) {
            int t = __shfl_down_sync(full, c, d, G);
            if (j + d < G) c = min(c, t);
        }
        int cex = __shfl_down_sync(full, c, 1, G);
        if (j > 0) {
            int cin = aex + lam * (E * (j - 1) + 1);  // value at position j*E
#pragma unroll
            for (int i = 0; i < EM; ++i)
                if (i < E) f[i] = min(f[i], cin + lam * i);
        }
        if (j < G - 1) {
            int cin = cex - lam * (j * E + E - 1);  // value at position j*E + E - 1
#pragma unroll
            for (int i = 0; i < EM; ++i)
                if (i < E) b[i] = min(b[i], cin + lam * (E - 1 - i));
        }
        for (int d = G >> 1; d >= 1; d >>= 1) lmin = min(lmin, __shfl_xor_sync(full, lmin, d, G));
    }
#pragma unroll
    for (int i = 0; i < EM; ++i)
        if (i < E) v[i] = min(f[i], b[i]);
    return lmin;
}

// Same transform on 64-bit keys (value << 32 | label index), so the minimum
// carries the lowest label index among equal values (lexicographic order).
// lam_k = lambda << 32.  Positions >= L must hold kBigKey.  Returns the
// lexicographic minimum key of the input line.
template <int EM>
__device__ __forceinline__ long long line_dt_key(long long (&v)[EM], int E, int G, int j,
                                                 long long lam_k) {
    const unsigned full = 0xffffffffu;
    long long f[EM], b[EM];
    long long lmin = kBigKey;
#pragma unroll
    for (int i = 0; i < EM; ++i)
        if (i < E) lmin = min(lmin, v[i]);
    f[0] = v[0];
#pragma unroll
    for (int i = 1; i < EM; ++i)
        if (i < E) f[i] = min(v[i], f[i - 1] + lam_k);
    long long last = v[0];
#pragma unroll
    for (int i = 0; i < EM; ++i)
        if (i == E - 1) last = v[i];
    b[EM - 1] = kBigKey;
#pragma unroll
    for (int i = EM - 1; i >= 0; --i) {
        if (i < E) {
            if (i == E - 1)
                b[i] = last;
            else
                b[i] = min(v[i], b[i + 1] + lam_k);
        }
    }
    if (G > 1) {
        long long F = f[0];
#pragma unroll
        for (int i = 0; i < EM; ++i)
            if (i == E - 1) F = f[i];
        long long a = F - lam_k * (long long)(E * j);
        for (int d = 1; d < G; d <<= 1) {
            long long t = __shfl_up_sync(full, a, d, G);
            if (j >= d) a = min(a, t);
        }
        long long aex = __shfl_up_sync(full, a, 1, G);
        long long c = b[0] + lam_k * (long long)(E * j);
        for (int d = 1; d < G; d <<= 1) {
            long long t = __shfl_down_sync(full, c, d, G);
            if (j + d < G) c = min(c, t);
        }
        long long cex = __shfl_down_sync(full, c, 1, G);
        if (j > 0) {
            long long cin = aex + lam_k * (long long)(E * (j - 1) + 1);
#pragma unroll
            for (int i = 0; i < EM; ++i)
                if (i < E) f[i] = min(f[i], cin + lam_k * (long long)i);
        }
        if (j < G - 1) {
            long long cin = cex - lam_k * (long long)(j * E + E - 1);
#pragma unroll
            for (int i = 0; i < EM; ++i)
                if (i < E) b[i] = min(b[i], cin + lam_k * (long long)(E - 1 - i));
        }
        for (int d = G >> 1; d >= 1; d >>= 1) lmin = min(lmin, __shfl_xor_sync(full, lmin, d, G));
    }
#pragma unroll
    for (int i = 0; i < EM; ++i)
        if (i < E) v[i] = min(f[i], b[i]);
    return lmin;
}

// Bounded spin on a progress counter written by another block with release
// semantics.  Returns the observed value once >= need, or -1 when `limit`
// polls pass without progress.
// Gives up early when the launch's status word is already non-zero (another
// block failed).
__device__ __forceinline__ long long wait_progress(const unsigned *p, unsigned need, long long limit,
                                                   const int *status) {
    unsigned v;
    long long n = 0;
    while (true) {
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
        if (v >= need) return v;
        if (++n > limit) return -1;
        if ((n & 255) == 0 && *(volatile const int *)status != 0) return -1;
        __nanosleep(32);
    }
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned sm_id() {
    unsigned v;
    asm volatile("mov.u32 %0, %smid;" : "=r"(v));
    return v;
}

__device__ __forceinline__ void publish_progress(unsigned *p, unsigned v) {
    __threadfence();
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Loads of data written by other blocks in this launch: L2, never L1.
__device__ __forceinline__ int ld_cg(const int *p) { return __ldcg(p); }

// 4-byte global -> shared asynchronous copy; zero-fills when !valid.
__device__ __forceinline__ void cp_async4(int *dst_smem, const int *src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    const int n = valid ? 4 : 0;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_n() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

}  // namespace edp
