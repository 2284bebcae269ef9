// net_tc.cu -- the 32 -> 32 channel 3x3 convolutions of the proposal network
// and their weight gradients on the 5th-generation tensor cores (tcgen05),
// sm_103a.
//
// Implicit GEMM per tile of 8 x 16 output pixels: D[m][n] = sum over k of
// A[m][k] B[k][n], M = 128 pixels, N = 32 output channels, K = 9 taps x 32
// input channels, bf16 operands, float32 accumulation in tensor memory.
// The tile's input halo (10 x 18 pixels, 32 channels) sits in shared memory
// in the no-swizzle K-major layout of the MMA operands: for halo row hy,
// channel chunk c (8 channels = 16 bytes) and halo column hx the chunk is at
// (hy * 4 + c) * 160 + hx * 16.  Eight consecutive output pixels of a tile
// row then read eight consecutive 16-byte rows, one core matrix, for every
// tap: the A operand of tap (dy, dx) is the same buffer seen through a
// descriptor starting at dy * 640 + dx * 16 (8-row groups 640 bytes apart,
// channel chunks 160 bytes apart), so no im2col copy is made.  The weights
// are prepared once per call in the same layout (B: N = 32 rows, K-major).
// One thread issues the 18 MMAs of a tile (9 taps x 2 chunk pairs of
// K = 16) and commits them to an mbarrier; the four warps then read the
// accumulator (warp w owns TMEM lanes 32w .. 32w + 31 = pixels 32w ..) and
// apply the epilogue: bias and ReLU (forward), or the ReLU mask of the
// layer below (input gradient).  Every wait is bounded; a wait that runs out
// sets the status word and the block stops after freeing its tensor memory.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "kernels.h"

namespace edp {
namespace {

constexpr int kTX = 8, kTY = 16;       // output tile (pixels)
constexpr int kHX = kTX + 2, kHY = kTY + 2;
constexpr int kChunkStride = kHX * 16;  // bytes between channel chunks of one halo row
constexpr int kRowStride = 4 * kChunkStride;
constexpr int kHaloBytes = kHY * kRowStride;          // 11520
constexpr int kBBytes = 9 * 32 * 32 * 2;              // 18432
constexpr int kSmem = kBBytes + 2 * kHaloBytes + 32;  // + two mbarriers, tensor-memory address
constexpr long long kSpin = 1LL << 24;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor (no swizzle): start address, the byte
// offset between core matrices along K (lbo) and along M / N (sbo), and the
// descriptor version bits of this architecture
__device__ __forceinline__ uint64_t mat_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}
// instruction descriptor: D float32, A and B bf16, both K-major, N = 32, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, bool acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(kIdesc), "r"((uint32_t)acc));
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (long long it = 0; it < kSpin; ++it) {
        uint32_t r;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(r)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (r) return true;
    }
    return false;
}

__device__ __forceinline__ void cp_async16_zfill(uint32_t dst, const void *src, bool ok) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(ok ? 16 : 0)
                 : "memory");
}

__device__ __forceinline__ __nv_bfloat16 f2bf(float v) { return __float2bfloat16_rn(v); }

// B image of one layer in global memory, laid out as the kernel's shared
// memory wants it: tap t, channel chunk c, row group g, row r, 8 bf16 at
// t * 1024 + c * 256 + g * 64 + r * 8 (elements).  Rows n are output
// channels, K = (tap, input channel).  flip: the input-gradient form, rows
// are the layer's input channels and K = (8 - tap, output channel).
__global__ void net_prep_tc(const float *w, int flip, __nv_bfloat16 *out) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 9 * 32 * 32; e += gridDim.x * blockDim.x) {
        const int tap = e % 9, ci = (e / 9) % 32, co = e / (9 * 32);  // w[co][ci][tap]
        const int t = flip ? 8 - tap : tap;
        const int n = flip ? ci : co, k = flip ? co : ci;
        const size_t o = (size_t)t * 1024 + (k / 8) * 256 + (n / 8) * 64 + (n % 8) * 8 + (k % 8);
        out[o] = f2bf(w[e]);
    }
}

// Epilogue of one tile: the accumulator (warp w: TMEM lanes 32w.. = pixels
// 32w..) to bf16 with bias + ReLU (MODE 0) or the ReLU mask of act (MODE 2).
template <int MODE>
__device__ __forceinline__ void tile_epilogue(uint32_t acc, int n, int x0, int y0, int H, int W,
                                              const float *bias, __nv_bfloat16 *out,
                                              const __nv_bfloat16 *act, int warp, int lane) {
    uint32_t v[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(acc + ((uint32_t)(32 * warp) << 16)));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    const int m = 32 * warp + lane, x = x0 + (m % kTX), y = y0 + m / kTX;
    if (x >= W || y >= H) return;
    const size_t o = (((size_t)n * H + y) * W + x) * 32;
    uint32_t pk[16];
    if (MODE == 0) {
#pragma unroll
        for (int c = 0; c < 32; c += 2) {
            const __nv_bfloat16 lo = f2bf(fmaxf(__uint_as_float(v[c]) + bias[c], 0.f));
            const __nv_bfloat16 hi = f2bf(fmaxf(__uint_as_float(v[c + 1]) + bias[c + 1], 0.f));
            pk[c / 2] = (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
        }
    } else {
        uint4 a4[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) a4[q] = reinterpret_cast<const uint4 *>(act + o)[q];
        const __nv_bfloat16 *ab = reinterpret_cast<const __nv_bfloat16 *>(a4);
#pragma unroll
        for (int c = 0; c < 32; c += 2) {
            const __nv_bfloat16 lo = f2bf(__bfloat162float(ab[c]) > 0.f ? __uint_as_float(v[c]) : 0.f);
            const __nv_bfloat16 hi = f2bf(__bfloat162float(ab[c + 1]) > 0.f ? __uint_as_float(v[c + 1]) : 0.f);
            pk[c / 2] = (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
        reinterpret_cast<uint4 *>(out + o)[q] = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
}

// Asynchronous copies of one tile's halo: 18 rows x 10 pixels x 4 chunks of
// 16 bytes, zero outside the image.
__device__ __forceinline__ void halo_load(uint32_t sH, const __nv_bfloat16 *in, int n, int x0, int y0, int H,
                                          int W, int tid) {
    for (int e = tid; e < kHY * kHX * 4; e += 128) {
        const int hy = e / (kHX * 4), r2 = e - hy * (kHX * 4), hx = r2 >> 2, c = r2 & 3;
        const int gy = y0 - 1 + hy, gx = x0 - 1 + hx;
        const bool inb = gy >= 0 && gy < H && gx >= 0 && gx < W;
        const __nv_bfloat16 *src = inb ? in + (((size_t)n * H + gy) * W + gx) * 32 + c * 8 : in;
        cp_async16_zfill(sH + (hy * 4 + c) * kChunkStride + hx * 16, src, inb);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// MODE 0: out = bf16(relu(z + bias)); MODE 2: out = bf16(z if act > 0 else 0).
// A block walks its tiles two deep: while the MMAs of tile i run, the halo
// of tile i + 1 is copied into the other buffer and tile i - 1's
// accumulator (the other half of the block's 64 tensor-memory columns)
// goes through the epilogue.
template <int MODE>
__global__ void __launch_bounds__(128) net_conv_tc(const __nv_bfloat16 *in, int N, int H, int W,
                                                   const __nv_bfloat16 *wB, const float *bias,
                                                   __nv_bfloat16 *out, const __nv_bfloat16 *act, int *status) {
    extern __shared__ __align__(128) unsigned char sm[];
    unsigned char *const Bs = sm;
    unsigned char *const halo = sm + kBBytes;  // two buffers
    unsigned long long *const mbar = reinterpret_cast<unsigned long long *>(sm + kBBytes + 2 * kHaloBytes);
    uint32_t *const taddr = reinterpret_cast<uint32_t *>(sm + kBBytes + 2 * kHaloBytes + 16);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    for (int e = tid; e < kBBytes / 16; e += blockDim.x)
        reinterpret_cast<uint4 *>(Bs)[e] = reinterpret_cast<const uint4 *>(wB)[e];
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(smem_u32(taddr)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar + 1)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *taddr;
    const uint32_t sB = smem_u32(Bs), sH0 = smem_u32(halo);

    const int tx_n = (W + kTX - 1) / kTX, ty_n = (H + kTY - 1) / kTY;
    const long long tiles = (long long)N * tx_n * ty_n;
    auto coords = [&](long long tile, int &n, int &x0, int &y0) {
        n = (int)(tile / ((long long)tx_n * ty_n));
        const int rem = (int)(tile - (long long)n * tx_n * ty_n);
        y0 = (rem / tx_n) * kTY;
        x0 = (rem % tx_n) * kTX;
    };
    const long long first = blockIdx.x, step = gridDim.x;
    if (first < tiles) {
        int n, x0, y0;
        coords(first, n, x0, y0);
        halo_load(sH0, in, n, x0, y0, H, W, tid);
    }
    bool ok = true;
    int pn = 0, px0 = 0, py0 = 0;  // the previous tile
    long long i = 0;
    for (long long tile = first; tile < tiles; tile += step, ++i) {
        const int b = (int)(i & 1);
        int n, x0, y0;
        coords(tile, n, x0, y0);
        // this tile's halo has arrived (only its copies are in flight)
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
            const uint32_t sH = sH0 + b * kHaloBytes, acc = tmem + 32 * b;
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                const int dy = t / 3, dx = t % 3;
#pragma unroll
                for (int cp = 0; cp < 2; ++cp) {
                    const uint64_t a = mat_desc(sH + dy * kRowStride + dx * 16 + cp * 2 * kChunkStride,
                                                kChunkStride, kRowStride);
                    const uint64_t bd = mat_desc(sB + t * 2048 + cp * 1024, 512, 128);
                    mma_bf16(acc, a, bd, t != 0 || cp != 0);
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(mbar + b))
                         : "memory");
        }
        if (i > 0) {
            // the previous tile's MMAs: done (its halo buffer and accumulator free up)
            const int pb = b ^ 1;
            ok = __syncthreads_and(mbar_wait(smem_u32(mbar + pb), (uint32_t)(((i - 1) >> 1) & 1))) != 0;
            if (!ok) break;
        }
        if (tile + step < tiles) {
            int n2, x2, y2;
            coords(tile + step, n2, x2, y2);
            halo_load(sH0 + (b ^ 1) * kHaloBytes, in, n2, x2, y2, H, W, tid);
        }
        if (i > 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            tile_epilogue<MODE>(tmem + 32 * (b ^ 1), pn, px0, py0, H, W, bias, out, act, warp, lane);
        }
        pn = n;
        px0 = x0;
        py0 = y0;
    }
    if (ok && i > 0) {  // the last tile
        const int lb = (int)((i - 1) & 1);
        ok = __syncthreads_and(mbar_wait(smem_u32(mbar + lb), (uint32_t)(((i - 1) >> 1) & 1))) != 0;
        if (ok) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            tile_epilogue<MODE>(tmem + 32 * lb, pn, px0, py0, H, W, bias, out, act, warp, lane);
        }
    }
    if (!ok && tid == 0) atomicCAS(status, 0, EDP_ERR_TIMEOUT_CODE);
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem));
}

// ---------------------------------------------------------------------------
// Weight and bias gradients of a 32 -> 32 layer:
//   dW[co][ci][dy][dx] = sum over pixels p of g[p][co] x[p + (dy-1, dx-1)][ci],
//   db[co] = sum over p of g[p][co].
// Per horizontal tap dx one GEMM with K = pixels: D[(dy, ci)][co], M = 128
// rows = 4 vertical offsets dy (the fourth, dy = 3, is padding and dropped)
// x 32 input channels, N = 32.  Both operands are MN-major (8 consecutive
// channels per 16-byte row, one row per pixel).  The A operand is the input
// halo (19 rows here) seen through a descriptor: channel chunk c of halo row
// (r + dy) sits at (r + dy) * 640 + c * 160, so the 16 groups (dy, c) are 160
// bytes apart and the pixels of tile row r 640 bytes apart; the B operand is
// the tile of g (tile row r, chunk c at r * 512 + c * 128).  Each block
// accumulates its tiles into three tensor-memory accumulators (one per dx)
// and adds them to dW at the end; db is summed on the CUDA cores from the
// same g tiles.
// ---------------------------------------------------------------------------
constexpr int kWHY = kTY + 3;                    // halo rows for dy = 0..3
constexpr int kWHaloBytes = kWHY * kRowStride;   // 12160
constexpr int kGBytes = kTY * 512;               // 8192
constexpr int kWStage = kWHaloBytes + kGBytes;   // one buffer: halo + g tile
constexpr int kWSmem = 2 * kWStage + 32;

__device__ __forceinline__ void wgrad_tile_load(uint32_t sH, uint32_t sG, const __nv_bfloat16 *x,
                                                const __nv_bfloat16 *g, int n, int x0, int y0, int H, int W,
                                                int tid) {
    for (int e = tid; e < kWHY * kHX * 4; e += 128) {
        const int hy = e / (kHX * 4), r2 = e - hy * (kHX * 4), hx = r2 >> 2, c = r2 & 3;
        const int gy = y0 - 1 + hy, gx = x0 - 1 + hx;
        const bool inb = gy >= 0 && gy < H && gx >= 0 && gx < W;
        const __nv_bfloat16 *src = inb ? x + (((size_t)n * H + gy) * W + gx) * 32 + c * 8 : x;
        cp_async16_zfill(sH + (hy * 4 + c) * kChunkStride + hx * 16, src, inb);
    }
    for (int e = tid; e < kTY * kTX * 4; e += 128) {
        const int r = e / (kTX * 4), r2 = e - r * (kTX * 4), px = r2 >> 2, c = r2 & 3;
        const int gy = y0 + r, gx = x0 + px;
        const bool inb = gy < H && gx < W;
        const __nv_bfloat16 *src = inb ? g + (((size_t)n * H + gy) * W + gx) * 32 + c * 8 : g;
        cp_async16_zfill(sG + r * 512 + c * 128 + px * 16, src, inb);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

constexpr int kPart = 32 * 32 * 9 + 32;  // floats of one block's partial gradients
constexpr int kWgradBlocksPerSm = 4;      // their tensor memory (128 columns each) fills the SM's 512
constexpr int kWgradMaxSms = 256;

__global__ void __launch_bounds__(128) net_wgrad_tc(const __nv_bfloat16 *g, const __nv_bfloat16 *x, int N, int H,
                                                    int W, float *part, int *status) {
    float *const dW = part + (size_t)blockIdx.x * kPart;  // this block's partial sums: [co][ci][9], then [co]
    float *const db = dW + 32 * 32 * 9;
    extern __shared__ __align__(128) unsigned char sm[];
    unsigned long long *const mbar = reinterpret_cast<unsigned long long *>(sm + 2 * kWStage);
    uint32_t *const taddr = reinterpret_cast<uint32_t *>(sm + 2 * kWStage + 16);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(smem_u32(taddr)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar + 1)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *taddr;
    const uint32_t s0 = smem_u32(sm);
    // instruction descriptor: as kIdesc with both operands MN-major
    constexpr uint32_t kIdescMN = kIdesc | (1u << 15) | (1u << 16);

    const int tx_n = (W + kTX - 1) / kTX, ty_n = (H + kTY - 1) / kTY;
    const long long tiles = (long long)N * tx_n * ty_n;
    auto coords = [&](long long tile, int &n, int &x0, int &y0) {
        n = (int)(tile / ((long long)tx_n * ty_n));
        const int rem = (int)(tile - (long long)n * tx_n * ty_n);
        y0 = (rem / tx_n) * kTY;
        x0 = (rem % tx_n) * kTX;
    };
    const long long first = blockIdx.x, step = gridDim.x;
    if (first < tiles) {
        int n, x0, y0;
        coords(first, n, x0, y0);
        wgrad_tile_load(s0, s0 + kWHaloBytes, x, g, n, x0, y0, H, W, tid);
    }
    float bsum[32];  // db partial sums of this thread's pixel (tile pixel tid)
#pragma unroll
    for (int c = 0; c < 32; ++c) bsum[c] = 0.f;
    bool ok = true;
    long long i = 0;
    for (long long tile = first; tile < tiles; tile += step, ++i) {
        const int b = (int)(i & 1);
        const uint32_t sH = s0 + b * kWStage, sG = sH + kWHaloBytes;
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
#pragma unroll
            for (int dx = 0; dx < 3; ++dx)
#pragma unroll
                for (int k = 0; k < kTY / 2; ++k) {  // 16 pixels (two tile rows) per MMA
                    const uint64_t a = mat_desc(sH + dx * 16 + k * 2 * kRowStride, kRowStride, kChunkStride);
                    const uint64_t bd = mat_desc(sG + k * 1024, 512, 128);
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem + 32 * dx),
                        "l"(a), "l"(bd), "r"(kIdescMN), "r"((uint32_t)(i > 0 || k > 0)));
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(mbar + b))
                         : "memory");
        }
        // db: this thread's pixel of the tile, all 32 channels (zero outside the image)
        {
            const unsigned char *gp = sm + b * kWStage + kWHaloBytes + (tid / kTX) * 512 + (tid % kTX) * 16;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const uint4 q = *reinterpret_cast<const uint4 *>(gp + c * 128);
                const __nv_bfloat16 *h = reinterpret_cast<const __nv_bfloat16 *>(&q);
#pragma unroll
                for (int e = 0; e < 8; ++e) bsum[c * 8 + e] += __bfloat162float(h[e]);
            }
        }
        if (i > 0) {
            ok = __syncthreads_and(mbar_wait(smem_u32(mbar + (b ^ 1)), (uint32_t)(((i - 1) >> 1) & 1))) != 0;
            if (!ok) break;
        }
        if (tile + step < tiles) {
            int n2, x2, y2;
            coords(tile + step, n2, x2, y2);
            const uint32_t nH = s0 + (b ^ 1) * kWStage;
            wgrad_tile_load(nH, nH + kWHaloBytes, x, g, n2, x2, y2, H, W, tid);
        }
    }
    if (ok && i > 0) {
        const int lb = (int)((i - 1) & 1);
        ok = __syncthreads_and(mbar_wait(smem_u32(mbar + lb), (uint32_t)(((i - 1) >> 1) & 1))) != 0;
    }
    if (ok && i > 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // warp w reads lanes 32w.. = rows (dy = w, ci = lane); dy = 3 is padding
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
            uint32_t v[32];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                  "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                  "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                : "r"(tmem + 32 * dx + ((uint32_t)(32 * warp) << 16)));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (warp < 3) {
                const int ci = lane, tap = warp * 3 + dx;
#pragma unroll
                for (int co = 0; co < 32; ++co) dW[((size_t)co * 32 + ci) * 9 + tap] = __uint_as_float(v[co]);
            }
        }
        // db: reduce the 128 pixels' sums per channel (warps through shared memory)
        float *const red = reinterpret_cast<float *>(sm);  // the stage buffers are free now
#pragma unroll
        for (int c = 0; c < 32; ++c) {
            float v = bsum[c];
            for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
            if (lane == 0) red[warp * 32 + c] = v;
        }
        __syncthreads();
        if (tid < 32) db[tid] = red[tid] + red[32 + tid] + red[64 + tid] + red[96 + tid];
    }
    if (!ok && tid == 0) atomicCAS(status, 0, EDP_ERR_TIMEOUT_CODE);
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem));
}

// grad[e] += sum over blocks of part[block][e] (blocks that ran no tile
// wrote nothing and are not counted: nb blocks ran one or more)
__global__ void net_wgrad_reduce(const float *part, int nb, float *grad) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < kPart; e += gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int b = 0; b < nb; ++b) s += part[(size_t)b * kPart + e];
        grad[e] += s;
    }
}

}  // namespace

int net_wgrad_tc_max_blocks() { return kWgradMaxSms * kWgradBlocksPerSm; }
int net_wgrad_tc_part_floats() { return kPart; }

int net_wgrad_tc_launch(const void *g, const void *x, int N, int H, int W, float *part, float *grad, int *status,
                        cudaStream_t st) {
    const long long tiles = (long long)N * ((W + kTX - 1) / kTX) * ((H + kTY - 1) / kTY);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long grid = std::min<long long>(
        std::min<long long>(tiles, (long long)std::max(1, sms) * kWgradBlocksPerSm), net_wgrad_tc_max_blocks());
    cudaFuncSetAttribute(net_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kWSmem);
    net_wgrad_tc<<<(unsigned)grid, 128, kWSmem, st>>>(static_cast<const __nv_bfloat16 *>(g),
                                                      static_cast<const __nv_bfloat16 *>(x), N, H, W, part, status);
    if (cudaGetLastError() != cudaSuccess) return -2;
    net_wgrad_reduce<<<(kPart + 255) / 256, 256, 0, st>>>(part, (int)grid, grad);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int net_prep_tc_launch(const float *w, int flip, void *out, cudaStream_t st) {
    net_prep_tc<<<36, 256, 0, st>>>(w, flip, static_cast<__nv_bfloat16 *>(out));
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int net_conv_tc_launch(const void *in, int N, int H, int W, const void *wB, const float *bias, int mode, void *out,
                       const void *act, int *status, cudaStream_t st) {
    const long long tiles = (long long)N * ((W + kTX - 1) / kTX) * ((H + kTY - 1) / kTY);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long grid = std::min<long long>(tiles, (long long)std::max(1, sms) * 5);
    const auto *i = static_cast<const __nv_bfloat16 *>(in);
    const auto *b = static_cast<const __nv_bfloat16 *>(wB);
    auto *o = static_cast<__nv_bfloat16 *>(out);
    const auto *a = static_cast<const __nv_bfloat16 *>(act);
    if (mode == 0) {
        cudaFuncSetAttribute(net_conv_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
        net_conv_tc<0><<<(unsigned)grid, 128, kSmem, st>>>(i, N, H, W, b, bias, o, nullptr, status);
    } else {
        cudaFuncSetAttribute(net_conv_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
        net_conv_tc<2><<<(unsigned)grid, 128, kSmem, st>>>(i, N, H, W, b, nullptr, o, a, status);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace edp
