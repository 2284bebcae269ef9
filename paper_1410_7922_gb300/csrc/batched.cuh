// batched.cuh -- the persistent kernel of the batched solve (batched.cu has
// the host side).  Each wave shape is instantiated in a translation unit of
// its own (batched_*.cu), so that the builds compile in parallel.
#pragma once
#include "pass_r1.cuh"
#include "pass_team.cuh"

namespace edp {

static_assert(sizeof(BatchArgs) <= 32000, "batch descriptors must fit the kernel parameter space");

// LM: lean line bound; GEN: generic team body built in; QUAD: quadratic-prior
// bodies built in (waves holding l1 = 2 problems)
template <int LM, bool GEN, bool QUAD>
__global__ void __launch_bounds__(256) edp_batched_kernel(const __grid_constant__ BatchArgs B) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item;
    __shared__ volatile int s_abort;
    const int tid = threadIdx.x;
    if (tid == 0) s_abort = (*(volatile int *)B.status != 0);
    __syncthreads();
    if (s_abort) return;
    const int total = B.slots * B.per_slot;
    while (true) {
        if (tid == 0) s_item = (int)atomicAdd(B.queue, 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= total) break;
        const int slot = item / B.per_slot;
        const int k = item - slot * B.per_slot;
        int i = 0;
        while (B.prefix[i + 1] <= k) ++i;
        const int band = k - B.prefix[i];
        const BatchProblem &P = B.p[i];
        // the previous pass of this problem must be complete
        if (slot > 0 && tid == 0) {
            const unsigned need = (unsigned)P.nbands;
            const long long got =
                wait_progress(B.done + (size_t)i * B.slots + (slot - 1), need, B.spin_limit, B.status);
            if (got < 0) {
                atomicCAS(B.status, 0, EDP_ERR_TIMEOUT_CODE);
                s_abort = 1;
            }
        }
        __syncthreads();
        if (s_abort) return;
        // slot: one pass, or with B.pairs one paired sweep (P1 + P2, P3 + P4)
        const int per_it = B.pairs ? 2 : 4;
        const int it = slot / per_it, kk = slot % per_it;
        const int pass = B.pairs ? 2 * kk : kk;
        const int pslot = it * 4 + pass;  // the first pass's slot: record tags, consumed counters
        const PassFlags f = pass_flags(it, pass, P.iters);
        const PassFlags f2 = pass_flags(it, B.pairs ? pass + 1 : pass, P.iters);
        bool ok;
        if (P.r1) {
            PassR1Args a = P.o;
            a.pass = pass;
            a.read_c = f.read_c;
            a.read_d = f.read_d;
            a.write_a = f.write_a;
            a.write_b = f.write_b;
            a.final_ = f.final_;
            a.pair = B.pairs;
            a.read_c2 = f2.read_c;
            a.write_a2 = f2.write_a;
            a.write_b2 = f2.write_b;
            a.final2 = f2.final_;
            a.tag = pslot + 1;
            if (QUAD && a.l1 == 2)
                ok = r1_dispatch(a.E, [&](auto e) {
                    return r1_band<decltype(e)::value, QUAD>(a, band, reinterpret_cast<int *>(smem_raw), &s_abort);
                });
            else
                ok = r1_dispatch(a.E, [&](auto e) {
                    return r1_band<decltype(e)::value, false>(a, band, reinterpret_cast<int *>(smem_raw), &s_abort);
                });
        } else {
            TeamArgs a = P.t;
            a.pass = pass;
            a.read_c = f.read_c;
            a.read_d = f.read_d;
            a.write_a = f.write_a;
            a.write_b = f.write_b;
            a.final_ = f.final_;
            a.pair = B.pairs;
            a.read_c2 = f2.read_c;
            a.write_a2 = f2.write_a;
            a.write_b2 = f2.write_b;
            a.final2 = f2.final_;
            a.cons = P.cons + (size_t)pslot * P.nbands;
            a.tag0 = 1 + pslot * P.laps;
            if (QUAD && a.lean && a.l1 == 2)
                ok = team_band<QUAD ? 2 : LM, true>(a, band, reinterpret_cast<int *>(smem_raw), &s_abort);
            else if (a.lean)
                ok = team_band<LM, true>(a, band, reinterpret_cast<int *>(smem_raw), &s_abort);
            else if constexpr (GEN)
                ok = team_band<33, false>(a, band, reinterpret_cast<int *>(smem_raw), &s_abort);
            else {
                // the host never puts a generic-body problem in a lean-only wave
                if (tid == 0) atomicCAS(B.status, 0, 2 /* EDP_ERR_UNSUPPORTED */);
                ok = false;
            }
        }
        if (!ok) return;
        // both bodies end with a block barrier: every write of this band is done
        if (tid == 0) {
            __threadfence();
            atomicAdd(B.done + (size_t)i * B.slots + slot, 1u);
        }
    }
}

}  // namespace edp
