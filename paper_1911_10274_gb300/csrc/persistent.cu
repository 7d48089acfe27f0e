// persistent.cu -- many time steps of one small system in one launch.
//
// For a system whose state and SELL rows fit in the shared memory of one
// thread-block cluster (up to 8 CTAs), launching one kernel per step leaves
// the GPU idle for most of each step (a step is a few hundred nanoseconds of
// work against microseconds of launch and drain).  This kernel instead loads
// the system once and runs a whole chunk of steps: CTA r of the cluster owns
// device masses [r P, (r + 1) P); at launch it copies their state and SELL rows
// (the simulation's own arrays, so parameter edits between launches are seen)
// into shared memory, then for every step first copies the current state of
// its halo - the masses of other CTAs its rows touch - out of their shared
// memory (distributed shared memory, one coalesced pass) into a local halo
// region, and evaluates each owned mass's row from local shared memory only,
// exactly as the launch kernels do (same entries, same order, same helpers:
// Sec. III-B, Eq. 1; Sec. III-A constraints; Eqs. 3-5 actuation); it writes
// the new state into the other shared buffer and meets one hardware cluster
// barrier.  The final state goes back to
// global memory.  No spin-wait of its own: the cluster barrier is hardware and
// all CTAs of a cluster are co-resident by construction.
#include <cooperative_groups.h>

#include <algorithm>

#include "layout.h"
#include "physics.cuh"
#include "titan_internal.h"

namespace cg = cooperative_groups;

namespace titan {

namespace {


template <bool HAS_C, bool HAS_ACT, bool GROUND>
__global__ void __launch_bounds__(512)
k_step_persist(const MassState *__restrict__ in, MassState *__restrict__ out, uint32_t n, PersistArgs pa,
               const uint32_t *__restrict__ slice_off, const uint16_t *__restrict__ slot,
               const uint32_t *__restrict__ halo, const float2 *__restrict__ kl, const float *__restrict__ cc,
               const float2 *__restrict__ act, StepConst c, const long long *__restrict__ step_in,
               long long *__restrict__ step_out, uint32_t n_steps) {
    extern __shared__ __align__(16) unsigned char sm[];
    const uint32_t per = pa.per_cta;
    const PersistLayout L = persist_layout(per, pa.max_halo, pa.max_entries, HAS_C, HAS_ACT);
    float4 *const a0 = reinterpret_cast<float4 *>(sm + L.a0), *const a1 = reinterpret_cast<float4 *>(sm + L.a1);
    float2 *const b0 = reinterpret_cast<float2 *>(sm + L.b0), *const b1 = reinterpret_cast<float2 *>(sm + L.b1);
    float *s_inv = reinterpret_cast<float *>(sm + L.inv);
    uint32_t *s_rel = reinterpret_cast<uint32_t *>(sm + L.rel);
    float2 *s_kl = reinterpret_cast<float2 *>(sm + L.kl);
    float2 *s_act = reinterpret_cast<float2 *>(sm + L.act);
    float *s_c = reinterpret_cast<float *>(sm + L.cc);
    uint16_t *s_slot = reinterpret_cast<uint16_t *>(sm + L.slot);

    cg::cluster_group cluster = cg::this_cluster();
    const uint32_t rank = pa.cluster > 1 ? cluster.block_rank() : 0;
    const uint32_t tid = threadIdx.x, nt = blockDim.x;
    const uint32_t m0 = rank * per;                                      // first device mass of this CTA
    const uint32_t count = m0 < n ? min(per, n - m0) : 0;                // masses owned
    const uint32_t n_sl = (count + 31) / 32;
    const uint32_t sl0 = m0 / 32;
    const uint32_t e_begin = n_sl ? slice_off[sl0] : 0;
    const uint32_t e_count = n_sl ? slice_off[sl0 + n_sl] - e_begin : 0;   // <= max_entries (host-checked)
    const uint32_t h_begin = pa.halo_off[rank], h_count = pa.halo_off[rank + 1] - h_begin;   // <= max_halo

    for (uint32_t s = tid; s <= n_sl; s += nt) s_rel[s] = slice_off[sl0 + s] - e_begin;
    for (uint32_t e = tid; e < e_count; e += nt) {
        s_kl[e] = kl[e_begin + e];
        s_slot[e] = slot[e_begin + e];
        if (HAS_C) s_c[e] = cc[e_begin + e];
        if (HAS_ACT) s_act[e] = act[e_begin + e];
    }
    for (uint32_t m = tid; m < count; m += nt) {
        float4 p, v;
        load_state(in + m0 + m, p, v);
        a0[m] = make_float4(p.x, p.y, p.z, v.x);
        b0[m] = make_float2(v.y, v.z);
        s_inv[m] = p.w;
    }
    // this thread's halo entries (the same every step)
    const long long step0 = *step_in;
    if (pa.cluster > 1) cluster.sync();     // every CTA's shared memory is loaded and alive
    else __syncthreads();

    int cur = 0;
    for (uint32_t k = 0; k < n_steps; ++k) {
        float4 *srcA = cur ? a1 : a0;
        float2 *srcB = cur ? b1 : b0;
        float4 *dstA = cur ? a0 : a1;
        float2 *dstB = cur ? b0 : b1;
        // halo: the current state of other CTAs' masses, copied into local slots per + h
        for (uint32_t h = tid; h < h_count; h += nt) {
            const uint32_t code = halo[h_begin + h];
            const uint32_t r = code >> 16, local = code & 0xffffu;
            srcA[per + h] = *cluster.map_shared_rank(srcA + local, r);
            srcB[per + h] = *cluster.map_shared_rank(srcB + local, r);
        }
        __syncthreads();
        const float clk = HAS_ACT ? actuation_clock(c, step0 + (long long)k) : 0.f;
        for (uint32_t m = tid; m < count; m += nt) {
            const float4 sA = srcA[m];
            const float2 sB = srcB[m];
            const float4 p = make_float4(sA.x, sA.y, sA.z, s_inv[m]);
            const float4 v = make_float4(sA.w, sB.x, sB.y, 0.f);
            float fx = 0.f, fy = 0.f, fz = 0.f;
            const uint32_t slice = m >> 5, lane = m & 31;
            const uint32_t e0 = s_rel[slice], width = (s_rel[slice + 1] - e0) >> 5;
            // widths are even: two entries per iteration, both neighbours read
            // before either force is formed (summation order as in the launch
            // kernels: entry t, then t + 1)
            for (uint32_t t = 0; t < width; t += 2) {
                const uint32_t e = e0 + t * 32 + lane;
                const uint32_t j0 = s_slot[e], j1 = s_slot[e + 32];
                const float4 qa0 = srcA[j0], qa1 = srcA[j1];
                const float2 qb0 = srcB[j0], qb1 = srcB[j1];
                const float2 k0 = s_kl[e], k1 = s_kl[e + 32];
                const float L0 = HAS_ACT ? actuated_length(c, k0.y, s_act[e], clk) : k0.y;
                const float L1 = HAS_ACT ? actuated_length(c, k1.y, s_act[e + 32], clk) : k1.y;
                spring_force(p, v, qa0, make_float4(qa0.w, qb0.x, qb0.y, 0.f), k0.x, L0,
                             HAS_C ? s_c[e] : c.c_uniform, fx, fy, fz);
                spring_force(p, v, qa1, make_float4(qa1.w, qb1.x, qb1.y, 0.f), k1.x, L1,
                             HAS_C ? s_c[e + 32] : c.c_uniform, fx, fy, fz);
            }
            MassState o;
            integrate<GROUND>(p, v, fx, fy, fz, c, &o);
            dstA[m] = make_float4(o.p.x, o.p.y, o.p.z, o.v.x);
            dstB[m] = make_float2(o.v.y, o.v.z);
        }
        // every CTA's new state is written before anyone copies it as halo,
        // and every halo copy of the old state is done before it is overwritten
        if (pa.cluster > 1) cluster.sync();
        else __syncthreads();
        cur ^= 1;
    }
    for (uint32_t m = tid; m < count; m += nt) {
        const float4 a = (cur ? a1 : a0)[m];
        const float2 b = (cur ? b1 : b0)[m];
        MassState o;
        o.p = make_float4(a.x, a.y, a.z, s_inv[m]);
        o.v = make_float4(a.w, b.x, b.y, 0.f);
        out[m0 + m] = o;
    }
    if (rank == 0 && tid == 0) *step_out = step0 + (long long)n_steps;
}

}  // namespace

cudaError_t launch_step_persistent(const MassState *in, MassState *out, uint32_t n, const PersistPlan &plan,
                                   const uint32_t *slice_off, const uint16_t *slot, const uint32_t *halo,
                                   const float2 *kl, const float *cc, const float2 *act, const StepConst &c,
                                   const long long *step_in, long long *step_out, uint32_t n_steps,
                                   cudaStream_t stream) {
    const bool hc = cc != nullptr, ha = act != nullptr, gr = c.ground != 0;
    PersistArgs pa;
    pa.cluster = plan.cluster;
    pa.per_cta = plan.per_cta;
    pa.max_entries = plan.max_entries;
    pa.max_halo = plan.max_halo;
    for (int r = 0; r < 9; ++r) pa.halo_off[r] = plan.halo_off[r];
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(plan.cluster);
    cfg.blockDim = dim3(plan.threads);
    cfg.dynamicSmemBytes = plan.smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = plan.cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    decltype(&k_step_persist<false, false, false>) kern;
    if (hc) {
        if (ha) kern = gr ? k_step_persist<true, true, true> : k_step_persist<true, true, false>;
        else    kern = gr ? k_step_persist<true, false, true> : k_step_persist<true, false, false>;
    } else {
        if (ha) kern = gr ? k_step_persist<false, true, true> : k_step_persist<false, true, false>;
        else    kern = gr ? k_step_persist<false, false, true> : k_step_persist<false, false, false>;
    }
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plan.smem);
    if (e != cudaSuccess) return e;
    return cudaLaunchKernelEx(&cfg, kern, in, out, n, pa, slice_off, slot, halo, kl, cc, act, c, step_in, step_out,
                              n_steps);
}

}  // namespace titan
