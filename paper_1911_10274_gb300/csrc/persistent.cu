// persistent.cu -- many time steps of one small system in one launch.
//
// For a system whose state and SELL rows fit in the shared memory of one
// thread-block cluster (up to 8 CTAs), launching one kernel per step leaves
// the GPU idle for most of each step (a step is a few hundred nanoseconds of
// work against microseconds of launch and drain).  This kernel instead loads
// the system once and runs a whole chunk of steps: CTA r of the cluster owns
// device masses [r P, (r + 1) P); at launch it copies their state and SELL rows
// (the simulation's own arrays, so parameter edits between launches are seen)
// into shared memory, then for every step evaluates each owned mass's row
// exactly as the launch kernels do (same entries, same order, same helpers:
// Sec. III-B, Eq. 1; Sec. III-A constraints; Eqs. 3-5 actuation), reading
// neighbours in its own shared memory or, for masses of another CTA, through
// distributed shared memory, writes the new state into the other shared
// buffer and meets one hardware cluster barrier.  The final state goes back to
// global memory.  No spin-wait of its own: the cluster barrier is hardware and
// all CTAs of a cluster are co-resident by construction.
#include <cooperative_groups.h>

#include <algorithm>

#include "physics.cuh"
#include "titan_internal.h"

namespace cg = cooperative_groups;

namespace titan {

namespace {

constexpr uint32_t kPersistLocalBits = 12;   // neighbour code = rank << 12 | local slot

struct PersistLayout {
    uint32_t a0, b0, a1, b1, inv, rel, kl, code, cc, act, total;
};

__host__ __device__ inline uint32_t al16(uint32_t x) { return (x + 15u) & ~15u; }

__host__ __device__ inline PersistLayout persist_layout(uint32_t slots, uint32_t entries, bool has_c, bool has_act) {
    PersistLayout L;
    L.a0 = 0;
    L.b0 = L.a0 + slots * 16;
    L.a1 = L.b0 + slots * 8;
    L.b1 = L.a1 + slots * 16;
    L.inv = L.b1 + slots * 8;
    L.rel = al16(L.inv + slots * 4);
    L.kl = al16(L.rel + 4 * (slots / 32 + 1));
    L.act = L.kl + entries * 8;
    L.cc = L.act + (has_act ? entries * 8 : 0);
    L.code = L.cc + (has_c ? entries * 4 : 0);
    L.total = al16(L.code + entries * 2);
    return L;
}

template <bool HAS_C, bool HAS_ACT, bool GROUND>
__global__ void __launch_bounds__(512)
k_step_persist(const MassState *__restrict__ in, MassState *__restrict__ out, uint32_t n, uint32_t per_cta,
               uint32_t max_entries, const uint32_t *__restrict__ slice_off, const uint16_t *__restrict__ code,
               const float2 *__restrict__ kl, const float *__restrict__ cc, const float2 *__restrict__ act,
               StepConst c, const long long *__restrict__ step_in, long long *__restrict__ step_out,
               uint32_t n_steps, uint32_t cluster_size) {
    extern __shared__ __align__(16) unsigned char sm[];
    const PersistLayout L = persist_layout(per_cta, max_entries, HAS_C, HAS_ACT);
    float4 *const a0 = reinterpret_cast<float4 *>(sm + L.a0), *const a1 = reinterpret_cast<float4 *>(sm + L.a1);
    float2 *const b0 = reinterpret_cast<float2 *>(sm + L.b0), *const b1 = reinterpret_cast<float2 *>(sm + L.b1);
    float *s_inv = reinterpret_cast<float *>(sm + L.inv);
    uint32_t *s_rel = reinterpret_cast<uint32_t *>(sm + L.rel);
    float2 *s_kl = reinterpret_cast<float2 *>(sm + L.kl);
    float2 *s_act = reinterpret_cast<float2 *>(sm + L.act);
    float *s_c = reinterpret_cast<float *>(sm + L.cc);
    uint16_t *s_code = reinterpret_cast<uint16_t *>(sm + L.code);

    cg::cluster_group cluster = cg::this_cluster();
    const uint32_t rank = cluster_size > 1 ? cluster.block_rank() : 0;
    const uint32_t tid = threadIdx.x, nt = blockDim.x;
    const uint32_t m0 = rank * per_cta;                                  // first device mass of this CTA
    const uint32_t count = m0 < n ? min(per_cta, n - m0) : 0;            // masses owned
    const uint32_t n_sl = (count + 31) / 32;
    const uint32_t sl0 = m0 / 32;
    const uint32_t e_begin = n_sl ? slice_off[sl0] : 0;
    const uint32_t e_count = n_sl ? slice_off[sl0 + n_sl] - e_begin : 0;   // <= max_entries (host-checked)

    for (uint32_t s = tid; s <= n_sl; s += nt) s_rel[s] = slice_off[sl0 + s] - e_begin;
    for (uint32_t e = tid; e < e_count; e += nt) {
        s_kl[e] = kl[e_begin + e];
        s_code[e] = code[e_begin + e];
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
    const long long step0 = *step_in;
    if (cluster_size > 1) cluster.sync();     // every CTA's shared memory is loaded and alive
    else __syncthreads();

    int cur = 0;
    for (uint32_t k = 0; k < n_steps; ++k) {
        const float clk = HAS_ACT ? actuation_clock(c, step0 + (long long)k) : 0.f;
        const float4 *srcA = cur ? a1 : a0;
        const float2 *srcB = cur ? b1 : b0;
        float4 *dstA = cur ? a0 : a1;
        float2 *dstB = cur ? b0 : b1;
        for (uint32_t m = tid; m < count; m += nt) {
            const float4 sA = srcA[m];
            const float2 sB = srcB[m];
            const float4 p = make_float4(sA.x, sA.y, sA.z, s_inv[m]);
            const float4 v = make_float4(sA.w, sB.x, sB.y, 0.f);
            float fx = 0.f, fy = 0.f, fz = 0.f;
            const uint32_t slice = m >> 5, lane = m & 31;
            const uint32_t e0 = s_rel[slice], width = (s_rel[slice + 1] - e0) >> 5;
            // widths are even: two entries per iteration, both neighbours
            // requested before either force is formed (same summation order
            // as the launch kernels: entry t, then t + 1)
            for (uint32_t t = 0; t < width; t += 2) {
                const uint32_t e = e0 + t * 32 + lane;
                float4 qa[2];
                float2 qb[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint32_t cd = s_code[e + 32 * h];
                    const uint32_t r = cd >> kPersistLocalBits, local = cd & ((1u << kPersistLocalBits) - 1);
                    if (r == rank) {
                        qa[h] = srcA[local];
                        qb[h] = srcB[local];
                    } else {
                        qa[h] = *cluster.map_shared_rank(srcA + local, r);
                        qb[h] = *cluster.map_shared_rank(srcB + local, r);
                    }
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float2 a = s_kl[e + 32 * h];
                    const float L0 = HAS_ACT ? actuated_length(c, a.y, s_act[e + 32 * h], clk) : a.y;
                    spring_force(p, v, qa[h], make_float4(qa[h].w, qb[h].x, qb[h].y, 0.f), a.x, L0,
                                 HAS_C ? s_c[e + 32 * h] : c.c_uniform, fx, fy, fz);
                }
            }
            MassState o;
            integrate<GROUND>(p, v, fx, fy, fz, c, &o);
            dstA[m] = make_float4(o.p.x, o.p.y, o.p.z, o.v.x);
            dstB[m] = make_float2(o.v.y, o.v.z);
        }
        if (cluster_size > 1) cluster.sync();
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

size_t persistent_smem_bytes(uint32_t per_cta, uint32_t max_entries, bool has_c, bool has_act) {
    return persist_layout(per_cta, max_entries, has_c, has_act).total;
}

bool plan_persistent(uint32_t n, const std::vector<uint32_t> &slice_off, const std::vector<uint32_t> &nbr,
                     bool has_c, bool has_act, size_t smem_limit, PersistPlan &plan,
                     std::vector<uint16_t> &code) {
    if (n == 0 || slice_off.size() != (size_t)(n + 31) / 32 + 1) return false;
    auto masses_per_cta = [&](uint32_t cl) { return ((n + cl - 1) / cl + 31) & ~31u; };
    auto entries_per_cta = [&](uint32_t cl) {
        const uint32_t per = masses_per_cta(cl);
        uint32_t max_e = 0;
        for (uint32_t r = 0; r < cl && r * per < n; ++r) {
            const uint32_t sl0 = r * per / 32, sl1 = (std::min(n, (r + 1) * per) + 31) / 32;
            max_e = std::max(max_e, slice_off[sl1] - slice_off[sl0]);
        }
        return max_e;
    };
    auto fits = [&](uint32_t cl) {
        const uint32_t per = masses_per_cta(cl);
        return per <= (1u << kPersistLocalBits) &&
               persistent_smem_bytes(per, entries_per_cta(cl), has_c, has_act) <= smem_limit;
    };
    // the smallest cluster that fits and gives each thread one mass (512 per
    // CTA); failing that, the smallest that fits at all
    uint32_t cl = 0;
    for (uint32_t c2 = 1; c2 <= 8 && !cl; c2 *= 2)
        if (masses_per_cta(c2) <= 512 && fits(c2)) cl = c2;
    for (uint32_t c2 = 1; c2 <= 8 && !cl; c2 *= 2)
        if (fits(c2)) cl = c2;
    if (!cl) return false;
    const uint32_t per = masses_per_cta(cl);
    plan.cluster = cl;
    plan.per_cta = per;
    plan.max_entries = entries_per_cta(cl);
    plan.smem = persistent_smem_bytes(per, plan.max_entries, has_c, has_act);
    plan.threads = std::min<uint32_t>(512, per);
    code.resize(nbr.size());
    for (size_t e = 0; e < nbr.size(); ++e) {
        const uint32_t j = nbr[e];
        code[e] = (uint16_t)(((j / per) << kPersistLocalBits) | (j % per));
    }
    return true;
}

cudaError_t launch_step_persistent(const MassState *in, MassState *out, uint32_t n, const PersistPlan &plan,
                                   const uint32_t *slice_off, const uint16_t *code, const float2 *kl,
                                   const float *cc, const float2 *act, const StepConst &c,
                                   const long long *step_in, long long *step_out, uint32_t n_steps,
                                   cudaStream_t stream) {
    const bool hc = cc != nullptr, ha = act != nullptr, gr = c.ground != 0;
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
    return cudaLaunchKernelEx(&cfg, kern, in, out, n, plan.per_cta, plan.max_entries, slice_off, code, kl, cc, act,
                              c, step_in, step_out, n_steps, plan.cluster);
}

}  // namespace titan
