// batch.cu -- many independent spring-mass systems ("robots") advanced for a
// whole rollout in one persistent launch per cluster size and shared-memory
// class (the host layout - clusters, rows, halos, launch groups - is built by
// build_batch in layout.cpp; this file validates, uploads and launches).
//
// The paper simulates hundreds of worms at once (Sec. V-B) and many agents in
// parallel (Sec. I).  Here every robot is owned by one thread-block cluster of
// C CTAs (C = 1, 2, 4 or 8, the smallest that holds it; one-CTA robots are
// plain launches).  Each CTA owns a contiguous range of the robot's masses,
// held in its slots by decreasing degree (rows of similar length share a
// SELL-32 slice): at launch it copies their state and half-edge rows into
// shared memory with 1-D TMA bulk copies (one mbarrier, bounded wait), then
// runs every time step of the rollout without touching global memory: each
// step first copies the current state of its halo - the masses of other CTAs
// of the cluster its rows touch - out of their shared memory (distributed
// shared memory, one coalesced pass), then reads every neighbour from its own
// shared memory; integration into the other state buffer; one hardware cluster
// barrier per step.  The final state goes back to global memory.  The step is
// the same as the single-system kernels' (Sec. III-B, Eq. 1 with the Sec. III-A
// constraints), including sinusoidal actuation, whose sin and cos are formed
// once per CTA and step.
#include <cooperative_groups.h>
#include <math.h>
#include <string.h>

#include <cmath>

#include <algorithm>
#include <atomic>
#include <string>
#include <vector>

#include "layout.h"
#include "physics.cuh"
#include "ptx.cuh"
#include "titan.h"
#include "titan_internal.h"

namespace cg = cooperative_groups;
using titan::MassState;

namespace titan {
void set_thread_error(const std::string &msg);   // runtime.cu
}

namespace {

using titan::BatchCta;
using titan::BatchSmem;
using titan::batch_smem_layout;

template <bool ACT, bool GROUND>
__global__ void __launch_bounds__(1024)
k_batch_rollout(const BatchCta *__restrict__ ctas, const MassState *__restrict__ state_in,
                MassState *__restrict__ state_out, const uint32_t *__restrict__ slice_rel,
                const float2 *__restrict__ kl, const float4 *__restrict__ kla,
                const uint16_t *__restrict__ nbr, const uint32_t *__restrict__ halo, titan::StepConst c,
                long long step0, uint32_t n_steps, uint32_t cluster_size, uint32_t tpm_max, uint32_t spin_limit,
                int *__restrict__ err) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ uint64_t bar;
    // sin and cos of the actuation phase, one pair per step parity: thread 0
    // forms step k + 1's pair during step k (the end-of-step barrier publishes
    // it; the slot it overwrites was last read before the previous barrier)
    __shared__ float2 s_sc[2];
    const BatchCta d = ctas[blockIdx.x];
    const BatchSmem L = batch_smem_layout(d.slot_count, d.halo_slots, d.n_slices, d.edge_count, ACT);
    float4 *const a0s = reinterpret_cast<float4 *>(sm + L.a0), *const a1s = reinterpret_cast<float4 *>(sm + L.a1);
    float2 *const b0s = reinterpret_cast<float2 *>(sm + L.b0), *const b1s = reinterpret_cast<float2 *>(sm + L.b1);
    float *s_inv = reinterpret_cast<float *>(sm + L.inv);
    const uint32_t *s_slice = reinterpret_cast<const uint32_t *>(sm + L.slices);
    const float2 *s_kl = reinterpret_cast<const float2 *>(sm + L.kl);      // not actuated
    const float4 *s_kla = reinterpret_cast<const float4 *>(sm + L.kl);     // actuated: {k, L0, A cos, A sin}
    const uint16_t *s_nbr = reinterpret_cast<const uint16_t *>(sm + L.nbr);
    const uint32_t tid = threadIdx.x;

    if (ACT && tid == 0) {
        float sp, cp;
        sincosf(titan::clock_phase(c, step0), &sp, &cp);
        s_sc[0] = make_float2(sp, cp);
    }
    if (tid == 0) {
        const uint32_t slice_bytes = 4 * ((d.n_slices + 1 + 3) & ~3u);
        const uint32_t bytes = slice_bytes + d.edge_count * (ACT ? 18 : 10);
        titan::ptx::mbar_init(&bar, 1);
        titan::ptx::fence_mbar_init();
        titan::ptx::mbar_arrive_expect_tx(&bar, bytes);
        // every size is a multiple of 16 bytes; zero-size copies are not issued
        titan::ptx::bulk_g2s(sm + L.slices, slice_rel + d.slice_base, slice_bytes, &bar);
        if (d.edge_count) {
            if (ACT) titan::ptx::bulk_g2s(sm + L.kl, kla + d.edge_off, d.edge_count * 16, &bar);
            else titan::ptx::bulk_g2s(sm + L.kl, kl + d.edge_off, d.edge_count * 8, &bar);
            titan::ptx::bulk_g2s(sm + L.nbr, nbr + d.edge_off, d.edge_count * 2, &bar);
        }
    }
    // the state goes through registers into the split layout while the bulk copies run
    for (uint32_t m = tid; m < d.slot_count; m += blockDim.x) {
        float4 p, v;
        titan::load_state(state_in + d.mass_begin + m, p, v);
        a0s[m] = make_float4(p.x, p.y, p.z, v.x);
        b0s[m] = make_float2(v.y, v.z);
        s_inv[m] = p.w;
    }
    __syncthreads();
    bool ok = titan::ptx::mbar_wait_bounded(&bar, 0, spin_limit);
    ok = __syncthreads_and(ok);
    if (!ok && tid == 0) {
        // the copy did not complete: record it, wait (bounded) for it, and compute nothing;
        // the CTA still meets every cluster barrier so the cluster's other CTAs finish
        atomicExch(err, 1);
        titan::ptx::mbar_wait_bounded(&bar, 0, spin_limit);
    }
    cg::cluster_group cluster = cg::this_cluster();
    if (cluster_size > 1) cluster.sync();       // all CTAs' shared memory is loaded and alive

    // threads per mass: the most (a power of two up to tpm_max) that still
    // give every mass of this CTA its own thread group in one pass
    uint32_t tpm = 1;
    while (tpm < tpm_max && 2 * tpm * d.slot_count <= blockDim.x) tpm *= 2;
    const uint32_t tpm_log = (uint32_t)__ffs((int)tpm) - 1;
    const uint32_t sub = tid & (tpm - 1);
    const uint32_t per_pass = blockDim.x >> tpm_log;
    const uint32_t passes = (d.slot_count + per_pass - 1) / per_pass;   // CTA-uniform
    int cur = 0;
    for (uint32_t k = 0; k < n_steps; ++k) {
        float sp = 0.f, cp = 1.f;
        if (ACT) {
            const float2 sc = s_sc[k & 1];
            sp = sc.x;
            cp = sc.y;
            if (tid == 0) {
                float sn, cs;
                sincosf(titan::clock_phase(c, step0 + (long long)k + 1), &sn, &cs);
                s_sc[(k + 1) & 1] = make_float2(sn, cs);
            }
        }
        float4 *srcA = cur ? a1s : a0s;
        float2 *srcB = cur ? b1s : b0s;
        float4 *dstA = cur ? a0s : a1s;
        float2 *dstB = cur ? b0s : b1s;
        if (d.halo_count) {
            // the halo's current state, copied out of the other CTAs' shared memory
            for (uint32_t h = tid; h < d.halo_count; h += blockDim.x) {
                const uint32_t code = halo[d.halo_off + h];
                const uint32_t rank = code >> 16, local = code & 0xffffu;
                srcA[d.slot_count + h] = *cluster.map_shared_rank(srcA + local, rank);
                srcB[d.slot_count + h] = *cluster.map_shared_rank(srcB + local, rank);
            }
            __syncthreads();
        }
        for (uint32_t pass = 0; ok && pass < passes; ++pass) {
            const uint32_t m = pass * per_pass + (tid >> tpm_log);
            const bool live = m < d.slot_count;
            float fx = 0.f, fy = 0.f, fz = 0.f;
            float4 p = make_float4(0.f, 0.f, 0.f, 0.f), v = p;
            if (live) {
                const uint32_t slice = m >> 5, lane = m & 31;
                const float4 a0 = srcA[m];
                const float2 b0 = srcB[m];
                p = make_float4(a0.x, a0.y, a0.z, s_inv[m]);
                v = make_float4(a0.w, b0.x, b0.y, 0.f);
                const uint32_t e0 = s_slice[slice] + lane;
                const uint32_t width = (s_slice[slice + 1] - s_slice[slice]) >> 5;
                // the neighbour's state and the spring's constants of row entry t
                auto load = [&](uint32_t t, float4 &qp, float4 &qv, float &k, float &L0) {
                    const uint32_t e = e0 + t * 32;
                    const uint32_t slot = s_nbr[e];         // own slot or halo slot
                    const float4 qa = srcA[slot];
                    const float2 qb = srcB[slot];
                    qp = make_float4(qa.x, qa.y, qa.z, 0.f);
                    qv = make_float4(qa.w, qb.x, qb.y, 0.f);
                    if (ACT) {
                        const float4 a = s_kla[e];
                        k = a.x;
                        L0 = a.y + a.y * (a.z * sp + a.w * cp);
                    } else {
                        const float2 a = s_kl[e];
                        k = a.x;
                        L0 = a.y;
                    }
                };
                // four entries in flight per thread (their shared-memory loads
                // overlap), added in row order like the one-at-a-time tail
                uint32_t t = sub;
                for (; t + 3 * tpm < width; t += 4 * tpm) {
                    float4 qp[4], qv[4];
                    float k[4], L0[4], f[4], ux[4], uy[4], uz[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) load(t + u * tpm, qp[u], qv[u], k[u], L0[u]);
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        titan::spring_terms(p, v, qp[u], qv[u], k[u], L0[u], c.c_uniform, f[u], ux[u], uy[u], uz[u]);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        fx = __fmaf_rn(f[u], ux[u], fx);
                        fy = __fmaf_rn(f[u], uy[u], fy);
                        fz = __fmaf_rn(f[u], uz[u], fz);
                    }
                }
                for (; t < width; t += tpm) {
                    float4 qp, qv;
                    float k, L0;
                    load(t, qp, qv, k, L0);
                    titan::spring_force(p, v, qp, qv, k, L0, c.c_uniform, fx, fy, fz);
                }
            }
            for (uint32_t o = 1; o < tpm; o <<= 1) {   // CTA-uniform: every lane takes part
                fx += __shfl_xor_sync(0xffffffffu, fx, o);
                fy += __shfl_xor_sync(0xffffffffu, fy, o);
                fz += __shfl_xor_sync(0xffffffffu, fz, o);
            }
            if (live && sub == 0) {
                MassState o;
                if (m < d.mass_count) titan::integrate<GROUND>(p, v, fx, fy, fz, c, &o);
                else { o.p = p; o.v = v; }
                dstA[m] = make_float4(o.p.x, o.p.y, o.p.z, o.v.x);
                dstB[m] = make_float2(o.v.y, o.v.z);
            }
        }
        if (cluster_size > 1) cluster.sync();
        else __syncthreads();
        cur ^= 1;
    }
    if (ok)
        for (uint32_t m = tid; m < d.mass_count; m += blockDim.x) {
            const float4 a = (cur ? a1s : a0s)[m];
            const float2 b = (cur ? b1s : b0s)[m];
            MassState o;
            o.p = make_float4(a.x, a.y, a.z, s_inv[m]);
            o.v = make_float4(a.w, b.x, b.y, 0.f);
            state_out[d.mass_begin + m] = o;
        }
}

// Per-robot centroid x, y, z (fixed summation order: mass by mass).
__global__ void k_batch_centroid(const uint32_t *__restrict__ mass_off, const uint32_t *__restrict__ mass_cnt,
                                 const MassState *__restrict__ state, uint32_t n_robots, float *__restrict__ out) {
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_robots) return;
    double sx = 0, sy = 0, sz = 0;
    const uint32_t o = mass_off[r], n = mass_cnt[r];
    for (uint32_t m = 0; m < n; ++m) {
        const float4 p = state[o + m].p;
        sx += p.x; sy += p.y; sz += p.z;
    }
    out[3 * r] = (float)(sx / n);
    out[3 * r + 1] = (float)(sy / n);
    out[3 * r + 2] = (float)(sz / n);
}

struct Group {
    uint32_t cluster = 1;
    uint32_t threads = 256;
    uint32_t tpm = 1;            // most threads per mass (each CTA takes the most that fit its masses)
    uint32_t cta_first = 0, cta_count = 0;
    size_t smem = 0;
};

}  // namespace

struct titan_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<cudaStream_t> group_streams;
    std::vector<cudaEvent_t> group_events;
    cudaEvent_t fork = nullptr;
    titan::StepConst c{};
    double dt = 0;
    bool has_act = false;
    uint32_t n_robots = 0;
    uint64_t steps = 0;
    uint32_t spin_limit = 1u << 22;
    std::vector<uint32_t> mass_off, mass_cnt;   // per robot, into the global mass slots
    std::vector<uint32_t> slot_of_mass;          // per robot's caller index (from caller_off): its slot - mass_off
    std::vector<size_t> caller_off;              // per robot, into slot_of_mass
    std::vector<float> init_state;               // caller-provided initial state, [slots][8] (x y z 1/m vx vy vz 0)
    std::vector<Group> groups;
    std::vector<uint32_t> group_of;              // per system: the launch group holding its cluster
    // device
    BatchCta *d_ctas = nullptr;
    MassState *d_state[2] = {nullptr, nullptr};
    int cur = 0;
    uint32_t *d_slice = nullptr;
    float2 *d_kl = nullptr;                      // not actuated: {k, L0} per entry
    float4 *d_kla = nullptr;                     // actuated: {k, L0, A cos phi, A sin phi} per entry
    uint16_t *d_nbr = nullptr;
    uint32_t *d_halo = nullptr;
    uint32_t *d_moff = nullptr, *d_mcnt = nullptr;
    float *d_centroid = nullptr;
    int *d_err = nullptr;
    uint32_t total_slots = 0;
    std::vector<void *> allocs;
    std::string error;
    std::atomic<bool> busy{false};
    cudaGraphExec_t graph = nullptr;
    uint64_t graph_steps = 0;
    int graph_cur = -1;
};

namespace {

titan_status bfail(titan_batch *b, titan_status st, const std::string &msg) {
    if (b) b->error = msg;
    else titan::set_thread_error(msg);
    return st;
}

titan_status bfail_cuda(titan_batch *b, cudaError_t e, const char *what) {
    return bfail(b, e == cudaErrorMemoryAllocation ? TITAN_E_OOM : TITAN_E_CUDA,
                 std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

#define BATCH_CK(b, call)                                                    \
    do {                                                                     \
        cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess) return bfail_cuda((b), e_, #call);            \
    } while (0)

struct BusyB {
    titan_batch *b;
    bool acquired;
    explicit BusyB(titan_batch *x) : b(x) { acquired = !b->busy.exchange(true); }
    ~BusyB() { if (acquired) b->busy.store(false); }
};

template <typename T>
cudaError_t balloc(titan_batch *b, T **p, size_t count) {
    void *raw = nullptr;
    cudaError_t e = cudaMalloc(&raw, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) return e;
    b->allocs.push_back(raw);
    *p = static_cast<T *>(raw);
    return cudaSuccess;
}

void release(titan_batch *b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (void *p : b->allocs) cudaFree(p);
    for (auto s : b->group_streams) cudaStreamDestroy(s);
    for (auto e : b->group_events) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
}

cudaError_t launch_group(titan_batch *b, const Group &g, cudaStream_t st, long long step0, uint32_t n_steps) {
    if (!g.cta_count) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(g.cta_count);
    cfg.blockDim = dim3(g.threads);
    cfg.dynamicSmemBytes = g.smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = g.cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = g.cluster > 1 ? 1 : 0;       // one-CTA robots: a plain launch
    const BatchCta *ctas = b->d_ctas + g.cta_first;
    const MassState *in = b->d_state[b->cur];
    MassState *out = b->d_state[b->cur ^ 1];
    void (*kern)(const BatchCta *, const MassState *, MassState *, const uint32_t *, const float2 *,
                 const float4 *, const uint16_t *, const uint32_t *, titan::StepConst, long long, uint32_t, uint32_t,
                 uint32_t, uint32_t, int *);
    if (b->has_act) kern = b->c.ground ? k_batch_rollout<true, true> : k_batch_rollout<true, false>;
    else kern = b->c.ground ? k_batch_rollout<false, true> : k_batch_rollout<false, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
    if (e != cudaSuccess) return e;
    return cudaLaunchKernelEx(&cfg, kern, ctas, in, out, (const uint32_t *)b->d_slice, (const float2 *)b->d_kl,
                              (const float4 *)b->d_kla, (const uint16_t *)b->d_nbr, (const uint32_t *)b->d_halo,
                              b->c, step0, n_steps,
                              g.cluster, g.tpm, b->spin_limit, b->d_err);
}

// All groups run concurrently (one stream each), forked from and joined into b->stream.
cudaError_t enqueue_rollout(titan_batch *b, cudaStream_t st, long long step0, uint32_t n_steps) {
    cudaError_t e = cudaEventRecord(b->fork, st);
    if (e != cudaSuccess) return e;
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
        cudaStream_t gs = b->group_streams[gi];
        if ((e = cudaStreamWaitEvent(gs, b->fork, 0)) != cudaSuccess) return e;
        if ((e = launch_group(b, b->groups[gi], gs, step0, n_steps)) != cudaSuccess) return e;
        if ((e = cudaEventRecord(b->group_events[gi], gs)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(st, b->group_events[gi], 0)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

extern "C" {

titan_status titan_batch_create(uint32_t n_systems, const titan_masses *masses, const titan_springs *springs,
                                const titan_actuation *act, const titan_params *p, titan_batch **out) {
    if (!out || !p || (n_systems && (!masses || !springs)))
        return bfail(nullptr, TITAN_E_INVALID, "titan_batch_create: null argument");
    if (!(p->dt > 0) || !std::isfinite(p->dt) || !(p->damping >= 0) || !std::isfinite(p->damping) ||
        !(p->ground_k >= 0) || !(p->mu >= 0))
        return bfail(nullptr, TITAN_E_INVALID, "titan_batch_create: invalid params (dt, damping, ground_k, mu)");
    // validation of every system, before any device work
    double freq = 0;
    bool any_act = false;
    for (uint32_t r = 0; r < n_systems; ++r) {
        const titan_masses &m = masses[r];
        const titan_springs &s = springs[r];
        const std::string at = " (system " + std::to_string(r) + ")";
        if (m.n == 0 || !m.pos || !m.mass) return bfail(nullptr, TITAN_E_INVALID, "empty system or null pos/mass" + at);
        if (m.n > titan::kBatchMaxCluster * titan::kBatchMaxPerCta)
            return bfail(nullptr, TITAN_E_INVALID, "system too large for one cluster" + at);
        if (s.n && (!s.ends || !s.k)) return bfail(nullptr, TITAN_E_INVALID, "null springs.ends or springs.k" + at);
        for (uint32_t i = 0; i < m.n; ++i) {
            if (!(m.mass[i] > 0) || !std::isfinite(m.mass[i])) return bfail(nullptr, TITAN_E_INVALID, "mass must be finite and > 0" + at);
            for (int a = 0; a < 3; ++a)
                if (!std::isfinite(m.pos[3 * (size_t)i + a]) || (m.vel && !std::isfinite(m.vel[3 * (size_t)i + a])))
                    return bfail(nullptr, TITAN_E_INVALID, "non-finite pos or vel" + at);
        }
        for (uint32_t q = 0; q < s.n; ++q) {
            const uint32_t i = s.ends[2 * (size_t)q], j = s.ends[2 * (size_t)q + 1];
            if (i >= m.n || j >= m.n || i == j) return bfail(nullptr, TITAN_E_INVALID, "bad spring ends" + at);
            if (!(s.k[q] >= 0) || !std::isfinite(s.k[q])) return bfail(nullptr, TITAN_E_INVALID, "bad spring k" + at);
            if (s.rest && (!(s.rest[q] >= 0) || !std::isfinite(s.rest[q]))) return bfail(nullptr, TITAN_E_INVALID, "bad rest length" + at);
        }
        if (s.damping) return bfail(nullptr, TITAN_E_UNSUPPORTED, "per-spring damping is not supported in batches; use params.damping" + at);
        if (act && act[r].amp) {
            if (!act[r].phase) return bfail(nullptr, TITAN_E_INVALID, "actuation phase is required" + at);
            for (uint32_t q = 0; q < s.n; ++q)
                if (!std::isfinite(act[r].amp[q]) || !std::isfinite(act[r].phase[q]))
                    return bfail(nullptr, TITAN_E_INVALID, "non-finite actuation" + at);
            if (any_act && act[r].freq_hz != freq)
                return bfail(nullptr, TITAN_E_UNSUPPORTED, "all systems of a batch share one actuation frequency" + at);
            freq = act[r].freq_hz;
            any_act = true;
        }
    }

    titan_batch *b = new titan_batch();
    b->device = p->device;
    b->n_robots = n_systems;
    b->dt = p->dt;
    b->has_act = any_act;
    b->spin_limit = p->spin_limit ? (uint32_t)std::min<uint64_t>(p->spin_limit, 0xffffffffull) : (1u << 22);
    titan::StepConst &c = b->c;
    c.dt = (float)p->dt; c.dt_d = p->dt;
    c.gx = (float)p->gravity[0]; c.gy = (float)p->gravity[1]; c.gz = (float)p->gravity[2];
    c.ground = p->ground ? 1 : 0; c.ground_k = (float)p->ground_k; c.mu = (float)p->mu;
    c.c_uniform = (float)p->damping;
    titan::set_act_clock(c, freq);
    int prev = -1;
    cudaGetDevice(&prev);
    // every failure after this point releases what was built and gives the
    // caller back its current device
    auto bail = [&](titan_status st) {
        titan::set_thread_error(b->error);
        release(b);
        delete b;
        if (prev >= 0) cudaSetDevice(prev);
        return st;
    };
#define CK(call)                                                             \
    do {                                                                     \
        cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess) return bail(bfail_cuda(b, e_, #call));        \
    } while (0)
    CK(cudaSetDevice(p->device));

    // ---- host layout (layout.cpp): clusters, per-CTA rows and halos, launch groups
    titan::BatchHost L;
    std::string why;
    if (!titan::build_batch(n_systems, masses, springs, act, L, &why))
        return bail(bfail(b, TITAN_E_UNSUPPORTED, why));
    b->mass_off = L.mass_off;
    b->mass_cnt = L.mass_cnt;
    b->caller_off.assign(n_systems + 1, 0);
    for (uint32_t r = 0; r < n_systems; ++r) b->caller_off[r + 1] = b->caller_off[r] + L.mass_cnt[r];
    b->slot_of_mass.assign(b->caller_off[n_systems], 0);
    for (uint32_t r = 0; r < n_systems; ++r)
        for (uint32_t k = 0; k < L.mass_cnt[r]; ++k) {
            const uint32_t i = L.mass_of_slot[L.mass_off[r] + k];    // real masses fill the first n slots
            b->slot_of_mass[b->caller_off[r] + i] = k;
        }
    b->init_state = std::move(L.init_state);
    b->total_slots = L.total_slots;
    b->group_of.assign(n_systems, UINT32_MAX);
    for (const titan::BatchGroup &lg : L.groups) {
        Group g;
        g.cluster = lg.cluster;
        g.cta_first = lg.cta_first;
        g.cta_count = lg.cta_count;
        g.smem = lg.smem;
        for (uint32_t q = lg.cta_first; q < lg.cta_first + lg.cta_count; ++q)
            b->group_of[L.ctas[q].robot] = (uint32_t)b->groups.size();
        b->groups.push_back(g);
    }

    // ---- device
    if (p->stream) b->stream = static_cast<cudaStream_t>(p->stream);
    else { CK(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking)); b->own_stream = true; }
    CK(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
        cudaStream_t s;
        cudaEvent_t e;
        CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        b->group_streams.push_back(s);
        CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        b->group_events.push_back(e);
    }
    static_assert(sizeof(MassState) == 8 * sizeof(float), "state slot = 8 floats");
    const size_t E = L.nbr.size();
    CK(balloc(b, &b->d_ctas, L.ctas.size()));
    CK(balloc(b, &b->d_state[0], b->total_slots));
    CK(balloc(b, &b->d_state[1], b->total_slots));
    CK(balloc(b, &b->d_slice, L.slices.size()));
    if (b->has_act) CK(balloc(b, &b->d_kla, E));
    else CK(balloc(b, &b->d_kl, E));
    CK(balloc(b, &b->d_nbr, E));
    CK(balloc(b, &b->d_halo, std::max<size_t>(L.halo.size(), 1)));
    CK(balloc(b, &b->d_moff, n_systems));
    CK(balloc(b, &b->d_mcnt, n_systems));
    CK(balloc(b, &b->d_centroid, 3 * (size_t)n_systems));
    CK(balloc(b, &b->d_err, 1));
    CK(cudaMemcpy(b->d_ctas, L.ctas.data(), L.ctas.size() * sizeof(BatchCta), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(b->d_state[0], b->init_state.data(), b->init_state.size() * sizeof(float), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(b->d_slice, L.slices.data(), L.slices.size() * 4, cudaMemcpyHostToDevice));
    if (b->has_act) {
        std::vector<float4> kla(E);
        for (size_t e = 0; e < E; ++e)
            kla[e] = make_float4(L.kl[2 * e], L.kl[2 * e + 1], L.act[2 * e], L.act[2 * e + 1]);
        CK(cudaMemcpy(b->d_kla, kla.data(), E * sizeof(float4), cudaMemcpyHostToDevice));
    } else {
        CK(cudaMemcpy(b->d_kl, L.kl.data(), L.kl.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
    CK(cudaMemcpy(b->d_nbr, L.nbr.data(), E * 2, cudaMemcpyHostToDevice));
    if (!L.halo.empty()) CK(cudaMemcpy(b->d_halo, L.halo.data(), L.halo.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(b->d_moff, b->mass_off.data(), n_systems * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(b->d_mcnt, b->mass_cnt.data(), n_systems * 4, cudaMemcpyHostToDevice));
    CK(cudaMemset(b->d_err, 0, sizeof(int)));
#undef CK
    if (prev >= 0) cudaSetDevice(prev);
    *out = b;
    return TITAN_OK;
}

titan_status titan_batch_rollout(titan_batch *b, uint64_t n_steps) {
    if (!b) return bfail(nullptr, TITAN_E_INVALID, "batch is null");
    BusyB g(b);
    if (!g.acquired) return bfail(b, TITAN_E_BUSY, "another call on this batch is in progress");
    if (n_steps > 0xffffffffull) return bfail(b, TITAN_E_INVALID, "n_steps must fit 32 bits");
    if (!n_steps || !b->n_robots) return TITAN_OK;
    int prev = -1;
    cudaGetDevice(&prev);
    BATCH_CK(b, cudaSetDevice(b->device));
    // one captured graph per (step count, parity): the fork/join of all groups
    if (!b->graph || b->graph_steps != n_steps || b->graph_cur != b->cur) {
        if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
        cudaStream_t cap;
        BATCH_CK(b, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        cudaError_t le = e == cudaSuccess ? enqueue_rollout(b, cap, 0, (uint32_t)n_steps) : e;
        cudaGraph_t gr = nullptr;
        e = cudaStreamEndCapture(cap, &gr);
        cudaStreamDestroy(cap);
        if (le != cudaSuccess) { if (gr) cudaGraphDestroy(gr); return bfail_cuda(b, le, "capture rollout"); }
        if (e != cudaSuccess) return bfail_cuda(b, e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&b->graph, gr, 0);
        cudaGraphDestroy(gr);
        if (e != cudaSuccess) return bfail_cuda(b, e, "cudaGraphInstantiate");
        b->graph_steps = n_steps;
        b->graph_cur = b->cur;
    }
    if (b->has_act && b->steps != 0) {
        // the captured graph starts its actuation clock at step 0: later rollouts launch directly
        BATCH_CK(b, enqueue_rollout(b, b->stream, (long long)b->steps, (uint32_t)n_steps));
    } else {
        BATCH_CK(b, cudaGraphLaunch(b->graph, b->stream));
    }
    b->cur ^= 1;
    b->steps += n_steps;
    if (prev >= 0) cudaSetDevice(prev);
    return TITAN_OK;
}

titan_status titan_batch_reset(titan_batch *b) {
    if (!b) return bfail(nullptr, TITAN_E_INVALID, "batch is null");
    BusyB g(b);
    if (!g.acquired) return bfail(b, TITAN_E_BUSY, "another call on this batch is in progress");
    BATCH_CK(b, cudaMemcpyAsync(b->d_state[b->cur], b->init_state.data(), b->init_state.size() * sizeof(float),
                                cudaMemcpyHostToDevice, b->stream));
    BATCH_CK(b, cudaStreamSynchronize(b->stream));
    b->steps = 0;
    return TITAN_OK;
}

titan_status titan_batch_sync(titan_batch *b) {
    if (!b) return bfail(nullptr, TITAN_E_INVALID, "batch is null");
    BATCH_CK(b, cudaStreamSynchronize(b->stream));
    int flag = 0;
    BATCH_CK(b, cudaMemcpy(&flag, b->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        cudaMemset(b->d_err, 0, sizeof(int));
        return bfail(b, TITAN_E_TIMEOUT, "a bounded device wait expired during a rollout");
    }
    return TITAN_OK;
}

titan_status titan_batch_read(titan_batch *b, uint32_t system, float *pos, float *vel) {
    if (!b || system >= b->n_robots) return bfail(b, TITAN_E_INVALID, "batch is null or system out of range");
    titan_status st = titan_batch_sync(b);
    if (st != TITAN_OK) return st;
    const uint32_t n = b->mass_cnt[system];
    std::vector<MassState> h(n);
    BATCH_CK(b, cudaMemcpy(h.data(), b->d_state[b->cur] + b->mass_off[system], n * sizeof(MassState),
                           cudaMemcpyDeviceToHost));
    const uint32_t *slot = b->slot_of_mass.data() + b->caller_off[system];
    for (uint32_t i = 0; i < n; ++i) {
        const MassState &x = h[slot[i]];
        if (pos) { pos[3 * i] = x.p.x; pos[3 * i + 1] = x.p.y; pos[3 * i + 2] = x.p.z; }
        if (vel) { vel[3 * i] = x.v.x; vel[3 * i + 1] = x.v.y; vel[3 * i + 2] = x.v.z; }
    }
    return TITAN_OK;
}

titan_status titan_batch_centroids(titan_batch *b, float *out) {
    if (!b || !out) return bfail(b, TITAN_E_INVALID, "batch or out is null");
    if (!b->n_robots) return TITAN_OK;
    k_batch_centroid<<<(b->n_robots + 127) / 128, 128, 0, b->stream>>>(b->d_moff, b->d_mcnt, b->d_state[b->cur],
                                                                       b->n_robots, b->d_centroid);
    BATCH_CK(b, cudaGetLastError());
    titan_status st = titan_batch_sync(b);
    if (st != TITAN_OK) return st;
    BATCH_CK(b, cudaMemcpy(out, b->d_centroid, 3 * sizeof(float) * b->n_robots, cudaMemcpyDeviceToHost));
    return TITAN_OK;
}

titan_status titan_batch_autotune(titan_batch *b, uint32_t probe_steps) {
    if (!b) return bfail(nullptr, TITAN_E_INVALID, "batch is null");
    BusyB g(b);
    if (!g.acquired) return bfail(b, TITAN_E_BUSY, "another call on this batch is in progress");
    if (!probe_steps) probe_steps = 50;
    cudaEvent_t e0, e1;
    BATCH_CK(b, cudaEventCreate(&e0));
    BATCH_CK(b, cudaEventCreate(&e1));
    const int cand_t[4] = {128, 256, 512, 1024};
    const int cand_m[4] = {1, 2, 4, 8};
    for (auto &grp : b->groups) {
        float best = INFINITY;
        uint32_t best_t = grp.threads, best_m = grp.tpm;
        for (int t : cand_t)
            for (int mm : cand_m) {
                grp.threads = (uint32_t)t;
                grp.tpm = (uint32_t)mm;
                float ms = 0;
                for (int rep = 0; rep < 2; ++rep) {   // first repetition warms up
                    BATCH_CK(b, cudaEventRecord(e0, b->stream));
                    BATCH_CK(b, launch_group(b, grp, b->stream, 0, probe_steps));
                    BATCH_CK(b, cudaEventRecord(e1, b->stream));
                    BATCH_CK(b, cudaEventSynchronize(e1));
                    BATCH_CK(b, cudaEventElapsedTime(&ms, e0, e1));
                }
                if (ms < best) { best = ms; best_t = (uint32_t)t; best_m = (uint32_t)mm; }
            }
        grp.threads = best_t;
        grp.tpm = best_m;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
    // the probes wrote into the other state buffer only; the current state is unchanged
    return TITAN_OK;
}

titan_status titan_batch_info(const titan_batch *b, uint32_t group, uint32_t *cluster, uint32_t *threads,
                              uint32_t *threads_per_mass, uint32_t *ctas) {
    if (!b || group >= b->groups.size()) return TITAN_E_INVALID;
    if (cluster) *cluster = b->groups[group].cluster;
    if (threads) *threads = b->groups[group].threads;
    if (threads_per_mass) *threads_per_mass = b->groups[group].tpm;
    if (ctas) *ctas = b->groups[group].cta_count;
    return TITAN_OK;
}

titan_status titan_batch_configure(titan_batch *b, uint32_t group, uint32_t threads, uint32_t threads_per_mass) {
    if (!b || group >= b->groups.size()) return bfail(b, TITAN_E_INVALID, "batch is null or group out of range");
    if (threads < 32 || threads > 1024 || threads % 32 ||
        !(threads_per_mass == 1 || threads_per_mass == 2 || threads_per_mass == 4 || threads_per_mass == 8))
        return bfail(b, TITAN_E_INVALID, "threads must be a multiple of 32 in [32, 1024] and threads_per_mass 1, 2, 4 or 8");
    b->groups[group].threads = threads;
    b->groups[group].tpm = threads_per_mass;
    if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
    return TITAN_OK;
}

uint32_t titan_batch_groups(const titan_batch *b) { return b ? (uint32_t)b->groups.size() : 0; }

titan_status titan_batch_system_group(const titan_batch *b, uint32_t system, uint32_t *group) {
    if (!b || !group || system >= b->group_of.size()) return TITAN_E_INVALID;
    *group = b->group_of[system];
    return TITAN_OK;
}

const char *titan_batch_last_error(const titan_batch *b) { return b ? b->error.c_str() : ""; }

titan_status titan_batch_destroy(titan_batch *b) {
    if (!b) return TITAN_OK;
    titan_status st = TITAN_OK;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) st = TITAN_E_CUDA;
    release(b);
    delete b;
    return st;
}

}  // extern "C"
