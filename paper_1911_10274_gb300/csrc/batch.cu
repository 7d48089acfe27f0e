// batch.cu -- many independent spring-mass systems ("robots") advanced for a
// whole rollout in one persistent launch per cluster size.
//
// The paper simulates hundreds of worms at once (Sec. V-B) and many agents in
// parallel (Sec. I).  Here every robot is owned by one thread-block cluster of
// C CTAs (C = 1, 2, 4 or 8, the smallest that holds it).  Each CTA owns a
// contiguous range of the robot's masses: at launch it copies its masses'
// state and their SELL-32 half-edge rows into shared memory with 1-D TMA bulk
// copies (one mbarrier, bounded wait), then runs every time step of the
// rollout without touching global memory: each step first copies the current
// state of its halo - the masses of other CTAs of the cluster its rows touch -
// out of their shared memory (distributed shared memory, one coalesced pass),
// then reads every neighbour from its own shared memory; integration into the
// other state buffer; one hardware cluster barrier per step.  The final state goes back to global
// memory.  The step is the same as the single-system kernels' (Sec. III-B,
// Eq. 1 with the Sec. III-A constraints), including sinusoidal actuation.
#include <cooperative_groups.h>
#include <math.h>
#include <string.h>

#include <cmath>

#include <algorithm>
#include <atomic>
#include <string>
#include <vector>

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

constexpr int kMaxCluster = 8;
constexpr uint32_t kMaxPerCta = 4096;             // masses per CTA
// A CTA's rows address its own masses at slots [0, slot_count) and its halo
// at [slot_count, slot_count + halo_count); a halo entry names the owner as
// rank << 16 | slot there.
constexpr size_t kBatchSmemLimit = 220 * 1024;

// Per-CTA descriptor.  All offsets are in elements of the arrays they index.
struct CtaDesc {
    uint32_t mass_begin;    // first global mass slot of this CTA
    uint32_t mass_count;    // masses owned (<= kMaxPerCta)
    uint32_t slot_count;    // mass_count rounded up to 32
    uint32_t edge_off;      // first SELL entry (multiple of 64)
    uint32_t edge_count;    // SELL entries (multiple of 64)
    uint32_t slice_base;    // first relative slice offset (multiple of 4)
    uint32_t n_slices;
    uint32_t robot;
    uint32_t halo_off;      // first entry of this CTA's halo list
    uint32_t halo_count;    // masses of other CTAs of the cluster its rows touch
    uint32_t halo_slots;    // halo slots in the layout: the largest halo_count of the robot's CTAs, so
                            // that every CTA of a cluster has its state buffers at the same offsets
};

// Shared-memory layout of one CTA (byte offsets; all 16-byte aligned).  The
// state is split per slot into (x, y, z, vx) float4 and (vy, vz) float2 arrays
// (two buffers) plus 1/m: 16-byte loads at a 16-byte stride keep consecutive
// slots in distinct banks (a 32-byte record read in two halves cannot).
struct SmemLayout {
    uint32_t a0, b0, a1, b1, inv, slices, kl, act, nbr, total;
};

__host__ __device__ inline uint32_t align16(uint32_t x) { return (x + 15u) & ~15u; }

__host__ __device__ inline SmemLayout smem_layout(uint32_t slots, uint32_t halo, uint32_t n_slices, uint32_t edges,
                                                  bool act) {
    const uint32_t tab = slots + halo;          // own masses, then the halo
    SmemLayout L;
    L.a0 = 0;
    L.b0 = L.a0 + tab * 16;
    L.a1 = align16(L.b0 + tab * 8);
    L.b1 = L.a1 + tab * 16;
    L.inv = align16(L.b1 + tab * 8);
    L.slices = align16(L.inv + slots * 4);
    L.kl = align16(L.slices + 4 * ((n_slices + 1 + 3) & ~3u));
    L.act = L.kl + edges * 8;
    L.nbr = L.act + (act ? edges * 8 : 0);
    L.total = align16(L.nbr + edges * 2);
    return L;
}

template <bool ACT, bool GROUND, int TPM>
__global__ void __launch_bounds__(512)
k_batch_rollout(const CtaDesc *__restrict__ ctas, const MassState *__restrict__ state_in,
                MassState *__restrict__ state_out, const uint32_t *__restrict__ slice_rel,
                const float2 *__restrict__ kl, const float2 *__restrict__ act,
                const uint16_t *__restrict__ nbr, const uint32_t *__restrict__ halo, titan::StepConst c,
                long long step0, uint32_t n_steps, uint32_t cluster_size, uint32_t spin_limit,
                int *__restrict__ err) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ uint64_t bar;
    const CtaDesc d = ctas[blockIdx.x];
    const SmemLayout L = smem_layout(d.slot_count, d.halo_slots, d.n_slices, d.edge_count, ACT);
    float4 *const a0s = reinterpret_cast<float4 *>(sm + L.a0), *const a1s = reinterpret_cast<float4 *>(sm + L.a1);
    float2 *const b0s = reinterpret_cast<float2 *>(sm + L.b0), *const b1s = reinterpret_cast<float2 *>(sm + L.b1);
    float *s_inv = reinterpret_cast<float *>(sm + L.inv);
    const uint32_t *s_slice = reinterpret_cast<const uint32_t *>(sm + L.slices);
    const float2 *s_kl = reinterpret_cast<const float2 *>(sm + L.kl);
    const float2 *s_act = reinterpret_cast<const float2 *>(sm + L.act);
    const uint16_t *s_nbr = reinterpret_cast<const uint16_t *>(sm + L.nbr);
    const uint32_t tid = threadIdx.x;

    if (tid == 0) {
        const uint32_t slice_bytes = 4 * ((d.n_slices + 1 + 3) & ~3u);
        const uint32_t bytes = slice_bytes + d.edge_count * (ACT ? 18 : 10);
        titan::ptx::mbar_init(&bar, 1);
        titan::ptx::fence_mbar_init();
        titan::ptx::mbar_arrive_expect_tx(&bar, bytes);
        // every size is a multiple of 16 bytes; zero-size copies are not issued
        titan::ptx::bulk_g2s(sm + L.slices, slice_rel + d.slice_base, slice_bytes, &bar);
        if (d.edge_count) {
            titan::ptx::bulk_g2s(sm + L.kl, kl + d.edge_off, d.edge_count * 8, &bar);
            if (ACT) titan::ptx::bulk_g2s(sm + L.act, act + d.edge_off, d.edge_count * 8, &bar);
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

    const uint32_t sub = tid % TPM;
    const uint32_t per_pass = blockDim.x / TPM;
    const uint32_t passes = (d.slot_count + per_pass - 1) / per_pass;   // CTA-uniform
    int cur = 0;
    for (uint32_t k = 0; k < n_steps; ++k) {
        float sp = 0.f, cp = 1.f;
        if (ACT) sincosf(titan::clock_phase(c, step0 + (long long)k), &sp, &cp);
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
            const uint32_t m = pass * per_pass + tid / TPM;
            const bool live = m < d.slot_count;
            float fx = 0.f, fy = 0.f, fz = 0.f;
            float4 p = make_float4(0.f, 0.f, 0.f, 0.f), v = p;
            if (live) {
                const uint32_t slice = m >> 5, lane = m & 31;
                const float4 a0 = srcA[m];
                const float2 b0 = srcB[m];
                p = make_float4(a0.x, a0.y, a0.z, s_inv[m]);
                v = make_float4(a0.w, b0.x, b0.y, 0.f);
                const uint32_t e0 = s_slice[slice];
                const uint32_t width = (s_slice[slice + 1] - e0) >> 5;
                for (uint32_t t = sub; t < width; t += TPM) {
                    const uint32_t e = e0 + t * 32 + lane;
                    const uint32_t slot = s_nbr[e];         // own slot or halo slot
                    const float4 qa = srcA[slot];
                    const float2 qb = srcB[slot];
                    const float4 qp = make_float4(qa.x, qa.y, qa.z, 0.f);
                    const float4 qv = make_float4(qa.w, qb.x, qb.y, 0.f);
                    const float2 a = s_kl[e];
                    float L0 = a.y;
                    if (ACT) {
                        const float2 s = s_act[e];               // (A cos phi, A sin phi)
                        L0 = a.y + a.y * (s.x * sp + s.y * cp);
                    }
                    titan::spring_force(p, v, qp, qv, a.x, L0, c.c_uniform, fx, fy, fz);
                }
            }
#pragma unroll
            for (int o = 1; o < TPM; o <<= 1) {
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
    uint32_t tpm = 1;            // threads per mass
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
    std::vector<MassState> init_state;           // caller-provided initial state (global slots)
    std::vector<Group> groups;
    // device
    CtaDesc *d_ctas = nullptr;
    MassState *d_state[2] = {nullptr, nullptr};
    int cur = 0;
    uint32_t *d_slice = nullptr;
    float2 *d_kl = nullptr, *d_act = nullptr;
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
    cfg.numAttrs = 1;
    const CtaDesc *ctas = b->d_ctas + g.cta_first;
    const MassState *in = b->d_state[b->cur];
    MassState *out = b->d_state[b->cur ^ 1];
    void (*kern)(const CtaDesc *, const MassState *, MassState *, const uint32_t *, const float2 *,
                 const float2 *, const uint16_t *, const uint32_t *, titan::StepConst, long long, uint32_t, uint32_t,
                 uint32_t, int *);
#define PICK(T)                                                                                   \
    if (b->has_act) kern = b->c.ground ? k_batch_rollout<true, true, T> : k_batch_rollout<true, false, T>; \
    else kern = b->c.ground ? k_batch_rollout<false, true, T> : k_batch_rollout<false, false, T>;
    if (g.tpm == 4) { PICK(4) } else if (g.tpm == 2) { PICK(2) } else { PICK(1) }
#undef PICK
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
    if (e != cudaSuccess) return e;
    return cudaLaunchKernelEx(&cfg, kern, ctas, in, out, (const uint32_t *)b->d_slice, (const float2 *)b->d_kl,
                              (const float2 *)b->d_act, (const uint16_t *)b->d_nbr, (const uint32_t *)b->d_halo,
                              b->c, step0, n_steps,
                              g.cluster, b->spin_limit, b->d_err);
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
        if (m.n > kMaxCluster * kMaxPerCta) return bfail(nullptr, TITAN_E_INVALID, "system too large for one cluster" + at);
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
    c.act_omega = 2.0 * 3.14159265358979323846 * freq;
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

    // ---- host layout: per robot, the cluster size and per-CTA SELL blocks
    struct CtaHost {
        CtaDesc d;
        std::vector<uint32_t> slices;
        std::vector<float2> kl, act;
        std::vector<uint16_t> nbr;   // own slot or halo slot per entry
        std::vector<uint32_t> halo;  // rank << 16 | slot of each halo mass in its owner CTA
    };
    std::vector<std::vector<CtaHost>> per_robot(n_systems);
    std::vector<uint32_t> cluster_of(n_systems);
    uint32_t slot_cursor = 0;
    for (uint32_t r = 0; r < n_systems; ++r) {
        const titan_masses &m = masses[r];
        const titan_springs &s = springs[r];
        // incidence in input order: row of mass i = its half-edges (neighbour, spring)
        std::vector<uint32_t> deg(m.n, 0);
        for (uint32_t q = 0; q < s.n; ++q) { ++deg[s.ends[2 * (size_t)q]]; ++deg[s.ends[2 * (size_t)q + 1]]; }
        std::vector<uint32_t> rowptr(m.n + 1, 0);
        for (uint32_t i = 0; i < m.n; ++i) rowptr[i + 1] = rowptr[i] + deg[i];
        std::vector<std::pair<uint32_t, uint32_t>> he(rowptr[m.n]);
        std::vector<uint32_t> cur(rowptr.begin(), rowptr.end() - 1);
        for (uint32_t q = 0; q < s.n; ++q) {
            const uint32_t i = s.ends[2 * (size_t)q], j = s.ends[2 * (size_t)q + 1];
            he[cur[i]++] = {j, q};
            he[cur[j]++] = {i, q};
        }
        for (uint32_t i = 0; i < m.n; ++i) std::sort(he.begin() + rowptr[i], he.begin() + rowptr[i + 1]);
        // distinct masses outside [q0, q1) that the rows of [q0, q1) touch
        std::vector<uint32_t> mark(m.n, UINT32_MAX);
        uint32_t gen = 0;
        auto halo_count = [&](uint32_t q0, uint32_t q1) {
            ++gen;                                    // a fresh mark for every call
            uint32_t cnt = 0;
            for (uint32_t i = q0; i < q1; ++i)
                for (uint32_t r2 = rowptr[i]; r2 < rowptr[i + 1]; ++r2) {
                    const uint32_t j = he[r2].first;
                    if ((j < q0 || j >= q1) && mark[j] != gen) { mark[j] = gen; ++cnt; }
                }
            return cnt;
        };
        // smallest cluster whose per-CTA shared memory fits
        uint32_t C = 1;
        for (;; C *= 2) {
            if (C > (uint32_t)kMaxCluster)
                return bail(bfail(b, TITAN_E_UNSUPPORTED, "system " + std::to_string(r) + " does not fit a cluster of 8 CTAs"));
            const uint32_t per = ((m.n + C - 1) / C + 31) & ~31u;
            if (per > kMaxPerCta) continue;
            // the layout of every CTA of the cluster reserves the largest halo
            uint32_t hc = 0;
            if (C > 1)
                for (uint32_t q0 = 0; q0 < m.n; q0 += per) hc = std::max(hc, halo_count(q0, std::min(m.n, q0 + per)));
            size_t worst = 0;
            for (uint32_t q0 = 0; q0 < m.n; q0 += per) {
                uint32_t edges = 0, ns = 0;
                for (uint32_t sl = q0; sl < std::min(m.n, q0 + per); sl += 32, ++ns) {
                    uint32_t w = 0;
                    for (uint32_t i = sl; i < std::min(m.n, sl + 32); ++i) w = std::max(w, deg[i]);
                    edges += 32 * ((w + 1) & ~1u);
                }
                edges = (edges + 63) & ~63u;
                worst = std::max<size_t>(worst, smem_layout(per, hc, ns, edges, any_act).total);
            }
            if (worst <= kBatchSmemLimit && per + hc <= 65535) break;
        }
        cluster_of[r] = C;
        const uint32_t per = ((m.n + C - 1) / C + 31) & ~31u;
        b->mass_off.push_back(slot_cursor);
        b->mass_cnt.push_back(m.n);
        for (uint32_t q = 0; q < C; ++q) {
            CtaHost h;
            const uint32_t m0 = std::min(m.n, q * per), m1 = std::min(m.n, m0 + per);
            h.d = CtaDesc{slot_cursor + m0, m1 - m0, per, 0, 0, 0, 0, r, 0, 0, 0};
            // SELL of the CTA's masses, neighbours as own slots (j - m0) or halo slots (per + h)
            std::fill(mark.begin(), mark.end(), UINT32_MAX);      // here: halo slot of a mass
            auto slot_of = [&](uint32_t j) -> uint16_t {
                if (j >= m0 && j < m1) return (uint16_t)(j - m0);
                if (mark[j] == UINT32_MAX) {
                    mark[j] = per + (uint32_t)h.halo.size();
                    h.halo.push_back(((j / per) << 16) | (j % per));
                }
                return (uint16_t)mark[j];
            };
            h.slices.push_back(0);
            for (uint32_t sl = m0; sl < m0 + per; sl += 32) {
                uint32_t w = 0;
                for (uint32_t i = sl; i < std::min(m1, sl + 32); ++i) w = std::max(w, deg[i]);
                w = (w + 1) & ~1u;
                const uint32_t base = (uint32_t)h.kl.size();
                h.kl.resize(base + 32 * w, make_float2(0.f, 0.f));
                h.act.resize(base + 32 * w, make_float2(0.f, 0.f));
                h.nbr.resize(base + 32 * w, 0);
                for (uint32_t l = 0; l < 32; ++l) {
                    const uint32_t i = sl + l;
                    for (uint32_t t = 0; t < w; ++t) {
                        const uint32_t e = base + 32 * t + l;
                        if (i < m1 && t < deg[i]) {
                            const auto &x = he[rowptr[i] + t];
                            const uint32_t j = x.first, q2 = x.second;
                            h.nbr[e] = slot_of(j);
                            double L;
                            if (s.rest) L = s.rest[q2];
                            else {
                                double d2 = 0;
                                for (int a = 0; a < 3; ++a) {
                                    const double dd = m.pos[3 * (size_t)j + a] - m.pos[3 * (size_t)i + a];
                                    d2 += dd * dd;
                                }
                                L = std::sqrt(d2);
                            }
                            h.kl[e] = make_float2((float)s.k[q2], (float)L);
                            if (any_act && act[r].amp)
                                h.act[e] = make_float2((float)(act[r].amp[q2] * std::cos(act[r].phase[q2])),
                                                       (float)(act[r].amp[q2] * std::sin(act[r].phase[q2])));
                        } else {
                            const uint32_t self = std::min(i, m.n - 1);   // zero-parameter padding
                            h.nbr[e] = slot_of(self);
                        }
                    }
                }
                h.slices.push_back((uint32_t)h.kl.size());
            }
            const uint32_t E = ((uint32_t)h.kl.size() + 63) & ~63u;
            h.kl.resize(E, make_float2(0.f, 0.f));
            h.act.resize(E, make_float2(0.f, 0.f));
            h.nbr.resize(E, 0);
            h.d.edge_count = E;
            h.d.n_slices = (uint32_t)h.slices.size() - 1;
            h.d.halo_count = (uint32_t)h.halo.size();
            per_robot[r].push_back(std::move(h));
        }
        uint32_t halo_slots = 0;
        for (const auto &hh : per_robot[r]) halo_slots = std::max(halo_slots, hh.d.halo_count);
        for (auto &hh : per_robot[r]) hh.d.halo_slots = halo_slots;
        slot_cursor += C * per;
        // initial state of every slot of this robot (padding slots: fixed, at rest)
        b->init_state.resize(slot_cursor);
        for (uint32_t k = 0; k < C * per; ++k) {
            MassState st{};
            if (k < m.n) {
                const double im = (m.fixed && m.fixed[k]) ? 0.0 : 1.0 / m.mass[k];
                st.p = make_float4((float)m.pos[3 * (size_t)k], (float)m.pos[3 * (size_t)k + 1], (float)m.pos[3 * (size_t)k + 2], (float)im);
                if (m.vel) st.v = make_float4((float)m.vel[3 * (size_t)k], (float)m.vel[3 * (size_t)k + 1], (float)m.vel[3 * (size_t)k + 2], 0.f);
            }
            b->init_state[b->mass_off[r] + k] = st;
        }
    }
    b->total_slots = slot_cursor;
    // Groups: one launch per (cluster size, shared-memory class).  A launch's
    // dynamic shared memory is the largest of its CTAs', so small robots get
    // a class of their own and several of their CTAs share an SM (class k: at
    // most 1/k of an SM's 228 KB); robots in decreasing size within a group.
    static const uint32_t kPerSm[] = {1, 2, 3, 4, 6, 8};
    auto smem_class = [&](uint32_t r) {
        size_t worst = 0;
        for (const auto &h : per_robot[r])
            worst = std::max<size_t>(worst, smem_layout(h.d.slot_count, h.d.halo_slots, h.d.n_slices, h.d.edge_count, any_act).total);
        uint32_t cls = 0;
        for (uint32_t k = 0; k < sizeof(kPerSm) / sizeof(kPerSm[0]); ++k)
            if (worst + 1024 <= 228u * 1024u / kPerSm[k]) cls = k;
        return cls;
    };
    std::vector<uint32_t> class_of(n_systems);
    for (uint32_t r = 0; r < n_systems; ++r) class_of[r] = smem_class(r);
    std::vector<uint32_t> order(n_systems);
    for (uint32_t r = 0; r < n_systems; ++r) order[r] = r;
    std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) {
        if (cluster_of[x] != cluster_of[y]) return cluster_of[x] > cluster_of[y];
        if (class_of[x] != class_of[y]) return class_of[x] < class_of[y];
        return masses[x].n > masses[y].n;
    });
    std::vector<CtaDesc> descs;
    std::vector<uint32_t> slices;
    std::vector<float2> kl, ac;
    std::vector<uint16_t> nb;
    std::vector<uint32_t> hl;
    for (uint32_t k = 0; k < n_systems; ++k) {
        const uint32_t r = order[k];
        if (b->groups.empty() || b->groups.back().cluster != cluster_of[r] || class_of[order[k - 1]] != class_of[r]) {
            Group g;
            g.cluster = cluster_of[r];
            g.cta_first = (uint32_t)descs.size();
            b->groups.push_back(g);
        }
        Group &g = b->groups.back();
        for (auto &h : per_robot[r]) {
            h.d.edge_off = (uint32_t)kl.size();
            while (slices.size() % 4) slices.push_back(0);
            h.d.slice_base = (uint32_t)slices.size();
            slices.insert(slices.end(), h.slices.begin(), h.slices.end());
            while (slices.size() % 4) slices.push_back(0);
            kl.insert(kl.end(), h.kl.begin(), h.kl.end());
            ac.insert(ac.end(), h.act.begin(), h.act.end());
            nb.insert(nb.end(), h.nbr.begin(), h.nbr.end());
            h.d.halo_off = (uint32_t)hl.size();
            hl.insert(hl.end(), h.halo.begin(), h.halo.end());
            descs.push_back(h.d);
            ++g.cta_count;
            g.smem = std::max<size_t>(g.smem, smem_layout(h.d.slot_count, h.d.halo_slots, h.d.n_slices, h.d.edge_count, any_act).total);
        }
        per_robot[r].clear();
    }
    for (auto &g : b->groups) g.threads = g.cluster > 1 ? 256 : 256;

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
    CK(balloc(b, &b->d_ctas, descs.size()));
    CK(balloc(b, &b->d_state[0], b->total_slots));
    CK(balloc(b, &b->d_state[1], b->total_slots));
    CK(balloc(b, &b->d_slice, slices.size()));
    CK(balloc(b, &b->d_kl, kl.size()));
    if (any_act) CK(balloc(b, &b->d_act, ac.size()));
    CK(balloc(b, &b->d_nbr, nb.size()));
    CK(balloc(b, &b->d_halo, std::max<size_t>(hl.size(), 1)));
    CK(balloc(b, &b->d_moff, n_systems));
    CK(balloc(b, &b->d_mcnt, n_systems));
    CK(balloc(b, &b->d_centroid, 3 * (size_t)n_systems));
    CK(balloc(b, &b->d_err, 1));
    CK(cudaMemcpy(b->d_ctas, descs.data(), descs.size() * sizeof(CtaDesc), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(b->d_state[0], b->init_state.data(), b->init_state.size() * sizeof(MassState), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(b->d_slice, slices.data(), slices.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(b->d_kl, kl.data(), kl.size() * sizeof(float2), cudaMemcpyHostToDevice));
    if (any_act) CK(cudaMemcpy(b->d_act, ac.data(), ac.size() * sizeof(float2), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(b->d_nbr, nb.data(), nb.size() * 2, cudaMemcpyHostToDevice));
    if (!hl.empty()) CK(cudaMemcpy(b->d_halo, hl.data(), hl.size() * 4, cudaMemcpyHostToDevice));
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
    BATCH_CK(b, cudaMemcpyAsync(b->d_state[b->cur], b->init_state.data(), b->init_state.size() * sizeof(MassState),
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
    for (uint32_t i = 0; i < n; ++i) {
        if (pos) { pos[3 * i] = h[i].p.x; pos[3 * i + 1] = h[i].p.y; pos[3 * i + 2] = h[i].p.z; }
        if (vel) { vel[3 * i] = h[i].v.x; vel[3 * i + 1] = h[i].v.y; vel[3 * i + 2] = h[i].v.z; }
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
    const int cand_t[3] = {128, 256, 512};
    const int cand_m[3] = {1, 2, 4};
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
    if (threads < 32 || threads > 512 || threads % 32 || !(threads_per_mass == 1 || threads_per_mass == 2 || threads_per_mass == 4))
        return bfail(b, TITAN_E_INVALID, "threads must be a multiple of 32 in [32, 512] and threads_per_mass 1, 2 or 4");
    b->groups[group].threads = threads;
    b->groups[group].tpm = threads_per_mass;
    if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
    return TITAN_OK;
}

uint32_t titan_batch_groups(const titan_batch *b) { return b ? (uint32_t)b->groups.size() : 0; }

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
