// runtime.cu -- the C ABI of libtitan (include/titan.h): handles, validation,
// device layout upload, the asynchronous step loop and snapshots.
//
// Asynchronous model (Titan Sec. III-D): titan_step only enqueues work on the
// simulation stream - one fused kernel per step, replayed from captured CUDA
// graphs of `graph_chunk` steps - and returns.  Snapshots copy the state on
// the simulation stream into a slot buffer (a gather into caller order, one
// small kernel) and move it to pinned host memory on a side stream, so the
// host reads state while later steps keep running.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <thread>
#include <atomic>
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "layout.h"
#include "sim_internal.h"
#include "titan.h"
#include "titan_internal.h"


namespace {

thread_local std::string g_thread_error = "";

constexpr uint32_t kHaloMaxSlots = 4096;     // 96 KiB of shared memory per CTA
constexpr size_t kHaloTmaMaxSmem = 112 * 1024;  // two CTAs per SM
constexpr size_t kBoxTmaMaxSmem = 74 * 1024;    // three CTAs per SM
constexpr size_t kPersistSmemLimit = 220 * 1024;  // persistent kernel: shared memory per CTA
// AUTO takes the persistent kernel only while each CTA holds at most this many
// masses (one per thread): beyond it a per-step launch over the whole GPU is
// faster than the few SMs of one cluster.
constexpr uint32_t kPersistAutoMaxPerCta = 512;
constexpr uint32_t kPersistChunk = 1u << 16;       // steps per persistent launch

struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

bool finite(double x) { return std::isfinite(x); }

}  // namespace

namespace titan {
// Lets other translation units of the library report an error through
// titan_last_error(NULL).
void set_thread_error(const std::string &msg) { g_thread_error = msg; }
}  // namespace titan


namespace {

struct BusyGuard {
    titan_sim *sim;
    bool acquired;
    explicit BusyGuard(titan_sim *s) : sim(s) { acquired = !sim->busy.exchange(true); }
    ~BusyGuard() {
        if (acquired) sim->busy.store(false);
    }
};

titan_status fail(titan_sim *sim, titan_status st, const std::string &msg) {
    if (sim) sim->error = msg;
    else g_thread_error = msg;
    return st;
}

titan_status fail_cuda(titan_sim *sim, cudaError_t e, const char *what) {
    std::string msg = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(sim, e == cudaErrorMemoryAllocation ? TITAN_E_OOM : TITAN_E_CUDA, msg);
}

#define TITAN_CK(sim, call)                                                  \
    do {                                                                     \
        cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess) return fail_cuda((sim), e_, #call);           \
    } while (0)

template <typename T>
cudaError_t dev_alloc(titan_sim *sim, T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    void *raw = nullptr;
    cudaError_t e = cudaMalloc(&raw, count * sizeof(T));
    if (e != cudaSuccess) return e;
    sim->allocations.push_back(raw);
    *p = static_cast<T *>(raw);
    return cudaSuccess;
}

template <typename T>
cudaError_t upload(T *dst, const std::vector<T> &src, cudaStream_t st) {
    if (src.empty()) return cudaSuccess;
    return cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, st);
}

void free_graphs(titan_sim *sim) {
    for (auto &lvl : sim->graph)
        for (auto &g : lvl) {
            if (g) cudaGraphExecDestroy(g);
            g = nullptr;
        }
    for (auto &x : sim->exact) {
        if (x.exec) cudaGraphExecDestroy(x.exec);
        x = SimCore::ExactGraph();
    }
    sim->graphs_built = false;
}

// Steps run by the captured graph of level L (0 when the level is unused).
int graph_steps(const titan_sim *sim, int L) {
    const int k = sim->graph_chunk >> L;
    if (sim->graph_chunk <= 0 || L >= kGraphLevels || k < 2 || (k << L) != sim->graph_chunk || (k & 1)) return 0;
    return k;
}

// The context-wide persisting-L2 limit is shared by every simulation that
// asks for it: raised while at least one lives, restored after the last.
std::mutex g_l2_mu;
int g_l2_users = 0;
size_t g_l2_prev = 0;

void l2_persist_on(titan_sim *sim) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, sim->device) != cudaSuccess) return;
    const size_t bytes = 2 * (size_t)sim->n_dev * sizeof(MassState);
    // only when the whole state fits the persisting part of L2: a partial
    // window (hit ratio below 1) was measured to slow the step down
    // (2M-point mesh, 128 MB of state: 112.8 against 97.7 us)
    if (prop.persistingL2CacheMaxSize <= 0 || bytes == 0 || bytes > (size_t)prop.persistingL2CacheMaxSize ||
        bytes > (size_t)prop.accessPolicyMaxWindowSize)
        return;
    std::lock_guard<std::mutex> lk(g_l2_mu);
    size_t cur = 0;
    if (cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize) != cudaSuccess) return;
    const size_t want = std::min<size_t>((size_t)prop.persistingL2CacheMaxSize, std::max(cur, bytes));
    if (want != cur && cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    if (g_l2_users++ == 0) g_l2_prev = cur;
    sim->l2win.base_ptr = sim->state[0];
    sim->l2win.num_bytes = bytes;
    sim->l2win.hitRatio = std::min(1.f, (float)((double)want / (double)bytes));
    sim->l2win.hitProp = cudaAccessPropertyPersisting;
    sim->l2win.missProp = cudaAccessPropertyStreaming;
    sim->l2_on = true;
}

void l2_persist_off(titan_sim *sim) {
    if (!sim->l2_on) return;
    sim->l2_on = false;
    std::lock_guard<std::mutex> lk(g_l2_mu);
    if (--g_l2_users == 0) {
        cudaCtxResetPersistingL2Cache();
        cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, g_l2_prev);
        cudaGetLastError();
    }
}

void release(titan_sim *sim) {
    l2_persist_off(sim);
    free_graphs(sim);
    if (sim->state_stage) cudaFreeHost(sim->state_stage);
    if (sim->state_staged) cudaEventDestroy(sim->state_staged);
    for (int b = 0; b < 2; ++b) {
        if (sim->snap_host[b]) cudaFreeHost(sim->snap_host[b]);
        if (sim->snap_ready[b]) cudaEventDestroy(sim->snap_ready[b]);
        if (sim->snap_done[b]) cudaEventDestroy(sim->snap_done[b]);
    }
    for (void *p : sim->allocations) cudaFree(p);
    sim->allocations.clear();
    if (sim->side) cudaStreamDestroy(sim->side);
    if (sim->capture) cudaStreamDestroy(sim->capture);
    if (sim->own_stream && sim->stream) cudaStreamDestroy(sim->stream);
}

titan_status validate(const titan_masses *m, const titan_springs *sp, const titan_params *p) {
    if (!m || !sp || !p) return fail(nullptr, TITAN_E_INVALID, "null masses, springs or params");
    if (m->n >= (1u << 31)) return fail(nullptr, TITAN_E_INVALID, "too many masses (>= 2^31)");
    if (sp->n >= (1u << 30)) return fail(nullptr, TITAN_E_INVALID, "too many springs (>= 2^30)");
    if (m->n && (!m->pos || !m->mass)) return fail(nullptr, TITAN_E_INVALID, "masses.pos and masses.mass are required");
    if (sp->n && (!sp->ends || !sp->k)) return fail(nullptr, TITAN_E_INVALID, "springs.ends and springs.k are required");
    if (!(finite(p->dt) && p->dt > 0)) return fail(nullptr, TITAN_E_INVALID, "params.dt must be finite and > 0");
    for (int a = 0; a < 3; ++a)
        if (!finite(p->gravity[a])) return fail(nullptr, TITAN_E_INVALID, "params.gravity must be finite");
    if (!(finite(p->ground_k) && p->ground_k >= 0)) return fail(nullptr, TITAN_E_INVALID, "params.ground_k must be finite and >= 0");
    if (!(finite(p->mu) && p->mu >= 0)) return fail(nullptr, TITAN_E_INVALID, "params.mu must be finite and >= 0");
    if (!(finite(p->damping) && p->damping >= 0)) return fail(nullptr, TITAN_E_INVALID, "params.damping must be finite and >= 0");
    if (p->accumulate != TITAN_ACCUM_CSR && p->accumulate != TITAN_ACCUM_ATOMIC)
        return fail(nullptr, TITAN_E_INVALID, "params.accumulate must be TITAN_ACCUM_CSR or TITAN_ACCUM_ATOMIC");
    if (p->order != TITAN_ORDER_INPUT && p->order != TITAN_ORDER_MORTON)
        return fail(nullptr, TITAN_E_INVALID, "params.order must be TITAN_ORDER_INPUT or TITAN_ORDER_MORTON");
    if (p->exec < TITAN_EXEC_AUTO || p->exec > TITAN_EXEC_PERSISTENT)
        return fail(nullptr, TITAN_E_INVALID, "params.exec out of range");
    if (p->device < 0) return fail(nullptr, TITAN_E_INVALID, "params.device must be >= 0");
    if (p->kernel_variant < 0 || p->kernel_variant > 8) return fail(nullptr, TITAN_E_INVALID, "params.kernel_variant must be 0..8");
    for (uint64_t i = 0; i < m->n; ++i) {
        for (int a = 0; a < 3; ++a) {
            if (!finite(m->pos[3 * i + a])) return fail(nullptr, TITAN_E_INVALID, "masses.pos has a non-finite value at mass " + std::to_string(i));
            if (m->vel && !finite(m->vel[3 * i + a])) return fail(nullptr, TITAN_E_INVALID, "masses.vel has a non-finite value at mass " + std::to_string(i));
        }
        if (!(finite(m->mass[i]) && m->mass[i] > 0)) return fail(nullptr, TITAN_E_INVALID, "masses.mass must be finite and > 0 (mass " + std::to_string(i) + ")");
    }
    for (uint64_t q = 0; q < sp->n; ++q) {
        const uint32_t i = sp->ends[2 * q], j = sp->ends[2 * q + 1];
        if (i >= m->n || j >= m->n) return fail(nullptr, TITAN_E_INVALID, "springs.ends index out of range at spring " + std::to_string(q));
        if (i == j) return fail(nullptr, TITAN_E_INVALID, "spring " + std::to_string(q) + " joins a mass to itself");
        if (!(finite(sp->k[q]) && sp->k[q] >= 0)) return fail(nullptr, TITAN_E_INVALID, "springs.k must be finite and >= 0 (spring " + std::to_string(q) + ")");
        if (sp->rest && !(finite(sp->rest[q]) && sp->rest[q] >= 0)) return fail(nullptr, TITAN_E_INVALID, "springs.rest must be finite and >= 0 (spring " + std::to_string(q) + ")");
        if (sp->damping && !(finite(sp->damping[q]) && sp->damping[q] >= 0)) return fail(nullptr, TITAN_E_INVALID, "springs.damping must be finite and >= 0 (spring " + std::to_string(q) + ")");
    }
    return TITAN_OK;
}

void fill_state(const titan_sim *sim, const double *pos, const double *vel, std::vector<MassState> &st) {
    st.resize(sim->n_dev);
    for (uint32_t d = 0; d < sim->n_dev; ++d) {
        const uint32_t i = sim->caller_of_dev[d];
        MassState m;
        if (i == UINT32_MAX) {            // hole: a fixed, unconnected slot
            m.p = make_float4(0.f, 0.f, 0.f, 0.f);
            m.v = make_float4(0.f, 0.f, 0.f, 0.f);
            st[d] = m;
            continue;
        }
        m.p = make_float4((float)pos[3 * (size_t)i], (float)pos[3 * (size_t)i + 1], (float)pos[3 * (size_t)i + 2], sim->inv_mass[i]);
        if (vel) m.v = make_float4((float)vel[3 * (size_t)i], (float)vel[3 * (size_t)i + 1], (float)vel[3 * (size_t)i + 2], 0.f);
        else m.v = make_float4(0.f, 0.f, 0.f, 0.f);
        st[d] = m;
    }
}

// fill_state into `out` ([n_dev]) on up to 16 host threads, each checking its
// masses' values; false (and `out` partly written) if one is not finite.
bool fill_state_parallel(const titan_sim *sim, const double *pos, const double *vel, MassState *out) {
    const uint32_t nd = sim->n_dev;
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const unsigned nt = (unsigned)std::min<uint64_t>(std::min(16u, hw), std::max<uint64_t>(1, nd / 65536));
    std::atomic<bool> ok{true};
    auto work = [&](unsigned t) {
        const uint32_t d0 = (uint32_t)((uint64_t)nd * t / nt), d1 = (uint32_t)((uint64_t)nd * (t + 1) / nt);
        for (uint32_t d = d0; d < d1; ++d) {
            const uint32_t i = sim->caller_of_dev[d];
            MassState m;
            if (i == UINT32_MAX) {            // hole: a fixed, unconnected slot
                m.p = make_float4(0.f, 0.f, 0.f, 0.f);
                m.v = make_float4(0.f, 0.f, 0.f, 0.f);
                out[d] = m;
                continue;
            }
            const double *x = pos + 3 * (size_t)i, *v = vel ? vel + 3 * (size_t)i : nullptr;
            if (!std::isfinite(x[0]) || !std::isfinite(x[1]) || !std::isfinite(x[2]) ||
                (v && (!std::isfinite(v[0]) || !std::isfinite(v[1]) || !std::isfinite(v[2])))) {
                ok.store(false, std::memory_order_relaxed);
                return;
            }
            m.p = make_float4((float)x[0], (float)x[1], (float)x[2], sim->inv_mass[i]);
            m.v = v ? make_float4((float)v[0], (float)v[1], (float)v[2], 0.f) : make_float4(0.f, 0.f, 0.f, 0.f);
            out[d] = m;
        }
    };
    if (nt == 1) {
        work(0);
    } else {
        std::vector<std::thread> pool;
        for (unsigned t = 1; t < nt; ++t) pool.emplace_back(work, t);
        work(0);
        for (auto &th : pool) th.join();
    }
    return ok.load();
}

// The cube kernel (8) runs from the cube stream.
bool uses_cube(const titan_sim *sim) { return sim->csr_kernel == 8; }


// Uploads the per-entry actuation arrays of the current layout.
// Mean position of each group of masses (caller indices first[g] ..
// first[g+1] - 1, clamped to n), summed in FP64 in caller order, minus the
// group's origin if given (an empty group: 0); one thread per group.
__global__ void k_group_centroid(const MassState *__restrict__ state, const uint32_t *__restrict__ dev_of_caller,
                                 uint32_t n, const uint32_t *__restrict__ first, uint32_t n_groups,
                                 const float *__restrict__ origin, float *__restrict__ out) {
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_groups) return;
    const uint32_t i0 = min(first[g], n), i1 = max(i0, min(first[g + 1], n));
    double sx = 0, sy = 0, sz = 0;
    for (uint32_t i = i0; i < i1; ++i) {
        const float4 p = state[dev_of_caller[i]].p;
        sx += p.x; sy += p.y; sz += p.z;
    }
    const double c = i1 > i0 ? 1.0 / (double)(i1 - i0) : 0.0;
    float o[3] = {0.f, 0.f, 0.f};
    if (origin && i1 > i0) { o[0] = origin[3 * g]; o[1] = origin[3 * g + 1]; o[2] = origin[3 * g + 2]; }
    out[3 * g] = (float)(sx * c - (double)o[0]);
    out[3 * g + 1] = (float)(sy * c - (double)o[1]);
    out[3 * g + 2] = (float)(sz * c - (double)o[2]);
}

// seed[i][axis] = w[g] / |group g| for the masses of group g; a warp per group.
__global__ void k_group_seed(const uint32_t *__restrict__ first, uint32_t n_groups, uint32_t n,
                             const float *__restrict__ w, int axis, float *__restrict__ seed) {
    const uint32_t g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (g >= n_groups) return;
    const uint32_t i0 = min(first[g], n), i1 = max(i0, min(first[g + 1], n));
    if (i1 == i0) return;
    const float v = (float)((double)w[g] / (double)(i1 - i0));
    for (uint32_t i = i0 + lane; i < i1; i += 32) seed[3 * (size_t)i + axis] = v;
}

// Brings act_amp / act_phase up to the values last set from device arrays.
cudaError_t fetch_act_host(titan_sim *sim) {
    if (!sim->act_host_stale) return cudaSuccess;
    sim->act_amp.resize(sim->s);
    sim->act_phase.resize(sim->s);
    cudaError_t e = cudaMemcpyAsync(sim->act_amp.data(), sim->d_act_amp, (size_t)sim->s * 4, cudaMemcpyDeviceToHost,
                                    sim->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sim->act_phase.data(), sim->d_act_phase, (size_t)sim->s * 4, cudaMemcpyDeviceToHost,
                            sim->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(sim->stream);
    if (e == cudaSuccess) sim->act_host_stale = false;
    return e;
}

cudaError_t upload_actuation(titan_sim *sim) {
    cudaError_t e;
    if ((e = fetch_act_host(sim)) != cudaSuccess) return e;
    if (sim->accumulate == TITAN_ACCUM_CSR) {
        if (!sim->d_act && (e = dev_alloc(sim, &sim->d_act, sim->sell.entries + titan::kStreamTail)) != cudaSuccess)
            return e;
        std::vector<float2> a(sim->sell.entries + titan::kStreamTail, make_float2(0.f, 0.f));
        for (uint32_t e2 = 0; e2 < sim->sell.entries; ++e2) {
            const uint32_t q = sim->sell.spring[e2];
            if (q != UINT32_MAX) a[e2] = make_float2(sim->act_amp[q], sim->act_phase[q]);
        }
        if ((e = upload(sim->d_act, a, sim->stream)) != cudaSuccess) return e;
        if (uses_cube(sim)) {
            if (!sim->d_cact && (e = dev_alloc(sim, &sim->d_cact, sim->cube.entries)) != cudaSuccess) return e;
            std::vector<float2> ca(sim->cube.entries, make_float2(0.f, 0.f));
            for (uint32_t e2 = 0; e2 < sim->cube.entries; ++e2) {
                const uint32_t q = sim->cube.spring[e2];
                if (q != UINT32_MAX) ca[e2] = make_float2(sim->act_amp[q], sim->act_phase[q]);
            }
            if ((e = upload(sim->d_cact, ca, sim->stream)) != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    if (!sim->d_ract && (e = dev_alloc(sim, &sim->d_ract, sim->s)) != cudaSuccess) return e;
    std::vector<float2> a(sim->s);
    for (uint32_t r = 0; r < sim->s; ++r) {
        const uint32_t q = sim->rec.order[r];
        a[r] = make_float2(sim->act_amp[q], sim->act_phase[q]);
    }
    return upload(sim->d_ract, a, sim->stream);
}

__global__ void k_count_nonfinite(const float *__restrict__ a, const float *__restrict__ b, uint32_t n,
                                  int *__restrict__ bad) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && !(isfinite(a[i]) && isfinite(b[i]))) atomicAdd(bad, 1);
}

// out[i] = (amp, phase) of the spring behind entry i, zero for padding.
__global__ void k_scatter_act(const uint32_t *__restrict__ spring_of, uint32_t n, const float *__restrict__ amp,
                              const float *__restrict__ phase, float2 *__restrict__ out) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t q = spring_of[i];
    out[i] = q != UINT32_MAX ? make_float2(amp[q], phase[q]) : make_float2(0.f, 0.f);
}

// Uploads the host map `map` into *dst once (spring of each entry).
cudaError_t ensure_map(titan_sim *sim, uint32_t **dst, const std::vector<uint32_t> &map) {
    if (*dst) return cudaSuccess;
    cudaError_t e = dev_alloc(sim, dst, map.size());
    if (e != cudaSuccess) return e;
    return map.empty() ? cudaSuccess
                       : cudaMemcpy(*dst, map.data(), map.size() * 4, cudaMemcpyHostToDevice);
}

// Fills the per-entry actuation arrays of the active layout from the
// caller-order device arrays d_act_amp / d_act_phase.
cudaError_t scatter_actuation_dev(titan_sim *sim) {
    cudaError_t e;
    auto run = [&](const uint32_t *map, uint32_t n, float2 *out) {
        if (n) k_scatter_act<<<(n + 255) / 256, 256, 0, sim->stream>>>(map, n, sim->d_act_amp, sim->d_act_phase, out);
        return cudaGetLastError();
    };
    if (sim->accumulate == TITAN_ACCUM_CSR) {
        if (!sim->d_act) {
            if ((e = dev_alloc(sim, &sim->d_act, sim->sell.entries + titan::kStreamTail)) != cudaSuccess) return e;
            if ((e = cudaMemsetAsync(sim->d_act, 0, (sim->sell.entries + titan::kStreamTail) * sizeof(float2),
                                     sim->stream)) != cudaSuccess)
                return e;
        }
        if ((e = ensure_map(sim, &sim->d_entry_spring, sim->sell.spring)) != cudaSuccess) return e;
        if ((e = run(sim->d_entry_spring, sim->sell.entries, sim->d_act)) != cudaSuccess) return e;
        if (uses_cube(sim)) {
            if (!sim->d_cact && (e = dev_alloc(sim, &sim->d_cact, sim->cube.entries)) != cudaSuccess) return e;
            if ((e = ensure_map(sim, &sim->d_cube_spring, sim->cube.spring)) != cudaSuccess) return e;
            if ((e = run(sim->d_cube_spring, sim->cube.entries, sim->d_cact)) != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    if (!sim->d_ract && (e = dev_alloc(sim, &sim->d_ract, sim->s)) != cudaSuccess) return e;
    if ((e = ensure_map(sim, &sim->d_rec_spring, sim->rec.order)) != cudaSuccess) return e;
    return run(sim->d_rec_spring, sim->s, sim->d_ract);
}

// after_step: the operation just before this one on `st` is this
// simulation's previous step kernel.  Only then may the step start early as a
// programmatic dependent (it waits for that kernel before reading the state);
// after a copy, a set_state or any other operation it is launched in plain
// stream order.
cudaError_t enqueue_step_io(titan_sim *sim, cudaStream_t st, const MassState *in, MassState *out,
                            const long long *si, long long *so, bool after_step) {
    const bool overlap = sim->launch_overlap && after_step;
    if (sim->accumulate == TITAN_ACCUM_CSR) {
        titan::SellView v{sim->d_slice_off, sim->d_nbr, sim->d_kl, sim->has_c ? sim->d_c : nullptr,
                          sim->has_act ? sim->d_act : nullptr, 0, sim->spin_limit, sim->d_err};
        if (sim->csr_kernel >= 6 && sim->csr_kernel <= 8) {
            titan::BoxView h{sim->d_col_off, sim->d_own_slot, sim->d_ext_off, sim->d_ext_idx, sim->d_ext_slot,
                             (sim->box.max_table + 1) & ~1u};
            if (uses_cube(sim)) {
                titan::CubeView cv{sim->d_cube_base, sim->d_cube_meta, sim->d_ckl, sim->has_c ? sim->d_cc : nullptr,
                                   sim->has_act ? sim->d_cact : nullptr};
                return titan::launch_step_cube(in, out, sim->n_dev, cv, h, sim->c, si, so, st,
                                               sim->l2_on ? &sim->l2win : nullptr);
            }
            if (sim->csr_kernel == 7)
                return titan::launch_step_box_tma(in, out, sim->n_dev, v, h, sim->halo_w_max, sim->c, si, so, st);
            return titan::launch_step_box(in, out, sim->n_dev, v, h, sim->c, si, so, st,
                                          sim->l2_on ? &sim->l2win : nullptr, overlap);
        }
        if (sim->csr_kernel == 4 || sim->csr_kernel == 5) {
            titan::HaloView h{sim->d_nslot, sim->d_own_slot, sim->d_ext_off, sim->d_ext_idx,
                              sim->d_ext_slot, sim->halo.max_table, sim->halo_ahead};
            if (sim->csr_kernel == 5)
                return titan::launch_step_halo_tma(in, out, sim->n_dev, v, h, sim->halo_w_max, sim->c, si,
                                                   so, st);
            return titan::launch_step_halo(in, out, sim->n_dev, v, h, sim->c, si, so, st,
                                           sim->l2_on ? &sim->l2win : nullptr, overlap);
        }
        v.variant = sim->csr_kernel == 3 ? 0 : sim->csr_kernel;   // launcher: 0 prefetch, 1 direct, 2 staged
        return titan::launch_step_sell(in, out, sim->n_dev, v, sim->c, si, so, st);
    }
    titan::AtomicView v{sim->d_rec, sim->has_c ? sim->d_rc : nullptr,
                        sim->has_act ? sim->d_ract : nullptr, sim->d_force, sim->s};
    return titan::launch_step_atomic(in, out, sim->n_dev, v, sim->c, si, so, st);
}

cudaError_t enqueue_step(titan_sim *sim, cudaStream_t st, int b, bool after_step) {
    return enqueue_step_io(sim, st, sim->state[b], sim->state[1 - b], sim->steps_dev + b, sim->steps_dev + (1 - b),
                           after_step);
}

// Staged columns per slice for the halo+TMA kernel: every slice if two CTAs
// per SM still fit, else the widest width that does (wider slices read their
// columns from global memory).  False if not even two columns fit.
bool choose_halo_width(titan_sim *sim) {
    uint32_t w_max = 0;
    for (size_t sl = 0; sl + 1 < sim->sell.slice_off.size(); ++sl)
        w_max = std::max(w_max, (sim->sell.slice_off[sl + 1] - sim->sell.slice_off[sl]) / 32);
    w_max = std::max(2u, (w_max + 1) & ~1u);
    auto bytes = [&](uint32_t w) {
        return titan::halo_tma_smem_bytes(sim->halo.max_table, w, sim->has_c, sim->has_act);
    };
    while (w_max > 2 && bytes(w_max) > kHaloTmaMaxSmem) w_max -= 2;
    if (bytes(w_max) > kHaloTmaMaxSmem) return false;
    sim->halo_w_max = w_max;
    return true;
}

// Staged columns per slice for the TMA-staged box kernel: every slice if three
// CTAs per SM still fit, else the widest width that does.  False if not even
// two columns fit.
bool choose_box_width(titan_sim *sim) {
    uint32_t w_max = 0;
    for (size_t sl = 0; sl + 1 < sim->sell.slice_off.size(); ++sl)
        w_max = std::max(w_max, (sim->sell.slice_off[sl + 1] - sim->sell.slice_off[sl]) / 32);
    w_max = std::max(2u, (w_max + 1) & ~1u);
    const uint32_t slots = (sim->box.max_table + 1) & ~1u;
    auto bytes = [&](uint32_t w) { return titan::box_tma_smem_bytes(slots, w, sim->has_c, sim->has_act); };
    while (w_max > 2 && bytes(w_max) > kBoxTmaMaxSmem) w_max -= 2;
    if (bytes(w_max) > kBoxTmaMaxSmem) return false;
    sim->halo_w_max = w_max;
    return true;
}

// Resolves params.exec for the current layout and entry size: the persistent
// cluster kernel when the system fits one cluster's shared memory and (AUTO)
// each CTA's rows are short enough that a few SMs beat a whole-GPU launch per
// step; else one launch per step.  Rewrites the neighbour codes if the plan
// changed.
cudaError_t resolve_exec(titan_sim *sim) {
    sim->persistent = false;
    if (sim->accumulate != TITAN_ACCUM_CSR || sim->exec_req == TITAN_EXEC_LAUNCH) return cudaSuccess;
    titan::PersistPlan plan;
    std::vector<uint16_t> slot;
    std::vector<uint32_t> halo;
    if (!titan::plan_persistent(sim->n_dev, sim->sell.slice_off, sim->sell.nbr, sim->has_c, sim->has_act,
                                kPersistSmemLimit, plan, slot, halo))
        return cudaSuccess;
    if (sim->exec_req == TITAN_EXEC_AUTO && plan.per_cta > kPersistAutoMaxPerCta) return cudaSuccess;
    cudaError_t e;
    if (!sim->d_pslot && (e = dev_alloc(sim, &sim->d_pslot, slot.size())) != cudaSuccess) return e;
    if (halo.size() > sim->phalo_cap) {
        if ((e = dev_alloc(sim, &sim->d_phalo, halo.size())) != cudaSuccess) return e;
        sim->phalo_cap = halo.size();
    }
    if ((e = upload(sim->d_pslot, slot, sim->stream)) != cudaSuccess) return e;
    if ((e = upload(sim->d_phalo, halo, sim->stream)) != cudaSuccess) return e;
    // the host vectors must outlive the asynchronous copies
    if ((e = cudaStreamSynchronize(sim->stream)) != cudaSuccess) return e;
    sim->plan = plan;
    sim->persistent = true;
    return cudaSuccess;
}

// After per-spring damping or actuation arrays appear (larger SELL entries).
cudaError_t entries_grew(titan_sim *sim) {
    if (sim->csr_kernel == 5 && !choose_halo_width(sim)) sim->csr_kernel = 4;
    if (sim->csr_kernel == 7 && !choose_box_width(sim)) sim->csr_kernel = 6;
    return resolve_exec(sim);
}

// Reads (and clears) the device error flag set by bounded waits that expired.
// The caller has synchronised the simulation stream.
titan_status check_device_error(titan_sim *sim) {
    int flag = 0;
    TITAN_CK(sim, cudaMemcpy(&flag, sim->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        TITAN_CK(sim, cudaMemset(sim->d_err, 0, sizeof(int)));
        return fail(sim, TITAN_E_TIMEOUT, "a bounded device wait expired; the affected steps did not complete");
    }
    return TITAN_OK;
}

}  // namespace

cudaError_t titan::enqueue_sim_step(titan_sim *sim, cudaStream_t st, int b, bool after_step) {
    return enqueue_step(sim, st, b, after_step);
}

cudaError_t titan::enqueue_sim_step_io(titan_sim *sim, cudaStream_t st, const MassState *in, MassState *out,
                                       const long long *step_in, long long *step_out, bool after_step) {
    return enqueue_step_io(sim, st, in, out, step_in, step_out, after_step);
}

namespace {

// Captures k_steps steps starting from state buffer b into *out.
cudaError_t capture_steps(titan_sim *sim, uint64_t k_steps, int b, cudaGraphExec_t *out) {
    cudaError_t e = cudaStreamBeginCapture(sim->capture, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t le = cudaSuccess;
    // the graph's first step follows whatever precedes the graph launch: plain order
    for (uint64_t k = 0; k < k_steps && le == cudaSuccess; ++k)
        le = enqueue_step(sim, sim->capture, b ^ (int)(k & 1), k > 0);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(sim->capture, &g);
    if (le != cudaSuccess) { if (g) cudaGraphDestroy(g); return le; }
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    return e;
}

cudaError_t capture_graph(titan_sim *sim, int L, int b) {
    return capture_steps(sim, (uint64_t)graph_steps(sim, L), b, &sim->graph[L][b]);
}

// The graph of exactly n steps from buffer b, captured on first use (n from
// 3 to twice the graph chunk that is not itself a ladder level); null if the
// count does not qualify or the capture failed (the ladder then runs it).
cudaGraphExec_t exact_graph(titan_sim *sim, uint64_t n, int b) {
    if (n < 3 || n > 2 * (uint64_t)sim->graph_chunk) return nullptr;
    for (int L = 0; L < kGraphLevels; ++L)
        if ((uint64_t)graph_steps(sim, L) == n) return nullptr;
    ++sim->exact_clock;
    SimCore::ExactGraph *slot = &sim->exact[0];
    for (auto &x : sim->exact) {
        if (x.exec && x.n == n && x.b == b) {
            x.last_use = sim->exact_clock;
            return x.exec;
        }
        if (!x.exec || (slot->exec && x.last_use < slot->last_use)) slot = &x;
    }
    if (slot->exec) cudaGraphExecDestroy(slot->exec);
    *slot = SimCore::ExactGraph();
    cudaGraphExec_t g = nullptr;
    if (capture_steps(sim, n, b, &g) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    slot->n = n;
    slot->b = b;
    slot->last_use = sim->exact_clock;
    slot->exec = g;
    return g;
}

// Captures every level's graph for both starting buffers at once (so that no
// later titan_step captures), on the first stepping call after a layout or
// constants change.  If capturing the programmatic launches fails, the step
// kernels fall back to plain stream order and the graphs are captured again.
cudaError_t ensure_graphs(titan_sim *sim) {
    if (sim->graphs_built || sim->graph_chunk <= 0) return cudaSuccess;
    for (int attempt = 0; attempt < 2; ++attempt) {
        cudaError_t e = cudaSuccess;
        for (int L = 0; L < kGraphLevels && e == cudaSuccess; ++L)
            for (int b = 0; b < 2 && e == cudaSuccess; ++b)
                if (graph_steps(sim, L)) e = capture_graph(sim, L, b);
        if (e == cudaSuccess) {
            sim->graphs_built = true;
            return cudaSuccess;
        }
        free_graphs(sim);
        cudaGetLastError();
        if (!sim->launch_overlap || attempt) return e;
        sim->launch_overlap = false;
    }
    return cudaErrorUnknown;
}

}  // namespace

extern "C" {

void titan_default_params(titan_params *p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->dt = 1e-4;
    p->gravity[2] = -9.81;
    p->ground = 0;
    p->ground_k = 1e5;
    p->mu = 0.5;
    p->damping = 0.0;
    p->accumulate = TITAN_ACCUM_CSR;
    p->order = TITAN_ORDER_MORTON;
    p->exec = TITAN_EXEC_AUTO;
    p->device = 0;
    p->stream = nullptr;
    p->spin_limit = 0;
    p->graph_chunk = 0;
    p->l2_persist = 1;
    p->launch_overlap = 1;
}

titan_status titan_create(const titan_masses *m, const titan_springs *sp, const titan_params *p,
                          titan_sim **out) {
    if (!out) return fail(nullptr, TITAN_E_INVALID, "out is null");
    titan_status vs = validate(m, sp, p);
    if (vs != TITAN_OK) return vs;

    DeviceGuard dg(p->device);
    if (!dg.ok) return fail(nullptr, TITAN_E_CUDA, "cannot select CUDA device " + std::to_string(p->device));
    titan_sim *sim = new titan_sim();
    sim->device = p->device;
    sim->n = m->n;
    sim->s = sp->n;
    sim->accumulate = p->accumulate;
    sim->dt = p->dt;
    sim->graph_chunk = p->graph_chunk == 0 ? kDefaultGraphChunk : (p->graph_chunk < 0 ? 0 : ((p->graph_chunk + 1) & ~1));
    sim->c.dt = (float)p->dt;
    sim->c.dt_d = p->dt;
    sim->c.gx = (float)p->gravity[0];
    sim->c.gy = (float)p->gravity[1];
    sim->c.gz = (float)p->gravity[2];
    sim->c.ground = p->ground ? 1 : 0;
    sim->c.ground_k = (float)p->ground_k;
    sim->c.mu = (float)p->mu;
    sim->c.c_uniform = (float)p->damping;
    sim->c.act_omega = 0.0;
    sim->kernel_variant = p->kernel_variant;
    sim->launch_overlap = p->launch_overlap != 0;
    sim->exec_req = p->exec;
    sim->spin_limit = p->spin_limit == 0 ? kDefaultSpinLimit
                                         : (uint32_t)(p->spin_limit > 0xffffffffull ? 0xffffffffull : p->spin_limit);

    auto bail = [&](titan_status st) {
        g_thread_error = sim->error;
        release(sim);
        delete sim;
        return st;
    };
#define CREATE_CK(call)                                                      \
    do {                                                                     \
        cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess) return bail(fail_cuda(sim, e_, #call));       \
    } while (0)

    if (p->stream) {
        sim->stream = static_cast<cudaStream_t>(p->stream);
    } else {
        CREATE_CK(cudaStreamCreateWithFlags(&sim->stream, cudaStreamNonBlocking));
        sim->own_stream = true;
    }
    CREATE_CK(cudaStreamCreateWithFlags(&sim->side, cudaStreamNonBlocking));
    CREATE_CK(cudaStreamCreateWithFlags(&sim->capture, cudaStreamNonBlocking));

    // ---- host-side layout
    const uint32_t n = m->n, s = sp->n;
    std::vector<int32_t> cells;           // grid cell per device index (grid-tile order only)
    if (p->order == TITAN_ORDER_MORTON) {
        // masses on a grid (pitch = shortest spring) get the grid-tile order, others Morton
        double h = INFINITY;
        for (uint32_t q = 0; q < s; ++q) {
            const uint32_t i = sp->ends[2 * (size_t)q], j = sp->ends[2 * (size_t)q + 1];
            double d2 = 0;
            for (int a = 0; a < 3; ++a) {
                const double d = m->pos[3 * (size_t)j + a] - m->pos[3 * (size_t)i + a];
                d2 += d * d;
            }
            if (d2 > 0) h = std::min(h, std::sqrt(d2));
        }
        sim->grid_order = s > 0 && titan::grid_tile_order(m->pos, n, h, sim->caller_of_dev, &cells) &&
                          sim->caller_of_dev.size() <= 2 * (size_t)n + 4096;
        if (!sim->grid_order) {
            cells.clear();
            titan::morton_order(m->pos, n, sim->caller_of_dev);
        }
    } else {
        sim->caller_of_dev.resize(n);
        for (uint32_t i = 0; i < n; ++i) sim->caller_of_dev[i] = i;
    }
    sim->n_dev = (uint32_t)sim->caller_of_dev.size();
    sim->dev_of_caller.resize(n);
    for (uint32_t d = 0; d < sim->n_dev; ++d)
        if (sim->caller_of_dev[d] != UINT32_MAX) sim->dev_of_caller[sim->caller_of_dev[d]] = d;
    sim->inv_mass.resize(n);
    for (uint32_t i = 0; i < n; ++i)
        sim->inv_mass[i] = (m->fixed && m->fixed[i]) ? 0.f : (float)(1.0 / m->mass[i]);
    sim->k.resize(s);
    sim->rest.resize(s);
    sim->damp.resize(s);
    bool uniform_c = true;
    for (uint32_t q = 0; q < s; ++q) {
        const uint32_t i = sp->ends[2 * (size_t)q], j = sp->ends[2 * (size_t)q + 1];
        sim->k[q] = (float)sp->k[q];
        double L;
        if (sp->rest) {
            L = sp->rest[q];
        } else {
            const double dx = m->pos[3 * (size_t)j] - m->pos[3 * (size_t)i];
            const double dy = m->pos[3 * (size_t)j + 1] - m->pos[3 * (size_t)i + 1];
            const double dz = m->pos[3 * (size_t)j + 2] - m->pos[3 * (size_t)i + 2];
            L = sqrt(dx * dx + dy * dy + dz * dz);
        }
        sim->rest[q] = (float)L;
        sim->damp[q] = (float)(sp->damping ? sp->damping[q] : p->damping);
        if (q && sim->damp[q] != sim->damp[0]) uniform_c = false;
    }
    sim->has_c = !uniform_c;
    if (uniform_c && s) sim->c.c_uniform = sim->damp[0];
    sim->params = *p;
    sim->h_mass.assign(m->mass, m->mass + n);
    sim->h_fixed.assign(n, 0);
    if (m->fixed)
        for (uint32_t i = 0; i < n; ++i) sim->h_fixed[i] = m->fixed[i] ? 1 : 0;
    sim->h_ends.assign(sp->ends, sp->ends + 2 * (size_t)s);
    sim->h_k.assign(sp->k, sp->k + s);
    sim->h_rest.resize(s);
    sim->h_damp.resize(s);
    for (uint32_t q = 0; q < s; ++q) {
        sim->h_rest[q] = sp->rest ? sp->rest[q] : (double)sim->rest[q];
        sim->h_damp[q] = sp->damping ? sp->damping[q] : p->damping;
    }
    if (!sp->rest) {          // keep the FP64 initial distances
        for (uint32_t q = 0; q < s; ++q) {
            const uint32_t i = sp->ends[2 * (size_t)q], j = sp->ends[2 * (size_t)q + 1];
            double d2 = 0;
            for (int a = 0; a < 3; ++a) {
                const double d = m->pos[3 * (size_t)j + a] - m->pos[3 * (size_t)i + a];
                d2 += d * d;
            }
            sim->h_rest[q] = std::sqrt(d2);
        }
    }
    sim->c.act_mode = 1;

    // ---- device state
    const uint32_t nd = sim->n_dev;
    CREATE_CK(dev_alloc(sim, &sim->state[0], 2 * (size_t)nd));   // both buffers in one range (L2 window)
    sim->state[1] = sim->state[0] + nd;
    CREATE_CK(dev_alloc(sim, &sim->steps_dev, 2));
    CREATE_CK(dev_alloc(sim, &sim->d_err, 1));
    CREATE_CK(cudaMemsetAsync(sim->d_err, 0, sizeof(int), sim->stream));
    CREATE_CK(dev_alloc(sim, &sim->d_dev_of_caller, n));
    {
        std::vector<MassState> st;
        fill_state(sim, m->pos, m->vel, st);
        CREATE_CK(upload(sim->state[0], st, sim->stream));
        CREATE_CK(upload(sim->state[1], st, sim->stream));
        CREATE_CK(upload(sim->d_dev_of_caller, sim->dev_of_caller, sim->stream));
        CREATE_CK(cudaMemsetAsync(sim->steps_dev, 0, 2 * sizeof(long long), sim->stream));
    }

    if (sim->accumulate == TITAN_ACCUM_CSR) {
        if (!titan::build_sell(nd, s, sp->ends, m->pos, sim->dev_of_caller, sim->sell,
                               sim->grid_order ? cells.data() : nullptr))
            return bail(fail(sim, TITAN_E_UNSUPPORTED, "padded incidence exceeds 2^32 entries"));
        const int want = p->kernel_variant;
        sim->csr_kernel = want == 0 ? (sim->grid_order ? 6 : 4) : want;
        if (sim->csr_kernel >= 6 && sim->csr_kernel <= 8 &&
            !(sim->grid_order && titan::build_box(nd, sim->sell, cells, sim->caller_of_dev, kHaloMaxSlots, sim->box))) {
            if (want >= 6)
                return bail(fail(sim, TITAN_E_UNSUPPORTED, "the grid box kernel needs masses on a grid whose "
                                                           "blocks' boxes fit " + std::to_string(kHaloMaxSlots) + " slots"));
            sim->csr_kernel = 4;
        }
        if (uses_cube(sim) &&
            !titan::build_cube(nd, s, sp->ends, sim->dev_of_caller, sim->sell, cells, sim->caller_of_dev, sim->box,
                               sim->cube)) {
            if (want == 8)
                return bail(fail(sim, TITAN_E_UNSUPPORTED, "the cube kernel needs 26-neighbour springs on a grid, "
                                                           "at most one per mass and offset"));
            sim->csr_kernel = 6;
        }
        if (sim->csr_kernel == 7 && !choose_box_width(sim)) {
            if (want == 7)
                return bail(fail(sim, TITAN_E_UNSUPPORTED, "the TMA-staged box kernel's shared memory does not fit"));
            sim->csr_kernel = 6;
        }
        if ((sim->csr_kernel == 4 || sim->csr_kernel == 5) &&
            !titan::build_halo(nd, sim->sell, kHaloMaxSlots, sim->grid_order, sim->halo)) {
            if (want == 4 || want == 5)
                return bail(fail(sim, TITAN_E_UNSUPPORTED, "a block's neighbourhood table exceeds " +
                                                               std::to_string(kHaloMaxSlots) + " slots"));
            sim->csr_kernel = 3;
        }
        if (sim->csr_kernel == 5 && !choose_halo_width(sim)) {
            if (want == 5)
                return bail(fail(sim, TITAN_E_UNSUPPORTED, "the halo+TMA kernel's shared memory does not fit"));
            sim->csr_kernel = 4;
        }
        const uint32_t E = sim->sell.entries;
        std::vector<float2> kl(E + titan::kStreamTail, make_float2(0.f, titan::kPadRest));
        std::vector<float> cc;
        if (sim->has_c) cc.assign(E + titan::kStreamTail, 0.f);
        for (uint32_t e = 0; e < E; ++e) {
            const uint32_t q = sim->sell.spring[e];
            if (q == UINT32_MAX) continue;
            kl[e] = make_float2(sim->k[q], sim->rest[q]);
            if (sim->has_c) cc[e] = sim->damp[q];
        }
        CREATE_CK(dev_alloc(sim, &sim->d_slice_off, sim->sell.slice_off.size()));
        CREATE_CK(dev_alloc(sim, &sim->d_kl, E + titan::kStreamTail));
        CREATE_CK(upload(sim->d_slice_off, sim->sell.slice_off, sim->stream));
        CREATE_CK(upload(sim->d_kl, kl, sim->stream));
        if (sim->csr_kernel >= 6 && sim->csr_kernel <= 8) {
            const titan::BoxHost &h = sim->box;
            CREATE_CK(dev_alloc(sim, &sim->d_col_off, h.col_off.size() + 2));      // + one word read ahead
            CREATE_CK(cudaMemsetAsync(sim->d_col_off, 0, (h.col_off.size() + 2) * sizeof(int16_t), sim->stream));
            CREATE_CK(dev_alloc(sim, &sim->d_own_slot, nd));
            CREATE_CK(dev_alloc(sim, &sim->d_ext_off, h.ext_off.size()));
            CREATE_CK(dev_alloc(sim, &sim->d_ext_idx, h.ext_idx.size()));
            CREATE_CK(dev_alloc(sim, &sim->d_ext_slot, h.ext_slot.size()));
            CREATE_CK(upload(sim->d_col_off, h.col_off, sim->stream));
            CREATE_CK(upload(sim->d_own_slot, h.own_slot, sim->stream));
            CREATE_CK(upload(sim->d_ext_off, h.ext_off, sim->stream));
            CREATE_CK(upload(sim->d_ext_idx, h.ext_idx, sim->stream));
            CREATE_CK(upload(sim->d_ext_slot, h.ext_slot, sim->stream));
            if (uses_cube(sim)) {
                const titan::CubeHost &cu = sim->cube;
                std::vector<float2> ckl(cu.entries, make_float2(0.f, titan::kPadRest));
                std::vector<float> c2;
                if (sim->has_c) c2.assign(cu.entries, 0.f);
                for (uint32_t e = 0; e < cu.entries; ++e) {
                    const uint32_t q = cu.spring[e];
                    if (q == UINT32_MAX) continue;
                    ckl[e] = make_float2(sim->k[q], sim->rest[q]);
                    if (sim->has_c) c2[e] = sim->damp[q];
                }
                std::vector<uint4> meta(cu.meta.size() / 4);
                memcpy(meta.data(), cu.meta.data(), cu.meta.size() * sizeof(uint32_t));
                CREATE_CK(dev_alloc(sim, &sim->d_cube_base, cu.base.size()));
                CREATE_CK(dev_alloc(sim, &sim->d_cube_meta, meta.size()));
                CREATE_CK(dev_alloc(sim, &sim->d_ckl, ckl.size()));
                CREATE_CK(upload(sim->d_cube_base, cu.base, sim->stream));
                CREATE_CK(upload(sim->d_cube_meta, meta, sim->stream));
                CREATE_CK(upload(sim->d_ckl, ckl, sim->stream));
                if (sim->has_c) {
                    CREATE_CK(dev_alloc(sim, &sim->d_cc, c2.size()));
                    CREATE_CK(upload(sim->d_cc, c2, sim->stream));
                }
                CREATE_CK(cudaStreamSynchronize(sim->stream));     // the host vectors go out of scope
            }
        } else if (sim->csr_kernel == 4 || sim->csr_kernel == 5) {
            sim->halo_ahead = 0;    // each warp prefetches its own slice
            const titan::HaloHost &h = sim->halo;
            CREATE_CK(dev_alloc(sim, &sim->d_nslot, E));
            CREATE_CK(dev_alloc(sim, &sim->d_own_slot, nd));
            CREATE_CK(dev_alloc(sim, &sim->d_ext_off, h.ext_off.size()));
            CREATE_CK(dev_alloc(sim, &sim->d_ext_idx, h.ext_idx.size()));
            CREATE_CK(dev_alloc(sim, &sim->d_ext_slot, h.ext_slot.size()));
            CREATE_CK(upload(sim->d_nslot, h.nbr_slot, sim->stream));
            CREATE_CK(upload(sim->d_own_slot, h.own_slot, sim->stream));
            CREATE_CK(upload(sim->d_ext_off, h.ext_off, sim->stream));
            CREATE_CK(upload(sim->d_ext_idx, h.ext_idx, sim->stream));
            CREATE_CK(upload(sim->d_ext_slot, h.ext_slot, sim->stream));
        } else {
            CREATE_CK(dev_alloc(sim, &sim->d_nbr, E));
            CREATE_CK(upload(sim->d_nbr, sim->sell.nbr, sim->stream));
        }
        if (sim->has_c) {
            CREATE_CK(dev_alloc(sim, &sim->d_c, E + titan::kStreamTail));
            CREATE_CK(upload(sim->d_c, cc, sim->stream));
        }
    } else {
        titan::build_records(s, sp->ends, sim->dev_of_caller, sim->rec);
        std::vector<uint4> r(s);
        std::vector<float> cc;
        if (sim->has_c) cc.resize(s);
        for (uint32_t k = 0; k < s; ++k) {
            const uint32_t q = sim->rec.order[k];
            uint32_t kb, lb;
            memcpy(&kb, &sim->k[q], 4);
            memcpy(&lb, &sim->rest[q], 4);
            r[k] = make_uint4(sim->dev_of_caller[sp->ends[2 * (size_t)q]], sim->dev_of_caller[sp->ends[2 * (size_t)q + 1]], kb, lb);
            if (sim->has_c) cc[k] = sim->damp[q];
        }
        CREATE_CK(dev_alloc(sim, &sim->d_rec, s));
        CREATE_CK(dev_alloc(sim, &sim->d_force, nd));
        CREATE_CK(upload(sim->d_rec, r, sim->stream));
        CREATE_CK(cudaMemsetAsync(sim->d_force, 0, (size_t)(nd ? nd : 1) * sizeof(float4), sim->stream));
        if (sim->has_c) {
            CREATE_CK(dev_alloc(sim, &sim->d_rc, s));
            CREATE_CK(upload(sim->d_rc, cc, sim->stream));
        }
    }
    if (p->l2_persist && sim->accumulate == TITAN_ACCUM_CSR) l2_persist_on(sim);
    CREATE_CK(resolve_exec(sim));
    if (p->exec == TITAN_EXEC_PERSISTENT && !sim->persistent)
        return bail(fail(sim, TITAN_E_UNSUPPORTED, "exec PERSISTENT: the system does not fit one cluster's shared "
                                                   "memory (or accumulation is atomic)"));
    CREATE_CK(cudaStreamSynchronize(sim->stream));
#undef CREATE_CK
    *out = sim;
    return TITAN_OK;
}

titan_status titan_step(titan_sim *sim, uint64_t n_steps) {
    if (!sim) return fail(nullptr, TITAN_E_INVALID, "sim is null");
    BusyGuard bg(sim);
    if (!bg.acquired) return fail(sim, TITAN_E_BUSY, "another call on this handle is in progress");
    DeviceGuard dg(sim->device);
    {
        titan_status es_ = titan::ensure_layout(sim);
        if (es_ != TITAN_OK) return es_;
    }
    TITAN_CK(sim, cudaGetLastError());
    while (n_steps > 0 && sim->persistent) {
        const uint32_t k = (uint32_t)std::min<uint64_t>(n_steps, kPersistChunk);
        const int b = sim->cur;
        TITAN_CK(sim, titan::launch_step_persistent(sim->state[b], sim->state[1 - b], sim->n_dev, sim->plan,
                                                    sim->d_slice_off, sim->d_pslot, sim->d_phalo, sim->d_kl,
                                                    sim->has_c ? sim->d_c : nullptr, sim->has_act ? sim->d_act : nullptr,
                                                    sim->c, sim->steps_dev + b, sim->steps_dev + (1 - b), k,
                                                    sim->stream));
        sim->cur ^= 1;
        n_steps -= k;
        sim->steps += k;
    }
    // whole graphs, largest level first (each an even step count: the buffer
    // parity is unchanged), then at most one single launch; a count of its
    // own (up to twice the chunk) replays one graph captured for it
    if (n_steps >= 2 && sim->graph_chunk > 0) TITAN_CK(sim, ensure_graphs(sim));
    if (sim->graph_chunk > 0 && sim->graphs_built) {
        if (cudaGraphExec_t g = exact_graph(sim, n_steps, sim->cur)) {
            TITAN_CK(sim, cudaGraphLaunch(g, sim->stream));
            sim->cur ^= (int)(n_steps & 1);
            sim->steps += n_steps;
            n_steps = 0;
        }
    }
    for (int L = 0; L < kGraphLevels && n_steps >= 2; ++L) {
        const uint64_t k = (uint64_t)graph_steps(sim, L);
        if (!k) continue;
        while (n_steps >= k) {
            TITAN_CK(sim, cudaGraphLaunch(sim->graph[L][sim->cur], sim->stream));
            n_steps -= k;
            sim->steps += k;
        }
    }
    for (bool first = true; n_steps > 0; first = false) {
        TITAN_CK(sim, enqueue_step(sim, sim->stream, sim->cur, !first));
        sim->cur ^= 1;
        --n_steps;
        ++sim->steps;
    }
    return TITAN_OK;
}

titan_status titan_snapshot_async(titan_sim *sim, void *stream, uint64_t *ticket) {
    if (!sim || !ticket) return fail(sim, TITAN_E_INVALID, "sim or ticket is null");
    BusyGuard bg(sim);
    if (!bg.acquired) return fail(sim, TITAN_E_BUSY, "another call on this handle is in progress");
    DeviceGuard dg(sim->device);
    {
        titan_status es_ = titan::ensure_layout(sim);
        if (es_ != TITAN_OK) return es_;
    }
    cudaStream_t side = stream ? static_cast<cudaStream_t>(stream) : sim->side;
    const uint64_t tk = sim->last_ticket + 1;
    const int slot = (int)(tk & 1);
    const size_t floats = 6 * (size_t)(sim->n ? sim->n : 1);
    if (!sim->snap_dev[slot]) {
        TITAN_CK(sim, dev_alloc(sim, &sim->snap_dev[slot], floats));
        TITAN_CK(sim, cudaHostAlloc((void **)&sim->snap_host[slot], floats * sizeof(float), cudaHostAllocDefault));
        TITAN_CK(sim, cudaEventCreateWithFlags(&sim->snap_ready[slot], cudaEventDisableTiming));
        TITAN_CK(sim, cudaEventCreateWithFlags(&sim->snap_done[slot], cudaEventDisableTiming));
    } else {
        // the slot's previous device-to-host copy must be done before it is overwritten
        TITAN_CK(sim, cudaStreamWaitEvent(sim->stream, sim->snap_done[slot], 0));
    }
    float *pos = sim->snap_dev[slot], *vel = pos + 3 * (size_t)sim->n;
    TITAN_CK(sim, titan::launch_unpermute(sim->state[sim->cur], sim->d_dev_of_caller, sim->n, pos, vel, sim->stream));
    TITAN_CK(sim, cudaEventRecord(sim->snap_ready[slot], sim->stream));
    TITAN_CK(sim, cudaStreamWaitEvent(side, sim->snap_ready[slot], 0));
    TITAN_CK(sim, cudaMemcpyAsync(sim->snap_host[slot], sim->snap_dev[slot], 6 * (size_t)sim->n * sizeof(float),
                                  cudaMemcpyDeviceToHost, side));
    TITAN_CK(sim, cudaEventRecord(sim->snap_done[slot], side));
    sim->snap_t[slot] = (double)sim->steps * sim->dt;
    sim->last_ticket = tk;
    *ticket = tk;
    return TITAN_OK;
}

titan_status titan_snapshot_wait(titan_sim *sim, uint64_t ticket, const float **pos, const float **vel,
                                 double *t) {
    if (!sim) return fail(nullptr, TITAN_E_INVALID, "sim is null");
    BusyGuard bg(sim);
    if (!bg.acquired) return fail(sim, TITAN_E_BUSY, "another call on this handle is in progress");
    if (ticket == 0 || ticket > sim->last_ticket || sim->last_ticket - ticket >= 2)
        return fail(sim, TITAN_E_INVALID, "snapshot ticket " + std::to_string(ticket) + " is unknown or overwritten");
    DeviceGuard dg(sim->device);
    const int slot = (int)(ticket & 1);
    TITAN_CK(sim, cudaEventSynchronize(sim->snap_done[slot]));
    {
        titan_status es = check_device_error(sim);
        if (es != TITAN_OK) return es;
    }
    if (pos) *pos = sim->snap_host[slot];
    if (vel) *vel = sim->snap_host[slot] + 3 * (size_t)sim->n;
    if (t) *t = sim->snap_t[slot];
    return TITAN_OK;
}

titan_status titan_set_actuation(titan_sim *sim, uint32_t n, const uint32_t *ids, const float *amp,
                                 const float *phase, float freq_hz) {
    if (!sim) return fail(nullptr, TITAN_E_INVALID, "sim is null");
    BusyGuard bg(sim);
    if (!bg.acquired) return fail(sim, TITAN_E_BUSY, "another call on this handle is in progress");
    if (n && (!ids || !amp || !phase)) return fail(sim, TITAN_E_INVALID, "spring_ids, amp and phase are required");
    if (!std::isfinite(freq_hz)) return fail(sim, TITAN_E_INVALID, "freq_hz must be finite");
    {
        titan_status es_ = titan::ensure_layout(sim);
        if (es_ != TITAN_OK) return es_;
    }
    for (uint32_t q = 0; q < n; ++q) {
        if (ids[q] >= sim->s) return fail(sim, TITAN_E_INVALID, "spring id out of range: " + std::to_string(ids[q]));
        if (!std::isfinite(amp[q]) || !std::isfinite(phase[q])) return fail(sim, TITAN_E_INVALID, "non-finite amp or phase");
    }
    DeviceGuard dg(sim->device);
    TITAN_CK(sim, fetch_act_host(sim));
    if (sim->act_amp.empty() || sim->act_mode != 1) {
        sim->act_amp.assign(sim->s, 0.f);
        sim->act_phase.assign(sim->s, 0.f);
    }
    for (uint32_t q = 0; q < n; ++q) {
        sim->act_amp[ids[q]] = amp[q];
        sim->act_phase[ids[q]] = phase[q];
    }
    titan::set_act_clock(sim->c, (double)freq_hz);
    sim->c.act_mode = 1;
    sim->act_mode = 1;
    TITAN_CK(sim, upload_actuation(sim));
    sim->has_act = true;
    TITAN_CK(sim, entries_grew(sim));   // larger entries
    free_graphs(sim);       // kernel variant and constants changed
    return TITAN_OK;
}

titan_status titan_set_actuation_dev(titan_sim *sim, uint32_t n, const float *amp_dev, const float *phase_dev,
                                     float freq_hz) {
    if (!sim) return fail(nullptr, TITAN_E_INVALID, "sim is null");
    BusyGuard bg(sim);
    if (!bg.acquired) return fail(sim, TITAN_E_BUSY, "another call on this handle is in progress");
    if (!std::isfinite(freq_hz)) return fail(sim, TITAN_E_INVALID, "freq_hz must be finite");
    {
        titan_status es_ = titan::ensure_layout(sim);
        if (es_ != TITAN_OK) return es_;
    }
    const uint32_t S = sim->s;
    if (n != S)
        return fail(sim, TITAN_E_INVALID, "n (" + std::to_string(n) + ") is not the spring count (" +
                                              std::to_string(S) + ")");
    if (S && (!amp_dev || !phase_dev)) return fail(sim, TITAN_E_INVALID, "amp and phase are required");
    DeviceGuard dg(sim->device);
    if (S) {
        // the arguments are checked on the device before anything changes
        if (!sim->d_check) TITAN_CK(sim, dev_alloc(sim, &sim->d_check, 1));
        TITAN_CK(sim, cudaMemsetAsync(sim->d_check, 0, sizeof(int), sim->stream));
        k_count_nonfinite<<<(S + 255) / 256, 256, 0, sim->stream>>>(amp_dev, phase_dev, S, sim->d_check);
        TITAN_CK(sim, cudaGetLastError());
        int bad = 0;
        TITAN_CK(sim, cudaMemcpyAsync(&bad, sim->d_check, sizeof(int), cudaMemcpyDeviceToHost, sim->stream));
        TITAN_CK(sim, cudaStreamSynchronize(sim->stream));
        if (bad) return fail(sim, TITAN_E_INVALID, "non-finite amp or phase (" + std::to_string(bad) + " springs)");
        if (!sim->d_act_amp) {
            TITAN_CK(sim, dev_alloc(sim, &sim->d_act_amp, S));
            TITAN_CK(sim, dev_alloc(sim, &sim->d_act_phase, S));
        }
        TITAN_CK(sim, cudaMemcpyAsync(sim->d_act_amp, amp_dev, (size_t)S * 4, cudaMemcpyDeviceToDevice, sim->stream));
        TITAN_CK(sim, cudaMemcpyAsync(sim->d_act_phase, phase_dev, (size_t)S * 4, cudaMemcpyDeviceToDevice, sim->stream));
        TITAN_CK(sim, cudaStreamSynchronize(sim->stream));   // the caller's arrays are free on return
    }
    titan::StepConst nc = sim->c;
    titan::set_act_clock(nc, (double)freq_hz);
    // captured step graphs hold the kernel variant and the clock constants
    const bool same = sim->has_act && sim->act_mode == 1 && sim->c.act_turns == nc.act_turns &&
                      sim->c.act_omega == nc.act_omega;
    sim->c = nc;
    sim->c.act_mode = 1;
    sim->act_mode = 1;
    sim->act_host_stale = S > 0;
    if (!S) {
        sim->act_amp.clear();
        sim->act_phase.clear();
    }
    TITAN_CK(sim, scatter_actuation_dev(sim));
    if (!same) {
        sim->has_act = true;
        TITAN_CK(sim, entries_grew(sim));
        free_graphs(sim);
    }
    return TITAN_OK;
}

titan_status titan_set_state(titan_sim *sim, const double *pos, const double *vel) {
    if (!sim) return fail(nullptr, TITAN_E_INVALID, "sim is null");
    BusyGuard bg(sim);
    if (!bg.acquired) return fail(sim, TITAN_E_BUSY, "another call on this handle is in progress");
    if (sim->n && !pos) return fail(sim, TITAN_E_INVALID, "pos is required");
    DeviceGuard dg(sim->device);
    {
        titan_status es_ = titan::ensure_layout(sim);
        if (es_ != TITAN_OK) return es_;
    }
    const size_t nd = sim->n_dev;
    if (nd == 0) return TITAN_OK;
    // a library-owned pinned staging buffer: the device-order states are
    // written there (validated and converted on several host threads) and
    // leave in one asynchronous copy; its previous copy must be done first
    if (sim->state_stage_cap < nd) {
        if (sim->state_stage) {
            TITAN_CK(sim, cudaEventSynchronize(sim->state_staged));
            cudaFreeHost(sim->state_stage);
            sim->state_stage = nullptr;
            sim->state_stage_cap = 0;
        }
        TITAN_CK(sim, cudaHostAlloc((void **)&sim->state_stage, nd * sizeof(MassState), cudaHostAllocDefault));
        sim->state_stage_cap = nd;
        if (!sim->state_staged) TITAN_CK(sim, cudaEventCreateWithFlags(&sim->state_staged, cudaEventDisableTiming));
    } else {
        TITAN_CK(sim, cudaEventSynchronize(sim->state_staged));
    }
    if (!fill_state_parallel(sim, pos, vel, sim->state_stage))
        return fail(sim, TITAN_E_INVALID, "non-finite pos or vel");
    TITAN_CK(sim, cudaMemcpyAsync(sim->state[sim->cur], sim->state_stage, nd * sizeof(MassState),
                                  cudaMemcpyHostToDevice, sim->stream));
    TITAN_CK(sim, cudaEventRecord(sim->state_staged, sim->stream));
    return TITAN_OK;
}

titan_status titan_read_state_dev(titan_sim *sim, float *pos_dev, float *vel_dev, void *stream) {
    if (!sim) return fail(nullptr, TITAN_E_INVALID, "sim is null");
    BusyGuard bg(sim);
    if (!bg.acquired) return fail(sim, TITAN_E_BUSY, "another call on this handle is in progress");
    DeviceGuard dg(sim->device);
    {
        titan_status es_ = titan::ensure_layout(sim);
        if (es_ != TITAN_OK) return es_;
    }
    TITAN_CK(sim, titan::launch_unpermute(sim->state[sim->cur], sim->d_dev_of_caller, sim->n, pos_dev,
                                          vel_dev, sim->stream));
    if (stream && static_cast<cudaStream_t>(stream) != sim->stream) {
        cudaEvent_t ev;
        TITAN_CK(sim, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        cudaError_t e = cudaEventRecord(ev, sim->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(static_cast<cudaStream_t>(stream), ev, 0);
        cudaEventDestroy(ev);
        TITAN_CK(sim, e);
    }
    return TITAN_OK;
}

titan_status titan_group_centroids(titan_sim *sim, uint32_t n_groups, const uint32_t *first_dev,
                                   const float *origin_dev, float *out_dev) {
    if (!sim) return fail(nullptr, TITAN_E_INVALID, "sim is null");
    BusyGuard bg(sim);
    if (!bg.acquired) return fail(sim, TITAN_E_BUSY, "another call on this handle is in progress");
    if (!n_groups) return TITAN_OK;
    if (!first_dev || !out_dev) return fail(sim, TITAN_E_INVALID, "first_dev and out_dev are required");
    DeviceGuard dg(sim->device);
    {
        titan_status es_ = titan::ensure_layout(sim);
        if (es_ != TITAN_OK) return es_;
    }
    k_group_centroid<<<(n_groups + 127) / 128, 128, 0, sim->stream>>>(sim->state[sim->cur], sim->d_dev_of_caller,
                                                                       sim->n, first_dev, n_groups, origin_dev,
                                                                       out_dev);
    TITAN_CK(sim, cudaGetLastError());
    return TITAN_OK;
}

titan_status titan_group_seed(titan_sim *sim, uint32_t n_groups, const uint32_t *first_dev, const float *w_dev,
                              int32_t axis, float *seed_dev) {
    if (!sim) return fail(nullptr, TITAN_E_INVALID, "sim is null");
    BusyGuard bg(sim);
    if (!bg.acquired) return fail(sim, TITAN_E_BUSY, "another call on this handle is in progress");
    if (axis < 0 || axis > 2) return fail(sim, TITAN_E_INVALID, "axis must be 0, 1 or 2");
    if (!seed_dev || (n_groups && (!first_dev || !w_dev)))
        return fail(sim, TITAN_E_INVALID, "seed_dev, first_dev and w_dev are required");
    DeviceGuard dg(sim->device);
    {
        titan_status es_ = titan::ensure_layout(sim);
        if (es_ != TITAN_OK) return es_;
    }
    if (!sim->n) return TITAN_OK;
    TITAN_CK(sim, cudaMemsetAsync(seed_dev, 0, (size_t)sim->n * 3 * sizeof(float), sim->stream));
    if (n_groups) {
        k_group_seed<<<(n_groups + 3) / 4, 128, 0, sim->stream>>>(first_dev, n_groups, sim->n, w_dev, axis, seed_dev);
        TITAN_CK(sim, cudaGetLastError());
    }
    return TITAN_OK;
}

titan_status titan_set_step(titan_sim *sim, uint64_t step) {
    if (!sim) return fail(nullptr, TITAN_E_INVALID, "sim is null");
    BusyGuard bg(sim);
    if (!bg.acquired) return fail(sim, TITAN_E_BUSY, "another call on this handle is in progress");
    DeviceGuard dg(sim->device);
    const long long v[2] = {(long long)step, (long long)step};
    TITAN_CK(sim, cudaMemcpyAsync(sim->steps_dev, v, sizeof(v), cudaMemcpyHostToDevice, sim->stream));
    sim->steps = step;
    return TITAN_OK;
}

titan_status titan_sync(titan_sim *sim) {
    if (!sim) return fail(nullptr, TITAN_E_INVALID, "sim is null");
    BusyGuard bg(sim);
    if (!bg.acquired) return fail(sim, TITAN_E_BUSY, "another call on this handle is in progress");
    DeviceGuard dg(sim->device);
    TITAN_CK(sim, cudaStreamSynchronize(sim->stream));
    TITAN_CK(sim, cudaStreamSynchronize(sim->side));
    return check_device_error(sim);
}

uint64_t titan_steps(const titan_sim *sim) { return sim ? sim->steps : 0; }

int32_t titan_exec_mode(const titan_sim *sim) {
    if (!sim) return -1;
    return sim->persistent ? TITAN_EXEC_PERSISTENT : TITAN_EXEC_LAUNCH;
}

int32_t titan_csr_kernel(const titan_sim *sim) {
    if (!sim) return -1;
    return sim->accumulate == TITAN_ACCUM_CSR ? sim->csr_kernel : 0;
}

const char *titan_last_error(const titan_sim *sim) {
    return sim ? sim->error.c_str() : g_thread_error.c_str();
}

titan_status titan_destroy(titan_sim *sim) {
    if (!sim) return TITAN_OK;
    titan_status st = TITAN_OK;
    {
        DeviceGuard dg(sim->device);
        if (cudaStreamSynchronize(sim->stream) != cudaSuccess) st = TITAN_E_CUDA;
        if (sim->side && cudaStreamSynchronize(sim->side) != cudaSuccess) st = TITAN_E_CUDA;
        release(sim);
    }
    delete sim;
    return st;
}

}  // extern "C"

// ------------------------------------------------------------------ topology and parameter edits

namespace {

// Writes 32-bit words in device memory: base[idx[k]] = val[k] (stream-ordered).
cudaError_t patch_words(titan_sim *sim, void *base, const std::vector<uint32_t> &idx,
                        const std::vector<uint32_t> &val) {
    if (idx.empty()) return cudaSuccess;
    uint32_t *d = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&d, idx.size() * 8, sim->stream);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(d, idx.data(), idx.size() * 4, cudaMemcpyHostToDevice, sim->stream)) == cudaSuccess &&
        (e = cudaMemcpyAsync(d + idx.size(), val.data(), idx.size() * 4, cudaMemcpyHostToDevice, sim->stream)) == cudaSuccess)
        e = titan::launch_patch_words(static_cast<uint32_t *>(base), d, d + idx.size(), (uint32_t)idx.size(), sim->stream);
    cudaFreeAsync(d, sim->stream);
    return e;
}

uint32_t fbits(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
}

// Turns the uniform dashpot into a per-entry array (needed once a spring's damping is edited).
cudaError_t enable_per_spring_damping(titan_sim *sim) {
    if (sim->has_c) return cudaSuccess;
    cudaError_t e;
    if (sim->accumulate == TITAN_ACCUM_CSR) {
        std::vector<float> cc(sim->sell.entries + titan::kStreamTail, 0.f);
        for (uint32_t e2 = 0; e2 < sim->sell.entries; ++e2)
            if (sim->sell.spring[e2] != UINT32_MAX) cc[e2] = sim->damp[sim->sell.spring[e2]];
        if (!sim->d_c && (e = dev_alloc(sim, &sim->d_c, sim->sell.entries + titan::kStreamTail)) != cudaSuccess)
            return e;
        if ((e = upload(sim->d_c, cc, sim->stream)) != cudaSuccess) return e;
        if (uses_cube(sim)) {
            std::vector<float> c2(sim->cube.entries, 0.f);
            for (uint32_t e2 = 0; e2 < sim->cube.entries; ++e2)
                if (sim->cube.spring[e2] != UINT32_MAX) c2[e2] = sim->damp[sim->cube.spring[e2]];
            if (!sim->d_cc && (e = dev_alloc(sim, &sim->d_cc, sim->cube.entries)) != cudaSuccess) return e;
            if ((e = upload(sim->d_cc, c2, sim->stream)) != cudaSuccess) return e;
        }
    } else {
        std::vector<float> cc(sim->s);
        for (uint32_t r = 0; r < sim->s; ++r) cc[r] = sim->damp[sim->rec.order[r]];
        if (!sim->d_rc && (e = dev_alloc(sim, &sim->d_rc, sim->s)) != cudaSuccess) return e;
        if ((e = upload(sim->d_rc, cc, sim->stream)) != cudaSuccess) return e;
    }
    sim->has_c = true;
    if ((e = entries_grew(sim)) != cudaSuccess) return e;
    free_graphs(sim);
    return cudaSuccess;
}

// Pushes the current host parameters of device springs `ids` into the device layout.
cudaError_t push_springs(titan_sim *sim, const std::vector<uint32_t> &ids, bool damping, bool actuation) {
    if (actuation) {
        cudaError_t fe = fetch_act_host(sim);
        if (fe != cudaSuccess) return fe;
    }
    std::vector<uint32_t> wi, wv, ci, cv, ai, av;
    std::vector<uint32_t> xwi, xwv, xci, xcv, xai, xav;      // the cube stream (cube kernel)
    for (uint32_t q : ids) {
        const float kf = sim->k[q], lf = sim->rest[q];
        if (sim->accumulate == TITAN_ACCUM_CSR) {
            for (int end = 0; end < 2; ++end) {
                const uint32_t e = sim->sell.entry_of_end[2 * (size_t)q + end];
                wi.push_back(2 * e); wv.push_back(fbits(kf));
                wi.push_back(2 * e + 1); wv.push_back(fbits(lf));
                if (damping) { ci.push_back(e); cv.push_back(fbits(sim->damp[q])); }
                if (actuation) { ai.push_back(2 * e); av.push_back(fbits(sim->act_amp[q])); }
                if (uses_cube(sim)) {
                    const uint32_t x = sim->cube.pos_of_end[2 * (size_t)q + end];
                    if (x == UINT32_MAX) continue;                  // this end receives the force
                    xwi.push_back(2 * x); xwv.push_back(fbits(kf));
                    xwi.push_back(2 * x + 1); xwv.push_back(fbits(lf));
                    if (damping) { xci.push_back(x); xcv.push_back(fbits(sim->damp[q])); }
                    if (actuation) { xai.push_back(2 * x); xav.push_back(fbits(sim->act_amp[q])); }
                }
            }
        } else {
            const uint32_t r = sim->rec.slot_of_spring[q];
            wi.push_back(4 * r + 2); wv.push_back(fbits(kf));
            wi.push_back(4 * r + 3); wv.push_back(fbits(lf));
            if (damping) { ci.push_back(r); cv.push_back(fbits(sim->damp[q])); }
            if (actuation) { ai.push_back(2 * r); av.push_back(fbits(sim->act_amp[q])); }
        }
    }
    cudaError_t e;
    void *words = sim->accumulate == TITAN_ACCUM_CSR ? (void *)sim->d_kl : (void *)sim->d_rec;
    if ((e = patch_words(sim, words, wi, wv)) != cudaSuccess) return e;
    if (damping && (e = patch_words(sim, sim->accumulate == TITAN_ACCUM_CSR ? (void *)sim->d_c : (void *)sim->d_rc, ci, cv)) != cudaSuccess)
        return e;
    if (actuation && (e = patch_words(sim, sim->accumulate == TITAN_ACCUM_CSR ? (void *)sim->d_act : (void *)sim->d_ract, ai, av)) != cudaSuccess)
        return e;
    if (!xwi.empty()) {
        if ((e = patch_words(sim, sim->d_ckl, xwi, xwv)) != cudaSuccess) return e;
        if (damping && (e = patch_words(sim, sim->d_cc, xci, xcv)) != cudaSuccess) return e;
        if (actuation && (e = patch_words(sim, sim->d_cact, xai, xav)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

// Rebuilds the device layout after masses or springs were added, keeping the
// state, the step counter and the actuation.  The handle stays valid;
// snapshots taken before become invalid.
titan_status titan::ensure_layout(titan_sim *sim) {
    if (!sim->dirty) return TITAN_OK;
    const uint32_t n_old = sim->n;
    const uint32_t n_tot = (uint32_t)sim->h_mass.size();
    const uint32_t s_tot = (uint32_t)sim->h_k.size();
    std::vector<double> pos(3 * (size_t)n_tot), vel(3 * (size_t)n_tot);
    if (n_old) {
        float *d = nullptr;
        std::vector<float> h(6 * (size_t)n_old);
        TITAN_CK(sim, cudaMallocAsync((void **)&d, h.size() * 4, sim->stream));
        cudaError_t e = titan::launch_unpermute(sim->state[sim->cur], sim->d_dev_of_caller, n_old, d,
                                                d + 3 * (size_t)n_old, sim->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d, h.size() * 4, cudaMemcpyDeviceToHost, sim->stream);
        cudaFreeAsync(d, sim->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(sim->stream);
        TITAN_CK(sim, e);
        for (size_t k = 0; k < 3 * (size_t)n_old; ++k) {
            pos[k] = h[k];
            vel[k] = h[3 * (size_t)n_old + k];
        }
    }
    for (size_t k = 0; k < sim->pend_pos.size(); ++k) {
        pos[3 * (size_t)n_old + k] = sim->pend_pos[k];
        vel[3 * (size_t)n_old + k] = sim->pend_vel[k];
    }
    std::vector<double> rest = sim->h_rest;
    for (uint32_t q = 0; q < s_tot; ++q)
        if (std::isnan(rest[q])) {          // added without a rest length: the current distance
            const uint32_t i = sim->h_ends[2 * (size_t)q], j = sim->h_ends[2 * (size_t)q + 1];
            double d2 = 0;
            for (int a = 0; a < 3; ++a) {
                const double d = pos[3 * (size_t)j + a] - pos[3 * (size_t)i + a];
                d2 += d * d;
            }
            rest[q] = std::sqrt(d2);
        }
    titan_masses ms{n_tot, pos.data(), vel.data(), sim->h_mass.data(), sim->h_fixed.data()};
    titan_springs ss{s_tot, sim->h_ends.data(), sim->h_k.data(), rest.data(), sim->h_damp.data()};
    titan_params p = sim->params;
    p.stream = sim->stream;
    titan_sim *fresh = nullptr;
    titan_status st = titan_create(&ms, &ss, &p, &fresh);
    if (st != TITAN_OK) return fail(sim, st, std::string("rebuild after a topology edit: ") + titan_last_error(nullptr));
    // carry the clock and the actuation across
    TITAN_CK(sim, fetch_act_host(sim));
    const uint64_t steps = sim->steps;
    std::vector<float> amp = sim->act_amp, phase = sim->act_phase;
    const int act_mode = sim->act_mode;
    const titan::StepConst oldc = sim->c;
    const bool own = sim->own_stream;
    std::swap(static_cast<SimCore &>(*sim), static_cast<SimCore &>(*fresh));
    sim->own_stream = own;
    fresh->own_stream = false;
    titan_destroy(fresh);
    sim->steps = steps;
    const long long v[2] = {(long long)steps, (long long)steps};
    TITAN_CK(sim, cudaMemcpyAsync(sim->steps_dev, v, sizeof(v), cudaMemcpyHostToDevice, sim->stream));
    if (act_mode) {
        amp.resize(s_tot, 0.f);
        phase.resize(s_tot, 0.f);
        sim->act_amp = amp;
        sim->act_phase = phase;
        sim->act_mode = act_mode;
        sim->c.act_mode = oldc.act_mode;
        sim->c.act_omega = oldc.act_omega;
        sim->c.act_turns = oldc.act_turns;
        sim->c.worm_omega = oldc.worm_omega;
        sim->c.worm_period = oldc.worm_period;
        sim->c.worm_turns = oldc.worm_turns;
        sim->c.worm_unit = oldc.worm_unit;
        TITAN_CK(sim, upload_actuation(sim));
        sim->has_act = true;
        TITAN_CK(sim, entries_grew(sim));
        free_graphs(sim);
    }
    TITAN_CK(sim, cudaStreamSynchronize(sim->stream));
    return TITAN_OK;
}

extern "C" {

titan_status titan_set_spring_params(titan_sim *sim, uint32_t n, const uint32_t *ids, const double *k,
                                     const double *rest, const double *damping) {
    if (!sim) return fail(nullptr, TITAN_E_INVALID, "sim is null");
    BusyGuard bg(sim);
    if (!bg.acquired) return fail(sim, TITAN_E_BUSY, "another call on this handle is in progress");
    if (n && !ids) return fail(sim, TITAN_E_INVALID, "spring ids are required");
    const uint32_t s_tot = (uint32_t)sim->h_k.size();
    for (uint32_t q = 0; q < n; ++q) {
        if (ids[q] >= s_tot) return fail(sim, TITAN_E_INVALID, "spring id out of range: " + std::to_string(ids[q]));
        if (k && !(std::isfinite(k[q]) && k[q] >= 0)) return fail(sim, TITAN_E_INVALID, "k must be finite and >= 0");
        if (rest && !(std::isfinite(rest[q]) && rest[q] >= 0)) return fail(sim, TITAN_E_INVALID, "rest must be finite and >= 0");
        if (damping && !(std::isfinite(damping[q]) && damping[q] >= 0)) return fail(sim, TITAN_E_INVALID, "damping must be finite and >= 0");
    }
    DeviceGuard dg(sim->device);
    std::vector<uint32_t> live;
    for (uint32_t q = 0; q < n; ++q) {
        const uint32_t id = ids[q];
        if (k) sim->h_k[id] = k[q];
        if (rest) sim->h_rest[id] = rest[q];
        if (damping) sim->h_damp[id] = damping[q];
        if (id < sim->s) {            // on the device already (else the next rebuild takes it)
            if (k) sim->k[id] = (float)k[q];
            if (rest) sim->rest[id] = (float)rest[q];
            if (damping) sim->damp[id] = (float)damping[q];
            live.push_back(id);
        }
    }
    if (damping && !live.empty()) TITAN_CK(sim, enable_per_spring_damping(sim));
    TITAN_CK(sim, push_springs(sim, live, damping != nullptr, false));
    return TITAN_OK;
}

titan_status titan_remove_springs(titan_sim *sim, uint32_t n, const uint32_t *ids) {
    if (!sim) return fail(nullptr, TITAN_E_INVALID, "sim is null");
    BusyGuard bg(sim);
    if (!bg.acquired) return fail(sim, TITAN_E_BUSY, "another call on this handle is in progress");
    if (n && !ids) return fail(sim, TITAN_E_INVALID, "spring ids are required");
    const uint32_t s_tot = (uint32_t)sim->h_k.size();
    for (uint32_t q = 0; q < n; ++q)
        if (ids[q] >= s_tot) return fail(sim, TITAN_E_INVALID, "spring id out of range: " + std::to_string(ids[q]));
    DeviceGuard dg(sim->device);
    TITAN_CK(sim, fetch_act_host(sim));
    std::vector<uint32_t> live;
    for (uint32_t q = 0; q < n; ++q) {
        const uint32_t id = ids[q];
        sim->h_k[id] = 0.0;
        sim->h_damp[id] = 0.0;
        if (id < sim->act_amp.size()) sim->act_amp[id] = 0.f;
        if (id < sim->s) {
            sim->k[id] = 0.f;
            sim->damp[id] = 0.f;
            live.push_back(id);
        }
    }
    if (!live.empty()) {
        const bool damped = sim->has_c || sim->c.c_uniform != 0.f;
        if (damped) TITAN_CK(sim, enable_per_spring_damping(sim));
        TITAN_CK(sim, push_springs(sim, live, damped, sim->has_act));
    }
    return TITAN_OK;
}

titan_status titan_add_springs(titan_sim *sim, uint32_t n, const uint32_t *ends, const double *k, const double *rest,
                               const double *damping, uint32_t *first_id) {
    if (!sim) return fail(nullptr, TITAN_E_INVALID, "sim is null");
    BusyGuard bg(sim);
    if (!bg.acquired) return fail(sim, TITAN_E_BUSY, "another call on this handle is in progress");
    if (n && (!ends || !k)) return fail(sim, TITAN_E_INVALID, "ends and k are required");
    const uint32_t n_tot = (uint32_t)sim->h_mass.size();
    if ((uint64_t)sim->h_k.size() + n >= (1u << 30)) return fail(sim, TITAN_E_INVALID, "too many springs");
    for (uint32_t q = 0; q < n; ++q) {
        const uint32_t i = ends[2 * (size_t)q], j = ends[2 * (size_t)q + 1];
        if (i >= n_tot || j >= n_tot || i == j) return fail(sim, TITAN_E_INVALID, "bad spring ends in addition " + std::to_string(q));
        if (!(std::isfinite(k[q]) && k[q] >= 0)) return fail(sim, TITAN_E_INVALID, "k must be finite and >= 0");
        if (rest && !(std::isfinite(rest[q]) && rest[q] >= 0)) return fail(sim, TITAN_E_INVALID, "rest must be finite and >= 0");
        if (damping && !(std::isfinite(damping[q]) && damping[q] >= 0)) return fail(sim, TITAN_E_INVALID, "damping must be finite and >= 0");
    }
    if (first_id) *first_id = (uint32_t)sim->h_k.size();
    for (uint32_t q = 0; q < n; ++q) {
        sim->h_ends.push_back(ends[2 * (size_t)q]);
        sim->h_ends.push_back(ends[2 * (size_t)q + 1]);
        sim->h_k.push_back(k[q]);
        sim->h_rest.push_back(rest ? rest[q] : NAN);
        sim->h_damp.push_back(damping ? damping[q] : sim->params.damping);
    }
    if (n) sim->dirty = true;
    return TITAN_OK;
}

titan_status titan_add_masses(titan_sim *sim, uint32_t n, const double *pos, const double *vel, const double *mass,
                              const uint8_t *fixed, uint32_t *first_id) {
    if (!sim) return fail(nullptr, TITAN_E_INVALID, "sim is null");
    BusyGuard bg(sim);
    if (!bg.acquired) return fail(sim, TITAN_E_BUSY, "another call on this handle is in progress");
    if (n && (!pos || !mass)) return fail(sim, TITAN_E_INVALID, "pos and mass are required");
    if ((uint64_t)sim->h_mass.size() + n >= (1u << 31)) return fail(sim, TITAN_E_INVALID, "too many masses");
    for (uint64_t i = 0; i < n; ++i) {
        if (!(std::isfinite(mass[i]) && mass[i] > 0)) return fail(sim, TITAN_E_INVALID, "mass must be finite and > 0");
        for (int a = 0; a < 3; ++a)
            if (!std::isfinite(pos[3 * i + a]) || (vel && !std::isfinite(vel[3 * i + a])))
                return fail(sim, TITAN_E_INVALID, "non-finite pos or vel");
    }
    if (first_id) *first_id = (uint32_t)sim->h_mass.size();
    for (uint64_t i = 0; i < n; ++i) {
        sim->h_mass.push_back(mass[i]);
        sim->h_fixed.push_back(fixed && fixed[i] ? 1 : 0);
        for (int a = 0; a < 3; ++a) {
            sim->pend_pos.push_back(pos[3 * i + a]);
            sim->pend_vel.push_back(vel ? vel[3 * i + a] : 0.0);
        }
    }
    if (n) sim->dirty = true;
    return TITAN_OK;
}

titan_status titan_set_fixed(titan_sim *sim, uint32_t n, const uint32_t *ids, const uint8_t *fixed) {
    if (!sim) return fail(nullptr, TITAN_E_INVALID, "sim is null");
    BusyGuard bg(sim);
    if (!bg.acquired) return fail(sim, TITAN_E_BUSY, "another call on this handle is in progress");
    if (n && (!ids || !fixed)) return fail(sim, TITAN_E_INVALID, "ids and fixed are required");
    const uint32_t n_tot = (uint32_t)sim->h_mass.size();
    for (uint32_t q = 0; q < n; ++q)
        if (ids[q] >= n_tot) return fail(sim, TITAN_E_INVALID, "mass id out of range: " + std::to_string(ids[q]));
    DeviceGuard dg(sim->device);
    std::vector<uint32_t> wi, wv;
    for (uint32_t q = 0; q < n; ++q) {
        const uint32_t i = ids[q];
        sim->h_fixed[i] = fixed[q] ? 1 : 0;
        if (i < sim->n) {
            sim->inv_mass[i] = fixed[q] ? 0.f : (float)(1.0 / sim->h_mass[i]);
            wi.push_back(8 * sim->dev_of_caller[i] + 3);     // MassState word 3 = p.w = 1/m
            wv.push_back(fbits(sim->inv_mass[i]));
        }
    }
    TITAN_CK(sim, patch_words(sim, sim->state[sim->cur], wi, wv));
    return TITAN_OK;
}

titan_status titan_set_worm_actuation(titan_sim *sim, uint32_t n, const uint32_t *ids, const float *c,
                                      const float *t_offset, float omega, float period) {
    if (!sim) return fail(nullptr, TITAN_E_INVALID, "sim is null");
    {
        BusyGuard bg(sim);
        if (!bg.acquired) return fail(sim, TITAN_E_BUSY, "another call on this handle is in progress");
        if (n && (!ids || !c || !t_offset)) return fail(sim, TITAN_E_INVALID, "ids, c and t_offset are required");
        if (!std::isfinite(omega) || !(period > 0) || !std::isfinite(period))
            return fail(sim, TITAN_E_INVALID, "omega must be finite and period > 0");
        titan_status es = titan::ensure_layout(sim);
        if (es != TITAN_OK) return es;
        for (uint32_t q = 0; q < n; ++q) {
            if (ids[q] >= sim->s) return fail(sim, TITAN_E_INVALID, "spring id out of range: " + std::to_string(ids[q]));
            if (!std::isfinite(c[q]) || !std::isfinite(t_offset[q])) return fail(sim, TITAN_E_INVALID, "non-finite c or t_offset");
        }
        DeviceGuard dg(sim->device);
        TITAN_CK(sim, fetch_act_host(sim));
        if (sim->act_amp.empty() || sim->act_mode != 2) {
            sim->act_amp.assign(sim->s, 0.f);
            sim->act_phase.assign(sim->s, 0.f);
        }
        for (uint32_t q = 0; q < n; ++q) {
            sim->act_amp[ids[q]] = c[q];
            const double to = (double)t_offset[q];
            sim->act_phase[ids[q]] = (float)(to - (double)period * std::floor(to / (double)period));   // in [0, t_p)
        }
        sim->c.act_mode = 2;
        titan::set_worm_clock(sim->c, (double)omega, (double)period);
        sim->act_mode = 2;
        TITAN_CK(sim, upload_actuation(sim));
        sim->has_act = true;
        TITAN_CK(sim, entries_grew(sim));
        free_graphs(sim);
    }
    return TITAN_OK;
}

}  // extern "C"
