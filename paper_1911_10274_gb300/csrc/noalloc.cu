// noalloc.cu -- one time step through the atomic-scatter kernels for callers
// that cannot allocate device memory.
//
// The atomic scatter needs a force accumulator per mass on top of its inputs
// and outputs.  titan_create allocates that accumulator with cudaMalloc; this
// entry point instead uses a fixed array that lives in the library itself
// (a file-scope __device__ array, loaded with the module), so a call allocates
// nothing: no cudaMalloc, no cudaFree, no allocating library routine.
//
// Who needs this: code that must not enter the CUDA allocator, such as a
// control loop with a hard per-step deadline (cudaMalloc/cudaFree can
// synchronise the device and take unbounded time), or a plug-in running inside
// a host framework that owns all device memory through its own pool and does
// not let plug-ins allocate outside it.
//
// Limits and sharing: at most kNoAllocMaxMasses masses (the array is 4 MiB and
// every GPU that loads the library holds it until the process exits).  All
// calls in the process share the one array per device: two calls whose work
// overlaps on the GPU (for example on two streams) race on it and both give
// wrong results; serialise them.  The array keeps whatever the last call left
// in it, so each call clears the part it uses before accumulating.
//
// Spring end indices live in device memory, so the host cannot check them
// before the launch.  The spring kernel checks them instead: a spring with an
// end >= n_masses, or with both ends on one mass, is skipped (nothing is read
// or written through it) and counted in a second file-scope word.  The next
// call reads that word first (waiting for the work already queued on its
// stream), clears it, and returns TITAN_E_INVALID without stepping.
#include <cuda.h>

#include <cmath>
#include <mutex>
#include <string>

#include "physics.cuh"
#include "titan.h"
#include "titan_internal.h"

namespace titan {
void set_thread_error(const std::string &msg);   // defined in runtime.cu
}

namespace {

using titan::MassState;
using titan::StepConst;
using titan::integrate;
using titan::spring_force;

constexpr uint32_t kNoAllocMaxMasses = 1u << 18;   // 262,144 masses
constexpr int kThreadsNA = 256;

// The accumulator: one float4 per mass, zeroed by each call before use.
static __device__ __align__(256) float4 g_noalloc_force[kNoAllocMaxMasses];
// Springs the last call skipped for bad end indices (read and cleared by the
// next call).
static __device__ unsigned int g_noalloc_bad_springs;

// Device address of g_noalloc_force per device ordinal, found with that device
// current and kept while the device's context lives: the cache is keyed on the
// context's unique id, so after a cudaDeviceReset (a new primary context, the
// module loaded again, possibly at another address) it is looked up anew.  In
// host code the symbol itself is only a host-side stand-in and must never be
// handed to a kernel.
struct ScratchAddr {
    unsigned long long ctx_id = 0;
    float4 *ptr = nullptr;
};
std::mutex g_addr_mu;
ScratchAddr g_addr[64];

// The driver's context queries, reached through the runtime (no link against
// libcuda): the id of the context current on this thread, 0 if none.
using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;
std::once_flag g_ctx_fns_once;

unsigned long long current_context_id() {
    std::call_once(g_ctx_fns_once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f);
    });
    if (!g_ctx_get_current || !g_ctx_get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
    if (g_ctx_get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

cudaError_t scratch_address(float4 **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_addr_mu);
    const unsigned long long id = current_context_id();
    if (id != 0 && g_addr[dev].ctx_id == id && g_addr[dev].ptr) {
        *out = g_addr[dev].ptr;
        return cudaSuccess;
    }
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_force);     // also makes the primary context current
    if (e != cudaSuccess) return e;
    g_addr[dev].ptr = static_cast<float4 *>(p);
    g_addr[dev].ctx_id = current_context_id();          // 0 (no id): looked up again next call
    *out = g_addr[dev].ptr;
    return cudaSuccess;
}

__device__ __forceinline__ MassState load_plain(const float *pos, const float *vel, const float *inv_mass,
                                                uint32_t i) {
    MassState m;
    m.p = make_float4(pos[3 * (size_t)i], pos[3 * (size_t)i + 1], pos[3 * (size_t)i + 2], inv_mass[i]);
    m.v = make_float4(vel[3 * (size_t)i], vel[3 * (size_t)i + 1], vel[3 * (size_t)i + 2], 0.f);
    return m;
}

__global__ void k_na_springs(const float *__restrict__ pos, const float *__restrict__ vel,
                             const float *__restrict__ inv_mass, const uint32_t *__restrict__ ends,
                             const float *__restrict__ k, const float *__restrict__ rest, float c,
                             uint32_t n_springs, uint32_t n_masses, float4 *__restrict__ force) {
    const uint32_t s = blockIdx.x * kThreadsNA + threadIdx.x;
    if (s >= n_springs) return;
    const uint32_t i = ends[2 * (size_t)s], j = ends[2 * (size_t)s + 1];
    if (i >= n_masses || j >= n_masses || i == j) {     // never read or write through a bad index
        atomicAdd(&g_noalloc_bad_springs, 1u);
        return;
    }
    const MassState a = load_plain(pos, vel, inv_mass, i), b = load_plain(pos, vel, inv_mass, j);
    float fx = 0.f, fy = 0.f, fz = 0.f;
    spring_force(a.p, a.v, b.p, b.v, k[s], rest[s], c, fx, fy, fz);
    atomicAdd(force + i, make_float4(fx, fy, fz, 0.f));
    atomicAdd(force + j, make_float4(-fx, -fy, -fz, 0.f));
}

template <bool GROUND>
__global__ void k_na_masses(const float *__restrict__ pos, const float *__restrict__ vel,
                            const float *__restrict__ inv_mass, const float4 *__restrict__ force,
                            uint32_t n, StepConst c, float *__restrict__ pos_out,
                            float *__restrict__ vel_out) {
    const uint32_t i = blockIdx.x * kThreadsNA + threadIdx.x;
    if (i >= n) return;
    const MassState m = load_plain(pos, vel, inv_mass, i);
    const float4 F = force[i];
    MassState o;
    integrate<GROUND>(m.p, m.v, F.x, F.y, F.z, c, &o);
    pos_out[3 * (size_t)i] = o.p.x; pos_out[3 * (size_t)i + 1] = o.p.y; pos_out[3 * (size_t)i + 2] = o.p.z;
    vel_out[3 * (size_t)i] = o.v.x; vel_out[3 * (size_t)i + 1] = o.v.y; vel_out[3 * (size_t)i + 2] = o.v.z;
}

titan_status na_fail(titan_status st, const std::string &msg) {
    titan::set_thread_error(msg);
    return st;
}

}  // namespace

extern "C" titan_status titan_step_atomic_noalloc(
    uint32_t n_masses, const float *pos_dev, const float *vel_dev, const float *inv_mass_dev,
    uint32_t n_springs, const uint32_t *ends_dev, const float *k_dev, const float *rest_dev,
    float damping, const titan_params *params, float *pos_out_dev, float *vel_out_dev, void *stream) {
    if (!params) return na_fail(TITAN_E_INVALID, "titan_step_atomic_noalloc: params is null");
    if (n_masses > kNoAllocMaxMasses)
        return na_fail(TITAN_E_INVALID, "titan_step_atomic_noalloc: " + std::to_string(n_masses) +
                                            " masses exceed the static scratch limit of " +
                                            std::to_string(kNoAllocMaxMasses));
    if (n_masses && (!pos_dev || !vel_dev || !inv_mass_dev || !pos_out_dev || !vel_out_dev))
        return na_fail(TITAN_E_INVALID, "titan_step_atomic_noalloc: null mass array");
    if (n_springs && (!ends_dev || !k_dev || !rest_dev))
        return na_fail(TITAN_E_INVALID, "titan_step_atomic_noalloc: null spring array");
    if (!(params->dt > 0) || !std::isfinite(params->dt) || !(damping >= 0) || !std::isfinite(damping))
        return na_fail(TITAN_E_INVALID, "titan_step_atomic_noalloc: dt must be > 0 and damping >= 0, finite");
    if (n_masses == 0) return TITAN_OK;

    float4 *force = nullptr;
    cudaError_t e = scratch_address(&force);
    if (e != cudaSuccess)
        return na_fail(TITAN_E_CUDA, std::string("titan_step_atomic_noalloc: cudaGetSymbolAddress: ") +
                                         cudaGetErrorString(e));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the previous call's count of skipped springs (its kernels ran on the GPU
    // after it returned): report it here, clear it, and do not step
    unsigned int bad = 0;
    e = cudaMemcpyFromSymbolAsync(&bad, g_noalloc_bad_springs, sizeof bad, 0, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && bad) {
        static const unsigned int zero = 0;
        e = cudaMemcpyToSymbolAsync(g_noalloc_bad_springs, &zero, sizeof zero, 0, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess)
            return na_fail(TITAN_E_INVALID, "titan_step_atomic_noalloc: the previous call skipped " +
                                                std::to_string(bad) + " spring(s) with an end index >= n_masses "
                                                "or both ends on one mass; this call did not step");
    }
    if (e != cudaSuccess)
        return na_fail(TITAN_E_CUDA, std::string("titan_step_atomic_noalloc: reading the error word: ") +
                                         cudaGetErrorString(e));
    titan::StepConst c{};
    c.dt = (float)params->dt;
    c.dt_d = params->dt;
    c.gx = (float)params->gravity[0];
    c.gy = (float)params->gravity[1];
    c.gz = (float)params->gravity[2];
    c.ground = params->ground ? 1 : 0;
    c.ground_k = (float)params->ground_k;
    c.mu = (float)params->mu;
    c.c_uniform = damping;

    e = cudaMemsetAsync(force, 0, (size_t)n_masses * sizeof(float4), st);
    if (e == cudaSuccess && n_springs) {
        const unsigned blocks = (unsigned)(((uint64_t)n_springs + kThreadsNA - 1) / kThreadsNA);
        k_na_springs<<<blocks, kThreadsNA, 0, st>>>(pos_dev, vel_dev, inv_mass_dev, ends_dev, k_dev, rest_dev,
                                                    damping, n_springs, n_masses, force);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        const unsigned g = (unsigned)(((uint64_t)n_masses + kThreadsNA - 1) / kThreadsNA);
        if (c.ground)
            k_na_masses<true><<<g, kThreadsNA, 0, st>>>(pos_dev, vel_dev, inv_mass_dev, force, n_masses, c,
                                                       pos_out_dev, vel_out_dev);
        else
            k_na_masses<false><<<g, kThreadsNA, 0, st>>>(pos_dev, vel_dev, inv_mass_dev, force, n_masses, c,
                                                        pos_out_dev, vel_out_dev);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess)
        return na_fail(TITAN_E_CUDA, std::string("titan_step_atomic_noalloc: ") + cudaGetErrorString(e));
    return TITAN_OK;
}
