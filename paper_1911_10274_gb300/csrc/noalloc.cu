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

// Device address of g_noalloc_force per device ordinal, found once with that
// device current.  In host code the symbol itself is only a host-side stand-in
// and must never be handed to a kernel.
std::mutex g_addr_mu;
float4 *g_addr[64] = {};

cudaError_t scratch_address(float4 **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_force);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<float4 *>(p);
    }
    *out = g_addr[dev];
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
                             uint32_t n_springs, float4 *__restrict__ force) {
    const uint32_t s = blockIdx.x * kThreadsNA + threadIdx.x;
    if (s >= n_springs) return;
    const uint32_t i = ends[2 * (size_t)s], j = ends[2 * (size_t)s + 1];
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
        k_na_springs<<<(n_springs + kThreadsNA - 1) / kThreadsNA, kThreadsNA, 0, st>>>(
            pos_dev, vel_dev, inv_mass_dev, ends_dev, k_dev, rest_dev, damping, n_springs, force);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        const unsigned g = (n_masses + kThreadsNA - 1) / kThreadsNA;
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
