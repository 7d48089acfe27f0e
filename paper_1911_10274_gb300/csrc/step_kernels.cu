// step_kernels.cu -- the per-time-step kernels of the spring-mass hot path.
//
// One time step (Titan Sec. III-B, Eq. 1; constraints and planes of Sec. III-A):
//   for every spring (i, j):  d = x_j - x_i, l = |d|, u = d / l,
//       f = k (l - L(t)) + c ((v_j - v_i) . u);  F_i += f u;  F_j -= f u
//   for every mass:  a = F / m + g  (+ ground penalty and Coulomb friction when
//       z < 0), v' = v + a dt, x' = x + v' dt; fixed masses keep x and get v = 0.
//
// K1 (k_step_sell) fuses both passes into one launch: one thread per mass
// gathers its incident springs from the SELL-32 incidence in a fixed order, so
// the sum, and hence the trajectory, is bit-identical from run to run.  Each
// spring is evaluated once from each end; both ends compute the same l, u and
// f bit for bit, so the pair of forces cancels exactly.
// K2 (k_springs_atomic + k_masses_atomic) is the paper's default scatter: one
// thread per spring adds f u to both masses with vector atomics, then one
// thread per mass integrates and clears the accumulator.
#include "titan_internal.h"

namespace titan {
namespace {

constexpr int kThreads = 256;
constexpr double kTwoPi = 6.283185307179586476925286766559;


// Phase of the actuation clock at step `step`: 2 pi f t mod 2 pi with
// t = step dt, formed in FP64 so that long runs keep full FP32 phase accuracy.
__device__ __forceinline__ float clock_phase(const StepConst &c, long long step) {
    double ph = c.act_omega * ((double)step * c.dt_d);
    ph -= kTwoPi * floor(ph / kTwoPi);
    return (float)ph;
}

// Force on the mass at (p, v) from one spring to the mass at (q, w):
// accumulates f u into (fx, fy, fz).  A zero-length spring contributes 0.
__device__ __forceinline__ void spring_force(const float4 &p, const float4 &v, const float4 &q,
                                             const float4 &w, float k, float L, float c,
                                             float &fx, float &fy, float &fz) {
    const float dx = q.x - p.x, dy = q.y - p.y, dz = q.z - p.z;
    const float l2 = dx * dx + dy * dy + dz * dz;
    const float l = sqrtf(l2);
    const float inv = l2 > 0.f ? 1.0f / l : 0.f;
    const float ux = dx * inv, uy = dy * inv, uz = dz * inv;
    const float rate = (w.x - v.x) * ux + (w.y - v.y) * uy + (w.z - v.z) * uz;
    const float f = k * (l - L) + c * rate;
    fx += f * ux;
    fy += f * uy;
    fz += f * uz;
}

// The mass pass for one mass: gravity, ground contact with capped Coulomb
// friction, velocity-first Euler, fixed-mass constraint.
template <bool GROUND>
__device__ __forceinline__ void integrate(const float4 &p, const float4 &v, float fx, float fy,
                                          float fz, const StepConst &c, MassState *out) {
    const float im = p.w;
    float4 xn, vn;
    if (im == 0.f) {
        xn = p;
        vn = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
        float ax = fx * im + c.gx, ay = fy * im + c.gy, az = fz * im + c.gz;
        if (GROUND && p.z < 0.f) {
            const float an = c.ground_k * (-p.z) * im;       // normal force / m
            az += an;
            const float vt = sqrtf(v.x * v.x + v.y * v.y);
            if (vt > 0.f) {
                const float fr = fminf(c.mu * an, vt / c.dt);  // |friction| / m, capped
                ax -= fr * (v.x / vt);
                ay -= fr * (v.y / vt);
            }
        }
        vn = make_float4(v.x + ax * c.dt, v.y + ay * c.dt, v.z + az * c.dt, 0.f);
        xn = make_float4(p.x + vn.x * c.dt, p.y + vn.y * c.dt, p.z + vn.z * c.dt, im);
    }
    out->p = xn;
    out->v = vn;
}

template <bool HAS_C, bool HAS_ACT, bool GROUND>
__global__ void __launch_bounds__(kThreads)
k_step_sell(const MassState *__restrict__ in, MassState *__restrict__ out, uint32_t n,
            const uint32_t *__restrict__ slice_off, const uint32_t *__restrict__ nbr,
            const float2 *__restrict__ kl, const float *__restrict__ cc,
            const float2 *__restrict__ act, StepConst c, const long long *__restrict__ step_in,
            long long *__restrict__ step_out) {
    const uint32_t i = blockIdx.x * kThreads + threadIdx.x;
    long long step = 0;
    if (HAS_ACT) step = *step_in;
    if (blockIdx.x == 0 && threadIdx.x == 0) *step_out = *step_in + 1;
    if (i >= n) return;

    const uint32_t sl = i >> 5, lane = i & 31;
    const uint32_t e0 = __ldg(slice_off + sl);
    const uint32_t width = (__ldg(slice_off + sl + 1) - e0) >> 5;   // even, warp-uniform
    const float4 p = __ldg(&in[i].p);
    const float4 v = __ldg(&in[i].v);
    const float ph = HAS_ACT ? clock_phase(c, step) : 0.f;

    float fx = 0.f, fy = 0.f, fz = 0.f;
    uint32_t e = e0 + lane;
    for (uint32_t t = 0; t < width; t += 2, e += 64) {
        const uint32_t j0 = __ldcs(nbr + e), j1 = __ldcs(nbr + e + 32);
        const float2 a0 = __ldcs(kl + e), a1 = __ldcs(kl + e + 32);
        float c0 = c.c_uniform, c1 = c.c_uniform;
        if (HAS_C) { c0 = __ldcs(cc + e); c1 = __ldcs(cc + e + 32); }
        float L0 = a0.y, L1 = a1.y;
        if (HAS_ACT) {
            const float2 s0 = __ldcs(act + e), s1 = __ldcs(act + e + 32);
            L0 = a0.y * (1.f + s0.x * sinf(ph + s0.y));
            L1 = a1.y * (1.f + s1.x * sinf(ph + s1.y));
        }
        const float4 q0 = __ldg(&in[j0].p), w0 = __ldg(&in[j0].v);
        const float4 q1 = __ldg(&in[j1].p), w1 = __ldg(&in[j1].v);
        spring_force(p, v, q0, w0, a0.x, L0, c0, fx, fy, fz);
        spring_force(p, v, q1, w1, a1.x, L1, c1, fx, fy, fz);
    }
    integrate<GROUND>(p, v, fx, fy, fz, c, out + i);
}

template <bool HAS_C, bool HAS_ACT>
__global__ void __launch_bounds__(kThreads)
k_springs_atomic(const MassState *__restrict__ in, const uint4 *__restrict__ rec,
                 const float *__restrict__ cc, const float2 *__restrict__ act,
                 float4 *__restrict__ force, uint32_t n_springs, StepConst c,
                 const long long *__restrict__ step_in) {
    const uint32_t s = blockIdx.x * kThreads + threadIdx.x;
    if (s >= n_springs) return;
    const uint4 r = __ldcs(rec + s);
    const float k = __uint_as_float(r.z);
    float L = __uint_as_float(r.w);
    if (HAS_ACT) {
        const float2 a = __ldcs(act + s);
        L = L * (1.f + a.x * sinf(clock_phase(c, *step_in) + a.y));
    }
    const float cs = HAS_C ? __ldcs(cc + s) : c.c_uniform;
    const float4 p = __ldg(&in[r.x].p), v = __ldg(&in[r.x].v);
    const float4 q = __ldg(&in[r.y].p), w = __ldg(&in[r.y].v);
    float fx = 0.f, fy = 0.f, fz = 0.f;
    spring_force(p, v, q, w, k, L, cs, fx, fy, fz);
    atomicAdd(force + r.x, make_float4(fx, fy, fz, 0.f));
    atomicAdd(force + r.y, make_float4(-fx, -fy, -fz, 0.f));
}

template <bool GROUND>
__global__ void __launch_bounds__(kThreads)
k_masses_atomic(const MassState *__restrict__ in, MassState *__restrict__ out,
                float4 *__restrict__ force, uint32_t n, StepConst c,
                const long long *__restrict__ step_in, long long *__restrict__ step_out) {
    const uint32_t i = blockIdx.x * kThreads + threadIdx.x;
    if (blockIdx.x == 0 && threadIdx.x == 0) *step_out = *step_in + 1;
    if (i >= n) return;
    const float4 F = force[i];
    force[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    integrate<GROUND>(__ldg(&in[i].p), __ldg(&in[i].v), F.x, F.y, F.z, c, out + i);
}

__global__ void k_unpermute(const MassState *__restrict__ state,
                            const uint32_t *__restrict__ dev_of_caller, uint32_t n,
                            float *__restrict__ pos, float *__restrict__ vel) {
    const uint32_t i = blockIdx.x * kThreads + threadIdx.x;
    if (i >= n) return;
    const uint32_t d = dev_of_caller[i];
    if (pos) {
        const float4 p = state[d].p;
        pos[3 * (size_t)i + 0] = p.x; pos[3 * (size_t)i + 1] = p.y; pos[3 * (size_t)i + 2] = p.z;
    }
    if (vel) {
        const float4 v = state[d].v;
        vel[3 * (size_t)i + 0] = v.x; vel[3 * (size_t)i + 1] = v.y; vel[3 * (size_t)i + 2] = v.z;
    }
}

inline unsigned blocks_for(uint64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

}  // namespace

cudaError_t launch_step_sell(const MassState *in, MassState *out, uint32_t n, const SellView &v,
                             const StepConst &c, const long long *step_in, long long *step_out,
                             cudaStream_t stream) {
    const unsigned g = n ? blocks_for(n) : 1;
    const bool hc = v.c != nullptr, ha = v.act != nullptr, gr = c.ground != 0;
#define TITAN_SELL(HC, HA, GR)                                                                   \
    k_step_sell<HC, HA, GR><<<g, kThreads, 0, stream>>>(in, out, n, v.slice_off, v.nbr, v.kl,  \
                                                        v.c, v.act, c, step_in, step_out)
    if (hc) {
        if (ha) { if (gr) TITAN_SELL(true, true, true); else TITAN_SELL(true, true, false); }
        else    { if (gr) TITAN_SELL(true, false, true); else TITAN_SELL(true, false, false); }
    } else {
        if (ha) { if (gr) TITAN_SELL(false, true, true); else TITAN_SELL(false, true, false); }
        else    { if (gr) TITAN_SELL(false, false, true); else TITAN_SELL(false, false, false); }
    }
#undef TITAN_SELL
    return cudaGetLastError();
}

cudaError_t launch_step_atomic(const MassState *in, MassState *out, uint32_t n,
                               const AtomicView &v, const StepConst &c, const long long *step_in,
                               long long *step_out, cudaStream_t stream) {
    if (v.n_springs) {
        const unsigned g = blocks_for(v.n_springs);
        const bool hc = v.c != nullptr, ha = v.act != nullptr;
#define TITAN_SPR(HC, HA)                                                                        \
    k_springs_atomic<HC, HA><<<g, kThreads, 0, stream>>>(in, v.rec, v.c, v.act, v.force,          \
                                                         v.n_springs, c, step_in)
        if (hc) { if (ha) TITAN_SPR(true, true); else TITAN_SPR(true, false); }
        else    { if (ha) TITAN_SPR(false, true); else TITAN_SPR(false, false); }
#undef TITAN_SPR
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const unsigned g = n ? blocks_for(n) : 1;
    if (c.ground)
        k_masses_atomic<true><<<g, kThreads, 0, stream>>>(in, out, v.force, n, c, step_in, step_out);
    else
        k_masses_atomic<false><<<g, kThreads, 0, stream>>>(in, out, v.force, n, c, step_in, step_out);
    return cudaGetLastError();
}

cudaError_t launch_unpermute(const MassState *state, const uint32_t *dev_of_caller, uint32_t n,
                             float *pos, float *vel, cudaStream_t stream) {
    if (!n) return cudaSuccess;
    k_unpermute<<<blocks_for(n), kThreads, 0, stream>>>(state, dev_of_caller, n, pos, vel);
    return cudaGetLastError();
}

}  // namespace titan
