// adjoint.cu -- reverse-mode derivative of a rollout with respect to the
// actuation amplitudes and phases (gradient-based design of actuated robots).
//
// Forward: the ordinary step (Titan Sec. III-B, Eq. 1; Sec. III-A contact,
// friction and constraints) with L = L0 (1 + A sin(2 pi f t + phi)).  The
// rollout runs forward once, keeping the state every `every` steps
// (checkpoints); then, segment by segment from the last, the segment's states
// are recomputed from its checkpoint and the step is reversed one step at a
// time.  Reversing a step takes two kernels:
//   k_adj_mass   - per mass: the adjoint of x' = x + v' dt, v' = v + a dt and
//                  a = F/m + g + contact/friction (the branch the forward step
//                  took at each kink), giving dJ/dF and the direct terms of
//                  dJ/dx, dJ/dv;
//   k_adj_spring - per mass, gathering its SELL row in the forward's fixed
//                  order: each spring's adjoint seen from this end (both ends
//                  compute the same spring scalars), added to this mass only;
//                  the half-edge of the spring's first end also adds dJ/dA and
//                  dJ/dphi to the spring's gradient (one owner: no atomics,
//                  a fixed summation order).
#include <math.h>

#include <algorithm>
#include <string>
#include <vector>

#include "physics.cuh"
#include "sim_internal.h"

namespace {

constexpr int kT = 256;
constexpr uint32_t kOwner = 0x80000000u;
constexpr uint32_t kNoSpring = 0xffffffffu;

template <bool GROUND>
__global__ void __launch_bounds__(kT)
k_adj_mass(const MassState *__restrict__ X, const float4 *__restrict__ xbo, const float4 *__restrict__ vbo,
           float4 *__restrict__ xb, float4 *__restrict__ vb, float4 *__restrict__ Fb, uint32_t n,
           titan::StepConst c) {
    const uint32_t i = blockIdx.x * kT + threadIdx.x;
    if (i >= n) return;
    const float4 p = X[i].p, v = X[i].v;
    const float4 xo = xbo[i], vo = vbo[i];
    const float im = p.w;
    if (im == 0.f) {                       // fixed: x' = x, v' = 0
        xb[i] = make_float4(xo.x, xo.y, xo.z, 0.f);
        vb[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        Fb[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    const float dt = c.dt;
    const float vtx = vo.x + dt * xo.x, vty = vo.y + dt * xo.y, vtz = vo.z + dt * xo.z;
    float4 x_b = make_float4(xo.x, xo.y, xo.z, 0.f);
    float4 v_b = make_float4(vtx, vty, vtz, 0.f);
    const float abx = dt * vtx, aby = dt * vty, abz = dt * vtz;
    Fb[i] = make_float4(abx * im, aby * im, abz * im, 0.f);
    if (GROUND && p.z < 0.f) {
        x_b.z += -c.ground_k * im * abz;                   // a_z += kg (-z) / m
        const float vt = sqrtf(v.x * v.x + v.y * v.y);
        if (vt > 0.f) {
            const float an = c.ground_k * (-p.z) * im;
            const bool capped = vt / c.dt < c.mu * an;      // the forward's fminf choice
            const float fr = capped ? vt / c.dt : c.mu * an;
            const float wx = v.x / vt, wy = v.y / vt;
            const float frb = -(abx * wx + aby * wy);      // a_t -= fr w
            const float wbx = -fr * abx, wby = -fr * aby;
            float vtb = 0.f;
            if (!capped) x_b.z += -c.mu * c.ground_k * im * frb;
            else vtb = frb / c.dt;
            const float wdot = wbx * wx + wby * wy;
            v_b.x += (wbx - wdot * wx) / vt + vtb * wx;
            v_b.y += (wby - wdot * wy) / vt + vtb * wy;
        }
    }
    xb[i] = x_b;
    vb[i] = v_b;
}

// The adjoint of one spring seen from the mass at (p, v): adds to x_b, v_b and,
// for the spring's owner half-edge, to the spring's (dJ/dA, dJ/dphi) kept at
// that half-edge's entry (coalesced with the rows; gathered per spring at the
// end).
template <bool HAS_C>
__device__ __forceinline__ void adj_half_edge(const float4 &p, const float4 &v, const float4 &Fi, const float4 &q,
                                              const float4 &w, const float4 &Fj, float2 a, float2 s, float cd,
                                              float ph, uint32_t spr, float4 &x_b, float4 &v_b,
                                              float2 *__restrict__ gacc) {
    const float dx = q.x - p.x, dy = q.y - p.y, dz = q.z - p.z;
    const float l2 = dx * dx + dy * dy + dz * dz;
    if (!(l2 > 0.f)) return;                              // zero length: no force
    const float inv = rsqrtf(l2);
    const float l = l2 * inv;
    const float ux = dx * inv, uy = dy * inv, uz = dz * inv;
    const float k = a.x;
    float sn, cs;
    sincosf(ph + s.y, &sn, &cs);
    const float L = a.y * (1.f + s.x * sn);
    const float dvx = w.x - v.x, dvy = w.y - v.y, dvz = w.z - v.z;
    const float rate = dvx * ux + dvy * uy + dvz * uz;
    const float f = k * (l - L) + cd * rate;
    const float gx = Fi.x - Fj.x, gy = Fi.y - Fj.y, gz = Fi.z - Fj.z;
    const float fb = gx * ux + gy * uy + gz * uz;
    const float lb = k * fb, Lb = -k * fb, rb = cd * fb;
    const float ubx = f * gx + rb * dvx, uby = f * gy + rb * dvy, ubz = f * gz + rb * dvz;
    v_b.x -= rb * ux; v_b.y -= rb * uy; v_b.z -= rb * uz;
    const float udot = ubx * ux + uby * uy + ubz * uz;
    x_b.x -= (ubx - udot * ux) * inv + lb * ux;
    x_b.y -= (uby - udot * uy) * inv + lb * uy;
    x_b.z -= (ubz - udot * uz) * inv + lb * uz;
    if (spr & kOwner) {                   // gacc points at this entry's accumulator
        float2 g = *gacc;
        g.x += Lb * a.y * sn;
        g.y += Lb * a.y * s.x * cs;
        *gacc = g;
    }
}

// Widths are even: two entries per iteration, every load of both issued
// before either is reversed (summation order unchanged: entry t, then t + 1).
template <bool HAS_C>
__global__ void __launch_bounds__(kT)
k_adj_spring(const MassState *__restrict__ X, const float4 *__restrict__ Fb, float4 *__restrict__ xb,
             float4 *__restrict__ vb, uint32_t n, const uint32_t *__restrict__ slice_off,
             const uint32_t *__restrict__ nbr, const uint32_t *__restrict__ spring,
             const float2 *__restrict__ kl, const float2 *__restrict__ act, const float *__restrict__ cc,
             titan::StepConst c, long long step, float2 *__restrict__ gacc) {
    const uint32_t i = blockIdx.x * kT + threadIdx.x;
    if (i >= n) return;
    const uint32_t sl = i >> 5, lane = i & 31;
    const uint32_t e0 = slice_off[sl];
    const uint32_t width = (slice_off[sl + 1] - e0) >> 5;
    float4 p, v;
    titan::load_state(X + i, p, v);
    const float4 Fi = Fb[i];
    float4 x_b = xb[i], v_b = vb[i];
    const float ph = titan::clock_phase(c, step);
    for (uint32_t t = 0; t < width; t += 2) {
        const uint32_t e = e0 + 32 * t + lane, f = e + 32;
        const uint32_t spr0 = __ldg(spring + e), spr1 = __ldg(spring + f);
        // padding entries point at the mass itself: their loads are harmless
        const uint32_t j0 = __ldg(nbr + e), j1 = __ldg(nbr + f);
        const float2 a0 = __ldg(kl + e), a1 = __ldg(kl + f), s0 = __ldg(act + e), s1 = __ldg(act + f);
        const float c0 = HAS_C ? __ldg(cc + e) : c.c_uniform, c1 = HAS_C ? __ldg(cc + f) : c.c_uniform;
        float4 q0, w0, q1, w1;
        titan::load_state(X + j0, q0, w0);
        titan::load_state(X + j1, q1, w1);
        const float4 F0 = __ldg(Fb + j0), F1 = __ldg(Fb + j1);
        if (spr0 != kNoSpring)
            adj_half_edge<HAS_C>(p, v, Fi, q0, w0, F0, a0, s0, c0, ph, spr0, x_b, v_b, gacc + e);
        if (spr1 != kNoSpring)
            adj_half_edge<HAS_C>(p, v, Fi, q1, w1, F1, a1, s1, c1, ph, spr1, x_b, v_b, gacc + f);
    }
    xb[i] = x_b;
    vb[i] = v_b;
}

// grad[q] = the accumulator of spring q's owner entry.
__global__ void k_adj_gather(const float2 *__restrict__ gacc, const uint32_t *__restrict__ owner, uint32_t S,
                             float *__restrict__ grad_amp, float *__restrict__ grad_phase) {
    const uint32_t q = blockIdx.x * kT + threadIdx.x;
    if (q >= S) return;
    const float2 g = gacc[owner[q]];
    grad_amp[q] = g.x;
    grad_phase[q] = g.y;
}

__global__ void k_adj_seed(const float *__restrict__ seed_pos, const float *__restrict__ seed_vel,
                           const uint32_t *__restrict__ dev_of_caller, uint32_t n, float4 *__restrict__ xb,
                           float4 *__restrict__ vb) {
    const uint32_t i = blockIdx.x * kT + threadIdx.x;
    if (i >= n) return;
    const uint32_t d = dev_of_caller[i];
    xb[d] = make_float4(seed_pos[3 * (size_t)i], seed_pos[3 * (size_t)i + 1], seed_pos[3 * (size_t)i + 2], 0.f);
    if (seed_vel)
        vb[d] = make_float4(seed_vel[3 * (size_t)i], seed_vel[3 * (size_t)i + 1], seed_vel[3 * (size_t)i + 2], 0.f);
}

titan_status afail(titan_sim *sim, titan_status st, const std::string &msg) {
    sim->error = msg;
    return st;
}

#define ADJ_CK(call)                                                                               \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) {                                                                   \
            st_ = afail(sim, e_ == cudaErrorMemoryAllocation ? TITAN_E_OOM : TITAN_E_CUDA,         \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                        \
            goto done;                                                                             \
        }                                                                                          \
    } while (0)

}  // namespace

extern "C" titan_status titan_adjoint(titan_sim *sim, uint64_t n_steps, uint32_t every,
                                      const float *seed_pos_dev, const float *seed_vel_dev,
                                      float *grad_amp_dev, float *grad_phase_dev) {
    if (!sim) return TITAN_E_INVALID;
    if (sim->busy.exchange(true)) return afail(sim, TITAN_E_BUSY, "another call on this handle is in progress");
    titan_status st_ = TITAN_OK;
    int prev = -1;
    const uint32_t nd = sim->n_dev, S = sim->s;
    const size_t state_bytes = (size_t)std::max(nd, 1u) * sizeof(MassState);
    const size_t vec_bytes = (size_t)std::max(nd, 1u) * sizeof(float4);
    cudaStream_t s = sim->stream;
    MassState *ckpt = nullptr, *seg = nullptr;
    float4 *xb[2] = {nullptr, nullptr}, *vb[2] = {nullptr, nullptr}, *Fb = nullptr;
    long long *seg_steps = nullptr;
    float2 *gacc = nullptr;
    uint64_t n_seg = 0;
    int cur = 0;
    if ((st_ = titan::ensure_layout(sim)) != TITAN_OK) goto out;
    if (sim->accumulate != TITAN_ACCUM_CSR) { st_ = afail(sim, TITAN_E_UNSUPPORTED, "the adjoint needs the CSR (deterministic) accumulation"); goto out; }
    if (sim->act_mode == 2) { st_ = afail(sim, TITAN_E_UNSUPPORTED, "the adjoint differentiates the sinusoidal actuation (mode 1) only"); goto out; }
    if (!sim->has_act) { st_ = afail(sim, TITAN_E_INVALID, "the adjoint differentiates the actuation: call titan_set_actuation first"); goto out; }
    if (!seed_pos_dev || (S && (!grad_amp_dev || !grad_phase_dev))) { st_ = afail(sim, TITAN_E_INVALID, "null seed or gradient array"); goto out; }
    if (every == 0) every = 50;
    cudaGetDevice(&prev);
    if (cudaSetDevice(sim->device) != cudaSuccess) { st_ = afail(sim, TITAN_E_CUDA, "cannot select the device"); goto out; }
    {
        // per-entry neighbour and spring ownership for the reverse gather (built once)
        if (!sim->d_adj_spring) {
            std::vector<uint32_t> spr(sim->sell.entries, kNoSpring);
            for (uint32_t e = 0; e < sim->sell.entries; ++e)
                if (sim->sell.spring[e] != UINT32_MAX) spr[e] = sim->sell.spring[e];
            for (uint32_t q = 0; q < S; ++q) spr[sim->sell.entry_of_end[2 * (size_t)q]] |= kOwner;
            void *p1 = nullptr;
            ADJ_CK(cudaMalloc(&p1, std::max<size_t>(spr.size(), 1) * 4));
            sim->allocations.push_back(p1);
            sim->d_adj_spring = static_cast<uint32_t *>(p1);
            ADJ_CK(cudaMemcpy(sim->d_adj_spring, spr.data(), spr.size() * 4, cudaMemcpyHostToDevice));
            std::vector<uint32_t> owner(S);
            for (uint32_t q = 0; q < S; ++q) owner[q] = sim->sell.entry_of_end[2 * (size_t)q];
            void *p3 = nullptr;
            ADJ_CK(cudaMalloc(&p3, std::max<size_t>(owner.size(), 1) * 4));
            sim->allocations.push_back(p3);
            sim->d_adj_owner = static_cast<uint32_t *>(p3);
            ADJ_CK(cudaMemcpy(sim->d_adj_owner, owner.data(), owner.size() * 4, cudaMemcpyHostToDevice));
            if (!sim->d_nbr) {
                void *p2 = nullptr;
                ADJ_CK(cudaMalloc(&p2, std::max<size_t>(sim->sell.nbr.size(), 1) * 4));
                sim->allocations.push_back(p2);
                sim->d_nbr = static_cast<uint32_t *>(p2);
                ADJ_CK(cudaMemcpy(sim->d_nbr, sim->sell.nbr.data(), sim->sell.nbr.size() * 4, cudaMemcpyHostToDevice));
            }
        }
        n_seg = (n_steps + every - 1) / every;
        const unsigned gm = (nd + kT - 1) / kT;
        ADJ_CK(cudaMallocAsync((void **)&ckpt, state_bytes * (n_seg + 1), s));
        ADJ_CK(cudaMallocAsync((void **)&seg, state_bytes * (every + 1), s));
        for (int b = 0; b < 2; ++b) {
            ADJ_CK(cudaMallocAsync((void **)&xb[b], vec_bytes, s));
            ADJ_CK(cudaMallocAsync((void **)&vb[b], vec_bytes, s));
        }
        ADJ_CK(cudaMallocAsync((void **)&Fb, vec_bytes, s));
        ADJ_CK(cudaMallocAsync((void **)&seg_steps, sizeof(long long) * (every + 1), s));
        ADJ_CK(cudaMallocAsync((void **)&gacc, std::max<size_t>(sim->sell.entries, 1) * sizeof(float2), s));
        ADJ_CK(cudaMemsetAsync(gacc, 0, std::max<size_t>(sim->sell.entries, 1) * sizeof(float2), s));
        const uint64_t step0 = sim->steps;
        // forward rollout through the ordinary step, keeping checkpoints
        ADJ_CK(cudaMemcpyAsync(ckpt, sim->state[sim->cur], state_bytes, cudaMemcpyDeviceToDevice, s));
        for (uint64_t g = 0; g < n_seg; ++g) {
            const uint64_t len = std::min<uint64_t>(every, n_steps - g * every);
            for (uint64_t k = 0; k < len; ++k) {
                ADJ_CK(titan::enqueue_sim_step(sim, s, sim->cur, k > 0));
                sim->cur ^= 1;
                ++sim->steps;
            }
            ADJ_CK(cudaMemcpyAsync(ckpt + (g + 1) * nd, sim->state[sim->cur], state_bytes, cudaMemcpyDeviceToDevice, s));
        }
        // seed dJ/dx_T, dJ/dv_T in device order; gradients start at zero
        ADJ_CK(cudaMemsetAsync(xb[0], 0, vec_bytes, s));
        ADJ_CK(cudaMemsetAsync(vb[0], 0, vec_bytes, s));
        if (sim->n) {
            k_adj_seed<<<(sim->n + kT - 1) / kT, kT, 0, s>>>(seed_pos_dev, seed_vel_dev, sim->d_dev_of_caller,
                                                             sim->n, xb[0], vb[0]);
            ADJ_CK(cudaGetLastError());
        }

        for (uint64_t g = n_seg; g-- > 0;) {
            const uint64_t len = std::min<uint64_t>(every, n_steps - g * every);
            const long long first = (long long)(step0 + g * every);
            ADJ_CK(cudaMemcpyAsync(seg, ckpt + g * nd, state_bytes, cudaMemcpyDeviceToDevice, s));
            ADJ_CK(cudaMemcpyAsync(seg_steps, &first, sizeof(long long), cudaMemcpyHostToDevice, s));
            // the simulation's own step kernel (every CSR kernel gives bit-identical states)
            for (uint64_t k = 0; k < len; ++k)
                ADJ_CK(titan::enqueue_sim_step_io(sim, s, seg + k * nd, seg + (k + 1) * nd, seg_steps + k,
                                                  seg_steps + k + 1, k > 0));
            for (uint64_t k = len; k-- > 0;) {
                const MassState *X = seg + k * nd;
                if (sim->c.ground)
                    k_adj_mass<true><<<gm, kT, 0, s>>>(X, xb[cur], vb[cur], xb[cur ^ 1], vb[cur ^ 1], Fb, nd, sim->c);
                else
                    k_adj_mass<false><<<gm, kT, 0, s>>>(X, xb[cur], vb[cur], xb[cur ^ 1], vb[cur ^ 1], Fb, nd, sim->c);
                ADJ_CK(cudaGetLastError());
                const long long stepk = first + (long long)k;
                if (sim->has_c)
                    k_adj_spring<true><<<gm, kT, 0, s>>>(X, Fb, xb[cur ^ 1], vb[cur ^ 1], nd, sim->d_slice_off, sim->d_nbr,
                                                         sim->d_adj_spring, sim->d_kl, sim->d_act, sim->d_c, sim->c,
                                                         stepk, gacc);
                else
                    k_adj_spring<false><<<gm, kT, 0, s>>>(X, Fb, xb[cur ^ 1], vb[cur ^ 1], nd, sim->d_slice_off, sim->d_nbr,
                                                          sim->d_adj_spring, sim->d_kl, sim->d_act, sim->d_c, sim->c,
                                                          stepk, gacc);
                ADJ_CK(cudaGetLastError());
                cur ^= 1;
            }
        }
        if (S) {
            k_adj_gather<<<(S + kT - 1) / kT, kT, 0, s>>>(gacc, sim->d_adj_owner, S, grad_amp_dev, grad_phase_dev);
            ADJ_CK(cudaGetLastError());
        }
    }
done:
    if (ckpt) cudaFreeAsync(ckpt, s);
    if (seg) cudaFreeAsync(seg, s);
    for (int b = 0; b < 2; ++b) {
        if (xb[b]) cudaFreeAsync(xb[b], s);
        if (vb[b]) cudaFreeAsync(vb[b], s);
    }
    if (Fb) cudaFreeAsync(Fb, s);
    if (seg_steps) cudaFreeAsync(seg_steps, s);
    if (gacc) cudaFreeAsync(gacc, s);
    if (prev >= 0) cudaSetDevice(prev);
out:
    sim->busy.store(false);
    return st_;
}
