// physics.cuh -- the arithmetic of one spring and one mass, shared by every
// kernel of the GPU path (Titan Sec. III-B, Eq. 1; Sec. III-A constraints).
#pragma once

#include "titan_internal.h"

namespace titan {

// One 256-bit read-only load of a mass's whole 32-byte state (sm_100+ vector
// width): one L1 request per neighbour gather instead of two.
__device__ __forceinline__ void load_state(const MassState *m, float4 &p, float4 &v) {
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(p.x), "=f"(p.y), "=f"(p.z), "=f"(p.w), "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
        : "l"(m));
}

// The same load through L2 only (.cg, never served from L1), ordered after
// every earlier memory operation of the thread (volatile, with a memory
// clobber): for a kernel whose CTAs start before the previous step has
// finished writing the state (a programmatic dependent launch), issued only
// after waiting for that step.
__device__ __forceinline__ void load_state_after_wait(const MassState *m, float4 &p, float4 &v) {
    asm volatile("ld.global.cg.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=f"(p.x), "=f"(p.y), "=f"(p.z), "=f"(p.w), "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(m)
                 : "memory");
}

// Phase of the actuation clock at step `step`: 2 pi f t mod 2 pi with
// t = step dt.  The turns step x (f dt) are formed modulo 1 exactly in 64-bit
// fixed point (integer products wrap modulo 2^64) and their top 24 bits give
// the phase, so long runs keep full FP32 phase accuracy without FP64.
__device__ __forceinline__ float clock_phase(const StepConst &c, long long step) {
    const unsigned long long fr = (unsigned long long)step * c.act_turns;
    return __fmul_rn((float)(fr >> 40), 3.74507028e-7f);      // 2 pi / 2^24
}

// Per-thread actuation clock for step `step`: mode 1 the phase 2 pi f t mod
// 2 pi, mode 2 (the worm of Sec. V-B, Eq. 3) the time t mod t_p (the same
// fixed-point turns, of dt / t_p).
__device__ __forceinline__ float actuation_clock(const StepConst &c, long long step) {
    if (c.act_mode == 2) {
        const unsigned long long fr = (unsigned long long)step * c.worm_turns;
        return __fmul_rn((float)(fr >> 40), c.worm_unit);
    }
    return clock_phase(c, step);
}

// Rest length of an actuated spring: a = (A, phi) in mode 1,
// (c, t_o mod t_p) in mode 2 where tau = (t - t_o) mod t_p (Eqs. 3-4).
__device__ __forceinline__ float actuated_length(const StepConst &c, float L0, float2 a, float clk) {
    if (c.act_mode == 2) {
        float tau = clk - a.y;
        if (tau < 0.f) tau += (float)c.worm_period;
        return L0 * (1.f + a.x * sinf(c.worm_omega * tau));
    }
    return L0 * (1.f + a.x * sinf(clk + a.y));
}

// The two factors of the force on the mass at (p, v) from one spring to the
// mass at (q, w): the scalar f = k (l - L) + c (w - v) . u and the unit axis u
// (the force is f u).  A zero-length spring has u = 0.  Seen from the other
// end, d, u and the relative velocity change sign exactly and f is
// bit-identical, so one end's (f, u) serves the other as (f, -u).
//
// Every rounding is written out (no product-sum is left for the compiler to
// fuse or not): l2 = fma(dz, dz, fma(dy, dy, dx dx)), rate = fma(dvz, uz,
// fma(dvy, uy, dvx ux)), f = fma(k, l - L, c rate): every kernel computes the
// same bits, whatever the compiler would have fused (measured 2 % faster on
// the 1M-mass lattice than the contracted form).
__device__ __forceinline__ void spring_terms(const float4 &p, const float4 &v, const float4 &q, const float4 &w,
                                             float k, float L, float c, float &f, float &ux, float &uy,
                                             float &uz) {
    const float dx = __fsub_rn(q.x, p.x), dy = __fsub_rn(q.y, p.y), dz = __fsub_rn(q.z, p.z);
    const float l2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
    // one reciprocal square root gives both 1/l and l = l2 / l; its error
    // (a few ulp) is below the rounding of the FP32 positions themselves
    const float inv = l2 > 0.f ? rsqrtf(l2) : 0.f;
    const float l = __fmul_rn(l2, inv);
    ux = __fmul_rn(dx, inv);
    uy = __fmul_rn(dy, inv);
    uz = __fmul_rn(dz, inv);
    const float dvx = __fsub_rn(w.x, v.x), dvy = __fsub_rn(w.y, v.y), dvz = __fsub_rn(w.z, v.z);
    const float rate = __fmaf_rn(dvz, uz, __fmaf_rn(dvy, uy, __fmul_rn(dvx, ux)));
    f = __fmaf_rn(k, __fsub_rn(l, L), __fmul_rn(c, rate));
}

// Force on the mass at (p, v) from one spring to the mass at (q, w):
// accumulates f u into (fx, fy, fz), one fused multiply-add per component.
// A zero-length spring contributes 0.
__device__ __forceinline__ void spring_force(const float4 &p, const float4 &v, const float4 &q,
                                             const float4 &w, float k, float L, float c,
                                             float &fx, float &fy, float &fz) {
    float f, ux, uy, uz;
    spring_terms(p, v, q, w, k, L, c, f, ux, uy, uz);
    fx = __fmaf_rn(f, ux, fx);
    fy = __fmaf_rn(f, uy, fy);
    fz = __fmaf_rn(f, uz, fz);
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

}  // namespace titan
