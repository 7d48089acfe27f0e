// step_cube2.cu -- the fused step with every spring inside a 256-mass cube
// read and evaluated once, forces exchanged through shared memory in a few
// direction groups (CSR kernel variant 10).
//
// One time step of Titan Sec. III-B (Eq. 1; the constraints, ground and
// friction of Sec. III-A) on a lattice whose springs join 26-neighbour cells,
// in the cube layout (layout.h: build_cube): one CTA per cube of 8 x 8 x 4
// cells, the cube's box table of states in shared memory, and per cube a
// dense "plus" stream [13 directions][256 masses] of each mass's +p spring
// plus a compact "ext" stream of the -p springs whose partner lies outside
// the cube.
//
// The 13 canonical directions are taken in G-direction groups.  Phase 1 of a
// group: every mass evaluates its +p spring of each direction of the group
// and writes (f, ux, uy, uz) - the force scalar and the unit axis seen from
// the mass - to shared memory; the threads also evaluate the group's ext
// springs, spread evenly over the CTA (each from the outside partner's side,
// so that it reads like the partner's +p spring).  After one barrier, phase 2:
// every mass adds, direction by direction, its +p term f u and its -p term
// f (-u) read from the in-cube partner's +p slot or from the ext slot - the
// order +p1, -p1, +p2, ... of its CSR row.  Seen from the two ends a spring
// has the same f bit for bit and exactly opposite axes, so every mass adds
// the same fused multiply-adds in the same order as the other CSR kernels:
// the trajectory is bit-identical to theirs.  Each spring costs one
// evaluation instead of two and the stream holds 8 bytes per spring end pair
// instead of per half-edge; the price is one barrier pair per group.
#include <algorithm>

#include "layout.h"
#include "physics.cuh"
#include "titan_internal.h"

namespace titan {
namespace {

constexpr int kC2Threads = 256;               // one CTA per cube of 256 cells (layout.h: kHaloBlock)
constexpr uint32_t kC2HoleSlot = 0xFFFF;      // own slot of a hole (layout.h: kBoxHole)
constexpr int kC2Dirs = 13;                   // canonical directions (layout.h: kCubePasses)

template <int G, bool HAS_C, bool HAS_ACT, bool GROUND, int MINB>
__global__ void __launch_bounds__(kC2Threads, MINB)
k_step_cube2(const MassState *__restrict__ in, MassState *__restrict__ out, uint32_t n,
             const uint32_t *__restrict__ cube_base, const uint4 *__restrict__ cube_meta,
             const uint32_t *__restrict__ ext_slot, const uint8_t *__restrict__ partner,
             const float2 *__restrict__ kl, const float *__restrict__ cc, const float2 *__restrict__ act,
             const uint16_t *__restrict__ own_slot, const uint32_t *__restrict__ ext_off,
             const uint32_t *__restrict__ ext_idx, const uint16_t *__restrict__ ext_tslot, uint32_t table_slots,
             uint32_t ext_cap, StepConst c, const long long *__restrict__ step_in, long long *__restrict__ step_out) {
    extern __shared__ float4 c2sm[];
    // the cube's pass metadata and the partner table, read many times per step, live in shared memory
    __shared__ uint4 smeta[kC2Dirs * (kC2Threads / 32)];
    __shared__ uint32_t sptab[kC2Dirs * kC2Threads / 4];
    float4 *tA = c2sm;
    float2 *tB = reinterpret_cast<float2 *>(c2sm + table_slots);
    float4 *store = reinterpret_cast<float4 *>(tB + table_slots);      // [G][256] plus terms, then ext terms
    float4 *ext_store = store + G * kC2Threads;
    const uint32_t zero_idx = G * kC2Threads + ext_cap;                 // a slot holding (0, 0, 0, 0)
    const uint8_t *ptab = reinterpret_cast<const uint8_t *>(sptab);
    const uint32_t b = blockIdx.x, tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const uint32_t i = b * kC2Threads + tid;
    long long step = 0;
    if (HAS_ACT) step = *step_in;
    if (b == 0 && tid == 0) *step_out = *step_in + 1;
    const uint32_t s_own = i < n ? own_slot[i] : kC2HoleSlot;
    const bool valid = s_own != kC2HoleSlot;
    const uint32_t base = __ldg(cube_base + b);
    const uint32_t ext0 = base + kC2Dirs * kC2Threads;
    const uint4 *mt = cube_meta + (size_t)b * kC2Dirs * (kC2Threads / 32);   // [dir][warp]
    if (tid < kC2Dirs * (kC2Threads / 32)) smeta[tid] = __ldg(mt + tid);
    for (uint32_t k = tid; k < kC2Dirs * kC2Threads / 4; k += kC2Threads)
        sptab[k] = __ldg(reinterpret_cast<const uint32_t *>(partner) + k);
    if (tid == 0) store[zero_idx] = make_float4(0.f, 0.f, 0.f, 0.f);

    // the first group's plus entries are requested before the table fill
    float2 pk[G], ps[G];
    float pc[G];
#pragma unroll
    for (int q = 0; q < G; ++q) {
        pk[q] = __ldcs(kl + base + q * kC2Threads + tid);
        if (HAS_C) pc[q] = __ldcs(cc + base + q * kC2Threads + tid);
        if (HAS_ACT) ps[q] = __ldcs(act + base + q * kC2Threads + tid);
    }
    float4 p = make_float4(0.f, 0.f, 0.f, 0.f), v = p;
    if (valid) {
        load_state(in + i, p, v);
        tA[s_own] = make_float4(p.x, p.y, p.z, v.x);
        tB[s_own] = make_float2(v.y, v.z);
    }
    const uint32_t h0 = __ldg(ext_off + b), h1 = __ldg(ext_off + b + 1);
    for (uint32_t h = h0 + tid; h < h1; h += kC2Threads) {
        float4 q, ww;
        load_state(in + __ldg(ext_idx + h), q, ww);
        const uint32_t s = __ldg(ext_tslot + h);
        tA[s] = make_float4(q.x, q.y, q.z, ww.x);
        tB[s] = make_float2(ww.y, ww.z);
    }
    __syncthreads();

    // the cube's ext entries, in direction order: the count from the last direction's last warp
    const uint4 m_last = smeta[kC2Dirs * (kC2Threads / 32) - 1];
    const uint32_t ext_total = m_last.z + __popc(m_last.y);
    const float clk = HAS_ACT ? actuation_clock(c, step) : 0.f;
    const uint32_t below = (1u << lane) - 1u;
    float fx = 0.f, fy = 0.f, fz = 0.f;
#pragma unroll 1
    for (int j0 = 0; j0 < kC2Dirs; j0 += G) {
        const int nd = min(G, kC2Dirs - j0);
        // ---- phase 1: this mass's +p springs of the group
#pragma unroll
        for (int q = 0; q < G; ++q) {
            if (q >= nd) break;
            const int j = j0 + q;
            const int32_t off = (int32_t)(int16_t)(smeta[j * (kC2Threads / 32)].w & 0xffffu);
            const float2 a = pk[q];
            float f = 0.f, ux = 0.f, uy = 0.f, uz = 0.f;
            if (valid && a.y >= 0.f) {                       // not padding (no +p spring)
                const uint32_t js = s_own + (uint32_t)off;
                const float4 qa = tA[js];
                const float2 qb = tB[js];
                const float L = HAS_ACT ? actuated_length(c, a.y, ps[q], clk) : a.y;
                spring_terms(p, v, qa, make_float4(qa.w, qb.x, qb.y, 0.f), a.x, L, HAS_C ? pc[q] : c.c_uniform,
                             f, ux, uy, uz);
            }
            store[q * kC2Threads + tid] = make_float4(f, ux, uy, uz);
        }
        // the group's ext springs, evaluated from the outside partner's side
        const uint32_t e_lo = smeta[j0 * (kC2Threads / 32)].z;
        const uint32_t e_hi = j0 + G < kC2Dirs ? smeta[(j0 + G) * (kC2Threads / 32)].z : ext_total;
        for (uint32_t e = e_lo + tid; e < e_hi; e += kC2Threads) {
            const uint32_t sl = __ldg(ext_slot + ext0 + e);
            const uint32_t so = sl & 0xffffu, sp = sl >> 16;          // receiving mass, outside partner
            const float2 a = __ldcs(kl + ext0 + e);
            const float cd = HAS_C ? __ldcs(cc + ext0 + e) : c.c_uniform;
            const float L = HAS_ACT ? actuated_length(c, a.y, __ldcs(act + ext0 + e), clk) : a.y;
            const float4 oa = tA[sp], ra = tA[so];
            const float2 ob = tB[sp], rb = tB[so];
            float f, ux, uy, uz;
            spring_terms(make_float4(oa.x, oa.y, oa.z, 0.f), make_float4(oa.w, ob.x, ob.y, 0.f), ra,
                         make_float4(ra.w, rb.x, rb.y, 0.f), a.x, L, cd, f, ux, uy, uz);
            ext_store[e - e_lo] = make_float4(f, ux, uy, uz);
        }
        __syncthreads();
        // the next group's plus entries are requested before this group's phase 2
        if (j0 + G < kC2Dirs) {
#pragma unroll
            for (int q = 0; q < G; ++q) {
                if (j0 + G + q >= kC2Dirs) break;
                pk[q] = __ldcs(kl + base + (j0 + G + q) * kC2Threads + tid);
                if (HAS_C) pc[q] = __ldcs(cc + base + (j0 + G + q) * kC2Threads + tid);
                if (HAS_ACT) ps[q] = __ldcs(act + base + (j0 + G + q) * kC2Threads + tid);
            }
        }
        // ---- phase 2: +p then -p of each direction, in row order
        if (valid) {
#pragma unroll
            for (int q = 0; q < G; ++q) {
                if (q >= nd) break;
                const int j = j0 + q;
                const float4 s = store[q * kC2Threads + tid];
                fx = fmaf(s.x, s.y, fx);
                fy = fmaf(s.x, s.z, fy);
                fz = fmaf(s.x, s.w, fz);
                const uint4 m = smeta[j * (kC2Threads / 32) + w];
                // -p partner in the cube: its +p slot; outside: the ext slot; none: the zero slot
                const uint32_t idx = ((m.x >> lane) & 1u) ? q * kC2Threads + ptab[j * kC2Threads + tid]
                                   : ((m.y >> lane) & 1u) ? G * kC2Threads + (m.z + __popc(m.y & below) - e_lo)
                                                          : zero_idx;
                const float4 g = store[idx];
                fx = fmaf(g.x, -g.y, fx);
                fy = fmaf(g.x, -g.z, fy);
                fz = fmaf(g.x, -g.w, fz);
            }
        }
        if (j0 + G < kC2Dirs) __syncthreads();        // the stores are refilled by the next group
    }
    if (!valid) return;
    integrate<GROUND>(p, v, fx, fy, fz, c, out + i);
}

template <int G, int MINB>
cudaError_t launch_c2(const MassState *in, MassState *out, uint32_t n, const Cube2View &v, const BoxView &h,
                      const StepConst &c, const long long *step_in, long long *step_out, cudaStream_t stream,
                      const cudaAccessPolicyWindow *l2win) {
    const bool hc = v.cube.c != nullptr, ha = v.cube.act != nullptr, gr = c.ground != 0;
    const unsigned g = n / kC2Threads;
    const size_t bytes = cube2_smem_bytes(h.table_slots, G, v.ext_cap);
#define TITAN_C2(HC, HA, GR)                                                                     \
    do {                                                                                         \
        auto kern = k_step_cube2<G, HC, HA, GR, MINB>;                                           \
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes); \
        if (e != cudaSuccess) return e;                                                          \
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,           \
                                 (int)cudaSharedmemCarveoutMaxShared);                            \
        if (e != cudaSuccess) return e;                                                          \
        cudaLaunchConfig_t cfg = {};                                                             \
        cfg.gridDim = dim3(g);                                                                   \
        cfg.blockDim = dim3(kC2Threads);                                                         \
        cfg.dynamicSmemBytes = bytes;                                                            \
        cfg.stream = stream;                                                                     \
        cudaLaunchAttribute attr[1];                                                             \
        if (l2win) {                                                                             \
            attr[0].id = cudaLaunchAttributeAccessPolicyWindow;                                  \
            attr[0].val.accessPolicyWindow = *l2win;                                             \
            cfg.attrs = attr;                                                                    \
            cfg.numAttrs = 1;                                                                    \
        }                                                                                        \
        e = cudaLaunchKernelEx(&cfg, kern, in, out, n, v.cube.base, v.cube.meta, v.ext_slot, v.partner, \
                               v.cube.kl, v.cube.c, v.cube.act, h.own_slot, h.ext_off, h.ext_idx, h.ext_slot, \
                               h.table_slots, v.ext_cap, c, step_in, step_out);                 \
        if (e != cudaSuccess) return e;                                                          \
    } while (0)
    if (hc) {
        if (ha) { if (gr) TITAN_C2(true, true, true); else TITAN_C2(true, true, false); }
        else    { if (gr) TITAN_C2(true, false, true); else TITAN_C2(true, false, false); }
    } else {
        if (ha) { if (gr) TITAN_C2(false, true, true); else TITAN_C2(false, true, false); }
        else    { if (gr) TITAN_C2(false, false, true); else TITAN_C2(false, false, false); }
    }
#undef TITAN_C2
    return cudaGetLastError();
}

}  // namespace

size_t cube2_smem_bytes(uint32_t table_slots, int group, uint32_t ext_cap) {
    return (size_t)table_slots * (sizeof(float4) + sizeof(float2)) +
           ((size_t)group * kC2Threads + ext_cap + 1) * sizeof(float4);
}

int cube2_group(int config) { return config == 2 ? 7 : config == 3 ? 13 : 4; }

cudaError_t launch_step_cube2(const MassState *in, MassState *out, uint32_t n, const Cube2View &v, const BoxView &h,
                              int config, const StepConst &c, const long long *step_in, long long *step_out,
                              cudaStream_t stream, const cudaAccessPolicyWindow *l2win) {
    if (n % kC2Threads || (h.table_slots & 1)) return cudaErrorInvalidValue;
    switch (config) {
        case 2: return launch_c2<7, 4>(in, out, n, v, h, c, step_in, step_out, stream, l2win);
        case 3: return launch_c2<13, 2>(in, out, n, v, h, c, step_in, step_out, stream, l2win);
        default: return launch_c2<4, 4>(in, out, n, v, h, c, step_in, step_out, stream, l2win);
    }
}

}  // namespace titan
