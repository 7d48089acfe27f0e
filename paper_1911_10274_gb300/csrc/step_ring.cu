// step_ring.cu -- the grid-box step kernel with its half-edge stream fed
// through a per-warp ring in shared memory (CSR kernel variant 9).
//
// One time step exactly as k_step_box computes it (Titan Sec. III-B, Eq. 1;
// Sec. III-A constraints, ground and friction): one CTA per 256-mass block of
// the grid order, the block's box table of states in shared memory, each
// thread summing its offset-aligned SELL row in the fixed row order, so the
// result is bit-identical to every other CSR kernel.  What changes is how the
// {k, L0} stream (plus c and actuation when present) reaches the threads.
// k_step_box loads each column pair one iteration ahead into registers: at six
// CTAs per SM that keeps about 25 KB per SM in flight, while the DRAM latency
// at the measured bandwidth needs roughly twice that.  Here lane 0 of each
// warp keeps RING stages of SC columns of its slice in flight as 1-D bulk
// copies into a per-warp ring (one mbarrier per stage), issuing the first
// RING before the table fill and refilling each stage as soon as the warp has
// consumed it; the threads read the stream from shared memory.
#include <algorithm>

#include "physics.cuh"
#include "ptx.cuh"
#include "titan_internal.h"

namespace titan {
namespace {

constexpr int kRingThreads = 256;            // one CTA per 256-mass block (layout.h: kHaloBlock)
constexpr uint32_t kRingHoleSlot = 0xFFFF;   // own slot of a hole (layout.h: kBoxHole)

template <bool HAS_C, bool HAS_ACT>
constexpr int ring_col_bytes() { return 32 * (8 + (HAS_ACT ? 8 : 0) + (HAS_C ? 4 : 0)); }

// Arms `bar` for `cols` columns starting at column col0 of the slice at entry
// e0 and issues their bulk copies into `stage`, laid out as
// [kl SC x 32 float2][act SC x 32 float2][c SC x 32 float].
template <int SC, bool HAS_C, bool HAS_ACT>
__device__ __forceinline__ void ring_issue(unsigned char *stage, uint64_t *bar, const float2 *kl, const float *cc,
                                           const float2 *act, uint32_t e0, uint32_t col0, uint32_t cols) {
    const uint32_t ne = cols * 32, e = e0 + col0 * 32;
    ptx::mbar_arrive_expect_tx(bar, ne * (8 + (HAS_ACT ? 8 : 0) + (HAS_C ? 4 : 0)));
    ptx::bulk_g2s(stage, kl + e, ne * 8, bar);
    if (HAS_ACT) ptx::bulk_g2s(stage + SC * 32 * 8, act + e, ne * 8, bar);
    if (HAS_C) ptx::bulk_g2s(stage + SC * 32 * (HAS_ACT ? 16 : 8), cc + e, ne * 4, bar);
}

// Holes stay in the loop (lane 0 must keep issuing) but evaluate nothing.
// Every stage wait is bounded by spin_limit polls; on expiry the warp records
// the error in *err, waits (bounded) for its copies in flight and leaves its
// masses unwritten.
template <bool HAS_C, bool HAS_ACT, bool GROUND, int RING, int SC, int MINB>
__global__ void __launch_bounds__(kRingThreads, MINB)
k_step_box_ring(const MassState *__restrict__ in, MassState *__restrict__ out, uint32_t n,
                const uint32_t *__restrict__ slice_off, const uint32_t *__restrict__ col_off2,
                const float2 *__restrict__ kl, const float *__restrict__ cc, const float2 *__restrict__ act,
                const uint16_t *__restrict__ own_slot, const uint32_t *__restrict__ ext_off,
                const uint32_t *__restrict__ ext_idx, const uint16_t *__restrict__ ext_slot, uint32_t table_slots,
                StepConst c, const long long *__restrict__ step_in, long long *__restrict__ step_out,
                uint32_t spin_limit, int *__restrict__ err) {
    constexpr uint32_t FULL = 0xffffffffu;
    constexpr int STAGE = SC * ring_col_bytes<HAS_C, HAS_ACT>();
    extern __shared__ float4 rtab[];
    __shared__ uint64_t bars[kRingThreads / 32][RING];
    float4 *tA = rtab;
    float2 *tB = reinterpret_cast<float2 *>(rtab + table_slots);       // table_slots even: ring 16-B aligned
    const uint32_t b = blockIdx.x, tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const uint32_t i = b * kRingThreads + tid, sl = i >> 5;
    const uint32_t n_slices = (n + 31) >> 5;
    unsigned char *ring = reinterpret_cast<unsigned char *>(tB + table_slots) + (size_t)w * RING * STAGE;
    uint64_t *bar = bars[w];

    long long step = 0;
    if (HAS_ACT) step = *step_in;
    if (b == 0 && tid == 0) *step_out = *step_in + 1;

    const bool warp_live = sl < n_slices;                    // warp-uniform
    uint32_t e0 = 0, width = 0;
    if (warp_live) {
        e0 = __ldg(slice_off + sl);
        width = (__ldg(slice_off + sl + 1) - e0) >> 5;      // even
    }
    const uint32_t n_chunks = (width + SC - 1) / SC;
    if (lane == 0 && n_chunks) {
        for (int r = 0; r < RING; ++r) ptx::mbar_init(&bar[r], 1);
        ptx::fence_mbar_init();
        for (uint32_t q = 0; q < (uint32_t)RING && q < n_chunks; ++q)
            ring_issue<SC, HAS_C, HAS_ACT>(ring + q * STAGE, &bar[q], kl, cc, act, e0, q * SC,
                                           min((uint32_t)SC, width - q * SC));
    }
    const uint32_t s_own = i < n ? own_slot[i] : kRingHoleSlot;
    const bool valid = s_own != kRingHoleSlot;
    float4 p = make_float4(0.f, 0.f, 0.f, 0.f), v = p;
    const uint32_t *co = col_off2 + (e0 >> 6);      // a pair of int16 column offsets per word
    uint32_t no = 0;
    if (n_chunks) no = __ldg(co);
    if (valid) {
        load_state(in + i, p, v);
        tA[s_own] = make_float4(p.x, p.y, p.z, v.x);
        tB[s_own] = make_float2(v.y, v.z);
    }
    const uint32_t h0 = __ldg(ext_off + b), h1 = __ldg(ext_off + b + 1);
    for (uint32_t h = h0 + tid; h < h1; h += kRingThreads) {
        float4 q, ww;
        load_state(in + __ldg(ext_idx + h), q, ww);
        const uint32_t s = __ldg(ext_slot + h);
        tA[s] = make_float4(q.x, q.y, q.z, ww.x);
        tB[s] = make_float2(ww.y, ww.z);
    }
    __syncthreads();                    // also publishes the mbarrier initialisation
    if (!warp_live) return;

    const float ph = HAS_ACT ? actuation_clock(c, step) : 0.f;
    const uint32_t n_pairs = width >> 1;
    float fx = 0.f, fy = 0.f, fz = 0.f;
    uint32_t r = 0, parity = 0, t = 0;              // ring slot and phase of chunk q; next column pair
    for (uint32_t q = 0; q < n_chunks; ++q) {
        bool done = false;
        for (uint32_t it = 0; it < spin_limit; ++it) {
            done = ptx::mbar_try_wait(&bar[r], parity);
            if (__all_sync(FULL, done)) break;
        }
        if (!__all_sync(FULL, done)) {
            if (lane == 0) {            // drain every chunk issued and not yet consumed
                atomicExch(err, 1);
                const uint32_t issued = min(n_chunks, q + (uint32_t)RING);
                for (uint32_t x = q; x < issued; ++x)
                    ptx::mbar_wait_bounded(&bar[x % RING], (x / RING) & 1u, spin_limit);
            }
            __syncwarp();
            return;
        }
        const unsigned char *stg = ring + r * STAGE;
        const float2 *s_kl = reinterpret_cast<const float2 *>(stg);
        const float2 *s_act = reinterpret_cast<const float2 *>(stg + SC * 32 * 8);
        const float *s_c = reinterpret_cast<const float *>(stg + SC * 32 * (HAS_ACT ? 16 : 8));
        const uint32_t cols = min((uint32_t)SC, width - q * SC);      // even
#pragma unroll
        for (uint32_t k = 0; k < (uint32_t)SC; k += 2) {
            if (k >= cols) break;
            const uint32_t o = no;
            ++t;
            if (t < n_pairs) no = __ldg(co + t);
            const float2 a0 = s_kl[k * 32 + lane], a1 = s_kl[k * 32 + 32 + lane];
            float c0 = c.c_uniform, c1 = c.c_uniform;
            if (HAS_C) { c0 = s_c[k * 32 + lane]; c1 = s_c[k * 32 + 32 + lane]; }
            float L0 = a0.y, L1 = a1.y;
            if (HAS_ACT) {
                L0 = actuated_length(c, a0.y, s_act[k * 32 + lane], ph);
                L1 = actuated_length(c, a1.y, s_act[k * 32 + 32 + lane], ph);
            }
            const uint32_t j0 = s_own + (uint32_t)(int32_t)(int16_t)(o & 0xffffu);
            const uint32_t j1 = s_own + (uint32_t)(int32_t)(int16_t)(o >> 16);
            if (valid && a0.y >= 0.f) {          // not padding (padding: rest length kPadRest < 0)
                const float4 qa = tA[j0];
                const float2 qb = tB[j0];
                spring_force(p, v, qa, make_float4(qa.w, qb.x, qb.y, 0.f), a0.x, L0, c0, fx, fy, fz);
            }
            if (valid && a1.y >= 0.f) {
                const float4 qa = tA[j1];
                const float2 qb = tB[j1];
                spring_force(p, v, qa, make_float4(qa.w, qb.x, qb.y, 0.f), a1.x, L1, c1, fx, fy, fz);
            }
        }
        // every lane has consumed this stage: its values fed the forces above
        __syncwarp();
        if (lane == 0 && q + RING < n_chunks)
            ring_issue<SC, HAS_C, HAS_ACT>(ring + r * STAGE, &bar[r], kl, cc, act, e0, (q + RING) * SC,
                                           min((uint32_t)SC, width - (q + RING) * SC));
        if (++r == (uint32_t)RING) { r = 0; parity ^= 1u; }
    }
    if (!valid) return;
    integrate<GROUND>(p, v, fx, fy, fz, c, out + i);
}

template <int RING, int SC, int MINB>
cudaError_t launch_ring(const MassState *in, MassState *out, uint32_t n, const SellView &v, const BoxView &h,
                        const StepConst &c, const long long *step_in, long long *step_out, cudaStream_t stream,
                        const cudaAccessPolicyWindow *l2win) {
    const bool hc = v.c != nullptr, ha = v.act != nullptr, gr = c.ground != 0;
    const unsigned g = n ? (n + kRingThreads - 1) / kRingThreads : 1;
    const size_t bytes = box_ring_smem_bytes(h.table_slots, RING * SC, hc, ha);
#define TITAN_RING(HC, HA, GR)                                                                   \
    do {                                                                                         \
        auto kern = k_step_box_ring<HC, HA, GR, RING, SC, MINB>;                                 \
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes); \
        if (e != cudaSuccess) return e;                                                          \
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,           \
                                 (int)cudaSharedmemCarveoutMaxShared);                            \
        if (e != cudaSuccess) return e;                                                          \
        cudaLaunchConfig_t cfg = {};                                                             \
        cfg.gridDim = dim3(g);                                                                   \
        cfg.blockDim = dim3(kRingThreads);                                                       \
        cfg.dynamicSmemBytes = bytes;                                                            \
        cfg.stream = stream;                                                                     \
        cudaLaunchAttribute attr[1];                                                             \
        if (l2win) {                                                                             \
            attr[0].id = cudaLaunchAttributeAccessPolicyWindow;                                  \
            attr[0].val.accessPolicyWindow = *l2win;                                             \
            cfg.attrs = attr;                                                                    \
            cfg.numAttrs = 1;                                                                    \
        }                                                                                        \
        e = cudaLaunchKernelEx(&cfg, kern, in, out, n, v.slice_off,                              \
                               reinterpret_cast<const uint32_t *>(h.col_off), v.kl, v.c, v.act, h.own_slot, \
                               h.ext_off, h.ext_idx, h.ext_slot, h.table_slots, c, step_in, step_out, \
                               v.spin_limit, v.err);                                             \
        if (e != cudaSuccess) return e;                                                          \
    } while (0)
    if (hc) {
        if (ha) { if (gr) TITAN_RING(true, true, true); else TITAN_RING(true, true, false); }
        else    { if (gr) TITAN_RING(true, false, true); else TITAN_RING(true, false, false); }
    } else {
        if (ha) { if (gr) TITAN_RING(false, true, true); else TITAN_RING(false, true, false); }
        else    { if (gr) TITAN_RING(false, false, true); else TITAN_RING(false, false, false); }
    }
#undef TITAN_RING
    return cudaGetLastError();
}

}  // namespace

size_t box_ring_smem_bytes(uint32_t table_slots, uint32_t ring_cols, bool has_c, bool has_act) {
    return (size_t)table_slots * (sizeof(float4) + sizeof(float2)) +
           (size_t)(kRingThreads / 32) * ring_cols * 32 * (8 + (has_c ? 4 : 0) + (has_act ? 8 : 0));
}

int box_ring_stages(int config) { return config == 2 ? 6 : config == 3 ? 3 : 4; }
int box_ring_cols(int config) { return config == 3 ? 4 : 2; }

cudaError_t launch_step_box_ring(const MassState *in, MassState *out, uint32_t n, const SellView &v, const BoxView &h,
                                 int config, const StepConst &c, const long long *step_in, long long *step_out,
                                 cudaStream_t stream, const cudaAccessPolicyWindow *l2win) {
    if (reinterpret_cast<uintptr_t>(h.col_off) & 3) return cudaErrorInvalidValue;
    if (h.table_slots & 1) return cudaErrorInvalidValue;      // the ring must start 16-byte aligned
    switch (config) {
        case 2: return launch_ring<6, 2, 5>(in, out, n, v, h, c, step_in, step_out, stream, l2win);
        case 3: return launch_ring<3, 4, 5>(in, out, n, v, h, c, step_in, step_out, stream, l2win);
        default: return launch_ring<4, 2, 6>(in, out, n, v, h, c, step_in, step_out, stream, l2win);
    }
}

}  // namespace titan
