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
#include <algorithm>
#include <atomic>

#include "physics.cuh"
#include "ptx.cuh"
#include "titan_internal.h"

namespace titan {
namespace {

constexpr int kThreads = 256;

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
    const float ph = HAS_ACT ? actuation_clock(c, step) : 0.f;

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
            L0 = actuated_length(c, a0.y, s0, ph);
            L1 = actuated_length(c, a1.y, s1, ph);
        }
        float4 q0, w0, q1, w1;
        load_state(in + j0, q0, w0);
        load_state(in + j1, q1, w1);
        spring_force(p, v, q0, w0, a0.x, L0, c0, fx, fy, fz);
        spring_force(p, v, q1, w1, a1.x, L1, c1, fx, fy, fz);
    }
    integrate<GROUND>(p, v, fx, fy, fz, c, out + i);
}

// K1, default form.  One thread per mass, one warp per SELL slice.  At entry
// lane 0 asks the TMA engine to prefetch the slice's whole half-edge stream
// (all columns of every array) into L2 in one bulk request per array, so the
// DRAM latency is paid once per slice instead of once per column; the loop
// then loads each column one iteration ahead of its use (register double
// buffering), overlapping the L2 latency of the stream with the neighbour
// gathers of the current column.
template <bool HAS_C, bool HAS_ACT, bool GROUND>
__global__ void __launch_bounds__(kThreads)
k_step_sell_pf(const MassState *__restrict__ in, MassState *__restrict__ out, uint32_t n,
               const uint32_t *__restrict__ slice_off, const uint32_t *__restrict__ nbr,
               const float2 *__restrict__ kl, const float *__restrict__ cc,
               const float2 *__restrict__ act, StepConst c, const long long *__restrict__ step_in,
               long long *__restrict__ step_out) {
    const uint32_t i = blockIdx.x * kThreads + threadIdx.x;
    long long step = 0;
    if (HAS_ACT) step = *step_in;
    if (blockIdx.x == 0 && threadIdx.x == 0) *step_out = *step_in + 1;
    const uint32_t sl = i >> 5, lane = i & 31;
    const uint32_t n_slices = (n + 31) >> 5;
    if (sl >= n_slices) return;
    const uint32_t e0 = __ldg(slice_off + sl);
    const uint32_t width = (__ldg(slice_off + sl + 1) - e0) >> 5;   // even, warp-uniform
    if (lane == 0 && width) {
        const uint32_t ne = width * 32;
        ptx::bulk_prefetch_l2(kl + e0, ne * 8);
        ptx::bulk_prefetch_l2(nbr + e0, ne * 4);
        if (HAS_C) ptx::bulk_prefetch_l2(cc + e0, ne * 4);
        if (HAS_ACT) ptx::bulk_prefetch_l2(act + e0, ne * 8);
    }
    if (i >= n) return;

    const float4 p = __ldg(&in[i].p);
    const float4 v = __ldg(&in[i].v);
    const float ph = HAS_ACT ? actuation_clock(c, step) : 0.f;
    float fx = 0.f, fy = 0.f, fz = 0.f;
    if (width) {
        uint32_t e = e0 + lane;
        uint32_t nj0 = __ldcs(nbr + e), nj1 = __ldcs(nbr + e + 32);
        float2 na0 = __ldcs(kl + e), na1 = __ldcs(kl + e + 32);
        float nc0 = c.c_uniform, nc1 = c.c_uniform;
        float2 ns0 = make_float2(0.f, 0.f), ns1 = ns0;
        if (HAS_C) { nc0 = __ldcs(cc + e); nc1 = __ldcs(cc + e + 32); }
        if (HAS_ACT) { ns0 = __ldcs(act + e); ns1 = __ldcs(act + e + 32); }
        for (uint32_t t = 0; t < width; t += 2) {
            const uint32_t j0 = nj0, j1 = nj1;
            const float2 a0 = na0, a1 = na1;
            const float c0 = nc0, c1 = nc1;
            const float2 s0 = ns0, s1 = ns1;
            float4 q0, w0, q1, w1;
            load_state(in + j0, q0, w0);
            load_state(in + j1, q1, w1);
            if (t + 2 < width) {
                e += 64;
                nj0 = __ldcs(nbr + e); nj1 = __ldcs(nbr + e + 32);
                na0 = __ldcs(kl + e); na1 = __ldcs(kl + e + 32);
                if (HAS_C) { nc0 = __ldcs(cc + e); nc1 = __ldcs(cc + e + 32); }
                if (HAS_ACT) { ns0 = __ldcs(act + e); ns1 = __ldcs(act + e + 32); }
            }
            float L0 = a0.y, L1 = a1.y;
            if (HAS_ACT) {
                L0 = actuated_length(c, a0.y, s0, ph);
                L1 = actuated_length(c, a1.y, s1, ph);
            }
            spring_force(p, v, q0, w0, a0.x, L0, c0, fx, fy, fz);
            spring_force(p, v, q1, w1, a1.x, L1, c1, fx, fy, fz);
        }
    }
    integrate<GROUND>(p, v, fx, fy, fz, c, out + i);
}

// K1, halo form (the default when the neighbourhood tables fit).  One CTA
// per block of kHaloThreads consecutive device masses.  The CTA first copies
// the state of every mass its half-edges touch - its own masses and the
// external halo - into a shared-memory table (a float4 (x, y, z, vx) and a
// float2 (vy, vz) per slot), then each thread runs its SELL row reading
// neighbours from that table through 16-bit slots.  Each neighbour state is
// fetched from global memory once per block instead of once per half-edge, and
// the slots are coloured so that a quarter-warp's 16-byte and a half-warp's
// 8-byte table reads fall in distinct banks.  The half-edge stream (u16 slot
// + {k, L0}, 10 bytes) is brought into L2 by TMA bulk prefetches: of the
// warp's own slice (ahead = 0, the default: prefetching further ahead was
// measured to lose lines to L2 eviction), or `ahead` blocks in advance.
constexpr int kHaloThreads = 256;

// A neighbour or own state read by a step kernel.  Launched as a programmatic
// dependent (OVERLAP), the kernel's CTAs may start while the previous step is
// still writing the state: after waiting for it they read through L2 only,
// since a line of that buffer left in L1 by an earlier step can be stale
// (measured: with cached loads the trajectory drifted by centimetres).
template <bool OVERLAP>
__device__ __forceinline__ void read_state(const MassState *m, float4 &p, float4 &v) {
    if (OVERLAP) load_state_after_wait(m, p, v);
    else load_state(m, p, v);
}

// The step counter the previous step wrote, read the same way (through L2
// only after the wait: neighbouring counters share a cache line, so an L1 copy
// of it can be a step or more out of date).
template <bool OVERLAP>
__device__ __forceinline__ long long read_step(const long long *p) {
    return OVERLAP ? __ldcg(p) : *p;
}
constexpr uint32_t kBoxHoleSlot = 0xFFFF;   // own slot of a hole (layout.h: kBoxHole)
constexpr int kHaloMinBlocks = 6;      // resident CTAs per SM of the coloured-table halo kernel
constexpr int kBoxMinBlocks = 6;       // resident CTAs per SM the register budget is sized for

template <bool HAS_C, bool HAS_ACT>
__device__ __forceinline__ void prefetch_slice(const uint32_t *slice_off, uint32_t sl, const uint16_t *nslot,
                                               const float2 *kl, const float *cc, const float2 *act) {
    const uint32_t e0 = __ldg(slice_off + sl);
    const uint32_t ne = __ldg(slice_off + sl + 1) - e0;
    if (!ne) return;
    ptx::bulk_prefetch_l2(kl + e0, ne * 8);
    ptx::bulk_prefetch_l2(nslot + e0, ne * 2);
    if (HAS_C) ptx::bulk_prefetch_l2(cc + e0, ne * 4);
    if (HAS_ACT) ptx::bulk_prefetch_l2(act + e0, ne * 8);
}

template <bool HAS_C, bool HAS_ACT, bool GROUND, bool OVERLAP>
__global__ void __launch_bounds__(kHaloThreads, kHaloMinBlocks)
k_step_halo(const MassState *__restrict__ in, MassState *__restrict__ out, uint32_t n,
            const uint32_t *__restrict__ slice_off, const uint16_t *__restrict__ nslot,
            const float2 *__restrict__ kl, const float *__restrict__ cc,
            const float2 *__restrict__ act, const uint16_t *__restrict__ own_slot,
            const uint32_t *__restrict__ ext_off, const uint32_t *__restrict__ ext_idx,
            const uint16_t *__restrict__ ext_slot, uint32_t table_slots, uint32_t ahead, StepConst c,
            const long long *__restrict__ step_in, long long *__restrict__ step_out) {
    extern __shared__ float4 tab4[];
    float4 *tA = tab4;
    float2 *tB = reinterpret_cast<float2 *>(tab4 + table_slots);
    const uint32_t b = blockIdx.x, tid = threadIdx.x;
    const uint32_t i = b * kHaloThreads + tid;
    const uint32_t lane = tid & 31, sl = i >> 5, w = tid >> 5;
    const uint32_t n_slices = (n + 31) >> 5;
    if (OVERLAP) ptx::grid_dep_launch();    // the next step's CTAs may take SM slots this tail frees
    const bool valid = i < n;

    if (lane == 0) {
        if (b < ahead || ahead == 0) {
            if (sl < n_slices) prefetch_slice<HAS_C, HAS_ACT>(slice_off, sl, nslot, kl, cc, act);
        }
        const uint32_t sl_next = (b + ahead) * (kHaloThreads / 32) + w;
        if (ahead && sl_next < n_slices) prefetch_slice<HAS_C, HAS_ACT>(slice_off, sl_next, nslot, kl, cc, act);
    }
    uint32_t e0 = 0, width = 0;
    float4 p = make_float4(0.f, 0.f, 0.f, 0.f), v = p;
    if (valid) {
        e0 = __ldg(slice_off + sl);
        width = (__ldg(slice_off + sl + 1) - e0) >> 5;
    }
    // the state and the step counter are written by the previous step
    if (OVERLAP) ptx::grid_dep_wait();
    long long step = 0;
    if (HAS_ACT || (b == 0 && tid == 0)) step = read_step<OVERLAP>(step_in);
    if (b == 0 && tid == 0) *step_out = step + 1;
    if (valid) {
        read_state<OVERLAP>(in + i, p, v);
        const uint32_t s = own_slot[i];
        tA[s] = make_float4(p.x, p.y, p.z, v.x);
        tB[s] = make_float2(v.y, v.z);
    }
    const uint32_t h0 = __ldg(ext_off + b), h1 = __ldg(ext_off + b + 1);
    for (uint32_t h = h0 + tid; h < h1; h += kHaloThreads) {
        float4 q, ww;
        read_state<OVERLAP>(in + __ldg(ext_idx + h), q, ww);
        const uint32_t s = __ldg(ext_slot + h);
        tA[s] = make_float4(q.x, q.y, q.z, ww.x);
        tB[s] = make_float2(ww.y, ww.z);
    }
    __syncthreads();
    if (!valid) return;

    const float ph = HAS_ACT ? actuation_clock(c, step) : 0.f;
    float fx = 0.f, fy = 0.f, fz = 0.f;
    if (width) {
        uint32_t e = e0 + lane;
        uint32_t n0 = __ldcs(nslot + e), n1 = __ldcs(nslot + e + 32);
        float2 na0 = __ldcs(kl + e), na1 = __ldcs(kl + e + 32);
        float nc0 = c.c_uniform, nc1 = c.c_uniform;
        float2 ns0 = make_float2(0.f, 0.f), ns1 = ns0;
        if (HAS_C) { nc0 = __ldcs(cc + e); nc1 = __ldcs(cc + e + 32); }
        if (HAS_ACT) { ns0 = __ldcs(act + e); ns1 = __ldcs(act + e + 32); }
        for (uint32_t t = 0; t < width; t += 2) {
            const uint32_t j0 = n0, j1 = n1;
            const float2 a0 = na0, a1 = na1;
            const float c0 = nc0, c1 = nc1;
            const float2 s0 = ns0, s1 = ns1;
            if (t + 2 < width) {
                e += 64;
                n0 = __ldcs(nslot + e); n1 = __ldcs(nslot + e + 32);
                na0 = __ldcs(kl + e); na1 = __ldcs(kl + e + 32);
                if (HAS_C) { nc0 = __ldcs(cc + e); nc1 = __ldcs(cc + e + 32); }
                if (HAS_ACT) { ns0 = __ldcs(act + e); ns1 = __ldcs(act + e + 32); }
            }
            const float4 qa0 = tA[j0], qa1 = tA[j1];
            const float2 qb0 = tB[j0], qb1 = tB[j1];
            float L0 = a0.y, L1 = a1.y;
            if (HAS_ACT) {
                L0 = actuated_length(c, a0.y, s0, ph);
                L1 = actuated_length(c, a1.y, s1, ph);
            }
            spring_force(p, v, qa0, make_float4(qa0.w, qb0.x, qb0.y, 0.f), a0.x, L0, c0, fx, fy, fz);
            spring_force(p, v, qa1, make_float4(qa1.w, qb1.x, qb1.y, 0.f), a1.x, L1, c1, fx, fy, fz);
        }
    }
    integrate<GROUND>(p, v, fx, fy, fz, c, out + i);
}

// K1, grid-box form: k_step_halo for masses on a grid.  The block's table is
// the box of cells around its masses (see build_box), so a neighbour's slot
// is the mass's own slot plus the column's offset (one int16 per SELL column,
// the same for every lane) and the half-edge stream carries only {k, L0}
// (8 bytes instead of 10).  It issues no bulk L2 prefetch: with the first
// stream loads issued ahead of the table fill, the prefetch was measured to
// cost more than it saved.  Padding entries ({k, L0} = {0, kPadRest}: a
// negative rest length, where every real spring, zero-rest-length ones
// included, has L0 >= 0) may point at an empty cell of the box, whose table
// slot holds whatever was there: they are skipped, never evaluated.  Holes -
// device slots of empty cells, marked by own slot 0xFFFF - do nothing at all.
template <bool HAS_C, bool HAS_ACT, bool GROUND, bool OVERLAP>
__global__ void __launch_bounds__(kHaloThreads, kBoxMinBlocks)
k_step_box(const MassState *__restrict__ in, MassState *__restrict__ out, uint32_t n,
           const uint32_t *__restrict__ slice_off, const uint32_t *__restrict__ col_off2,
           const float2 *__restrict__ kl, const float *__restrict__ cc, const float2 *__restrict__ act,
           const uint16_t *__restrict__ own_slot, const uint32_t *__restrict__ ext_off,
           const uint32_t *__restrict__ ext_idx, const uint16_t *__restrict__ ext_slot, uint32_t table_slots,
           StepConst c, const long long *__restrict__ step_in, long long *__restrict__ step_out) {
    extern __shared__ float4 tab4[];
    float4 *tA = tab4;
    float2 *tB = reinterpret_cast<float2 *>(tab4 + table_slots);
    const uint32_t b = blockIdx.x, tid = threadIdx.x;
    const uint32_t i = b * kHaloThreads + tid;
    const uint32_t lane = tid & 31, sl = i >> 5;
    if (OVERLAP) ptx::grid_dep_launch();    // the next step's CTAs may take SM slots this tail frees
    // holes (empty cells of the block's cube) have no springs and never move:
    // their state is neither read nor written
    const uint32_t s_own = i < n ? own_slot[i] : kBoxHoleSlot;
    const bool valid = s_own != kBoxHoleSlot;

    uint32_t e0 = 0, width = 0;
    float4 p = make_float4(0.f, 0.f, 0.f, 0.f), v = p;
    const uint32_t *co = col_off2;
    uint32_t e = 0, no = 0;
    float2 na0 = make_float2(0.f, 0.f), na1 = na0;
    float nc0 = c.c_uniform, nc1 = c.c_uniform;
    float2 ns0 = make_float2(0.f, 0.f), ns1 = ns0;
    if (valid) {
        e0 = __ldg(slice_off + sl);
        width = (__ldg(slice_off + sl + 1) - e0) >> 5;
        // the first pair of columns is requested before the table fill so its
        // latency overlaps the fill; widths are even and slices start at even
        // column counts, so a pair of int16 column offsets is one aligned word
        co = col_off2 + (e0 >> 6);
        e = e0 + lane;
        if (width) {
            no = __ldg(co);
            na0 = __ldcs(kl + e); na1 = __ldcs(kl + e + 32);
            if (HAS_C) { nc0 = __ldcs(cc + e); nc1 = __ldcs(cc + e + 32); }
            if (HAS_ACT) { ns0 = __ldcs(act + e); ns1 = __ldcs(act + e + 32); }
        }
    }
    const uint32_t h0 = __ldg(ext_off + b), h1 = __ldg(ext_off + b + 1);
    // everything above reads layout data only; the state and the step counter
    // are written by the previous step, which must have completed
    if (OVERLAP) ptx::grid_dep_wait();
    long long step = 0;
    if (HAS_ACT || (b == 0 && tid == 0)) step = read_step<OVERLAP>(step_in);
    if (b == 0 && tid == 0) *step_out = step + 1;
    if (valid) {
        read_state<OVERLAP>(in + i, p, v);
        tA[s_own] = make_float4(p.x, p.y, p.z, v.x);
        tB[s_own] = make_float2(v.y, v.z);
    }
    for (uint32_t h = h0 + tid; h < h1; h += kHaloThreads) {
        float4 q, ww;
        read_state<OVERLAP>(in + __ldg(ext_idx + h), q, ww);
        const uint32_t s = __ldg(ext_slot + h);
        tA[s] = make_float4(q.x, q.y, q.z, ww.x);
        tB[s] = make_float2(ww.y, ww.z);
    }
    __syncthreads();
    if (!valid) return;

    const float ph = HAS_ACT ? actuation_clock(c, step) : 0.f;
    float fx = 0.f, fy = 0.f, fz = 0.f;
    if (width) {
        for (uint32_t t = 0; t < width; t += 2) {
            const uint32_t o = no;
            const float2 a0 = na0, a1 = na1;
            const float c0 = nc0, c1 = nc1;
            const float2 s0 = ns0, s1 = ns1;
            // the next pair, unconditionally: past the slice's last pair this
            // reads the next slice's entries or the arrays' tail (kStreamTail),
            // values never used
            e += 64;
            no = __ldg(co + (t >> 1) + 1);
            na0 = __ldcs(kl + e); na1 = __ldcs(kl + e + 32);
            if (HAS_C) { nc0 = __ldcs(cc + e); nc1 = __ldcs(cc + e + 32); }
            if (HAS_ACT) { ns0 = __ldcs(act + e); ns1 = __ldcs(act + e + 32); }
            const uint32_t j0 = s_own + (uint32_t)(int32_t)(int16_t)(o & 0xffffu);
            const uint32_t j1 = s_own + (uint32_t)(int32_t)(int16_t)(o >> 16);
            float L0 = a0.y, L1 = a1.y;
            if (HAS_ACT) {
                L0 = actuated_length(c, a0.y, s0, ph);
                L1 = actuated_length(c, a1.y, s1, ph);
            }
            if (a0.y >= 0.f) {          // not padding
                const float4 qa = tA[j0];
                const float2 qb = tB[j0];
                spring_force(p, v, qa, make_float4(qa.w, qb.x, qb.y, 0.f), a0.x, L0, c0, fx, fy, fz);
            }
            if (a1.y >= 0.f) {
                const float4 qa = tA[j1];
                const float2 qb = tB[j1];
                spring_force(p, v, qa, make_float4(qa.w, qb.x, qb.y, 0.f), a1.x, L1, c1, fx, fy, fz);
            }
        }
    }
    integrate<GROUND>(p, v, fx, fy, fz, c, out + i);
}

// K1, cube form (the default for 26-neighbourhood lattices): as k_step_box,
// but each spring inside the block's cube is read and evaluated once.  The
// step runs 13 passes, one per canonical direction p (layout.h: kCubeDirs);
// in pass j every mass evaluates its +p spring from the dense plus stream and
// publishes (f, u) in shared memory; after one barrier, a mass whose -p
// partner lies in the cube adds that force with u negated - exactly what it
// would have computed itself (the spring's scalar is the same from both ends
// and its axis changes sign exactly) - and one whose -p partner is outside
// evaluates the spring from the cube's compact ext stream.  Each mass adds
// +p1, -p1, +p2, ... in its row order, so the trajectory is bit-identical to
// the other CSR kernels.  Stream: 143 MB instead of 208 MB on the 1M lattice,
// but the 13 barriers per block and the divergent outside-partner path cost
// more than the bytes saved (measured 84.4 us/step against 59.8 for
// k_step_box): kernel variant 8, taken only when asked for.
// The pass directions of layout.h's kCubeDirs, as (dx + 1) | (dy + 1) << 2 | (dz + 1) << 4.
__constant__ uint8_t c_cube_dir[13] = {0x16, 0x18, 0x19, 0x1a, 0x20, 0x21, 0x22, 0x24, 0x25, 0x26, 0x28, 0x29, 0x2a};
__device__ __forceinline__ int3 cube_dir(int j) {
    const uint32_t d = c_cube_dir[j];
    return make_int3((int)(d & 3) - 1, (int)((d >> 2) & 3) - 1, (int)((d >> 4) & 3) - 1);
}
constexpr int kCubeP = 13;

constexpr int kCubeMinBlocks = 5;      // resident CTAs per SM the register budget is sized for

template <bool HAS_C, bool HAS_ACT, bool GROUND>
__global__ void __launch_bounds__(kHaloThreads, kCubeMinBlocks)
k_step_cube(const MassState *__restrict__ in, MassState *__restrict__ out, uint32_t n,
            const uint32_t *__restrict__ cube_base, const uint4 *__restrict__ cube_meta,
            const float2 *__restrict__ kl, const float *__restrict__ cc, const float2 *__restrict__ act,
            const uint16_t *__restrict__ own_slot, const uint32_t *__restrict__ ext_off,
            const uint32_t *__restrict__ ext_idx, const uint16_t *__restrict__ ext_slot, uint32_t table_slots,
            StepConst c, const long long *__restrict__ step_in, long long *__restrict__ step_out) {
    extern __shared__ float4 ctab[];
    float4 *tA = ctab;
    float2 *tB = reinterpret_cast<float2 *>(ctab + table_slots);
    float4 *xch = reinterpret_cast<float4 *>(tB + table_slots);    // [2][256] (f, ux, uy, uz); slots even
    const uint32_t b = blockIdx.x, tid = threadIdx.x;
    const uint32_t i = b * kHaloThreads + tid;
    const uint32_t lane = tid & 31, w = tid >> 5;
    long long step = 0;
    if (HAS_ACT) step = *step_in;
    if (b == 0 && tid == 0) *step_out = *step_in + 1;
    const uint32_t s_own = i < n ? own_slot[i] : kBoxHoleSlot;
    const bool valid = s_own != kBoxHoleSlot;

    const uint32_t base = __ldg(cube_base + b);
    const uint32_t ext0 = base + kCubeP * kHaloThreads;
    const uint4 *mt = cube_meta + (size_t)b * kCubeP * (kHaloThreads / 32) + w;   // [pass][warp]
    // the first pass's entries are requested before the table fill
    float2 a_n = make_float2(0.f, 0.f), s_n = a_n;
    float c_n = c.c_uniform;
    if (valid) {
        a_n = __ldcs(kl + base + tid);
        if (HAS_C) c_n = __ldcs(cc + base + tid);
        if (HAS_ACT) s_n = __ldcs(act + base + tid);
    }
    // pass metadata runs two passes ahead of its use, the plus entries one
    uint4 m_n = __ldg(mt), m_nn = __ldg(mt + (kHaloThreads / 32));
    float4 p = make_float4(0.f, 0.f, 0.f, 0.f), v = p;
    if (valid) {
        load_state(in + i, p, v);
        tA[s_own] = make_float4(p.x, p.y, p.z, v.x);
        tB[s_own] = make_float2(v.y, v.z);
    }
    const uint32_t h0 = __ldg(ext_off + b), h1 = __ldg(ext_off + b + 1);
    for (uint32_t h = h0 + tid; h < h1; h += kHaloThreads) {
        float4 q, ww;
        load_state(in + __ldg(ext_idx + h), q, ww);
        const uint32_t s = __ldg(ext_slot + h);
        tA[s] = make_float4(q.x, q.y, q.z, ww.x);
        tB[s] = make_float2(ww.y, ww.z);
    }
    __syncthreads();

    // this mass's cell within the cube (grid order: tile = warp, lane = cell in the tile)
    const int cx = 4 * (int)(w & 1) + (int)(lane & 3), cy = 4 * (int)((w >> 1) & 1) + (int)((lane >> 2) & 3),
              cz = 2 * (int)(w >> 2) + (int)(lane >> 4);
    const float clk = HAS_ACT ? actuation_clock(c, step) : 0.f;
    const uint32_t below = (1u << lane) - 1u;
    float fx = 0.f, fy = 0.f, fz = 0.f;
#pragma unroll 1
    for (int j = 0; j < kCubeP; ++j) {
        const float2 a = a_n, sa = s_n;
        const float ca = c_n;
        const uint4 m = m_n;
        // this pass's ext entry is requested before the +p work and the barrier
        const bool take_ext = valid && !((m.x >> lane) & 1u) && ((m.y >> lane) & 1u);
        const uint32_t ex = ext0 + m.z + __popc(m.y & below);
        float2 a2 = make_float2(0.f, 0.f), s2 = a2;
        float c2 = c.c_uniform;
        if (take_ext) {
            a2 = __ldcs(kl + ex);
            if (HAS_C) c2 = __ldcs(cc + ex);
            if (HAS_ACT) s2 = __ldcs(act + ex);
        }
        if (j + 1 < kCubeP) {
            if (valid) {
                a_n = __ldcs(kl + base + (j + 1) * kHaloThreads + tid);
                if (HAS_C) c_n = __ldcs(cc + base + (j + 1) * kHaloThreads + tid);
                if (HAS_ACT) s_n = __ldcs(act + base + (j + 1) * kHaloThreads + tid);
            }
            m_n = m_nn;
            if (j + 2 < kCubeP) m_nn = __ldg(mt + (j + 2) * (kHaloThreads / 32));
        }
        const int32_t off = (int32_t)(int16_t)(m.w & 0xffffu);
        float f = 0.f, ux = 0.f, uy = 0.f, uz = 0.f;
        if (valid && a.y >= 0.f) {                          // +p (not padding): evaluate and publish
            const uint32_t js = s_own + (uint32_t)off;
            const float4 qa = tA[js];
            const float2 qb = tB[js];
            const float L = HAS_ACT ? actuated_length(c, a.y, sa, clk) : a.y;
            spring_terms(p, v, qa, make_float4(qa.w, qb.x, qb.y, 0.f), a.x, L, ca, f, ux, uy, uz);
            fx = fmaf(f, ux, fx);
            fy = fmaf(f, uy, fy);
            fz = fmaf(f, uz, fz);
        }
        float4 *X = xch + (j & 1) * kHaloThreads;
        X[tid] = make_float4(f, ux, uy, uz);
        __syncthreads();
        if (valid) {
            if ((m.x >> lane) & 1u) {                       // -p from the in-cube partner
                const int3 d = cube_dir(j);
                const int px = cx - d.x, py = cy - d.y, pz = cz - d.z;
                const int pt = ((((px >> 2) & 1) | (((py >> 2) & 1) << 1) | (((pz >> 1) & 1) << 2)) << 5) +
                               (px & 3) + 4 * (py & 3) + 16 * (pz & 1);
                const float4 g = X[pt];
                fx = fmaf(g.x, -g.y, fx);
                fy = fmaf(g.x, -g.z, fy);
                fz = fmaf(g.x, -g.w, fz);
            } else if (take_ext) {                          // -p from outside the cube
                const uint32_t js = s_own - (uint32_t)off;
                const float4 qa = tA[js];
                const float2 qb = tB[js];
                const float L = HAS_ACT ? actuated_length(c, a2.y, s2, clk) : a2.y;
                spring_force(p, v, qa, make_float4(qa.w, qb.x, qb.y, 0.f), a2.x, L, c2, fx, fy, fz);
            }
        }
    }
    if (!valid) return;
    integrate<GROUND>(p, v, fx, fy, fz, c, out + i);
}

// K1, grid-box form with the stream staged by TMA: as k_step_box, but lane 0
// of each warp first copies its slice's {k, L0} (and c, actuation) columns
// into shared memory with 1-D bulk copies on one mbarrier per warp, so a
// whole slice's stream is in flight at once while the table fills; the row
// loop then reads only shared memory.  Slices wider than the staging buffer
// (w_max columns) read their columns from global memory.  The mbarrier wait
// is bounded by spin_limit polls; on expiry the warp records the error in
// *err, waits (bounded) for its copies and leaves its masses unwritten.
template <bool HAS_C, bool HAS_ACT>
constexpr int box_entry_bytes() { return 8 + (HAS_C ? 4 : 0) + (HAS_ACT ? 8 : 0); }

template <bool HAS_C, bool HAS_ACT, bool GROUND>
__global__ void __launch_bounds__(kHaloThreads, 3)
k_step_box_tma(const MassState *__restrict__ in, MassState *__restrict__ out, uint32_t n,
               const uint32_t *__restrict__ slice_off, const uint32_t *__restrict__ col_off2,
               const float2 *__restrict__ kl, const float *__restrict__ cc, const float2 *__restrict__ act,
               const uint16_t *__restrict__ own_slot, const uint32_t *__restrict__ ext_off,
               const uint32_t *__restrict__ ext_idx, const uint16_t *__restrict__ ext_slot, uint32_t table_slots,
               uint32_t w_max, StepConst c, const long long *__restrict__ step_in, long long *__restrict__ step_out,
               uint32_t spin_limit, int *__restrict__ err) {
    constexpr uint32_t FULL = 0xffffffffu;
    constexpr int EB = box_entry_bytes<HAS_C, HAS_ACT>();
    extern __shared__ float4 btab[];
    __shared__ uint64_t bars[kHaloThreads / 32];
    float4 *tA = btab;
    float2 *tB = reinterpret_cast<float2 *>(btab + table_slots);
    const uint32_t b = blockIdx.x, tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const uint32_t i = b * kHaloThreads + tid, sl = i >> 5;
    const uint32_t n_slices = (n + 31) >> 5;
    // per-warp staging buffer after the table: [kl float2 | act float2 | c float] x (w_max * 32)
    unsigned char *wb = reinterpret_cast<unsigned char *>(tB + table_slots) + (size_t)w * w_max * 32 * EB;
    float2 *s_kl = reinterpret_cast<float2 *>(wb);
    float2 *s_act = reinterpret_cast<float2 *>(wb + (size_t)w_max * 32 * 8);
    float *s_c = reinterpret_cast<float *>(wb + (size_t)w_max * 32 * (HAS_ACT ? 16 : 8));

    long long step = 0;
    if (HAS_ACT) step = *step_in;
    if (b == 0 && tid == 0) *step_out = *step_in + 1;

    const bool warp_live = sl < n_slices;                    // warp-uniform
    uint32_t e0 = 0, width = 0;
    if (warp_live) {
        e0 = __ldg(slice_off + sl);
        width = (__ldg(slice_off + sl + 1) - e0) >> 5;
    }
    const bool staged = warp_live && width > 0 && width <= w_max;
    if (staged && lane == 0) {
        const uint32_t ne = width * 32;
        ptx::mbar_init(&bars[w], 1);
        ptx::fence_mbar_init();
        ptx::mbar_arrive_expect_tx(&bars[w], ne * EB);
        ptx::bulk_g2s(s_kl, kl + e0, ne * 8, &bars[w]);
        if (HAS_ACT) ptx::bulk_g2s(s_act, act + e0, ne * 8, &bars[w]);
        if (HAS_C) ptx::bulk_g2s(s_c, cc + e0, ne * 4, &bars[w]);
    }
    const uint32_t s_own = i < n ? own_slot[i] : kBoxHoleSlot;
    const bool valid = s_own != kBoxHoleSlot;
    float4 p = make_float4(0.f, 0.f, 0.f, 0.f), v = p;
    if (valid) {
        load_state(in + i, p, v);
        tA[s_own] = make_float4(p.x, p.y, p.z, v.x);
        tB[s_own] = make_float2(v.y, v.z);
    }
    const uint32_t h0 = __ldg(ext_off + b), h1 = __ldg(ext_off + b + 1);
    for (uint32_t h = h0 + tid; h < h1; h += kHaloThreads) {
        float4 q, ww;
        load_state(in + __ldg(ext_idx + h), q, ww);
        const uint32_t s = __ldg(ext_slot + h);
        tA[s] = make_float4(q.x, q.y, q.z, ww.x);
        tB[s] = make_float2(ww.y, ww.z);
    }
    __syncthreads();                    // also publishes the mbarrier initialisation
    if (!warp_live) return;
    if (staged) {
        bool done = false;
        for (uint32_t it = 0; it < spin_limit; ++it) {
            done = ptx::mbar_try_wait(&bars[w], 0);
            if (__all_sync(FULL, done)) break;
        }
        if (!__all_sync(FULL, done)) {
            if (lane == 0) {
                atomicExch(err, 1);
                ptx::mbar_wait_bounded(&bars[w], 0, spin_limit);
            }
            __syncwarp();
            return;
        }
    }
    if (!valid) return;

    const float ph = HAS_ACT ? actuation_clock(c, step) : 0.f;
    float fx = 0.f, fy = 0.f, fz = 0.f;
    const uint32_t *co = col_off2 + (e0 >> 6);      // even widths: a pair of int16 offsets per word
    for (uint32_t t = 0; t < width; t += 2) {
        const uint32_t a = t * 32 + lane, bb = a + 32;
        float2 a0, a1, s0 = make_float2(0.f, 0.f), s1 = s0;
        float c0 = c.c_uniform, c1 = c.c_uniform;
        if (staged) {
            a0 = s_kl[a]; a1 = s_kl[bb];
            if (HAS_C) { c0 = s_c[a]; c1 = s_c[bb]; }
            if (HAS_ACT) { s0 = s_act[a]; s1 = s_act[bb]; }
        } else {
            a0 = __ldcs(kl + e0 + a); a1 = __ldcs(kl + e0 + bb);
            if (HAS_C) { c0 = __ldcs(cc + e0 + a); c1 = __ldcs(cc + e0 + bb); }
            if (HAS_ACT) { s0 = __ldcs(act + e0 + a); s1 = __ldcs(act + e0 + bb); }
        }
        const uint32_t o = __ldg(co + (t >> 1));
        const uint32_t j0 = s_own + (uint32_t)(int32_t)(int16_t)(o & 0xffffu);
        const uint32_t j1 = s_own + (uint32_t)(int32_t)(int16_t)(o >> 16);
        float L0 = a0.y, L1 = a1.y;
        if (HAS_ACT) {
            L0 = actuated_length(c, a0.y, s0, ph);
            L1 = actuated_length(c, a1.y, s1, ph);
        }
        if (a0.y >= 0.f) {          // not padding
            const float4 qa = tA[j0];
            const float2 qb = tB[j0];
            spring_force(p, v, qa, make_float4(qa.w, qb.x, qb.y, 0.f), a0.x, L0, c0, fx, fy, fz);
        }
        if (a1.y >= 0.f) {
            const float4 qa = tA[j1];
            const float2 qb = tB[j1];
            spring_force(p, v, qa, make_float4(qa.w, qb.x, qb.y, 0.f), a1.x, L1, c1, fx, fy, fz);
        }
    }
    integrate<GROUND>(p, v, fx, fy, fz, c, out + i);
}

// K1, halo + TMA form.  As k_step_halo, but the half-edge stream of each
// warp's slice (all columns of every array) is copied into shared memory by
// the TMA engine (1-D bulk copies on one mbarrier per warp), issued before the
// halo fill so the DRAM transfer overlaps it; the hot loop then reads only
// shared memory.  Slices wider than the staging buffer (w_max columns) read
// their columns from global memory instead.  The mbarrier wait is bounded by
// spin_limit polls; on expiry the warp records the error in *err, waits
// (bounded) for its copies and leaves its masses unwritten.
template <bool HAS_C, bool HAS_ACT>
constexpr int halo_entry_bytes() { return 10 + (HAS_C ? 4 : 0) + (HAS_ACT ? 8 : 0); }

template <bool HAS_C, bool HAS_ACT, bool GROUND>
__global__ void __launch_bounds__(kHaloThreads, 2)
k_step_halo_tma(const MassState *__restrict__ in, MassState *__restrict__ out, uint32_t n,
                const uint32_t *__restrict__ slice_off, const uint16_t *__restrict__ nslot,
                const float2 *__restrict__ kl, const float *__restrict__ cc,
                const float2 *__restrict__ act, const uint16_t *__restrict__ own_slot,
                const uint32_t *__restrict__ ext_off, const uint32_t *__restrict__ ext_idx,
                const uint16_t *__restrict__ ext_slot, uint32_t table_slots, uint32_t w_max,
                StepConst c, const long long *__restrict__ step_in, long long *__restrict__ step_out,
                uint32_t spin_limit, int *__restrict__ err) {
    constexpr uint32_t FULL = 0xffffffffu;
    constexpr int EB = halo_entry_bytes<HAS_C, HAS_ACT>();
    extern __shared__ __align__(16) unsigned char hsm[];
    __shared__ uint64_t bars[kHaloThreads / 32];
    float2 *tA = reinterpret_cast<float2 *>(hsm);
    float2 *tB = tA + table_slots, *tC = tB + table_slots;
    const uint32_t b = blockIdx.x, tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const uint32_t i = b * kHaloThreads + tid, sl = i >> 5;
    const uint32_t n_slices = (n + 31) >> 5;
    // per-warp staging buffer: [kl float2 | act float2 | c float | slot u16] x (w_max * 32)
    const size_t per_warp = (size_t)w_max * 32 * EB;
    unsigned char *wb = hsm + (size_t)3 * table_slots * sizeof(float2) + (size_t)w * per_warp;
    float2 *s_kl = reinterpret_cast<float2 *>(wb);
    float2 *s_act = reinterpret_cast<float2 *>(wb + (size_t)w_max * 32 * 8);
    float *s_c = reinterpret_cast<float *>(wb + (size_t)w_max * 32 * (HAS_ACT ? 16 : 8));
    uint16_t *s_slot = reinterpret_cast<uint16_t *>(wb + (size_t)w_max * 32 * (8 + (HAS_ACT ? 8 : 0) + (HAS_C ? 4 : 0)));

    long long step = 0;
    if (HAS_ACT) step = *step_in;
    if (b == 0 && tid == 0) *step_out = *step_in + 1;

    const bool warp_live = sl < n_slices;                    // warp-uniform
    uint32_t e0 = 0, width = 0;
    if (warp_live) {
        e0 = __ldg(slice_off + sl);
        width = (__ldg(slice_off + sl + 1) - e0) >> 5;
    }
    const bool staged = warp_live && width > 0 && width <= w_max;
    if (staged && lane == 0) {
        const uint32_t ne = width * 32;
        ptx::mbar_init(&bars[w], 1);
        ptx::fence_mbar_init();
        ptx::mbar_arrive_expect_tx(&bars[w], ne * EB);
        ptx::bulk_g2s(s_kl, kl + e0, ne * 8, &bars[w]);
        if (HAS_ACT) ptx::bulk_g2s(s_act, act + e0, ne * 8, &bars[w]);
        if (HAS_C) ptx::bulk_g2s(s_c, cc + e0, ne * 4, &bars[w]);
        ptx::bulk_g2s(s_slot, nslot + e0, ne * 2, &bars[w]);
    }
    const bool valid = i < n;
    float4 p = make_float4(0.f, 0.f, 0.f, 0.f), v = p;
    if (valid) {
        load_state(in + i, p, v);
        const uint32_t s = own_slot[i];
        tA[s] = make_float2(p.x, p.y);
        tB[s] = make_float2(p.z, v.x);
        tC[s] = make_float2(v.y, v.z);
    }
    const uint32_t h0 = __ldg(ext_off + b), h1 = __ldg(ext_off + b + 1);
    for (uint32_t h = h0 + tid; h < h1; h += kHaloThreads) {
        float4 q, ww;
        load_state(in + __ldg(ext_idx + h), q, ww);
        const uint32_t s = __ldg(ext_slot + h);
        tA[s] = make_float2(q.x, q.y);
        tB[s] = make_float2(q.z, ww.x);
        tC[s] = make_float2(ww.y, ww.z);
    }
    __syncthreads();                    // also publishes the mbarrier initialisation
    if (!warp_live) return;
    if (staged) {
        bool done = false;
        for (uint32_t it = 0; it < spin_limit; ++it) {
            done = ptx::mbar_try_wait(&bars[w], 0);
            if (__all_sync(FULL, done)) break;
        }
        if (!__all_sync(FULL, done)) {
            if (lane == 0) {
                atomicExch(err, 1);
                ptx::mbar_wait_bounded(&bars[w], 0, spin_limit);
            }
            __syncwarp();
            return;
        }
    }
    if (!valid) return;

    const float ph = HAS_ACT ? actuation_clock(c, step) : 0.f;
    float fx = 0.f, fy = 0.f, fz = 0.f;
    for (uint32_t t = 0; t < width; t += 2) {
        const uint32_t a = t * 32 + lane, bb = a + 32;
        uint32_t j0, j1;
        float2 a0, a1, s0 = make_float2(0.f, 0.f), s1 = s0;
        float c0 = c.c_uniform, c1 = c.c_uniform;
        if (staged) {
            j0 = s_slot[a]; j1 = s_slot[bb];
            a0 = s_kl[a]; a1 = s_kl[bb];
            if (HAS_C) { c0 = s_c[a]; c1 = s_c[bb]; }
            if (HAS_ACT) { s0 = s_act[a]; s1 = s_act[bb]; }
        } else {
            j0 = __ldcs(nslot + e0 + a); j1 = __ldcs(nslot + e0 + bb);
            a0 = __ldcs(kl + e0 + a); a1 = __ldcs(kl + e0 + bb);
            if (HAS_C) { c0 = __ldcs(cc + e0 + a); c1 = __ldcs(cc + e0 + bb); }
            if (HAS_ACT) { s0 = __ldcs(act + e0 + a); s1 = __ldcs(act + e0 + bb); }
        }
        const float2 qa0 = tA[j0], qb0 = tB[j0], qc0 = tC[j0];
        const float2 qa1 = tA[j1], qb1 = tB[j1], qc1 = tC[j1];
        float L0 = a0.y, L1 = a1.y;
        if (HAS_ACT) {
            L0 = actuated_length(c, a0.y, s0, ph);
            L1 = actuated_length(c, a1.y, s1, ph);
        }
        spring_force(p, v, make_float4(qa0.x, qa0.y, qb0.x, 0.f), make_float4(qb0.y, qc0.x, qc0.y, 0.f),
                     a0.x, L0, c0, fx, fy, fz);
        spring_force(p, v, make_float4(qa1.x, qa1.y, qb1.x, 0.f), make_float4(qb1.y, qc1.x, qc1.y, 0.f),
                     a1.x, L1, c1, fx, fy, fz);
    }
    integrate<GROUND>(p, v, fx, fy, fz, c, out + i);
}

// K1, TMA-staged form.  One warp owns one SELL slice (32 masses).  Lane 0
// streams the slice's half-edge columns into a per-warp ring of shared-memory
// stages with 1-D bulk copies (TMA), kStagesK1 chunks of kChunkCols columns
// ahead, each stage guarded by an mbarrier; the warp computes from shared
// memory while later chunks are in flight, so DRAM streaming no longer waits
// on the neighbour gathers.  Every mbarrier wait is bounded by spin_limit
// polls; on expiry the warp records the error in *err, waits (bounded) for its
// copies in flight and leaves its masses unwritten.
constexpr int kWarpsK1 = 4;
constexpr int kChunkCols = 8;
constexpr int kStagesK1 = 2;
constexpr int kChunkEntries = kChunkCols * 32;

template <bool HAS_C, bool HAS_ACT>
constexpr int entry_bytes() { return 12 + (HAS_C ? 4 : 0) + (HAS_ACT ? 8 : 0); }

template <bool HAS_C, bool HAS_ACT>
constexpr int staged_smem_bytes() { return kWarpsK1 * kStagesK1 * kChunkEntries * entry_bytes<HAS_C, HAS_ACT>(); }

template <bool HAS_C, bool HAS_ACT, bool GROUND>
__global__ void __launch_bounds__(kWarpsK1 * 32)
k_step_sell_staged(const MassState *__restrict__ in, MassState *__restrict__ out, uint32_t n,
                   uint32_t n_slices, const uint32_t *__restrict__ slice_off,
                   const uint32_t *__restrict__ nbr, const float2 *__restrict__ kl,
                   const float *__restrict__ cc, const float2 *__restrict__ act, StepConst c,
                   const long long *__restrict__ step_in, long long *__restrict__ step_out,
                   uint32_t spin_limit, int *__restrict__ err) {
    constexpr int EB = entry_bytes<HAS_C, HAS_ACT>();
    constexpr uint32_t FULL = 0xffffffffu;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bars[kWarpsK1][kStagesK1];

    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t sl = blockIdx.x * kWarpsK1 + w;
    long long step = 0;
    if (HAS_ACT) step = *step_in;
    if (blockIdx.x == 0 && threadIdx.x == 0) *step_out = *step_in + 1;
    if (sl >= n_slices) return;                 // whole warp; no CTA-wide barrier follows

    // stage s of this warp: [kl float2 | act float2 | nbr u32 | c float] x kChunkEntries
    unsigned char *wbase = smem + (size_t)w * kStagesK1 * kChunkEntries * EB;
    auto st_kl = [&](int s) { return reinterpret_cast<float2 *>(wbase + (size_t)s * kChunkEntries * EB); };
    auto st_act = [&](int s) { return reinterpret_cast<float2 *>(wbase + (size_t)s * kChunkEntries * EB + kChunkEntries * 8); };
    auto st_nbr = [&](int s) {
        return reinterpret_cast<uint32_t *>(wbase + (size_t)s * kChunkEntries * EB + kChunkEntries * (HAS_ACT ? 16 : 8));
    };
    auto st_c = [&](int s) {
        return reinterpret_cast<float *>(wbase + (size_t)s * kChunkEntries * EB + kChunkEntries * (HAS_ACT ? 20 : 12));
    };

    const uint32_t e0 = __ldg(slice_off + sl);
    const uint32_t width = (__ldg(slice_off + sl + 1) - e0) >> 5;
    const uint32_t n_chunks = (width + kChunkCols - 1) / kChunkCols;

    if (lane == 0) {
        for (int s = 0; s < kStagesK1; ++s) ptx::mbar_init(&bars[w][s], 1);
        ptx::fence_mbar_init();
    }
    __syncwarp();

    auto issue = [&](uint32_t ch) {            // lane 0 only
        const int s = ch % kStagesK1;
        const uint32_t cols = min((uint32_t)kChunkCols, width - ch * kChunkCols);
        const uint32_t ne = cols * 32, eb = e0 + ch * kChunkEntries;
        ptx::mbar_arrive_expect_tx(&bars[w][s], ne * EB);
        ptx::bulk_g2s(st_kl(s), kl + eb, ne * 8, &bars[w][s]);
        if (HAS_ACT) ptx::bulk_g2s(st_act(s), act + eb, ne * 8, &bars[w][s]);
        ptx::bulk_g2s(st_nbr(s), nbr + eb, ne * 4, &bars[w][s]);
        if (HAS_C) ptx::bulk_g2s(st_c(s), cc + eb, ne * 4, &bars[w][s]);
    };
    uint32_t issued = 0;
    if (lane == 0)
        for (; issued < n_chunks && issued < (uint32_t)kStagesK1; ++issued) issue(issued);
    issued = __shfl_sync(FULL, issued, 0);

    const uint32_t i = sl * 32 + lane;
    const bool valid = i < n;
    float4 p = make_float4(0.f, 0.f, 0.f, 0.f), v = p;
    if (valid) {
        p = __ldg(&in[i].p);
        v = __ldg(&in[i].v);
    }
    const float ph = HAS_ACT ? actuation_clock(c, step) : 0.f;
    float fx = 0.f, fy = 0.f, fz = 0.f;

    for (uint32_t ch = 0; ch < n_chunks; ++ch) {
        const int s = ch % kStagesK1;
        const uint32_t parity = (ch / kStagesK1) & 1;
        bool done = false;
        for (uint32_t it = 0; it < spin_limit; ++it) {
            done = ptx::mbar_try_wait(&bars[w][s], parity);
            if (__all_sync(FULL, done)) break;
        }
        if (!__all_sync(FULL, done)) {
            if (lane == 0) {
                atomicExch(err, 1);
                for (uint32_t k = ch; k < issued; ++k)
                    ptx::mbar_wait_bounded(&bars[w][k % kStagesK1], (k / kStagesK1) & 1, spin_limit);
            }
            __syncwarp();
            return;
        }
        const uint32_t cols = min((uint32_t)kChunkCols, width - ch * kChunkCols);
        if (valid) {
            const float2 *skl = st_kl(s);
            const uint32_t *snb = st_nbr(s);
            for (uint32_t t = 0; t < cols; t += 2) {
                const uint32_t a = t * 32 + lane, b = a + 32;
                const uint32_t j0 = snb[a], j1 = snb[b];
                const float2 a0 = skl[a], a1 = skl[b];
                float c0 = c.c_uniform, c1 = c.c_uniform;
                if (HAS_C) { c0 = st_c(s)[a]; c1 = st_c(s)[b]; }
                float L0 = a0.y, L1 = a1.y;
                if (HAS_ACT) {
                    const float2 s0 = st_act(s)[a], s1 = st_act(s)[b];
                    L0 = actuated_length(c, a0.y, s0, ph);
                    L1 = actuated_length(c, a1.y, s1, ph);
                }
                float4 q0, w0, q1, w1;
                load_state(in + j0, q0, w0);
                load_state(in + j1, q1, w1);
                spring_force(p, v, q0, w0, a0.x, L0, c0, fx, fy, fz);
                spring_force(p, v, q1, w1, a1.x, L1, c1, fx, fy, fz);
            }
        }
        __syncwarp();
        if (lane == 0 && issued < n_chunks) {
            ptx::fence_proxy_async_smem();
            issue(issued);
            ++issued;
        }
        issued = __shfl_sync(FULL, issued, 0);
    }
    if (valid) integrate<GROUND>(p, v, fx, fy, fz, c, out + i);
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
        L = actuated_length(c, L, a, actuation_clock(c, *step_in));
    }
    const float cs = HAS_C ? __ldcs(cc + s) : c.c_uniform;
    float4 p, v, q, w;
    load_state(in + r.x, p, v);
    load_state(in + r.y, q, w);
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
    const bool hc = v.c != nullptr, ha = v.act != nullptr, gr = c.ground != 0;
    if (v.variant == 0 || v.variant == 1) {
        const unsigned g = n ? blocks_for(n) : 1;
#define TITAN_SELL(HC, HA, GR)                                                                   \
    do {                                                                                         \
        if (v.variant == 0)                                                                      \
            k_step_sell_pf<HC, HA, GR><<<g, kThreads, 0, stream>>>(in, out, n, v.slice_off, v.nbr, \
                                                                 v.kl, v.c, v.act, c, step_in, step_out); \
        else                                                                                     \
            k_step_sell<HC, HA, GR><<<g, kThreads, 0, stream>>>(in, out, n, v.slice_off, v.nbr, v.kl, \
                                                                v.c, v.act, c, step_in, step_out); \
    } while (0)
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
    const uint32_t n_slices = (n + 31) / 32;
    const unsigned g = n_slices ? (n_slices + kWarpsK1 - 1) / kWarpsK1 : 1;
#define TITAN_STAGED(HC, HA, GR)                                                                 \
    do {                                                                                         \
        auto kern = k_step_sell_staged<HC, HA, GR>;                                              \
        constexpr int bytes = staged_smem_bytes<HC, HA>();                                       \
        static std::atomic<uint64_t> attr_set{0};                                                \
        int dev_ = 0;                                                                            \
        cudaGetDevice(&dev_);                                                                    \
        const uint64_t bit_ = 1ull << (dev_ & 63);                                               \
        if (!(attr_set.load() & bit_)) {                                                         \
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes); \
            if (e != cudaSuccess) return e;                                                      \
            attr_set.fetch_or(bit_);                                                             \
        }                                                                                        \
        kern<<<g, kWarpsK1 * 32, bytes, stream>>>(in, out, n, n_slices, v.slice_off, v.nbr, v.kl, \
                                                  v.c, v.act, c, step_in, step_out, v.spin_limit, v.err); \
    } while (0)
    if (hc) {
        if (ha) { if (gr) TITAN_STAGED(true, true, true); else TITAN_STAGED(true, true, false); }
        else    { if (gr) TITAN_STAGED(true, false, true); else TITAN_STAGED(true, false, false); }
    } else {
        if (ha) { if (gr) TITAN_STAGED(false, true, true); else TITAN_STAGED(false, true, false); }
        else    { if (gr) TITAN_STAGED(false, false, true); else TITAN_STAGED(false, false, false); }
    }
#undef TITAN_STAGED
    return cudaGetLastError();
}

// Shared-memory carveout for a kernel whose CTAs each hold `bytes` of dynamic
// shared memory and of which `resident` fit an SM by registers: shared memory
// for those CTAs (each also holds 1 KB reserved by the system), the rest of the
// SM's unified L1 / shared memory left to L1, where the halo and state gathers
// then hit more often.  At least 50 %: with six 17 KB tables per SM that was
// measured 5 % faster than the largest shared carveout on the 1M-mass lattice.
// The carveout is a hint: the driver always gives a single CTA what it needs.
static int carveout_for(size_t bytes, int resident) {
    int dev = 0, max_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&max_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess || max_sm <= 0)
        return (int)cudaSharedmemCarveoutMaxShared;
    const size_t need = (size_t)resident * (bytes + 1024);
    return (int)std::min<size_t>(100, std::max<size_t>(50, (100 * need + (size_t)max_sm - 1) / (size_t)max_sm));
}

// The launch attributes of a step kernel: the L2 window (optional) and
// programmatic stream serialization (overlap).
static unsigned step_attrs(cudaLaunchAttribute *attr, const cudaAccessPolicyWindow *l2win, bool overlap) {
    unsigned k = 0;
    if (l2win) {
        attr[k].id = cudaLaunchAttributeAccessPolicyWindow;
        attr[k].val.accessPolicyWindow = *l2win;
        ++k;
    }
    if (overlap) {
        attr[k].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[k].val.programmaticStreamSerializationAllowed = 1;
        ++k;
    }
    return k;
}

cudaError_t launch_step_halo(const MassState *in, MassState *out, uint32_t n, const SellView &v,
                             const HaloView &h, const StepConst &c, const long long *step_in,
                             long long *step_out, cudaStream_t stream, const cudaAccessPolicyWindow *l2win,
                             bool overlap) {
    const bool hc = v.c != nullptr, ha = v.act != nullptr, gr = c.ground != 0;
    const unsigned g = n ? (n + kHaloThreads - 1) / kHaloThreads : 1;
    const size_t bytes = (size_t)h.table_slots * (sizeof(float4) + sizeof(float2));
    const int carveout = carveout_for(bytes, kHaloMinBlocks);
#define TITAN_HALO(HC, HA, GR)                                                                   \
    do {                                                                                         \
        auto kern = overlap ? k_step_halo<HC, HA, GR, true> : k_step_halo<HC, HA, GR, false>;   \
        if (bytes > 48 * 1024) {                                                                 \
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes); \
            if (e != cudaSuccess) return e;                                                      \
        }                                                                                        \
        {                                                                                        \
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, \
                                                 carveout);            \
            if (e != cudaSuccess) return e;                                                      \
        }                                                                                        \
        cudaLaunchConfig_t cfg = {};                                                             \
        cfg.gridDim = dim3(g);                                                                   \
        cfg.blockDim = dim3(kHaloThreads);                                                       \
        cfg.dynamicSmemBytes = bytes;                                                            \
        cfg.stream = stream;                                                                     \
        cudaLaunchAttribute attr[2];                                                             \
        cfg.attrs = attr;                                                                        \
        cfg.numAttrs = step_attrs(attr, l2win, overlap);                                         \
        cudaError_t e = cudaLaunchKernelEx(&cfg, kern, in, out, n, v.slice_off, h.nslot, v.kl, v.c, v.act, \
                                           h.own_slot, h.ext_off, h.ext_idx, h.ext_slot, h.table_slots, \
                                           h.ahead, c, step_in, step_out);                       \
        if (e != cudaSuccess) return e;                                                          \
    } while (0)
    if (hc) {
        if (ha) { if (gr) TITAN_HALO(true, true, true); else TITAN_HALO(true, true, false); }
        else    { if (gr) TITAN_HALO(true, false, true); else TITAN_HALO(true, false, false); }
    } else {
        if (ha) { if (gr) TITAN_HALO(false, true, true); else TITAN_HALO(false, true, false); }
        else    { if (gr) TITAN_HALO(false, false, true); else TITAN_HALO(false, false, false); }
    }
#undef TITAN_HALO
    return cudaGetLastError();
}

cudaError_t launch_step_box(const MassState *in, MassState *out, uint32_t n, const SellView &v, const BoxView &h,
                            const StepConst &c, const long long *step_in, long long *step_out,
                            cudaStream_t stream, const cudaAccessPolicyWindow *l2win, bool overlap) {
    const bool hc = v.c != nullptr, ha = v.act != nullptr, gr = c.ground != 0;
    const unsigned g = n ? (n + kHaloThreads - 1) / kHaloThreads : 1;
    const size_t bytes = (size_t)h.table_slots * (sizeof(float4) + sizeof(float2));
    if (reinterpret_cast<uintptr_t>(h.col_off) & 3) return cudaErrorInvalidValue;
    const int carveout = carveout_for(bytes, kBoxMinBlocks);
#define TITAN_BOX(HC, HA, GR)                                                                    \
    do {                                                                                         \
        auto kern = overlap ? k_step_box<HC, HA, GR, true> : k_step_box<HC, HA, GR, false>;     \
        if (bytes > 48 * 1024) {                                                                 \
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes); \
            if (e != cudaSuccess) return e;                                                      \
        }                                                                                        \
        {                                                                                        \
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, \
                                                 carveout);                                      \
            if (e != cudaSuccess) return e;                                                      \
        }                                                                                        \
        cudaLaunchConfig_t cfg = {};                                                             \
        cfg.gridDim = dim3(g);                                                                   \
        cfg.blockDim = dim3(kHaloThreads);                                                       \
        cfg.dynamicSmemBytes = bytes;                                                            \
        cfg.stream = stream;                                                                     \
        cudaLaunchAttribute attr[2];                                                             \
        cfg.attrs = attr;                                                                        \
        cfg.numAttrs = step_attrs(attr, l2win, overlap);                                         \
        cudaError_t e = cudaLaunchKernelEx(&cfg, kern, in, out, n, v.slice_off,                  \
                                           reinterpret_cast<const uint32_t *>(h.col_off), v.kl, v.c, v.act, \
                                           h.own_slot, h.ext_off, h.ext_idx, h.ext_slot, h.table_slots, c, \
                                           step_in, step_out);                                   \
        if (e != cudaSuccess) return e;                                                          \
    } while (0)
    if (hc) {
        if (ha) { if (gr) TITAN_BOX(true, true, true); else TITAN_BOX(true, true, false); }
        else    { if (gr) TITAN_BOX(true, false, true); else TITAN_BOX(true, false, false); }
    } else {
        if (ha) { if (gr) TITAN_BOX(false, true, true); else TITAN_BOX(false, true, false); }
        else    { if (gr) TITAN_BOX(false, false, true); else TITAN_BOX(false, false, false); }
    }
#undef TITAN_BOX
    return cudaGetLastError();
}

cudaError_t launch_step_halo_tma(const MassState *in, MassState *out, uint32_t n, const SellView &v,
                                 const HaloView &h, uint32_t w_max, const StepConst &c,
                                 const long long *step_in, long long *step_out, cudaStream_t stream) {
    const bool hc = v.c != nullptr, ha = v.act != nullptr, gr = c.ground != 0;
    const unsigned g = n ? (n + kHaloThreads - 1) / kHaloThreads : 1;
#define TITAN_HTMA(HC, HA, GR)                                                                   \
    do {                                                                                         \
        auto kern = k_step_halo_tma<HC, HA, GR>;                                                 \
        const size_t bytes = (size_t)3 * h.table_slots * sizeof(float2) +                         \
                             (size_t)(kHaloThreads / 32) * w_max * 32 * halo_entry_bytes<HC, HA>(); \
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes); \
        if (e != cudaSuccess) return e;                                                          \
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,           \
                                 (int)cudaSharedmemCarveoutMaxShared);                            \
        if (e != cudaSuccess) return e;                                                          \
        kern<<<g, kHaloThreads, bytes, stream>>>(in, out, n, v.slice_off, h.nslot, v.kl, v.c, v.act, \
                                                 h.own_slot, h.ext_off, h.ext_idx, h.ext_slot,   \
                                                 h.table_slots, w_max, c, step_in, step_out,     \
                                                 v.spin_limit, v.err);                           \
    } while (0)
    if (hc) {
        if (ha) { if (gr) TITAN_HTMA(true, true, true); else TITAN_HTMA(true, true, false); }
        else    { if (gr) TITAN_HTMA(true, false, true); else TITAN_HTMA(true, false, false); }
    } else {
        if (ha) { if (gr) TITAN_HTMA(false, true, true); else TITAN_HTMA(false, true, false); }
        else    { if (gr) TITAN_HTMA(false, false, true); else TITAN_HTMA(false, false, false); }
    }
#undef TITAN_HTMA
    return cudaGetLastError();
}

cudaError_t launch_step_cube(const MassState *in, MassState *out, uint32_t n, const CubeView &v, const BoxView &h,
                             const StepConst &c, const long long *step_in, long long *step_out, cudaStream_t stream,
                             const cudaAccessPolicyWindow *l2win) {
    if (n % kHaloThreads || (h.table_slots & 1)) return cudaErrorInvalidValue;
    const bool hc = v.c != nullptr, ha = v.act != nullptr, gr = c.ground != 0;
    const unsigned g = n ? n / kHaloThreads : 1;
    const size_t bytes = (size_t)h.table_slots * (sizeof(float4) + sizeof(float2)) + 2 * kHaloThreads * sizeof(float4);
#define TITAN_CUBE(HC, HA, GR)                                                                   \
    do {                                                                                         \
        auto kern = k_step_cube<HC, HA, GR>;                                                     \
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, \
                                             (int)cudaSharedmemCarveoutMaxShared);                \
        if (e != cudaSuccess) return e;                                                          \
        cudaLaunchConfig_t cfg = {};                                                             \
        cfg.gridDim = dim3(g);                                                                   \
        cfg.blockDim = dim3(kHaloThreads);                                                       \
        cfg.dynamicSmemBytes = bytes;                                                            \
        cfg.stream = stream;                                                                     \
        cudaLaunchAttribute attr[1];                                                             \
        if (l2win) {                                                                             \
            attr[0].id = cudaLaunchAttributeAccessPolicyWindow;                                  \
            attr[0].val.accessPolicyWindow = *l2win;                                             \
            cfg.attrs = attr;                                                                    \
            cfg.numAttrs = 1;                                                                    \
        }                                                                                        \
        e = cudaLaunchKernelEx(&cfg, kern, in, out, n, v.base, v.meta, v.kl, v.c, v.act, h.own_slot, \
                               h.ext_off, h.ext_idx, h.ext_slot, h.table_slots, c, step_in, step_out); \
        if (e != cudaSuccess) return e;                                                          \
    } while (0)
    if (hc) {
        if (ha) { if (gr) TITAN_CUBE(true, true, true); else TITAN_CUBE(true, true, false); }
        else    { if (gr) TITAN_CUBE(true, false, true); else TITAN_CUBE(true, false, false); }
    } else {
        if (ha) { if (gr) TITAN_CUBE(false, true, true); else TITAN_CUBE(false, true, false); }
        else    { if (gr) TITAN_CUBE(false, false, true); else TITAN_CUBE(false, false, false); }
    }
#undef TITAN_CUBE
    return cudaGetLastError();
}

size_t box_tma_smem_bytes(uint32_t table_slots, uint32_t w_max, bool has_c, bool has_act) {
    return (size_t)table_slots * (sizeof(float4) + sizeof(float2)) +
           (size_t)(kHaloThreads / 32) * w_max * 32 * (8 + (has_c ? 4 : 0) + (has_act ? 8 : 0));
}

cudaError_t launch_step_box_tma(const MassState *in, MassState *out, uint32_t n, const SellView &v,
                                const BoxView &h, uint32_t w_max, const StepConst &c, const long long *step_in,
                                long long *step_out, cudaStream_t stream) {
    const bool hc = v.c != nullptr, ha = v.act != nullptr, gr = c.ground != 0;
    const unsigned g = n ? (n + kHaloThreads - 1) / kHaloThreads : 1;
    const size_t bytes = box_tma_smem_bytes(h.table_slots, w_max, hc, ha);
    if (reinterpret_cast<uintptr_t>(h.col_off) & 3) return cudaErrorInvalidValue;
    // the tables end on a 16-byte boundary only if the float2 part has an even slot count
    if (h.table_slots & 1) return cudaErrorInvalidValue;
#define TITAN_BTMA(HC, HA, GR)                                                                   \
    do {                                                                                         \
        auto kern = k_step_box_tma<HC, HA, GR>;                                                  \
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes); \
        if (e != cudaSuccess) return e;                                                          \
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,           \
                                 (int)cudaSharedmemCarveoutMaxShared);                            \
        if (e != cudaSuccess) return e;                                                          \
        kern<<<g, kHaloThreads, bytes, stream>>>(in, out, n, v.slice_off,                        \
                                                 reinterpret_cast<const uint32_t *>(h.col_off), v.kl, v.c, \
                                                 v.act, h.own_slot, h.ext_off, h.ext_idx, h.ext_slot, \
                                                 h.table_slots, w_max, c, step_in, step_out,     \
                                                 v.spin_limit, v.err);                           \
    } while (0)
    if (hc) {
        if (ha) { if (gr) TITAN_BTMA(true, true, true); else TITAN_BTMA(true, true, false); }
        else    { if (gr) TITAN_BTMA(true, false, true); else TITAN_BTMA(true, false, false); }
    } else {
        if (ha) { if (gr) TITAN_BTMA(false, true, true); else TITAN_BTMA(false, true, false); }
        else    { if (gr) TITAN_BTMA(false, false, true); else TITAN_BTMA(false, false, false); }
    }
#undef TITAN_BTMA
    return cudaGetLastError();
}

size_t halo_tma_smem_bytes(uint32_t table_slots, uint32_t w_max, bool has_c, bool has_act) {
    return (size_t)3 * table_slots * sizeof(float2) +
           (size_t)(kHaloThreads / 32) * w_max * 32 * (10 + (has_c ? 4 : 0) + (has_act ? 8 : 0));
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

__global__ void k_patch_words(uint32_t *__restrict__ base, const uint32_t *__restrict__ idx,
                              const uint32_t *__restrict__ val, uint32_t n) {
    const uint32_t i = blockIdx.x * kThreads + threadIdx.x;
    if (i < n) base[idx[i]] = val[i];
}

cudaError_t launch_patch_words(uint32_t *base, const uint32_t *idx, const uint32_t *val, uint32_t n,
                               cudaStream_t stream) {
    if (!n) return cudaSuccess;
    k_patch_words<<<blocks_for(n), kThreads, 0, stream>>>(base, idx, val, n);
    return cudaGetLastError();
}

cudaError_t launch_unpermute(const MassState *state, const uint32_t *dev_of_caller, uint32_t n,
                             float *pos, float *vel, cudaStream_t stream) {
    if (!n) return cudaSuccess;
    k_unpermute<<<blocks_for(n), kThreads, 0, stream>>>(state, dev_of_caller, n, pos, vel);
    return cudaGetLastError();
}

}  // namespace titan
