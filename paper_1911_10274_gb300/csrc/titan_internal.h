// titan_internal.h -- device layouts and kernel launchers of libtitan (GPU path only).
//
// Device layout (all in HBM, cudaMalloc'd, 256-byte aligned):
//   MassState[n]  32 B per mass {x, y, z, 1/m | vx, vy, vz, 0}; one neighbour
//                 gather is one 32-byte L2 sector.  1/m == 0 marks a fixed mass.
//                 Two copies (ping-pong): step n reads one and writes the other.
//   SELL-32 incidence (deterministic gather, K1): masses are taken in slices of
//                 32 consecutive device indices; slice s holds W_s columns of 32
//                 half-edge entries (column-major, entry = off[s] + 32 t + lane),
//                 W_s = the slice's largest degree rounded up to even (on a grid:
//                 its number of offset-aligned columns, see layout.h).  Per
//                 entry: nbr (u32 device index) and {k, L0} (float2), optionally
//                 c (float) and actuation {A, phi} (float2).  Padding entries
//                 point at the mass itself with k = c = A = 0 and the rest
//                 length kPadRest (negative, so never a real spring's: rest
//                 lengths are >= 0).  Evaluated, a padding entry gives an exactly
//                 zero force (a zero-length spring has no axis); the grid
//                 kernels, whose padding may address an empty table slot, skip
//                 it by the sign of its rest length.
//   Spring records (atomic scatter, K2): {i, j, k, L0} as one uint4 (128-bit
//                 load), sorted by the lower device index, plus a float4 force
//                 accumulator per mass.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <vector>

namespace titan {

// Rest length stored in the {k, L0} of a padding entry.  Real springs have
// L0 >= 0 (zero is legal: a zero-rest-length spring pulls with k l), so a
// negative value marks padding unambiguously.
constexpr float kPadRest = -1.0f;

// Entries past the end of the SELL stream arrays ({k, L0}, c, actuation):
// padding a kernel may read ahead into, so that its loop needs no bounds test
// for the next column pair of the last slice.  The column-offset array of the
// grid-box kernels likewise carries one word past its end.
constexpr uint32_t kStreamTail = 64;

struct __align__(16) MassState {
    float4 p;   // x, y, z, 1/m (0: fixed)
    float4 v;   // vx, vy, vz, unused (0)
};
static_assert(sizeof(MassState) == 32, "MassState must be one 32-byte sector");

// Per-step constants shared by every kernel of one simulation.
struct StepConst {
    float dt;
    float gx, gy, gz;
    float ground_k;
    float mu;
    float c_uniform;      // dashpot when there is no per-spring damping array
    int32_t ground;
    double act_omega;     // 2 pi f (rad/s) of the sinusoidal actuation
    double dt_d;          // dt in FP64
    int32_t act_mode;     // 1: L0 (1 + A sin(2 pi f t + phi)); 2: worm, L0 (1 + c sin(w tau))
    float worm_omega;     // mode 2: w (rad/s)
    double worm_period;   // mode 2: t_p (s); per-spring offsets are stored reduced to [0, t_p)
    // the actuation clocks as fixed-point turns per step (fractional part, in
    // units of 2^-64): step x turns wraps modulo 2^64 exactly, so the phase
    // of any step costs one 64-bit integer product (no FP64 on the device)
    unsigned long long act_turns;    // mode 1: f dt
    unsigned long long worm_turns;   // mode 2: dt / t_p
    float worm_unit;                 // mode 2: t_p / 2^24 (s per clock unit)
};

// The fractional part of x (turns per step, x >= 0) in units of 2^-64.
inline unsigned long long turns_fraction(double x) {
    const double f = x - floor(x);
    const double q = ldexp(f, 64);
    return q >= 18446744073709549568.0 ? 0xFFFFFFFFFFFFF800ull : (unsigned long long)q;
}

// Sets the sinusoidal clock (mode 1) of c for frequency freq_hz.
inline void set_act_clock(StepConst &c, double freq_hz) {
    c.act_omega = 2.0 * 3.14159265358979323846 * freq_hz;
    c.act_turns = turns_fraction(freq_hz * c.dt_d);
}

// Sets the worm clock (mode 2) of c: w and t_p.
inline void set_worm_clock(StepConst &c, double omega, double period) {
    c.worm_omega = (float)omega;
    c.worm_period = period;
    c.worm_turns = turns_fraction(c.dt_d / period);
    c.worm_unit = (float)(period / 16777216.0);
}

struct SellView {
    const uint32_t *slice_off;   // [n_slices + 1] entry offsets
    const uint32_t *nbr;         // [E]
    const float2 *kl;            // [E] {k, L0}
    const float *c;              // [E] or nullptr (uniform c)
    const float2 *act;           // [E] {A, phi} or nullptr (no actuation)
    int variant;                 // 0: bulk L2 prefetch (default), 1: direct loads, 2: smem-staged
    uint32_t spin_limit;         // bound on mbarrier polls
    int *err;                    // set to 1 when a bounded wait expires
};

struct HaloView {
    const uint16_t *nslot;       // [E] neighbour slot in the block's table
    const uint16_t *own_slot;    // [n] slot of each mass in its block's table
    const uint32_t *ext_off;     // [n_blocks + 1]
    const uint32_t *ext_idx;     // external entries: device index
    const uint16_t *ext_slot;    //                   and slot
    uint32_t table_slots;        // slots per block table (shared memory = 24 B each)
    uint32_t ahead;              // blocks between a CTA and the block whose stream it prefetches
};

struct BoxView {
    const int16_t *col_off;      // [E / 32] slot offset per SELL column (4-byte aligned)
    const uint16_t *own_slot;    // [n] slot of each mass in its block's box
    const uint32_t *ext_off;     // [n_blocks + 1]
    const uint32_t *ext_idx;     // external entries: device index
    const uint16_t *ext_slot;    //                   and slot
    uint32_t table_slots;        // slots per box (shared memory = 24 B each)
};

struct CubeView {
    const uint32_t *base;        // [n_cubes + 1] first stream entry of each cube
    const uint4 *meta;           // [n_cubes][13][8]: recv mask, ext mask, ext base, +p slot offset
    const float2 *kl;            // cube stream {k, L0}
    const float *c;              // or nullptr (uniform c)
    const float2 *act;           // or nullptr (no actuation)
};

struct AtomicView {
    const uint4 *rec;            // [S] {i, j, bits(k), bits(L0)}
    const float *c;              // [S] or nullptr
    const float2 *act;           // [S] or nullptr
    float4 *force;               // [n] accumulators, zero between steps
    uint32_t n_springs;
};

// Step counters: steps[b] is the step index of the state in buffer b.  A step
// that reads buffer b writes steps[1 - b] = steps[b] + 1.
cudaError_t launch_step_sell(const MassState *in, MassState *out, uint32_t n, const SellView &v,
                             const StepConst &c, const long long *step_in, long long *step_out,
                             cudaStream_t stream);

// Halo form of the fused CSR step (see step_kernels.cu).
cudaError_t launch_step_halo(const MassState *in, MassState *out, uint32_t n, const SellView &v,
                             const HaloView &h, const StepConst &c, const long long *step_in,
                             long long *step_out, cudaStream_t stream,
                             const cudaAccessPolicyWindow *l2win = nullptr, bool overlap = false);

// Grid-box form of the halo kernel (see step_kernels.cu).  l2win (optional):
// an L2 access-policy window attached to the launch.  overlap: launched as a
// programmatic dependent of the previous kernel in the stream (its CTAs start
// early and wait for that kernel before reading the state).
cudaError_t launch_step_box(const MassState *in, MassState *out, uint32_t n, const SellView &v, const BoxView &h,
                            const StepConst &c, const long long *step_in, long long *step_out,
                            cudaStream_t stream, const cudaAccessPolicyWindow *l2win = nullptr,
                            bool overlap = false);

// Cube form (26-neighbourhood lattices): springs inside a block's cube read
// and evaluated once (see step_kernels.cu).  n a multiple of 256.
cudaError_t launch_step_cube(const MassState *in, MassState *out, uint32_t n, const CubeView &v, const BoxView &h,
                             const StepConst &c, const long long *step_in, long long *step_out, cudaStream_t stream,
                             const cudaAccessPolicyWindow *l2win = nullptr);

// Grid-box form with the stream staged into shared memory by TMA bulk copies;
// slices wider than w_max columns read from global memory.
cudaError_t launch_step_box_tma(const MassState *in, MassState *out, uint32_t n, const SellView &v,
                                const BoxView &h, uint32_t w_max, const StepConst &c, const long long *step_in,
                                long long *step_out, cudaStream_t stream);
size_t box_tma_smem_bytes(uint32_t table_slots, uint32_t w_max, bool has_c, bool has_act);

// Halo form with the half-edge stream staged into shared memory by TMA bulk
// copies; slices wider than w_max columns read from global memory.
cudaError_t launch_step_halo_tma(const MassState *in, MassState *out, uint32_t n, const SellView &v,
                                 const HaloView &h, uint32_t w_max, const StepConst &c,
                                 const long long *step_in, long long *step_out, cudaStream_t stream);
size_t halo_tma_smem_bytes(uint32_t table_slots, uint32_t w_max, bool has_c, bool has_act);

cudaError_t launch_step_atomic(const MassState *in, MassState *out, uint32_t n,
                               const AtomicView &v, const StepConst &c, const long long *step_in,
                               long long *step_out, cudaStream_t stream);

// The plan's scalars as the kernel receives them (by value).
struct PersistArgs {
    uint32_t cluster, per_cta, max_entries, max_halo;
    uint32_t halo_off[9];
};

// n_steps steps in one launch: reads `in`, writes `out` once at the end;
// step_out = step_in + n_steps.
struct PersistPlan;
cudaError_t launch_step_persistent(const MassState *in, MassState *out, uint32_t n, const PersistPlan &plan,
                                   const uint32_t *slice_off, const uint16_t *slot, const uint32_t *halo,
                                   const float2 *kl, const float *cc, const float2 *act, const StepConst &c,
                                   const long long *step_in, long long *step_out, uint32_t n_steps,
                                   cudaStream_t stream);

// base[idx[k]] = val[k] for 32-bit words (in-place parameter edits).
cudaError_t launch_patch_words(uint32_t *base, const uint32_t *idx, const uint32_t *val, uint32_t n,
                               cudaStream_t stream);

// Gathers device-order state into caller order: pos/vel [n][3] float.
cudaError_t launch_unpermute(const MassState *state, const uint32_t *dev_of_caller, uint32_t n,
                             float *pos, float *vel, cudaStream_t stream);

}  // namespace titan
