// sim_internal.h -- the titan_sim handle, shared by the translation units of
// the single-system path (runtime.cu, adjoint.cu).  GPU path only.
#pragma once

#include <atomic>
#include <string>
#include <vector>

#include "layout.h"
#include "titan.h"
#include "titan_internal.h"

using titan::MassState;

constexpr int kDefaultGraphChunk = 64;
constexpr int kGraphLevels = 8;
constexpr int kExactGraphs = 4;          // step counts with a graph of their own (least recently used replaced)
constexpr uint32_t kDefaultSpinLimit = 1u << 22;

// Everything a simulation owns; titan_sim adds the per-handle lock and error
// text.  A topology rebuild builds a fresh core and swaps it in, so the
// caller's handle stays valid.
struct SimCore {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t side = nullptr;       // snapshot device-to-host copies
    cudaStream_t capture = nullptr;    // graph capture
    uint32_t n = 0, s = 0;
    uint32_t n_dev = 0;                   // device slots (>= n: grid-tile order leaves holes)
    bool grid_order = false;
    int accumulate = TITAN_ACCUM_CSR;
    titan::StepConst c{};
    bool has_c = false, has_act = false;
    double dt = 0;

    std::vector<uint32_t> caller_of_dev, dev_of_caller;
    std::vector<float> inv_mass;          // caller order
    std::vector<float> k, rest, damp;     // caller spring order
    std::vector<float> act_amp, act_phase;
    titan::SellHost sell;
    titan::HaloHost halo;
    titan::BoxHost box;
    titan::CubeHost cube;
    titan::RecordsHost rec;
    int csr_kernel = 0;                   // resolved: 1 direct, 2 smem-staged, 3 bulk-prefetch, 4 halo, 5 halo+TMA,
                                          // 6 grid box, 7 grid box+TMA, 8 cube
    uint32_t halo_w_max = 0;              // staged columns per slice (halo+TMA kernel)
    uint32_t halo_ahead = 0;              // L2 prefetch distance in blocks (halo kernel)
    int exec_req = TITAN_EXEC_AUTO;       // params.exec
    bool l2_on = false;                   // the step kernels carry an L2 persistence window
    cudaAccessPolicyWindow l2win{};       // over both state buffers (one allocation)
    bool persistent = false;              // resolved: whole chunks of steps in one cluster launch
    titan::PersistPlan plan;
    uint16_t *d_pslot = nullptr;          // persistent kernel: neighbour slot per SELL entry
    uint32_t *d_phalo = nullptr;          // persistent kernel: halo list
    size_t phalo_cap = 0;

    MassState *state[2] = {nullptr, nullptr};
    long long *steps_dev = nullptr;       // [2]
    int cur = 0;
    uint64_t steps = 0;
    uint32_t *d_dev_of_caller = nullptr;

    uint32_t *d_slice_off = nullptr, *d_nbr = nullptr;
    uint16_t *d_nslot = nullptr, *d_own_slot = nullptr, *d_ext_slot = nullptr;
    uint32_t *d_ext_off = nullptr, *d_ext_idx = nullptr;   // halo or box tables (whichever kernel runs)
    int16_t *d_col_off = nullptr;         // box kernel: slot offset per SELL column
    uint32_t *d_cube_base = nullptr;      // cube kernel: stream start of each cube
    uint4 *d_cube_meta = nullptr;         //              per (cube, pass, warp) masks, ext base, offset
    float2 *d_ckl = nullptr, *d_cact = nullptr;   //      cube stream {k, L0}, actuation
    float *d_cc = nullptr;                //              cube stream damping
    float2 *d_kl = nullptr, *d_act = nullptr;
    float *d_c = nullptr;

    uint4 *d_rec = nullptr;
    float *d_rc = nullptr;
    float2 *d_ract = nullptr;
    float4 *d_force = nullptr;

    int graph_chunk = kDefaultGraphChunk;
    int kernel_variant = 0;
    bool launch_overlap = true;           // programmatic dependent launches of the step kernels
    uint32_t spin_limit = kDefaultSpinLimit;
    int *d_err = nullptr;                 // device error flag (bounded waits)
    // captured step loops: level L runs graph_chunk >> L steps (levels while
    // that count is even and >= 2), one graph per starting buffer
    cudaGraphExec_t graph[kGraphLevels][2] = {};
    bool graphs_built = false;
    // whole step counts that are not one ladder level (a caller stepping by a
    // fixed count, e.g. 20 = 16 + 4), captured on first use: one graph
    // replaces several, so one fewer step per call starts in plain order
    struct ExactGraph {
        uint64_t n = 0;
        int b = 0;
        uint64_t last_use = 0;
        cudaGraphExec_t exec = nullptr;
    };
    ExactGraph exact[kExactGraphs];
    uint64_t exact_clock = 0;

    // snapshots: slot = ticket & 1
    float *snap_dev[2] = {nullptr, nullptr};     // [2][n][3] pos then vel, caller order
    float *snap_host[2] = {nullptr, nullptr};    // pinned, same layout
    titan::MassState *state_stage = nullptr;     // pinned staging of titan_set_state ([n_dev])
    size_t state_stage_cap = 0;
    cudaEvent_t state_staged = nullptr;          // the staging buffer's last upload is done
    cudaEvent_t snap_ready[2] = {nullptr, nullptr};
    cudaEvent_t snap_done[2] = {nullptr, nullptr};
    double snap_t[2] = {0, 0};
    uint64_t last_ticket = 0;

    uint32_t *d_adj_spring = nullptr;     // adjoint: spring id per SELL entry (+ owner bit)
    uint32_t *d_adj_owner = nullptr;      // adjoint: owner SELL entry of each spring

    std::vector<void *> allocations;

    // host copies kept for topology edits (FP64, caller order)
    titan_params params{};
    std::vector<double> h_mass;
    std::vector<uint8_t> h_fixed;
    std::vector<uint32_t> h_ends;
    std::vector<double> h_k, h_rest, h_damp;
    bool dirty = false;                   // masses or springs were added: rebuild before next use
    std::vector<double> pend_pos, pend_vel;   // initial state of masses added since the last rebuild
    int act_mode = 0;                     // 0 none, 1 sinusoid, 2 worm (Eqs. 3-4)
    // actuation set from device arrays (titan_set_actuation_dev): the
    // caller-order values stay on the device, and act_amp / act_phase follow
    // them only when host code needs them (act_host_stale until then)
    float *d_act_amp = nullptr, *d_act_phase = nullptr;
    bool act_host_stale = false;
    uint32_t *d_entry_spring = nullptr;   // spring of each SELL entry (UINT32_MAX: padding)
    uint32_t *d_cube_spring = nullptr;    // spring of each cube-stream entry
    uint32_t *d_rec_spring = nullptr;     // spring of each record (atomic path)
    int *d_check = nullptr;               // non-finite count of the last device-array argument check
};

struct titan_sim : SimCore {
    std::string error;
    std::atomic<bool> busy{false};
};

namespace titan {
// Enqueues one fused step reading state buffer b of the simulation (runtime.cu).
// after_step: the operation just before it on st is this simulation's previous
// step kernel (only then may it start early, as a programmatic dependent).
cudaError_t enqueue_sim_step(titan_sim *sim, cudaStream_t st, int b, bool after_step);
// The same step kernel between caller-chosen buffers (adjoint recomputation).
cudaError_t enqueue_sim_step_io(titan_sim *sim, cudaStream_t st, const MassState *in, MassState *out,
                                const long long *step_in, long long *step_out, bool after_step);
void set_thread_error(const std::string &msg);
// Rebuilds the device layout if masses or springs were added (runtime.cu).
titan_status ensure_layout(titan_sim *sim);
}  // namespace titan
