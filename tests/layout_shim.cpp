// layout_shim.cpp -- exposes the library's host-side layout builders
// (paper_1911_10274_gb300/csrc/layout.cpp: single-system tables, the
// persistent plan and the batch layout) through a C interface so that the
// CPU tests can check the device layouts without a GPU.  Test infrastructure:
// compiled by tests/test_layout_host.py together with layout.cpp.
#include <cstring>
#include <string>
#include <vector>

#include "layout.h"

namespace {
struct Built {
    std::vector<uint32_t> caller_of_dev, dev_of_caller;
    std::vector<int32_t> cell;
    titan::SellHost sell;
    titan::HaloHost halo;
    titan::BoxHost box;
    titan::CubeHost cube;
    int cube_ok = 0;
    titan::PersistPlan plan;
    std::vector<uint16_t> pslot;
    std::vector<uint32_t> phalo;
    int grid = 0, box_ok = 0, halo_ok = 0, plan_ok = 0;
} g;

template <typename T>
void copy_out(const std::vector<T> &v, void *dst) {
    if (!v.empty()) std::memcpy(dst, v.data(), v.size() * sizeof(T));
}
}  // namespace

extern "C" {

// Orders the masses as titan_create does (grid-tile order on a grid of pitch
// h, else Morton), builds the SELL incidence and both neighbourhood tables.
// Returns 0 on success, 1 if the SELL could not be built.
int shim_build(const double *pos, uint32_t n, const uint32_t *ends, uint32_t s, double h, uint32_t max_slots) {
    g = Built();
    g.grid = titan::grid_tile_order(pos, n, h, g.caller_of_dev, &g.cell) ? 1 : 0;
    if (!g.grid) titan::morton_order(pos, n, g.caller_of_dev);
    const uint32_t nd = (uint32_t)g.caller_of_dev.size();
    g.dev_of_caller.assign(n, 0);
    for (uint32_t d = 0; d < nd; ++d)
        if (g.caller_of_dev[d] != UINT32_MAX) g.dev_of_caller[g.caller_of_dev[d]] = d;
    if (!titan::build_sell(nd, s, ends, pos, g.dev_of_caller, g.sell, g.grid ? g.cell.data() : nullptr)) return 1;
    g.halo_ok = titan::build_halo(nd, g.sell, max_slots, g.grid != 0, g.halo) ? 1 : 0;
    g.box_ok = g.grid && titan::build_box(nd, g.sell, g.cell, g.caller_of_dev, max_slots, g.box) ? 1 : 0;
    g.cube_ok = g.box_ok && titan::build_cube(nd, s, ends, g.dev_of_caller, g.sell, g.cell, g.caller_of_dev, g.box,
                                              g.cube) ? 1 : 0;
    return 0;
}

// Plans persistent execution of the last built layout within smem_limit
// bytes per CTA.  Returns 1 if it fits one cluster.
int shim_plan(uint64_t smem_limit, int has_c, int has_act) {
    g.plan_ok = titan::plan_persistent((uint32_t)g.caller_of_dev.size(), g.sell.slice_off, g.sell.nbr, has_c != 0,
                                       has_act != 0, (size_t)smem_limit, g.plan, g.pslot, g.phalo) ? 1 : 0;
    return g.plan_ok;
}

// Plan scalars: 0 cluster, 1 per_cta, 2 threads, 3 max_entries, 4 max_halo, 5 smem, 10 + r: halo_off[r].
uint64_t shim_plan_scalar(int which) {
    switch (which) {
        case 0: return g.plan.cluster;
        case 1: return g.plan.per_cta;
        case 2: return g.plan.threads;
        case 3: return g.plan.max_entries;
        case 4: return g.plan.max_halo;
        case 5: return g.plan.smem;
        default: return (which >= 10 && which < 19) ? g.plan.halo_off[which - 10] : 0;
    }
}

// Scalars: 0 n_dev, 1 entries, 2 grid, 3 box_ok, 4 halo_ok, 5 box max_table, 6 halo max_table,
// 7 cube_ok, 8 cube stream entries.
uint64_t shim_scalar(int which) {
    switch (which) {
        case 0: return g.caller_of_dev.size();
        case 1: return g.sell.entries;
        case 2: return (uint64_t)g.grid;
        case 3: return (uint64_t)g.box_ok;
        case 4: return (uint64_t)g.halo_ok;
        case 5: return g.box.max_table;
        case 6: return g.halo.max_table;
        case 7: return (uint64_t)g.cube_ok;
        case 8: return g.cube.entries;
        default: return 0;
    }
}

// Array lengths and copies, by name.
uint64_t shim_len(const char *name) {
    const std::string k(name);
    if (k == "caller_of_dev") return g.caller_of_dev.size();
    if (k == "cell") return g.cell.size();
    if (k == "slice_off") return g.sell.slice_off.size();
    if (k == "nbr") return g.sell.nbr.size();
    if (k == "spring") return g.sell.spring.size();
    if (k == "entry_of_end") return g.sell.entry_of_end.size();
    if (k == "col_off") return g.box.col_off.size();
    if (k == "box_own_slot") return g.box.own_slot.size();
    if (k == "box_ext_off") return g.box.ext_off.size();
    if (k == "box_ext_idx") return g.box.ext_idx.size();
    if (k == "box_ext_slot") return g.box.ext_slot.size();
    if (k == "cube_base") return g.cube.base.size();
    if (k == "cube_meta") return g.cube.meta.size();
    if (k == "cube_spring") return g.cube.spring.size();
    if (k == "cube_pos_of_end") return g.cube.pos_of_end.size();
    if (k == "box_dims") return g.box.dims.size();
    if (k == "pslot") return g.pslot.size();
    if (k == "phalo") return g.phalo.size();
    return 0;
}

void shim_get(const char *name, void *dst) {
    const std::string k(name);
    if (k == "caller_of_dev") copy_out(g.caller_of_dev, dst);
    if (k == "cell") copy_out(g.cell, dst);
    if (k == "slice_off") copy_out(g.sell.slice_off, dst);
    if (k == "nbr") copy_out(g.sell.nbr, dst);
    if (k == "spring") copy_out(g.sell.spring, dst);
    if (k == "entry_of_end") copy_out(g.sell.entry_of_end, dst);
    if (k == "col_off") copy_out(g.box.col_off, dst);
    if (k == "box_own_slot") copy_out(g.box.own_slot, dst);
    if (k == "box_ext_off") copy_out(g.box.ext_off, dst);
    if (k == "box_ext_idx") copy_out(g.box.ext_idx, dst);
    if (k == "box_ext_slot") copy_out(g.box.ext_slot, dst);
    if (k == "cube_base") copy_out(g.cube.base, dst);
    if (k == "cube_meta") copy_out(g.cube.meta, dst);
    if (k == "cube_spring") copy_out(g.cube.spring, dst);
    if (k == "cube_pos_of_end") copy_out(g.cube.pos_of_end, dst);
    if (k == "box_dims") copy_out(g.box.dims, dst);
    if (k == "pslot") copy_out(g.pslot, dst);
    if (k == "phalo") copy_out(g.phalo, dst);
}

// Spring records of the atomic path for the last built ordering: order[r] is
// the caller spring held by record r, slot[q] the record of caller spring q.
void shim_records(uint32_t s, const uint32_t *ends, uint32_t *order, uint32_t *slot) {
    titan::RecordsHost rec;
    titan::build_records(s, ends, g.dev_of_caller, rec);
    copy_out(rec.order, order);
    copy_out(rec.slot_of_spring, slot);
}

// ---- batch layout (titan_batch_create's host part)

namespace {
titan::BatchHost bh;
std::string bwhy;
}  // namespace

// Builds the batch layout of n systems.  Returns 1 on success, 0 if refused
// (reason: shim_batch_why).
int shim_build_batch(uint32_t n, const titan_masses *m, const titan_springs *s, const titan_actuation *a) {
    bwhy.clear();
    return titan::build_batch(n, m, s, a, bh, &bwhy) ? 1 : 0;
}

const char *shim_batch_why() { return bwhy.c_str(); }

// 0 total_slots, 1 any_act, 2 CTAs, 3 groups.
uint64_t shim_batch_scalar(int which) {
    switch (which) {
        case 0: return bh.total_slots;
        case 1: return bh.any_act ? 1 : 0;
        case 2: return bh.ctas.size();
        case 3: return bh.groups.size();
        default: return 0;
    }
}

// Shared memory of one CTA image (the kernel's own formula).
uint64_t shim_batch_smem(uint32_t slots, uint32_t halo, uint32_t n_slices, uint32_t edges, int act) {
    return titan::batch_smem_layout(slots, halo, n_slices, edges, act != 0).total;
}

// Arrays: "ctas" as 11 uint32 per CTA (BatchCta field order), "groups" as 4
// uint64 per group (cluster, cta_first, cta_count, smem), then slices, kl,
// act, nbr, halo, mass_off, mass_cnt, init_state, mass_of_slot as stored.
uint64_t shim_batch_len(const char *name) {
    const std::string k(name);
    if (k == "ctas") return bh.ctas.size() * 11;
    if (k == "groups") return bh.groups.size() * 4;
    if (k == "slices") return bh.slices.size();
    if (k == "kl") return bh.kl.size();
    if (k == "act") return bh.act.size();
    if (k == "nbr") return bh.nbr.size();
    if (k == "halo") return bh.halo.size();
    if (k == "mass_off") return bh.mass_off.size();
    if (k == "mass_cnt") return bh.mass_cnt.size();
    if (k == "init_state") return bh.init_state.size();
    if (k == "mass_of_slot") return bh.mass_of_slot.size();
    return 0;
}

void shim_batch_get(const char *name, void *dst) {
    const std::string k(name);
    static_assert(sizeof(titan::BatchCta) == 11 * sizeof(uint32_t), "BatchCta is 11 words");
    if (k == "ctas") copy_out(bh.ctas, dst);
    if (k == "groups") {
        uint64_t *o = static_cast<uint64_t *>(dst);
        for (size_t g = 0; g < bh.groups.size(); ++g) {
            o[4 * g] = bh.groups[g].cluster;
            o[4 * g + 1] = bh.groups[g].cta_first;
            o[4 * g + 2] = bh.groups[g].cta_count;
            o[4 * g + 3] = bh.groups[g].smem;
        }
    }
    if (k == "slices") copy_out(bh.slices, dst);
    if (k == "kl") copy_out(bh.kl, dst);
    if (k == "act") copy_out(bh.act, dst);
    if (k == "nbr") copy_out(bh.nbr, dst);
    if (k == "halo") copy_out(bh.halo, dst);
    if (k == "mass_off") copy_out(bh.mass_off, dst);
    if (k == "mass_cnt") copy_out(bh.mass_cnt, dst);
    if (k == "init_state") copy_out(bh.init_state, dst);
    if (k == "mass_of_slot") copy_out(bh.mass_of_slot, dst);
}

}  // extern "C"
