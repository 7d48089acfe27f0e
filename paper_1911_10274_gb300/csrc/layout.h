// layout.h -- host-side builders of the device layouts (see layout.cpp).
#pragma once

#include <stddef.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "titan.h"

namespace titan {

// caller_of_dev[d] = caller index of the mass placed at device index d.
void morton_order(const double *pos, uint32_t n, std::vector<uint32_t> &caller_of_dev);

// Grid-tile order for masses that sit on a cubic grid of pitch h (every
// coordinate within 1e-3 h of lo + integer x h, at most one mass per cell):
// cells are grouped in tiles of 4 x 4 x 2 and tiles in cubes of 2 x 2 x 2
// (8 x 8 x 4 cells); cubes are ordered along a Morton curve and each
// occupied cube gets 256 device slots, 32 per tile, so that a block of 256
// device masses is one cube.  The mass in cell (x, y, z) of a tile goes to lane
// (x & 3) + 4 (y & 3) + 16 (z & 1) of that tile's 32 slots.  Slots of empty
// cells are holes (caller_of_dev = UINT32_MAX).  Consequences used by the
// halo and box kernels: the 16 lanes of a half-warp are a 4 x 4 x 1 layer of
// cells, any translate of such a layer covers each value of (device index
// mod 16) once, and a block's box is 8 x 8 x 4 cells plus its halo.  Returns
// false (leaving the output empty) if the masses are not on such a grid.
// cell_of_dev (optional) receives the integer cell (x, y, z) of every device
// index, holes included, relative to the lowest occupied cell.
bool grid_tile_order(const double *pos, uint32_t n, double h, std::vector<uint32_t> &caller_of_dev,
                     std::vector<int32_t> *cell_of_dev = nullptr);

struct SellHost {
    std::vector<uint32_t> slice_off;      // [n_slices + 1]
    std::vector<uint32_t> nbr;            // [E] neighbour device index (self for padding)
    std::vector<uint32_t> spring;         // [E] caller spring index (UINT32_MAX for padding)
    std::vector<uint32_t> entry_of_end;   // [2 S] entry holding end 0 (i) / end 1 (j) of a spring
    uint32_t entries = 0;
};

// Returns false if the padded incidence does not fit 32-bit entry offsets.
// pos: caller-order positions [n][3], used only to order each row by direction.
// cell (optional, [n][3] per device index): grid cells; columns are then
// offset-aligned - every non-padding entry of a column of a slice points at
// the same cell offset - which the box kernel relies on.
bool build_sell(uint32_t n, uint32_t s, const uint32_t *ends, const double *pos,
                const std::vector<uint32_t> &dev_of, SellHost &out, const int32_t *cell = nullptr);

// Per-block neighbourhood tables for the halo kernel.  Block b is the CTA of
// kHaloBlock consecutive device masses; its table holds the state of every mass
// the block's half-edges touch (its own masses and the external "halo"), in
// shared memory, one slot each.  Slots are chosen by a greedy colouring so that
// the 16 lanes of each half-warp that gather in the same SELL column read
// distinct slots modulo 16 (no shared-memory bank conflicts for 8-byte loads)
// whenever the colouring finds such an assignment.
constexpr uint32_t kHaloBlock = 256;

struct HaloHost {
    std::vector<uint16_t> nbr_slot;      // [E] slot of the neighbour in its block's table
    std::vector<uint16_t> own_slot;      // [n] slot of each mass in its own block's table
    std::vector<uint32_t> ext_off;       // [n_blocks + 1] offsets into ext_idx / ext_slot
    std::vector<uint32_t> ext_idx;       // device index of each external table entry
    std::vector<uint16_t> ext_slot;      // its slot
    uint32_t max_table = 0;              // largest table (slots) over all blocks
    double conflict_ways = 0;            // mean wavefronts per half-warp 8-byte gather (1 = none)
};

// Builds the tables; returns false if some block's table exceeds max_slots.
// grid_colours: the device order is a grid-tile order, so (device index mod
// 16) is already a conflict-free colour; otherwise a greedy colouring is used.
bool build_halo(uint32_t n, const SellHost &sell, uint32_t max_slots, bool grid_colours, HaloHost &out);

// Box tables for the grid form of the halo kernel (masses in grid-tile order,
// SELL built with offset-aligned columns).  Block b's table covers the box of
// cells from its masses' lowest cell minus the largest spring offset to their
// highest cell plus it; the cell (x, y, z) has slot
// (x - x0) + X (y - y0) + X Y (z - z0), with the row length X padded to 4
// modulo 8 so that a quarter-warp (a 4 x 2 patch of cells) reads 16-byte
// entries in distinct banks and a half-warp (4 x 4) reads 8-byte entries in
// distinct banks.  A neighbour's slot is then the mass's own slot plus the
// column's offset, and the half-edge stream needs no neighbour index.
struct BoxHost {
    std::vector<int16_t> col_off;        // [E / 32] slot offset of every SELL column
    std::vector<uint16_t> own_slot;      // [n] (kBoxHole for holes)
    std::vector<uint32_t> ext_off;       // [n_blocks + 1]
    std::vector<uint32_t> ext_idx;       // device index of each external table entry
    std::vector<uint16_t> ext_slot;      // its slot
    std::vector<uint32_t> dims;          // [n_blocks][2] row length X and rows per layer Y of each box
    uint32_t max_table = 0;              // largest box (slots) over all blocks
};

// Returns false if some box exceeds max_slots or a column is not
// offset-aligned.  Checks that every entry's table read, padding included,
// stays inside its block's box.
// caller_of_dev marks holes (UINT32_MAX): they get own_slot = kBoxHole and
// no table slot; the box kernel neither reads nor writes their state.
constexpr uint16_t kBoxHole = 0xFFFF;
bool build_box(uint32_t n, const SellHost &sell, const std::vector<int32_t> &cell,
               const std::vector<uint32_t> &caller_of_dev, uint32_t max_slots, BoxHost &out);

// Cube-pair layout (the cube kernel; masses in grid order, 26-neighbourhood
// springs, at most one spring per mass and offset).  A block of 256 device
// masses is one cube of 8 x 8 x 4 cells; its step runs 13 passes, one per
// canonical direction p (kCubeDirs, the paired row order).  In pass j every
// mass evaluates its +p spring from the dense "plus" stream and publishes the
// force in shared memory; a mass whose -p partner is in the cube takes that
// force (negated) instead of evaluating the spring again, and one whose -p
// partner is outside reads the spring from the cube's compact "ext" stream.
// Springs inside a cube are thus read and evaluated once, and each mass still
// adds its forces in its row order (+p1, -p1, +p2, ...), so the result is
// bit-identical to the other CSR kernels.
constexpr int kCubeDirs[13][3] = {{1, 0, 0},  {-1, 1, 0}, {0, 1, 0},  {1, 1, 0},  {-1, -1, 1}, {0, -1, 1}, {1, -1, 1},
                                  {-1, 0, 1}, {0, 0, 1},  {1, 0, 1},  {-1, 1, 1}, {0, 1, 1},  {1, 1, 1}};
constexpr uint32_t kCubePasses = 13;

struct CubeHost {
    std::vector<uint32_t> base;       // [n_cubes + 1] first stream entry of each cube (plus, then ext)
    std::vector<uint32_t> meta;       // [n_cubes][13][8 warps][4]: recv mask, ext mask, ext base (from
                                      // the cube's ext start), box slot offset of +p (int16 in 32 bits)
    std::vector<uint32_t> spring;     // [entries] caller spring of each stream entry (UINT32_MAX: padding)
    std::vector<uint32_t> pos_of_end; // [2 S] stream entry of each spring end (UINT32_MAX: received)
    uint32_t entries = 0;
};

// Returns false unless every spring joins two masses of the grid at one of
// the 26 neighbour offsets, no mass has two springs with the same offset, and
// the blocks are cubes (grid order).  Needs the SELL (paired grid order) and
// the box tables of the same layout.
bool build_cube(uint32_t n, uint32_t s, const uint32_t *ends, const std::vector<uint32_t> &dev_of,
                const SellHost &sell, const std::vector<int32_t> &cell, const std::vector<uint32_t> &caller_of_dev,
                const BoxHost &box, CubeHost &out);

struct RecordsHost {
    std::vector<uint32_t> order;            // [S] record r holds caller spring order[r]
    std::vector<uint32_t> slot_of_spring;   // [S] inverse of order
};

void build_records(uint32_t s, const uint32_t *ends, const std::vector<uint32_t> &dev_of,
                   RecordsHost &out);

// ---- persistent execution of one small system (see persistent.cu)

#if defined(__CUDACC__)
#define TITAN_HD __host__ __device__
#else
#define TITAN_HD
#endif

// Shared memory of one CTA: two state buffers of (own + halo) slots, split
// (x, y, z, vx) / (vy, vz) for conflict-free 16- and 8-byte reads; 1/m of the
// own slots; the relative slice offsets and the rows (slot per entry, {k, L0},
// optional c and actuation).
struct PersistLayout {
    uint32_t a0, b0, a1, b1, inv, rel, kl, slot, cc, act, total;
};

TITAN_HD inline uint32_t al16(uint32_t x) { return (x + 15u) & ~15u; }

TITAN_HD inline PersistLayout persist_layout(uint32_t own, uint32_t halo, uint32_t entries, bool has_c,
                                                        bool has_act) {
    const uint32_t slots = own + halo;
    PersistLayout L;
    L.a0 = 0;
    L.b0 = L.a0 + slots * 16;
    L.a1 = al16(L.b0 + slots * 8);
    L.b1 = L.a1 + slots * 16;
    L.inv = al16(L.b1 + slots * 8);
    L.rel = al16(L.inv + own * 4);
    L.kl = al16(L.rel + 4 * (own / 32 + 1));
    L.act = L.kl + entries * 8;
    L.cc = L.act + (has_act ? entries * 8 : 0);
    L.slot = L.cc + (has_c ? entries * 4 : 0);
    L.total = al16(L.slot + entries * 2);
    return L;
}

// One cluster of `cluster` CTAs, CTA r owning device masses
// [r per_cta, (r + 1) per_cta) and a halo of other CTAs' masses,
// halo_off[r] .. halo_off[r + 1] in the halo list.
struct PersistPlan {
    uint32_t cluster = 0;       // CTAs (1, 2, 4 or 8)
    uint32_t per_cta = 0;       // masses per CTA (multiple of 32, <= 4096)
    uint32_t threads = 0;
    uint32_t max_entries = 0;   // largest SELL entry count of one CTA
    uint32_t max_halo = 0;      // largest halo of one CTA
    uint32_t halo_off[9] = {};
    size_t smem = 0;            // dynamic shared memory per CTA
};

size_t persistent_smem_bytes(uint32_t per_cta, uint32_t max_halo, uint32_t max_entries, bool has_c, bool has_act);

// Picks the smallest cluster whose CTAs fit smem_limit (preferring one mass
// per thread, 512 per CTA) and writes, per SELL entry, the neighbour's slot in
// its CTA's local table (own masses first, then the halo), and the halo list
// (rank << 16 | local slot in the owning CTA).  False if the system does not
// fit one cluster of 8.
bool plan_persistent(uint32_t n, const std::vector<uint32_t> &slice_off, const std::vector<uint32_t> &nbr,
                     bool has_c, bool has_act, size_t smem_limit, PersistPlan &plan,
                     std::vector<uint16_t> &slot, std::vector<uint32_t> &halo);

// ---- batches of independent systems (see batch.cu)
//
// Every system is owned by one thread-block cluster of C CTAs (C = 1, 2, 4 or
// 8, the smallest whose CTAs fit kBatchSmemLimit).  CTA q of a system owns its
// masses [q P, (q + 1) P) in caller order, P = ceil(n / C) rounded up to 32,
// at global state slots mass_begin .. mass_begin + P (slots past the system's
// last mass are padding: fixed, at rest).  The CTA's rows are SELL-32 over its
// P slots (slices of 32 masses, widths even, padding entries {k, L0} = {0, 0}
// pointing at the mass itself, or at the system's last mass for slots past
// it); each entry names its neighbour by a slot of the CTA's table: own
// masses at [0, P), other CTAs' masses - the halo - at [P, P + halo_count),
// halo entry h being (owner rank << 16 | owner slot).  A row keeps its
// springs in the order of (neighbour, spring) in caller numbering.

constexpr uint32_t kBatchMaxCluster = 8;
constexpr uint32_t kBatchMaxPerCta = 4096;          // masses per CTA
constexpr size_t kBatchSmemLimit = 220 * 1024;      // shared memory per CTA

// Per-CTA descriptor.  All offsets are in elements of the arrays they index.
struct BatchCta {
    uint32_t mass_begin;    // first global state slot of this CTA
    uint32_t mass_count;    // masses owned (<= kBatchMaxPerCta)
    uint32_t slot_count;    // P, a multiple of 32 (the same for every CTA of a system)
    uint32_t edge_off;      // first SELL entry (multiple of 64)
    uint32_t edge_count;    // SELL entries (multiple of 64)
    uint32_t slice_base;    // first relative slice offset (multiple of 4)
    uint32_t n_slices;      // P / 32
    uint32_t robot;         // system index
    uint32_t halo_off;      // first entry of this CTA's halo list
    uint32_t halo_count;    // masses of other CTAs of the cluster its rows touch
    uint32_t halo_slots;    // halo slots in the layout: the largest halo_count of the system's CTAs, so
                            // that every CTA of a cluster has its state buffers at the same offsets
};

// Shared-memory image of one CTA (byte offsets, all 16-byte aligned): two
// state buffers of (own + halo) slots split into (x, y, z, vx) float4 and
// (vy, vz) float2 arrays, 1/m of the own slots, the relative slice offsets,
// per entry {k, L0} - or, when the batch is actuated, {k, L0, A cos phi,
// A sin phi} (one 16-byte load) - then the slot per entry.  (`act` names the
// same offset as `kl`: the actuation pair is interleaved there.)
struct BatchSmem {
    uint32_t a0, b0, a1, b1, inv, slices, kl, act, nbr, total;
};

TITAN_HD inline BatchSmem batch_smem_layout(uint32_t slots, uint32_t halo, uint32_t n_slices, uint32_t edges,
                                            bool act) {
    const uint32_t tab = slots + halo;
    BatchSmem L;
    L.a0 = 0;
    L.b0 = L.a0 + tab * 16;
    L.a1 = al16(L.b0 + tab * 8);
    L.b1 = L.a1 + tab * 16;
    L.inv = al16(L.b1 + tab * 8);
    L.slices = al16(L.inv + slots * 4);
    L.kl = al16(L.slices + 4 * ((n_slices + 1 + 3) & ~3u));
    L.act = L.kl;
    L.nbr = L.kl + edges * (act ? 16 : 8);
    L.total = al16(L.nbr + edges * 2);
    return L;
}

// One launch: the CTAs [cta_first, cta_first + cta_count) of clusters of
// `cluster` CTAs, dynamic shared memory `smem` (the largest of its CTAs).
// Launches are split by cluster size and by shared-memory class (at most 1/k
// of an SM's 228 KB, k = 1, 2, 3, 4, 6, 8) so small systems share an SM.
struct BatchGroup {
    uint32_t cluster = 1;
    uint32_t cta_first = 0, cta_count = 0;
    size_t smem = 0;
};

struct BatchHost {
    std::vector<BatchCta> ctas;          // launch order: by group, systems in decreasing size within a group
    std::vector<BatchGroup> groups;
    std::vector<uint32_t> slices;        // relative slice offsets of every CTA (each run padded to 4)
    std::vector<float> kl;               // [E][2] {k, L0}
    std::vector<float> act;              // [E][2] {A cos phi, A sin phi} (empty if no system is actuated)
    std::vector<uint16_t> nbr;           // [E] table slot of the neighbour
    std::vector<uint32_t> halo;          // halo lists of every CTA
    std::vector<uint32_t> mass_off;      // [systems] first global state slot
    std::vector<uint32_t> mass_cnt;      // [systems] masses
    std::vector<float> init_state;       // [slots][8] x, y, z, 1/m, vx, vy, vz, 0 (FP32 of the caller's values)
    std::vector<uint32_t> mass_of_slot;  // [slots] caller index (within its system) of the mass in each slot,
                                         // UINT32_MAX for padding: each CTA holds its masses by decreasing
                                         // degree, so that its SELL slices hold rows of similar length
    uint32_t total_slots = 0;
    bool any_act = false;
};

// Builds the layout of n_systems validated systems (act may be null; act[r].amp
// null: system r is not actuated).  False, with the reason in *why, if a
// system fits no cluster of kBatchMaxCluster CTAs.
bool build_batch(uint32_t n_systems, const titan_masses *masses, const titan_springs *springs,
                 const titan_actuation *act, BatchHost &out, std::string *why);

}  // namespace titan
