// layout.h -- host-side builders of the device layouts (see layout.cpp).
#pragma once

#include <stdint.h>

#include <vector>

namespace titan {

// caller_of_dev[d] = caller index of the mass placed at device index d.
void morton_order(const double *pos, uint32_t n, std::vector<uint32_t> &caller_of_dev);

// Grid-tile order for masses that sit on a cubic grid of pitch h (every
// coordinate within 1e-3 h of lo + integer x h, at most one mass per cell):
// cells are grouped in tiles of 4 x 4 x 2, tiles are ordered along a Morton
// curve, and the mass in cell (x, y, z) of a tile goes to lane
// (x & 3) + 4 (y & 3) + 16 (z & 1) of that tile's 32 device slots.  Slots of
// empty cells are holes (caller_of_dev = UINT32_MAX).  Consequence used by the
// halo kernel: the 16 lanes of a half-warp are a 4 x 4 x 1 layer of cells, and
// any translate of such a layer covers each value of (device index mod 16)
// once.  Returns false (leaving the output empty) if the masses are not on
// such a grid.
bool grid_tile_order(const double *pos, uint32_t n, double h, std::vector<uint32_t> &caller_of_dev);

struct SellHost {
    std::vector<uint32_t> slice_off;      // [n_slices + 1]
    std::vector<uint32_t> nbr;            // [E] neighbour device index (self for padding)
    std::vector<uint32_t> spring;         // [E] caller spring index (UINT32_MAX for padding)
    std::vector<uint32_t> entry_of_end;   // [2 S] entry holding end 0 (i) / end 1 (j) of a spring
    uint32_t entries = 0;
};

// Returns false if the padded incidence does not fit 32-bit entry offsets.
// pos: caller-order positions [n][3], used only to order each row by direction.
bool build_sell(uint32_t n, uint32_t s, const uint32_t *ends, const double *pos,
                const std::vector<uint32_t> &dev_of, SellHost &out);

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

struct RecordsHost {
    std::vector<uint32_t> order;            // [S] record r holds caller spring order[r]
    std::vector<uint32_t> slot_of_spring;   // [S] inverse of order
};

void build_records(uint32_t s, const uint32_t *ends, const std::vector<uint32_t> &dev_of,
                   RecordsHost &out);

}  // namespace titan
