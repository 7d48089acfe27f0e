// layout.h -- host-side builders of the device layouts (see layout.cpp).
#pragma once

#include <stdint.h>

#include <vector>

namespace titan {

// caller_of_dev[d] = caller index of the mass placed at device index d.
void morton_order(const double *pos, uint32_t n, std::vector<uint32_t> &caller_of_dev);

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

struct RecordsHost {
    std::vector<uint32_t> order;            // [S] record r holds caller spring order[r]
    std::vector<uint32_t> slot_of_spring;   // [S] inverse of order
};

void build_records(uint32_t s, const uint32_t *ends, const std::vector<uint32_t> &dev_of,
                   RecordsHost &out);

}  // namespace titan
