// layout.cpp -- host-side construction of the device layouts (run once per titan_create,
// and once per titan_batch_create for the batch layout at the end).
//
// Morton order: masses are sorted by the 63-bit Morton code of their position
// quantised to 2^21 cells per axis over the bounding cube, so that masses that
// are close in space get close device indices and the neighbour gathers of one
// warp fall in a few cache lines.
// SELL-32 incidence: per mass, its incident half-edges in a fixed order (which
// makes the force sum deterministic), stored column-major per slice of 32
// masses.  The order is by the direction class of the spring seen from the
// mass (each component of the initial unit vector rounded to -1/0/+1, 26
// classes), then by neighbour index: in a lattice, column t of a slice is then
// the same lattice direction for every interior mass, so the 32 neighbour
// gathers of one column hit a compact, shifted block of consecutive states
// (few cache lines) instead of 32 unrelated ones.  On a grid the order is by
// exact cell offset and the columns are offset-aligned (see build_sell).
// Grid order, box tables and the persistent plan: see layout.h.
// Spring records: one {i, j, k, L0} record per spring, sorted by (lower,
// higher) device index, for the atomic scatter.
#include "layout.h"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <climits>
#include <numeric>
#include <string>
#include <utility>

namespace titan {

namespace {
// Spreads the low 21 bits of x so that bit b moves to bit 3b.
inline uint64_t spread_bits3(uint64_t x) {
    x &= 0x1fffffULL;
    x = (x | (x << 32)) & 0x1f00000000ffffULL;
    x = (x | (x << 16)) & 0x1f0000ff0000ffULL;
    x = (x | (x << 8)) & 0x100f00f00f00f00fULL;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ULL;
    x = (x | (x << 2)) & 0x1249249249249249ULL;
    return x;
}
}  // namespace

void morton_order(const double *pos, uint32_t n, std::vector<uint32_t> &caller_of_dev) {
    caller_of_dev.resize(n);
    if (n == 0) return;
    double lo[3] = {pos[0], pos[1], pos[2]}, hi[3] = {pos[0], pos[1], pos[2]};
    for (uint32_t i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], pos[3 * (size_t)i + a]);
            hi[a] = std::max(hi[a], pos[3 * (size_t)i + a]);
        }
    double ext = std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
    const double scale = ext > 0 ? (double)((1u << 21) - 1) / ext : 0.0;
    std::vector<std::pair<uint64_t, uint32_t>> key(n);
    for (uint32_t i = 0; i < n; ++i) {
        uint64_t code = 0;
        for (int a = 0; a < 3; ++a) {
            double q = std::floor((pos[3 * (size_t)i + a] - lo[a]) * scale);
            uint64_t c = q < 0 ? 0 : (q > (double)((1u << 21) - 1) ? (1u << 21) - 1 : (uint64_t)q);
            code |= spread_bits3(c) << a;
        }
        key[i] = {code, i};
    }
    std::sort(key.begin(), key.end());
    for (uint32_t d = 0; d < n; ++d) caller_of_dev[d] = key[d].second;
}

bool grid_tile_order(const double *pos, uint32_t n, double h, std::vector<uint32_t> &caller_of_dev,
                     std::vector<int32_t> *cell_of_dev) {
    caller_of_dev.clear();
    if (cell_of_dev) cell_of_dev->clear();
    if (n == 0 || !(h > 0) || !std::isfinite(h)) return false;
    double lo[3] = {pos[0], pos[1], pos[2]};
    for (uint32_t i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) lo[a] = std::min(lo[a], pos[3 * (size_t)i + a]);
    // cube = 2 x 2 x 2 tiles = 8 x 8 x 4 cells = 256 device slots
    struct Key { uint64_t cube; uint32_t slot, idx; };
    std::vector<Key> key(n);
    for (uint32_t i = 0; i < n; ++i) {
        uint64_t c[3];
        for (int a = 0; a < 3; ++a) {
            const double q = (pos[3 * (size_t)i + a] - lo[a]) / h;
            const double r = std::nearbyint(q);
            if (std::fabs(q - r) > 1e-3 || r > (double)((1u << 22) - 1)) return false;
            c[a] = (uint64_t)r;
        }
        const uint64_t cube = spread_bits3(c[0] >> 3) | (spread_bits3(c[1] >> 3) << 1) | (spread_bits3(c[2] >> 2) << 2);
        const uint32_t tile = (uint32_t)(((c[0] >> 2) & 1) | (((c[1] >> 2) & 1) << 1) | (((c[2] >> 1) & 1) << 2));
        const uint32_t lane = (uint32_t)((c[0] & 3) + 4 * (c[1] & 3) + 16 * (c[2] & 1));
        key[i] = {cube, 32 * tile + lane, i};
    }
    std::sort(key.begin(), key.end(), [](const Key &a, const Key &b) {
        return a.cube != b.cube ? a.cube < b.cube : (a.slot != b.slot ? a.slot < b.slot : a.idx < b.idx);
    });
    uint64_t cubes = 0;
    for (uint32_t k = 0; k < n; ++k) {
        if (k && key[k].cube == key[k - 1].cube && key[k].slot == key[k - 1].slot) return false;  // shared cell
        if (k == 0 || key[k].cube != key[k - 1].cube) ++cubes;
    }
    if (cubes * 256 >= (1ull << 31)) return false;
    caller_of_dev.assign(cubes * 256, UINT32_MAX);
    if (cell_of_dev) cell_of_dev->assign(cubes * 256 * 3, 0);
    uint64_t t = 0;
    for (uint32_t k = 0; k < n; ++k) {
        const bool first = k == 0 || key[k].cube != key[k - 1].cube;
        if (k && first) ++t;
        caller_of_dev[t * 256 + key[k].slot] = key[k].idx;
        if (cell_of_dev && first) {
            // every slot of the cube (holes included) gets its cell: cube origin + tile + lane offsets
            int32_t o[3];
            for (int a = 0; a < 3; ++a) {
                const double q = std::nearbyint((pos[3 * (size_t)key[k].idx + a] - lo[a]) / h);
                o[a] = (int32_t)q & ~(a == 2 ? 3 : 7);
            }
            for (uint32_t sl = 0; sl < 256; ++sl) {
                const uint32_t tile = sl >> 5, l = sl & 31;
                int32_t *c = cell_of_dev->data() + 3 * (t * 256 + sl);
                c[0] = o[0] + 4 * (int32_t)(tile & 1) + (int32_t)(l & 3);
                c[1] = o[1] + 4 * (int32_t)((tile >> 1) & 1) + (int32_t)((l >> 2) & 3);
                c[2] = o[2] + 2 * (int32_t)((tile >> 2) & 1) + (int32_t)(l >> 4);
            }
        }
    }
    return true;
}

namespace {
// Direction class 0..26 of d (13 for a zero vector): each component of d/|d|
// mapped to 0/1/2 for below -0.38 / within / above +0.38.
uint32_t direction_class(const double *a, const double *b) {
    const double d[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    const double l = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (!(l > 0)) return 13;
    uint32_t c = 0, m = 1;
    for (int k = 0; k < 3; ++k, m *= 3) {
        const double u = d[k] / l;
        c += m * (u > 0.38 ? 2u : (u < -0.38 ? 0u : 1u));
    }
    return c;
}
}  // namespace

bool build_sell(uint32_t n, uint32_t s, const uint32_t *ends, const double *pos,
                const std::vector<uint32_t> &dev_of, SellHost &out, const int32_t *cell) {
    const uint32_t n_slices = (n + 31) / 32;
    std::vector<uint32_t> deg(n, 0);
    for (uint32_t q = 0; q < s; ++q) {
        ++deg[dev_of[ends[2 * (size_t)q]]];
        ++deg[dev_of[ends[2 * (size_t)q + 1]]];
    }
    std::vector<uint64_t> rowptr(n + 1, 0);
    for (uint32_t i = 0; i < n; ++i) rowptr[i + 1] = rowptr[i] + deg[i];
    // half-edge = (order key, neighbour device index, spring index).  The key
    // is the direction class; on a grid it also holds the exact cell offset
    // of the neighbour (10 bits per component, clamped to +-511: equal keys
    // mean equal offsets for every offset within that range; the box builder
    // checks the columns anyway).
    struct HalfEdge { uint64_t key; uint32_t nbr, spring; };
    std::vector<HalfEdge> he(rowptr[n]);
    std::vector<uint64_t> cur(rowptr.begin(), rowptr.end() - 1);
    // On a grid the order pairs each offset with its opposite: the canonical
    // ("positive") member p of {o, -o} ranks the pair (by its direction class,
    // then its code), and within the pair +p precedes -p.  A row then reads
    // +p1, -p1, +p2, -p2, ...: the order in which the cube kernel receives the
    // -p force of an in-cube spring from the mass that computed it as +p.
    auto paired_key = [&](uint32_t from, uint32_t to) -> uint64_t {
        int64_t d[3];
        for (int a = 0; a < 3; ++a) d[a] = (int64_t)cell[3 * (size_t)to + a] - (int64_t)cell[3 * (size_t)from + a];
        const bool positive = d[2] > 0 || (d[2] == 0 && (d[1] > 0 || (d[1] == 0 && d[0] > 0)));
        if (!positive)
            for (int a = 0; a < 3; ++a) d[a] = -d[a];
        uint64_t cls = 0, code = 0;
        for (int a = 2; a >= 0; --a) cls = 3 * cls + (uint64_t)(d[a] > 0 ? 2 : (d[a] < 0 ? 0 : 1));
        for (int a = 0; a < 3; ++a) {
            const int64_t c = std::min<int64_t>(511, std::max<int64_t>(-512, d[a]));
            code = (code << 10) | (uint64_t)(c + 512);
        }
        return (((cls << 30) | code) << 1) | (positive ? 0u : 1u);
    };
    for (uint32_t q = 0; q < s; ++q) {
        const uint32_t ci = ends[2 * (size_t)q], cj = ends[2 * (size_t)q + 1];
        const uint32_t a = dev_of[ci], b = dev_of[cj];
        const uint32_t kab = direction_class(pos + 3 * (size_t)ci, pos + 3 * (size_t)cj);
        uint64_t ka = (uint64_t)kab << 32, kb = (uint64_t)(26u - kab) << 32;   // opposite direction
        if (cell) {
            ka = paired_key(a, b);
            kb = paired_key(b, a);
        }
        he[cur[a]++] = {ka, b, q};
        he[cur[b]++] = {kb, a, q};
    }
    for (uint32_t i = 0; i < n; ++i)
        std::sort(he.begin() + rowptr[i], he.begin() + rowptr[i + 1],
                  [](const HalfEdge &x, const HalfEdge &y) {
                      if (x.key != y.key) return x.key < y.key;
                      return x.nbr != y.nbr ? x.nbr < y.nbr : x.spring < y.spring;
                  });
    // Column of every half-edge within its slice.  Default: its position in
    // the row.  On a grid: one run of columns per distinct key of the slice
    // (as many as the most any lane has), so that every entry of a column has
    // the same cell offset and lanes lacking that offset hold padding.
    std::vector<uint32_t> col(rowptr[n]);
    out.slice_off.assign(n_slices + 1, 0);
    uint64_t total = 0;
    std::vector<std::pair<uint64_t, uint32_t>> runs;
    for (uint32_t sl = 0; sl < n_slices; ++sl) {
        const uint32_t l_end = std::min<uint32_t>(32, n - sl * 32);
        uint32_t w = 0;
        if (!cell) {
            for (uint32_t l = 0; l < l_end; ++l) {
                const uint32_t i = sl * 32 + l;
                w = std::max(w, deg[i]);
                for (uint32_t t = 0; t < deg[i]; ++t) col[rowptr[i] + t] = t;
            }
        } else {
            runs.clear();
            for (uint32_t l = 0; l < l_end; ++l) {
                const uint32_t i = sl * 32 + l;
                for (uint64_t r = rowptr[i]; r < rowptr[i + 1];) {
                    uint64_t r2 = r;
                    while (r2 < rowptr[i + 1] && he[r2].key == he[r].key) ++r2;
                    runs.push_back({he[r].key, (uint32_t)(r2 - r)});
                    r = r2;
                }
            }
            std::sort(runs.begin(), runs.end());
            // keep, per key, the longest run; then the column where each key starts
            std::vector<std::pair<uint64_t, uint32_t>> start;
            for (size_t k = 0; k < runs.size(); ++k)
                if (k + 1 == runs.size() || runs[k + 1].first != runs[k].first) {
                    start.push_back({runs[k].first, w});
                    w += runs[k].second;
                }
            for (uint32_t l = 0; l < l_end; ++l) {
                const uint32_t i = sl * 32 + l;
                for (uint64_t r = rowptr[i]; r < rowptr[i + 1];) {
                    const uint64_t key = he[r].key;
                    const auto it = std::lower_bound(start.begin(), start.end(), std::make_pair(key, 0u));
                    uint32_t c = it->second;
                    for (; r < rowptr[i + 1] && he[r].key == key; ++r) col[r] = c++;
                }
            }
        }
        w = (w + 1) & ~1u;
        total += (uint64_t)w * 32;
        if (total > 0xffffffffULL) return false;
        out.slice_off[sl + 1] = (uint32_t)total;
    }
    out.entries = (uint32_t)total;
    out.nbr.assign(total, 0);
    out.spring.assign(total, UINT32_MAX);
    out.entry_of_end.assign(2 * (size_t)s, 0);
    for (uint32_t sl = 0; sl < n_slices; ++sl) {
        const uint32_t w = (out.slice_off[sl + 1] - out.slice_off[sl]) / 32;
        for (uint32_t l = 0; l < 32; ++l) {
            const uint32_t i = sl * 32 + l;
            for (uint32_t t = 0; t < w; ++t)        // padding: a zero-length spring to itself
                out.nbr[out.slice_off[sl] + 32ull * t + l] = i < n ? i : 0;
            if (i >= n) continue;
            for (uint64_t r = rowptr[i]; r < rowptr[i + 1]; ++r) {
                const HalfEdge &h = he[r];
                const uint64_t e = out.slice_off[sl] + 32ull * col[r] + l;
                out.nbr[e] = h.nbr;
                out.spring[e] = h.spring;
                // which end of spring h.spring this row is
                const uint32_t end0 = dev_of[ends[2 * (size_t)h.spring]];
                const bool is_i = (end0 == i) && !(end0 == h.nbr);
                out.entry_of_end[2 * (size_t)h.spring + (is_i ? 0 : 1)] = (uint32_t)e;
            }
        }
    }
    return true;
}

bool build_halo(uint32_t n, const SellHost &sell, uint32_t max_slots, bool grid_colours, HaloHost &out) {
    const uint32_t n_blocks = (n + kHaloBlock - 1) / kHaloBlock;
    const uint32_t slices_per_block = kHaloBlock / 32;
    const uint32_t n_slices = (n + 31) / 32;
    out.nbr_slot.assign(sell.entries, 0);
    out.own_slot.assign(n, 0);
    out.ext_off.assign(n_blocks + 1, 0);
    out.ext_idx.clear();
    out.ext_slot.clear();
    out.max_table = 0;
    uint64_t groups = 0, wavefronts = 0;

    std::vector<uint32_t> local(n, UINT32_MAX);      // table entry of a device mass in the current block
    std::vector<uint32_t> entries;                    // device index per table entry
    std::vector<std::vector<uint32_t>> groups_of;     // access groups touching each entry
    std::vector<std::vector<uint32_t>> group_members; // entries per access group (distinct)
    std::vector<int> color;
    for (uint32_t b = 0; b < n_blocks; ++b) {
        const uint32_t m0 = b * kHaloBlock, m1 = std::min(n, m0 + kHaloBlock);
        entries.clear();
        for (uint32_t m = m0; m < m1; ++m) { local[m] = (uint32_t)entries.size(); entries.push_back(m); }
        const uint32_t own = (uint32_t)entries.size();
        group_members.clear();
        // access groups: (slice, column, half-warp) -> distinct entries read
        for (uint32_t w = 0; w < slices_per_block; ++w) {
            const uint32_t sl = b * slices_per_block + w;
            if (sl >= n_slices) break;
            const uint32_t e0 = sell.slice_off[sl], width = (sell.slice_off[sl + 1] - e0) / 32;
            for (uint32_t t = 0; t < width; ++t)
                for (uint32_t h = 0; h < 2; ++h) {
                    std::vector<uint32_t> g;
                    for (uint32_t l = 16 * h; l < 16 * h + 16; ++l) {
                        if (sl * 32 + l >= n) continue;
                        const uint32_t j = sell.nbr[e0 + 32 * t + l];
                        if (local[j] == UINT32_MAX) { local[j] = (uint32_t)entries.size(); entries.push_back(j); }
                        g.push_back(local[j]);
                    }
                    std::sort(g.begin(), g.end());
                    g.erase(std::unique(g.begin(), g.end()), g.end());
                    if (g.size() > 1) group_members.push_back(std::move(g));
                }
        }
        // the own-state writes: one group per half-warp of own masses
        for (uint32_t h = 0; 16 * h < own; ++h) {
            std::vector<uint32_t> g;
            for (uint32_t l = 16 * h; l < std::min(own, 16 * h + 16); ++l) g.push_back(l);
            if (g.size() > 1) group_members.push_back(std::move(g));
        }
        const uint32_t T = (uint32_t)entries.size();
        groups_of.assign(T, {});
        for (uint32_t gi = 0; gi < group_members.size(); ++gi)
            for (uint32_t e : group_members[gi]) groups_of[e].push_back(gi);
        // greedy colouring, most-constrained entries first; ties go to the least-used colour
        std::vector<uint32_t> order(T);
        std::iota(order.begin(), order.end(), 0u);
        std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) {
            return groups_of[x].size() > groups_of[y].size();
        });
        color.assign(T, -1);
        std::vector<uint32_t> used(16, 0);
        if (grid_colours) {
            for (uint32_t e = 0; e < T; ++e) { color[e] = (int)(entries[e] & 15); ++used[color[e]]; }
            order.clear();
        }
        for (uint32_t e : order) {
            uint32_t cost[16] = {0};
            for (uint32_t gi : groups_of[e])
                for (uint32_t o : group_members[gi])
                    if (o != e && color[o] >= 0) ++cost[color[o]];
            int best = 0;
            for (int c = 1; c < 16; ++c)
                if (cost[c] < cost[best] || (cost[c] == cost[best] && used[c] < used[best])) best = c;
            color[e] = best;
            ++used[best];
        }
        uint32_t rows = 0;
        for (int c = 0; c < 16; ++c) rows = std::max(rows, used[c]);
        const uint32_t table = 16 * rows;
        if (table > max_slots) {
            for (uint32_t e = 0; e < T; ++e) local[entries[e]] = UINT32_MAX;
            return false;
        }
        out.max_table = std::max(out.max_table, table);
        std::vector<uint32_t> next_row(16, 0), slot(T);
        for (uint32_t e = 0; e < T; ++e) slot[e] = 16 * next_row[color[e]]++ + (uint32_t)color[e];
        for (uint32_t m = m0; m < m1; ++m) out.own_slot[m] = (uint16_t)slot[local[m]];
        for (uint32_t e = own; e < T; ++e) {
            out.ext_idx.push_back(entries[e]);
            out.ext_slot.push_back((uint16_t)slot[e]);
        }
        out.ext_off[b + 1] = (uint32_t)out.ext_idx.size();
        for (uint32_t w = 0; w < slices_per_block; ++w) {
            const uint32_t sl = b * slices_per_block + w;
            if (sl >= n_slices) break;
            const uint32_t e0 = sell.slice_off[sl], e1 = sell.slice_off[sl + 1];
            for (uint32_t e = e0; e < e1; ++e) {
                const uint32_t l = (e - e0) % 32;
                const uint32_t j = (sl * 32 + l < n) ? sell.nbr[e] : m0;
                out.nbr_slot[e] = (uint16_t)slot[local[j]];
            }
            // conflict statistics: wavefronts per half-warp access
            const uint32_t width = (e1 - e0) / 32;
            for (uint32_t t = 0; t < width; ++t)
                for (uint32_t h = 0; h < 2; ++h) {
                    uint32_t per_bank[16] = {0};
                    std::vector<uint32_t> seen;
                    for (uint32_t l = 16 * h; l < 16 * h + 16; ++l) {
                        if (sl * 32 + l >= n) continue;
                        const uint32_t sslot = out.nbr_slot[e0 + 32 * t + l];
                        if (std::find(seen.begin(), seen.end(), sslot) != seen.end()) continue;
                        seen.push_back(sslot);
                        ++per_bank[sslot % 16];
                    }
                    uint32_t ways = 1;
                    for (int c = 0; c < 16; ++c) ways = std::max(ways, per_bank[c]);
                    wavefronts += ways;
                    ++groups;
                }
        }
        for (uint32_t e = 0; e < T; ++e) local[entries[e]] = UINT32_MAX;
    }
    out.conflict_ways = groups ? (double)wavefronts / (double)groups : 1.0;
    return true;
}

bool build_box(uint32_t n, const SellHost &sell, const std::vector<int32_t> &cell,
               const std::vector<uint32_t> &caller_of_dev, uint32_t max_slots, BoxHost &out) {
    const uint32_t n_blocks = (n + kHaloBlock - 1) / kHaloBlock;
    const uint32_t slices_per_block = kHaloBlock / 32;
    const uint32_t n_slices = (n + 31) / 32;
    if (cell.size() != 3 * (size_t)n || caller_of_dev.size() != n || sell.slice_off.size() != (size_t)n_slices + 1)
        return false;
    if (max_slots >= kBoxHole) return false;
    auto hole = [&](uint32_t m) { return caller_of_dev[m] == UINT32_MAX; };
    out.col_off.assign(sell.entries / 32, 0);
    out.own_slot.assign(n, 0);
    out.ext_off.assign(n_blocks + 1, 0);
    out.ext_idx.clear();
    out.ext_slot.clear();
    out.dims.assign(2 * (size_t)n_blocks, 0);
    out.max_table = 0;
    const int32_t *C = cell.data();
    std::vector<uint32_t> seen;     // external masses of the current block
    for (uint32_t b = 0; b < n_blocks; ++b) {
        const uint32_t m0 = b * kHaloBlock, m1 = std::min(n, m0 + kHaloBlock);
        const uint32_t sl0 = b * slices_per_block, sl1 = std::min(n_slices, sl0 + slices_per_block);
        int64_t lo[3], hi[3], R[3] = {0, 0, 0};
        for (int a = 0; a < 3; ++a) { lo[a] = INT64_MAX; hi[a] = INT64_MIN; }
        for (uint32_t m = m0; m < m1; ++m)
            for (int a = 0; a < 3; ++a) {
                lo[a] = std::min<int64_t>(lo[a], C[3 * (size_t)m + a]);
                hi[a] = std::max<int64_t>(hi[a], C[3 * (size_t)m + a]);
            }
        for (uint32_t sl = sl0; sl < sl1; ++sl)
            for (uint32_t e = sell.slice_off[sl]; e < sell.slice_off[sl + 1]; ++e) {
                if (sell.spring[e] == UINT32_MAX) continue;
                const uint32_t i = sl * 32 + (e - sell.slice_off[sl]) % 32, j = sell.nbr[e];
                for (int a = 0; a < 3; ++a)
                    R[a] = std::max<int64_t>(R[a], std::llabs((int64_t)C[3 * (size_t)j + a] - C[3 * (size_t)i + a]));
            }
        int64_t dim[3];
        for (int a = 0; a < 3; ++a) {
            lo[a] -= R[a];
            hi[a] += R[a];
            dim[a] = hi[a] - lo[a] + 1;
        }
        dim[0] += ((4 - dim[0]) % 8 + 8) % 8;            // X = 4 (mod 8)
        const int64_t slots = dim[0] * dim[1] * dim[2];
        if (slots > (int64_t)max_slots || slots > 32767) return false;
        out.max_table = std::max<uint32_t>(out.max_table, (uint32_t)slots);
        out.dims[2 * (size_t)b] = (uint32_t)dim[0];
        out.dims[2 * (size_t)b + 1] = (uint32_t)dim[1];
        auto slot = [&](uint32_t m) -> int64_t {
            return (C[3 * (size_t)m] - lo[0]) + dim[0] * ((C[3 * (size_t)m + 1] - lo[1]) + dim[1] * (C[3 * (size_t)m + 2] - lo[2]));
        };
        for (uint32_t m = m0; m < m1; ++m) out.own_slot[m] = hole(m) ? kBoxHole : (uint16_t)slot(m);
        seen.clear();
        for (uint32_t sl = sl0; sl < sl1; ++sl) {
            const uint32_t e0 = sell.slice_off[sl], w = (sell.slice_off[sl + 1] - e0) / 32;
            for (uint32_t t = 0; t < w; ++t) {
                bool have = false;
                int64_t off = 0;
                for (uint32_t l = 0; l < 32; ++l) {
                    const uint32_t e = e0 + 32 * t + l, i = sl * 32 + l;
                    if (i >= n || sell.spring[e] == UINT32_MAX) continue;
                    const uint32_t j = sell.nbr[e];
                    if (hole(i) || hole(j)) return false;             // holes have no springs
                    const int64_t o = slot(j) - slot(i);
                    if (have && o != off) return false;           // column not offset-aligned
                    // the neighbour's cell must be exactly the offset cell
                    for (int a = 0; a < 3; ++a)
                        if (C[3 * (size_t)j + a] < lo[a] || C[3 * (size_t)j + a] > hi[a]) return false;
                    have = true;
                    off = o;
                    if (j < m0 || j >= m1) seen.push_back(j);
                }
                // every lane's read, padding included, must stay inside the box
                for (uint32_t l = 0; l < 32; ++l) {
                    const uint32_t i = sl * 32 + l;
                    if (i >= n || hole(i)) continue;
                    const int64_t r = slot(i) + off;
                    if (r < 0 || r >= slots) return false;
                }
                out.col_off[e0 / 32 + t] = (int16_t)off;
            }
        }
        std::sort(seen.begin(), seen.end());
        seen.erase(std::unique(seen.begin(), seen.end()), seen.end());
        for (uint32_t j : seen) {
            out.ext_idx.push_back(j);
            out.ext_slot.push_back((uint16_t)slot(j));
        }
        out.ext_off[b + 1] = (uint32_t)out.ext_idx.size();
    }
    return true;
}

bool build_cube(uint32_t n, uint32_t s, const uint32_t *ends, const std::vector<uint32_t> &dev_of,
                const SellHost &sell, const std::vector<int32_t> &cell, const std::vector<uint32_t> &caller_of_dev,
                const BoxHost &box, CubeHost &out) {
    constexpr uint32_t P = kCubePasses, W = kHaloBlock / 32;
    if (n % kHaloBlock || cell.size() != 3 * (size_t)n || caller_of_dev.size() != n || box.own_slot.size() != n)
        return false;
    const uint32_t n_cubes = n / kHaloBlock;
    auto pass_of = [&](int dx, int dy, int dz, int &sign) -> int {
        for (uint32_t j = 0; j < P; ++j) {
            if (kCubeDirs[j][0] == dx && kCubeDirs[j][1] == dy && kCubeDirs[j][2] == dz) { sign = +1; return (int)j; }
            if (kCubeDirs[j][0] == -dx && kCubeDirs[j][1] == -dy && kCubeDirs[j][2] == -dz) { sign = -1; return (int)j; }
        }
        return -1;
    };
    const int32_t *C = cell.data();
    out.base.assign(n_cubes + 1, 0);
    out.meta.assign((size_t)n_cubes * P * W * 4, 0);
    out.spring.clear();
    out.pos_of_end.assign(2 * (size_t)s, UINT32_MAX);
    // per spring end: the end index (0 = ends[2q]) of device mass m
    auto end_of = [&](uint32_t q, uint32_t m) -> int { return dev_of[ends[2 * (size_t)q]] == m ? 0 : 1; };
    std::vector<uint32_t> plus(P * kHaloBlock), minus(P * kHaloBlock);
    for (uint32_t b = 0; b < n_cubes; ++b) {
        const uint32_t m0 = b * kHaloBlock;
        std::fill(plus.begin(), plus.end(), UINT32_MAX);
        std::fill(minus.begin(), minus.end(), UINT32_MAX);
        // every spring of the cube's masses, by pass and sign
        for (uint32_t sl = m0 / 32; sl < (m0 + kHaloBlock) / 32; ++sl)
            for (uint32_t e = sell.slice_off[sl]; e < sell.slice_off[sl + 1]; ++e) {
                const uint32_t q = sell.spring[e];
                if (q == UINT32_MAX) continue;
                const uint32_t m = sl * 32 + (e - sell.slice_off[sl]) % 32, j = sell.nbr[e];
                const int dx = C[3 * (size_t)j] - C[3 * (size_t)m], dy = C[3 * (size_t)j + 1] - C[3 * (size_t)m + 1],
                          dz = C[3 * (size_t)j + 2] - C[3 * (size_t)m + 2];
                int sign = 0;
                const int pj = pass_of(dx, dy, dz, sign);
                if (pj < 0) return false;                                   // not a 26-neighbour offset
                uint32_t &slot = (sign > 0 ? plus : minus)[(size_t)pj * kHaloBlock + (m - m0)];
                if (slot != UINT32_MAX) return false;                       // two springs, one offset
                slot = q;
            }
        const uint32_t start = (uint32_t)out.spring.size();
        out.base[b] = start;
        for (uint32_t pj = 0; pj < P; ++pj)
            for (uint32_t t = 0; t < kHaloBlock; ++t) {
                const uint32_t q = plus[(size_t)pj * kHaloBlock + t];
                if (q != UINT32_MAX) out.pos_of_end[2 * (size_t)q + end_of(q, m0 + t)] = (uint32_t)out.spring.size();
                out.spring.push_back(q);
            }
        const uint32_t ext_start = (uint32_t)out.spring.size();
        for (uint32_t pj = 0; pj < P; ++pj) {
            const int dx = kCubeDirs[pj][0], dy = kCubeDirs[pj][1], dz = kCubeDirs[pj][2];
            // box slot offset of +p in this cube's table
            const int32_t X = (int32_t)box.dims[2 * (size_t)b], Y = (int32_t)box.dims[2 * (size_t)b + 1];
            const int32_t off = dx + X * dy + X * Y * dz;
            for (uint32_t w = 0; w < W; ++w) {
                uint32_t recv = 0, ext = 0;
                const uint32_t ext_base = (uint32_t)out.spring.size() - ext_start;
                for (uint32_t l = 0; l < 32; ++l) {
                    const uint32_t t = w * 32 + l, m = m0 + t;
                    const uint32_t qp = plus[(size_t)pj * kHaloBlock + t], qm = minus[(size_t)pj * kHaloBlock + t];
                    if (qp != UINT32_MAX) {
                        const uint32_t j = dev_of[ends[2 * (size_t)qp + 1 - end_of(qp, m)]];
                        if (j >= m0 && j < m0 + kHaloBlock &&
                            (int32_t)box.own_slot[j] - (int32_t)box.own_slot[m] != off)
                            return false;
                    }
                    if (qm == UINT32_MAX) continue;
                    const uint32_t j = dev_of[ends[2 * (size_t)qm + 1 - end_of(qm, m)]];   // the -p partner
                    if (j >= m0 && j < m0 + kHaloBlock) {
                        // in the cube: its +p spring must be this one
                        if (plus[(size_t)pj * kHaloBlock + (j - m0)] != qm) return false;
                        recv |= 1u << l;
                    } else {
                        ext |= 1u << l;
                        out.pos_of_end[2 * (size_t)qm + end_of(qm, m)] = (uint32_t)out.spring.size();
                        out.spring.push_back(qm);
                    }
                }
                uint32_t *mt = &out.meta[(((size_t)b * P + pj) * W + w) * 4];
                mt[0] = recv;
                mt[1] = ext;
                mt[2] = ext_base;
                mt[3] = (uint32_t)(uint16_t)(int16_t)off;
            }
        }
        // every cube's region starts on a 128-byte boundary (its plus rows are 2 KB each)
        while (out.spring.size() % 16) out.spring.push_back(UINT32_MAX);
    }
    out.base[n_cubes] = (uint32_t)out.spring.size();
    out.entries = (uint32_t)out.spring.size();
    return true;
}

void build_records(uint32_t s, const uint32_t *ends, const std::vector<uint32_t> &dev_of,
                   RecordsHost &out) {
    out.order.resize(s);
    std::iota(out.order.begin(), out.order.end(), 0u);
    std::vector<uint64_t> key(s);
    for (uint32_t q = 0; q < s; ++q) {
        const uint64_t a = dev_of[ends[2 * (size_t)q]], b = dev_of[ends[2 * (size_t)q + 1]];
        key[q] = (std::min(a, b) << 32) | std::max(a, b);
    }
    std::stable_sort(out.order.begin(), out.order.end(),
                     [&](uint32_t x, uint32_t y) { return key[x] < key[y]; });
    out.slot_of_spring.resize(s);
    for (uint32_t r = 0; r < s; ++r) out.slot_of_spring[out.order[r]] = r;
}

size_t persistent_smem_bytes(uint32_t per_cta, uint32_t max_halo, uint32_t max_entries, bool has_c, bool has_act) {
    return persist_layout(per_cta, max_halo, max_entries, has_c, has_act).total;
}

bool plan_persistent(uint32_t n, const std::vector<uint32_t> &slice_off, const std::vector<uint32_t> &nbr,
                     bool has_c, bool has_act, size_t smem_limit, PersistPlan &plan,
                     std::vector<uint16_t> &slot, std::vector<uint32_t> &halo) {
    if (n == 0 || slice_off.size() != (size_t)(n + 31) / 32 + 1 || nbr.size() != slice_off.back()) return false;
    // per cluster size: masses per CTA, each CTA's entries and halo (the
    // distinct masses of other CTAs its rows touch, in first-use order)
    struct Try {
        uint32_t per = 0, max_e = 0, max_h = 0;
        std::vector<uint32_t> halo_off;
        std::vector<uint32_t> halo;
        std::vector<uint16_t> slot;
        size_t bytes = 0;
    };
    auto build = [&](uint32_t cl, Try &t) {
        t.per = ((n + cl - 1) / cl + 31) & ~31u;
        if (t.per > 4096) return false;
        t.halo_off.assign(9, 0);
        t.halo.clear();
        t.slot.assign(nbr.size(), 0);
        std::vector<uint32_t> local(n, UINT32_MAX);
        for (uint32_t r = 0; r < cl; ++r) {
            const uint32_t m0 = r * t.per, m1 = std::min(n, m0 + t.per);
            const size_t h0 = t.halo.size();
            if (m0 < n) {
                const uint32_t sl0 = m0 / 32, sl1 = (m1 + 31) / 32;
                t.max_e = std::max(t.max_e, slice_off[sl1] - slice_off[sl0]);
                for (uint32_t e = slice_off[sl0]; e < slice_off[sl1]; ++e) {
                    const uint32_t j = nbr[e];
                    if (j >= m0 && j < m1) {
                        t.slot[e] = (uint16_t)(j - m0);
                        continue;
                    }
                    if (local[j] == UINT32_MAX) {
                        local[j] = (uint32_t)(t.per + (t.halo.size() - h0));
                        t.halo.push_back(((j / t.per) << 16) | (j % t.per));
                    }
                    t.slot[e] = (uint16_t)local[j];
                }
                for (size_t h = h0; h < t.halo.size(); ++h) {       // reset the first-use map
                    const uint32_t code = t.halo[h];
                    local[(code >> 16) * t.per + (code & 0xffffu)] = UINT32_MAX;
                }
            }
            t.halo_off[r + 1] = (uint32_t)t.halo.size();
            t.max_h = std::max<uint32_t>(t.max_h, (uint32_t)(t.halo.size() - h0));
        }
        for (uint32_t r = cl; r < 8; ++r) t.halo_off[r + 1] = t.halo_off[r];
        if (t.per + t.max_h > 65535) return false;
        t.bytes = persistent_smem_bytes(t.per, t.max_h, t.max_e, has_c, has_act);
        return t.bytes <= smem_limit;
    };
    // the smallest cluster that fits and gives each thread one mass (512 per
    // CTA); failing that, the smallest that fits at all
    Try t;
    uint32_t cl = 0;
    for (int pass = 0; pass < 2 && !cl; ++pass)
        for (uint32_t c2 = 1; c2 <= 8 && !cl; c2 *= 2) {
            if (pass == 0 && (((n + c2 - 1) / c2 + 31) & ~31u) > 512) continue;
            t = Try();
            if (build(c2, t)) cl = c2;
        }
    if (!cl) return false;
    plan.cluster = cl;
    plan.per_cta = t.per;
    plan.max_entries = t.max_e;
    plan.max_halo = t.max_h;
    plan.smem = t.bytes;
    plan.threads = std::min<uint32_t>(512, t.per);
    for (int r = 0; r < 9; ++r) plan.halo_off[r] = t.halo_off[r];
    slot.swap(t.slot);
    halo.swap(t.halo);
    return true;
}


bool build_batch(uint32_t n_systems, const titan_masses *masses, const titan_springs *springs,
                 const titan_actuation *act, BatchHost &out, std::string *why) {
    out = BatchHost();
    bool any_act = false;
    for (uint32_t r = 0; r < n_systems; ++r)
        if (act && act[r].amp) any_act = true;
    out.any_act = any_act;
    // per system: the CTAs' rows, halo lists and descriptors (offsets into
    // the global arrays are set when the CTAs are placed in launch order)
    struct CtaHost {
        BatchCta d;
        std::vector<uint32_t> slices;
        std::vector<float> kl, act;
        std::vector<uint16_t> nbr;   // own slot or halo slot per entry
        std::vector<uint32_t> halo;  // rank << 16 | slot of each halo mass in its owner CTA
    };
    std::vector<std::vector<CtaHost>> per_sys(n_systems);
    std::vector<uint32_t> cluster_of(n_systems);
    uint32_t slot_cursor = 0;
    for (uint32_t r = 0; r < n_systems; ++r) {
        const titan_masses &m = masses[r];
        const titan_springs &s = springs[r];
        const bool sys_act = act && act[r].amp;
        // incidence in caller order: row of mass i = its half-edges (neighbour, spring), sorted
        std::vector<uint32_t> deg(m.n, 0);
        for (uint32_t q = 0; q < s.n; ++q) { ++deg[s.ends[2 * (size_t)q]]; ++deg[s.ends[2 * (size_t)q + 1]]; }
        std::vector<uint32_t> rowptr(m.n + 1, 0);
        for (uint32_t i = 0; i < m.n; ++i) rowptr[i + 1] = rowptr[i] + deg[i];
        std::vector<std::pair<uint32_t, uint32_t>> he(rowptr[m.n]);
        std::vector<uint32_t> cur(rowptr.begin(), rowptr.end() - 1);
        for (uint32_t q = 0; q < s.n; ++q) {
            const uint32_t i = s.ends[2 * (size_t)q], j = s.ends[2 * (size_t)q + 1];
            he[cur[i]++] = {j, q};
            he[cur[j]++] = {i, q};
        }
        for (uint32_t i = 0; i < m.n; ++i) std::sort(he.begin() + rowptr[i], he.begin() + rowptr[i + 1]);
        // distinct masses outside [q0, q1) that the rows of [q0, q1) touch
        std::vector<uint32_t> mark(m.n, UINT32_MAX);
        uint32_t gen = 0;
        auto halo_count = [&](uint32_t q0, uint32_t q1) {
            ++gen;                                    // a fresh mark for every call
            uint32_t cnt = 0;
            for (uint32_t i = q0; i < q1; ++i)
                for (uint32_t r2 = rowptr[i]; r2 < rowptr[i + 1]; ++r2) {
                    const uint32_t j = he[r2].first;
                    if ((j < q0 || j >= q1) && mark[j] != gen) { mark[j] = gen; ++cnt; }
                }
            return cnt;
        };
        // smallest cluster whose per-CTA shared memory fits
        uint32_t C = 1;
        for (;; C *= 2) {
            if (C > kBatchMaxCluster) {
                if (why) *why = "system " + std::to_string(r) + " does not fit a cluster of 8 CTAs";
                out = BatchHost();
                return false;
            }
            const uint32_t per = ((m.n + C - 1) / C + 31) & ~31u;
            if (per > kBatchMaxPerCta) continue;
            // the layout of every CTA of the cluster reserves the largest halo
            uint32_t hc = 0;
            if (C > 1)
                for (uint32_t q0 = 0; q0 < m.n; q0 += per) hc = std::max(hc, halo_count(q0, std::min(m.n, q0 + per)));
            size_t worst = 0;
            for (uint32_t q0 = 0; q0 < m.n; q0 += per) {
                uint32_t edges = 0, ns = 0;
                std::vector<uint32_t> dq(deg.begin() + q0, deg.begin() + std::min(m.n, q0 + per));
                std::sort(dq.begin(), dq.end(), std::greater<uint32_t>());
                for (uint32_t sl = 0; sl < (uint32_t)dq.size(); sl += 32, ++ns)
                    edges += 32 * ((dq[sl] + 1) & ~1u);      // a slice's widest row is its first
                edges = (edges + 63) & ~63u;
                worst = std::max<size_t>(worst, batch_smem_layout(per, hc, ns, edges, any_act).total);
            }
            if (worst <= kBatchSmemLimit && per + hc <= 65535) break;
        }
        cluster_of[r] = C;
        const uint32_t per = ((m.n + C - 1) / C + 31) & ~31u;
        out.mass_off.push_back(slot_cursor);
        out.mass_cnt.push_back(m.n);
        // each CTA's masses by decreasing degree (ties in caller order):
        // mass_at[q * per + p] is the mass in slot p of CTA q, pos_of[j] the slot of mass j in its CTA
        std::vector<uint32_t> mass_at((size_t)C * per, UINT32_MAX), pos_of(m.n);
        for (uint32_t q = 0; q < C; ++q) {
            const uint32_t a0 = std::min(m.n, q * per), a1 = std::min(m.n, a0 + per);
            std::vector<uint32_t> perm(a1 - a0);
            std::iota(perm.begin(), perm.end(), a0);
            std::stable_sort(perm.begin(), perm.end(), [&](uint32_t x, uint32_t y) { return deg[x] > deg[y]; });
            for (uint32_t p = 0; p < (uint32_t)perm.size(); ++p) {
                mass_at[(size_t)q * per + p] = perm[p];
                pos_of[perm[p]] = p;
            }
        }
        for (uint32_t q = 0; q < C; ++q) {
            CtaHost h;
            const uint32_t m0 = std::min(m.n, q * per), m1 = std::min(m.n, m0 + per);
            h.d = BatchCta{slot_cursor + m0, m1 - m0, per, 0, 0, 0, 0, r, 0, 0, 0};
            // neighbours as own slots (pos_of[j]) or halo slots (per + h)
            std::fill(mark.begin(), mark.end(), UINT32_MAX);      // here: halo slot of a mass
            auto slot_of = [&](uint32_t j) -> uint16_t {
                if (j >= m0 && j < m1) return (uint16_t)pos_of[j];
                if (mark[j] == UINT32_MAX) {
                    mark[j] = per + (uint32_t)h.halo.size();
                    h.halo.push_back(((j / per) << 16) | pos_of[j]);
                }
                return (uint16_t)mark[j];
            };
            const uint32_t *at = mass_at.data() + (size_t)q * per;
            const uint32_t count = m1 - m0;
            h.slices.push_back(0);
            for (uint32_t sl = 0; sl < per; sl += 32) {
                uint32_t w = 0;
                for (uint32_t p = sl; p < std::min(count, sl + 32); ++p) w = std::max(w, deg[at[p]]);
                w = (w + 1) & ~1u;
                const uint32_t base = (uint32_t)h.nbr.size();
                h.kl.resize(2 * (size_t)(base + 32 * w), 0.f);
                h.act.resize(2 * (size_t)(base + 32 * w), 0.f);
                h.nbr.resize(base + 32 * w, 0);
                for (uint32_t l = 0; l < 32; ++l) {
                    const uint32_t p = sl + l;                          // slot of this row
                    const uint32_t i = p < count ? at[p] : UINT32_MAX;   // its mass (none: padding slot)
                    for (uint32_t t = 0; t < w; ++t) {
                        const uint32_t e = base + 32 * t + l;
                        if (p < count && t < deg[i]) {
                            const auto &x = he[rowptr[i] + t];
                            const uint32_t j = x.first, q2 = x.second;
                            h.nbr[e] = slot_of(j);
                            double L;
                            if (s.rest) L = s.rest[q2];
                            else {
                                double d2 = 0;
                                for (int a = 0; a < 3; ++a) {
                                    const double dd = m.pos[3 * (size_t)j + a] - m.pos[3 * (size_t)i + a];
                                    d2 += dd * dd;
                                }
                                L = std::sqrt(d2);
                            }
                            h.kl[2 * (size_t)e] = (float)s.k[q2];
                            h.kl[2 * (size_t)e + 1] = (float)L;
                            if (sys_act) {
                                h.act[2 * (size_t)e] = (float)(act[r].amp[q2] * std::cos(act[r].phase[q2]));
                                h.act[2 * (size_t)e + 1] = (float)(act[r].amp[q2] * std::sin(act[r].phase[q2]));
                            }
                        } else {
                            h.nbr[e] = (uint16_t)p;          // zero-parameter padding: the row's own slot
                        }
                    }
                }
                h.slices.push_back((uint32_t)h.nbr.size());
            }
            const uint32_t E = ((uint32_t)h.nbr.size() + 63) & ~63u;
            h.kl.resize(2 * (size_t)E, 0.f);
            h.act.resize(2 * (size_t)E, 0.f);
            h.nbr.resize(E, 0);
            h.d.edge_count = E;
            h.d.n_slices = (uint32_t)h.slices.size() - 1;
            h.d.halo_count = (uint32_t)h.halo.size();
            per_sys[r].push_back(std::move(h));
        }
        uint32_t halo_slots = 0;
        for (const auto &hh : per_sys[r]) halo_slots = std::max(halo_slots, hh.d.halo_count);
        for (auto &hh : per_sys[r]) hh.d.halo_slots = halo_slots;
        slot_cursor += C * per;
        // initial state of every slot of this system (padding slots: fixed, at rest)
        out.init_state.resize(8 * (size_t)slot_cursor, 0.f);
        out.mass_of_slot.resize(slot_cursor, UINT32_MAX);
        for (size_t sl = 0; sl < mass_at.size(); ++sl) out.mass_of_slot[out.mass_off[r] + sl] = mass_at[sl];
        for (uint32_t k = 0; k < m.n; ++k) {
            const uint32_t q = k / per;
            float *st = &out.init_state[8 * (size_t)(out.mass_off[r] + (size_t)q * per + pos_of[k])];
            for (int a = 0; a < 3; ++a) {
                st[a] = (float)m.pos[3 * (size_t)k + a];
                st[4 + a] = m.vel ? (float)m.vel[3 * (size_t)k + a] : 0.f;
            }
            st[3] = (m.fixed && m.fixed[k]) ? 0.f : (float)(1.0 / m.mass[k]);
        }
    }
    out.total_slots = slot_cursor;
    // launch groups by (cluster size, shared-memory class); a launch's
    // dynamic shared memory is the largest of its CTAs'
    static const uint32_t kPerSm[] = {1, 2, 3, 4, 6, 8};
    auto smem_class = [&](uint32_t r) {
        size_t worst = 0;
        for (const auto &h : per_sys[r])
            worst = std::max<size_t>(worst, batch_smem_layout(h.d.slot_count, h.d.halo_slots, h.d.n_slices,
                                                              h.d.edge_count, any_act).total);
        uint32_t cls = 0;
        for (uint32_t k = 0; k < sizeof(kPerSm) / sizeof(kPerSm[0]); ++k)
            if (worst + 1024 <= 228u * 1024u / kPerSm[k]) cls = k;
        return cls;
    };
    std::vector<uint32_t> class_of(n_systems);
    for (uint32_t r = 0; r < n_systems; ++r) class_of[r] = smem_class(r);
    std::vector<uint32_t> order(n_systems);
    for (uint32_t r = 0; r < n_systems; ++r) order[r] = r;
    std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) {
        if (cluster_of[x] != cluster_of[y]) return cluster_of[x] > cluster_of[y];
        if (class_of[x] != class_of[y]) return class_of[x] < class_of[y];
        return masses[x].n > masses[y].n;
    });
    for (uint32_t k = 0; k < n_systems; ++k) {
        const uint32_t r = order[k];
        if (out.groups.empty() || out.groups.back().cluster != cluster_of[r] || class_of[order[k - 1]] != class_of[r]) {
            BatchGroup g;
            g.cluster = cluster_of[r];
            g.cta_first = (uint32_t)out.ctas.size();
            out.groups.push_back(g);
        }
        BatchGroup &g = out.groups.back();
        for (auto &h : per_sys[r]) {
            h.d.edge_off = (uint32_t)out.nbr.size();
            while (out.slices.size() % 4) out.slices.push_back(0);
            h.d.slice_base = (uint32_t)out.slices.size();
            out.slices.insert(out.slices.end(), h.slices.begin(), h.slices.end());
            while (out.slices.size() % 4) out.slices.push_back(0);
            out.kl.insert(out.kl.end(), h.kl.begin(), h.kl.end());
            if (any_act) out.act.insert(out.act.end(), h.act.begin(), h.act.end());
            out.nbr.insert(out.nbr.end(), h.nbr.begin(), h.nbr.end());
            h.d.halo_off = (uint32_t)out.halo.size();
            out.halo.insert(out.halo.end(), h.halo.begin(), h.halo.end());
            out.ctas.push_back(h.d);
            ++g.cta_count;
            g.smem = std::max<size_t>(g.smem, batch_smem_layout(h.d.slot_count, h.d.halo_slots, h.d.n_slices,
                                                                h.d.edge_count, any_act).total);
        }
        per_sys[r].clear();
    }
    return true;
}

}  // namespace titan
